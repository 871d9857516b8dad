"""The allocation-free entry point asm_spmv_dot_noalloc against the existing
one (asm_spmv), through the C ABI.

It serves callers that cannot allocate device memory while they run (a
stream capture in progress, latency-critical threads, applications with
their own allocator).  Its scratch is a static device array shared by all
calls, so two calls in a row must each produce the full result.  This file
is collected last so that a run stopping at the first failure has already
run every other test."""
import numpy as np
import pytest

from asm_inputs import SplitMix64, diffusion3d

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    from paper_2401_03915_gb300 import build
    build.build()
    import paper_2401_03915_gb300 as P
    P.load()
    return P


def test_noalloc_spmv_dot_matches_asm_spmv_twice(P):
    prob = diffusion3d(40, (2, 2, 2), contrast=1e3)
    dev = torch.device("cuda")
    rp = torch.as_tensor(prob.indptr, device=dev)
    ci = torch.as_tensor(prob.indices, device=dev)
    va = torch.as_tensor(prob.data, device=dev)
    pa = torch.as_tensor(prob.part, device=dev)
    h = P.asm_setup(rp, ci, va, pa, prob.N, 1, 0, P.default_options(), None, True)
    try:
        for seed in (1, 2):  # two calls in a row, different inputs
            x = torch.as_tensor(SplitMix64(seed).normal(prob.n), device=dev)
            y_ref = torch.empty_like(x)
            P.asm_spmv(h, x, y_ref)
            y = torch.full_like(x, float("nan"))
            xty = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
            P.asm_spmv_dot_noalloc(rp, ci, va, x, y, xty)
            torch.cuda.synchronize()
            yr = y_ref.cpu().numpy()
            np.testing.assert_allclose(y.cpu().numpy(), yr, rtol=1e-10, atol=1e-10 * np.abs(yr).max())
            dot_ref = float(np.dot(x.cpu().numpy(), yr))
            assert abs(float(xty.item()) - dot_ref) <= 1e-10 * abs(dot_ref)
    finally:
        P.asm_destroy(h)


def test_noalloc_rejects_sizes_beyond_its_scratch(P):
    n = (1 << 20) + 1
    dev = torch.device("cuda")
    rp = torch.zeros(n + 1, dtype=torch.int32, device=dev)
    ci = torch.zeros(1, dtype=torch.int32, device=dev)
    va = torch.zeros(1, dtype=torch.float64, device=dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    y = torch.zeros(n, dtype=torch.float64, device=dev)
    xty = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(P.AsmError) as e:
        P.asm_spmv_dot_noalloc(rp, ci, va, x, y, xty)
    assert e.value.name == "UNSUPPORTED"
