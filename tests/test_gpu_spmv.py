"""The CSR SpMV kernels (asm_csr_spmv through the C ABI) against SciPy.

Short rows (at most about 12 entries on average) take the one-thread-per-row
kernel, which loads a row's first 8 entries at once and finishes longer rows
in a loop; longer rows on average take the lane-group kernel.  The sums run
in a different order from SciPy's, so each row is compared within 1e-14 of
sum_k |a_rk x_k|.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from asm_inputs import SplitMix64, diffusion3d, elasticity3d

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    from paper_2401_03915_gb300 import build
    build.build()
    import paper_2401_03915_gb300 as P
    P.load()
    return P


def check(P, A, seed=3):
    A = sp.csr_matrix(A)
    n = A.shape[0]
    dev = torch.device("cuda")
    rp = torch.as_tensor(A.indptr.astype(np.int32), device=dev)
    ci = torch.as_tensor(A.indices.astype(np.int32), device=dev)
    va = torch.as_tensor(A.data.astype(np.float64), device=dev)
    x = SplitMix64(seed).normal(n)
    xt = torch.as_tensor(x, device=dev)
    yt = torch.full((n,), np.nan, dtype=torch.float64, device=dev)
    P.asm_csr_spmv(rp, ci, va, xt, yt)
    y = yt.cpu().numpy()
    ref = A @ x
    scale = abs(A) @ np.abs(x)
    assert np.all(np.abs(y - ref) <= 1e-14 * scale + 1e-300), np.max(np.abs(y - ref) / (scale + 1e-300))


def test_spmv_stencil_short_rows(P):
    check(P, diffusion3d(24, (3, 3, 3), contrast=1e6).csr())


def test_spmv_long_rows(P):
    check(P, elasticity3d(6, (2, 2, 2)).csr())


def _ragged(n, long_rows, seed):
    r = SplitMix64(seed)
    lens = r.integers(0, 7, n)
    lens[long_rows] = 200
    lens[::97] = 0
    rows = np.repeat(np.arange(n), lens)
    cols = np.concatenate([np.sort(r.integers(0, n - 1, int(k))) if k else np.zeros(0, np.int64) for k in lens])
    A = sp.coo_matrix((r.normal(len(rows)), (rows, cols)), shape=(n, n)).tocsr()
    A.sum_duplicates()
    return A


def test_spmv_ragged_short_rows_with_a_few_long_ones(P):
    """One thread per row (about 4 entries on average): n not a multiple of
    the 256-thread block, empty rows, 20 rows of 200 entries (beyond the 8
    loaded up front)."""
    A = _ragged(4001, slice(1000, 1020), 11)
    assert A.nnz / A.shape[0] <= 12
    check(P, A)


def test_spmv_ragged_long_rows(P):
    """Lane groups (about 44 entries on average), empty rows, ragged n."""
    A = _ragged(1000, slice(300, 512), 12)
    assert A.nnz / A.shape[0] > 12
    check(P, A)


def test_spmv_tiny(P):
    check(P, sp.csr_matrix(np.array([[2.0]])))
    check(P, sp.diags([1.0, -2.0, 3.0]).tocsr())


def test_pcg_spmv_timing_helper(P):
    """asm_time_spmv runs the PCG loop's fused q = A p, p.q launch."""
    prob = diffusion3d(16, (2, 2, 2), contrast=1e3, nev=4)
    A = prob.csr()
    pre = P.TwoLevelSchwarz(A.indptr, A.indices, A.data, prob.part, prob.N, 1, 4)
    dev = torch.device("cuda")
    p = torch.as_tensor(SplitMix64(4).normal(prob.n), device=dev)
    q = torch.empty_like(p)
    ms = P.asm_time_spmv(pre.h, p, q, 10)
    assert ms > 0
    ref = A @ p.cpu().numpy()
    np.testing.assert_allclose(q.cpu().numpy(), ref, rtol=0, atol=1e-14 * np.abs(ref).max() * 10)
    pre.close()

