"""Full-size runs of the elasticity (3D Q1, nev 24) and convection-diffusion
(upwind, overlap 2, general path, FGMRES(30)) workloads through the C ABI.

Checked against the oracle: the overlap bit-exact on sampled subdomains, and
against tests/golden/c3_oracle_reference.json / c4_oracle_reference.json
(written by tests/golden/make_config_reference.py, which calls only the
oracle) the kept local values of EVERY subdomain, their counts, n_C and the
Krylov iteration count; plus the true residual of the solve.

Tolerance of the values: with eig_tol = 1e-3 (set here; the library's
single-precision default is 4e-3) the subspace iteration stops when every kept
Ritz pair has a relative eigen-residual ||K z - mu z|| / mu below 1e-3; for a symmetric operator some eigenvalue then lies within 1e-3 mu of
mu (Bauer-Fike for normal matrices), so the sorted values agree to a relative
1e-3 where the kept values are separated.  The iteration count is within 10%
of the FP64 oracle's (the target for the single-precision local work)."""
import json
import os

import numpy as np
import pytest

import oracle as O
from asm_inputs import config

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    from paper_2401_03915_gb300 import build
    build.build()
    import paper_2401_03915_gb300 as P
    P.load()
    return P


def _setup(P, prob, **kw):
    return P.TwoLevelSchwarz(prob.indptr, prob.indices, prob.data, prob.part, prob.N, prob.delta, prob.nev, **kw)


def _check_overlap_sampled(P, h, ovs, sample):
    sub, lay, om = P.asm_get_overlap(h)
    for i in sample:
        np.testing.assert_array_equal(lay[i], ovs[i].offsets)
        np.testing.assert_array_equal(om[sub[i]:sub[i + 1]], ovs[i].omega)


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, f"{name}_oracle_reference.json")) as f:
        return json.load(f)


def _check_values_all(vals, cnt, ref, rtol):
    assert len(ref["values"]) == len(cnt)
    bad = []
    for i, rv in enumerate(ref["values"]):
        rv = np.asarray(rv)
        if int(cnt[i]) != len(rv):
            bad.append((i, "count", int(cnt[i]), len(rv)))
            continue
        if not np.allclose(vals[i, :len(rv)], rv, rtol=rtol, atol=0):
            bad.append((i, float(np.max(np.abs(vals[i, :len(rv)] / rv - 1)))))
    assert not bad, bad[:10]


def _true_relres(prob, x):
    A = prob.csr()
    return np.linalg.norm(prob.b - A @ x) / np.linalg.norm(prob.b)


def test_c3_elasticity_full_size(P):
    prob = config("c3")
    ref = _golden("c3")
    A = prob.csr()
    pre = _setup(P, prob, precision="fp32", eig_tol=1e-3)
    ovs = O.overlap(A, prob.part, prob.N, prob.delta)
    sample = [0, prob.N // 2, prob.N - 1]
    _check_overlap_sampled(P, pre.h, ovs, sample)
    vals, cnt = P.asm_get_local_values(pre.h)
    _check_values_all(vals, cnt, ref, 1e-3)
    assert pre.info.n_C == ref["n_C"]
    x, info = pre.solve(torch.as_tensor(prob.b, device="cuda"))
    rel = _true_relres(prob, x.cpu().numpy())
    assert info.converged and rel <= 1.5e-8, (info.iterations, rel)
    assert abs(info.iterations - ref["iterations"]) <= 0.1 * ref["iterations"], (info.iterations, ref["iterations"])
    pre.close()


def test_c4_convdiff_full_size(P):
    prob = config("c4")
    ref = _golden("c4")
    A = prob.csr()
    pre = _setup(P, prob, spd=False, precision="fp32", eig_tol=1e-3)
    ovs = O.overlap(A, prob.part, prob.N, prob.delta)
    sample = [0, 517, prob.N - 1]
    _check_overlap_sampled(P, pre.h, ovs, sample)
    vals, cnt = P.asm_get_local_values(pre.h)
    # singular values of D_i Pi_i: the same residual argument on X_p X_p^T
    _check_values_all(vals, cnt, ref, 1e-3)
    assert pre.info.n_C == ref["n_C"]
    x, info = pre.solve(torch.as_tensor(prob.b, device="cuda"))
    rel = _true_relres(prob, x.cpu().numpy())
    # FGMRES stops on its least-squares estimate; the true residual follows it
    assert info.converged and rel <= 1e-7, (info.iterations, rel)
    assert abs(info.iterations - ref["iterations"]) <= 0.1 * ref["iterations"], (info.iterations, ref["iterations"])
    pre.close()


def test_c3_elasticity_bf16_subspace_iteration(P):
    """ASM_PREC_FP32_B16: the subspace iteration's operator applications on
    BF16 operands with FP32 accumulation.  Rounding U and the block to BF16
    (2^-9 relative each) perturbs the operator K = U A^_II U^T by at most
    about 2^-7 ||K|| (two roundings in each of its two products), so each kept
    value moves by at most that much: |mu~_k - mu_k| <= 2^-6 mu_1 per
    subdomain with a factor-two margin; counts, n_C and the iteration count
    within 10% of the oracle's as for FP32."""
    prob = config("c3")
    ref = _golden("c3")
    pre = _setup(P, prob, precision="fp32b")
    vals, cnt = P.asm_get_local_values(pre.h)
    errs = []
    for i, rv in enumerate(ref["values"]):
        rv = np.asarray(rv)
        assert int(cnt[i]) == len(rv), (i, int(cnt[i]), len(rv))
        errs.append(np.max(np.abs(vals[i, :len(rv)] - rv)) / rv[0])
    assert max(errs) <= 2.0 ** -6, max(errs)
    assert pre.info.n_C == ref["n_C"]
    x, info = pre.solve(torch.as_tensor(prob.b, device="cuda"))
    rel = _true_relres(prob, x.cpu().numpy())
    assert info.converged and rel <= 1.5e-8, (info.iterations, rel)
    assert abs(info.iterations - ref["iterations"]) <= 0.1 * ref["iterations"], (info.iterations, ref["iterations"])
    pre.close()
