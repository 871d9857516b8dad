"""Selection of the coarse vectors by the threshold tau on the CUDA path
(Prop. 5.1: eigenvalues of eq. gevpsvd above tau^2; Section 5.2: singular
values of D_i Pi_i above tau), against the oracle's selection."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from asm_inputs import poisson2d, convdiff2d

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FP64 = dict(precision="fp64", eig_tol=1e-11, max_sweeps=400)


@pytest.fixture(scope="module")
def P():
    from paper_2401_03915_gb300 import build
    build.build()
    import paper_2401_03915_gb300 as P
    P.load()
    return P


def make(P, A, part, N, delta, nev, **kw):
    A = sp.csr_matrix(A)
    return P.TwoLevelSchwarz(A.indptr, A.indices, A.data, part, N, delta, nev, **kw)


def _near_threshold(values, thr):
    return np.any(np.abs(values - thr) <= 1e-8 * thr)


@pytest.mark.parametrize("delta", [1, 2])
def test_threshold_counts_match_oracle(P, delta):
    prob = poisson2d(64, 64, 4, 4, nev=4)
    A = prob.csr()
    tau, nev = 0.3, 40
    st = O.setup(A, prob.part, prob.N, delta, nev, tau=tau)
    pre = make(P, A, prob.part, prob.N, delta, nev, tau=tau, **FP64)
    vals, cnt = P.asm_get_local_values(pre.h)
    checked = 0
    for i, loc in enumerate(st.locals):
        if _near_threshold(loc.all_values[:nev + 1], tau * tau):
            continue
        k = len(loc.values)
        assert cnt[i] == k, (i, cnt[i], k)
        np.testing.assert_allclose(vals[i, :k], loc.values, rtol=1e-9)
        checked += 1
    assert checked >= prob.N - 2
    assert 0 < pre.info.n_C < nev * prob.N  # the threshold, not the cap, decided
    x, info = pre.solve(torch.as_tensor(prob.b, device="cuda"))
    rel = np.linalg.norm(prob.b - A @ x.cpu().numpy()) / np.linalg.norm(prob.b)
    assert info.converged and rel <= 1.5e-8
    pre.close()


def test_more_overlap_contributes_fewer_vectors_at_fixed_tau(P):
    prob = poisson2d(48, 48, 3, 3, nev=4)
    A = prob.csr()
    sizes = []
    for delta in (1, 2, 3):
        pre = make(P, A, prob.part, prob.N, delta, 80, tau=0.25, precision="fp32")
        sizes.append(pre.info.n_C)
        pre.close()
    assert sizes[0] > sizes[1] > sizes[2] > 0, sizes


def test_threshold_general_path(P):
    prob = convdiff2d(64, (4, 4), peclet=1e3, delta=2, nev=6)
    A = prob.csr()
    tau = 0.5
    st = O.setup(A, prob.part, prob.N, 2, 30, spd=False, tau=tau)
    pre = make(P, A, prob.part, prob.N, 2, 30, spd=False, tau=tau, precision="fp64", eig_tol=1e-11, max_sweeps=200)
    vals, cnt = P.asm_get_local_values(pre.h)
    for i, loc in enumerate(st.locals):
        if _near_threshold(loc.all_values[:31], tau):
            continue
        assert cnt[i] == len(loc.values), (i, cnt[i], len(loc.values))
    x, info = pre.solve(torch.as_tensor(prob.b, device="cuda"))
    rel = np.linalg.norm(prob.b - A @ x.cpu().numpy()) / np.linalg.norm(prob.b)
    assert info.converged and rel <= 1e-7
    pre.close()


def test_negative_tau_rejected(P):
    prob = poisson2d(16, 16, 2, 2, nev=2)
    with pytest.raises(P.AsmError) as e:
        make(P, prob.csr(), prob.part, prob.N, 1, 2, tau=-1.0)
    assert e.value.name == "INVALID_ARG"
