"""Pins of the oracle's restricted one-level part (eq. onelevelras) and of the
deflated coarse correction that the experiments of Section 6 combine it with.

The closed form is derived by hand below; the deflation identities follow
from Q = Z E^{-1} Z^T with E = Z^T A Z and hold for any one-level part.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
from asm_inputs import poisson2d, convdiff2d


def _path4():
    A = sp.diags([-np.ones(3), 2 * np.ones(4), -np.ones(3)], [-1, 0, 1]).tocsr()
    return A, np.array([0, 0, 1, 1])


def test_ras_closed_form_on_a_four_node_path():
    # A = tridiag(-1, 2, -1) on 4 nodes, I_0 = {0, 1}, I_1 = {2, 3}, delta = 1:
    # Omega_0 = (0, 1, 2), Omega_1 = (2, 3, 1).  Both A_ii are the 3-node path
    # matrix, whose inverse (in path order) is [[3,2,1],[2,4,2],[1,2,3]]/4.
    # D_i keeps the rows of I_i: nodes 0, 1 take rows 0, 1 of the first
    # inverse (path 0-1-2), nodes 2, 3 rows 1, 2 of the second (path 1-2-3).
    A, part = _path4()
    st = O.setup(A, part, 2, 1, 0)
    assert st.n_C == 0
    M = np.column_stack([st.apply_one_level_ras(e) for e in np.eye(4)])
    expect = np.array([[3, 2, 1, 0],
                       [2, 4, 2, 0],
                       [0, 2, 4, 2],
                       [0, 1, 2, 3]]) / 4.0
    np.testing.assert_allclose(M, expect, atol=1e-14)
    # restricted: not symmetric, unlike the additive one-level part
    M_asm = np.column_stack([st.apply_one_level(e) for e in np.eye(4)])
    np.testing.assert_allclose(M_asm, M_asm.T, atol=1e-14)
    assert abs(M[3, 1] - M[1, 3]) > 0.2


def test_ras_is_exact_on_a_single_subdomain():
    p = poisson2d(8, 8, 1, 1, nev=0)
    A = p.csr()
    st = O.setup(A, p.part, 1, 1, 0)
    r = np.random.default_rng(0).standard_normal(p.n)
    np.testing.assert_allclose(st.apply_one_level_ras(r), spla.spsolve(A.tocsc(), r), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("one_level", ["asm", "ras"])
def test_deflated_correction_identities(one_level):
    p = poisson2d(16, 16, 2, 2, nev=3)
    A = p.csr()
    st = O.setup(A, p.part, p.N, 1, 3)
    Z = st.Z.toarray()
    rng = np.random.default_rng(1)
    # M^{-1} A Z = Z: the deflated preconditioner inverts A on range(Z)
    c = rng.standard_normal(st.n_C)
    np.testing.assert_allclose(st.apply_variant(A @ (Z @ c), one_level, "deflated"), Z @ c, rtol=1e-9, atol=1e-9)
    # the one-level part sees r - A Q r, which is orthogonal to range(Z)
    r = rng.standard_normal(p.n)
    w = r - A @ st.apply_coarse(r)
    assert np.linalg.norm(Z.T @ w) <= 1e-10 * np.linalg.norm(Z.T @ r)
    # and the additive combination is the sum of the two parts
    one = st.apply_one_level_ras if one_level == "ras" else st.apply_one_level
    np.testing.assert_allclose(st.apply_variant(r, one_level, "additive"), one(r) + st.apply_coarse(r),
                               rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("spd", [True, False])
def test_ras_deflated_fgmres_matches_direct(spd):
    if spd:
        p = poisson2d(32, 32, 4, 4, nev=4)
    else:
        p = convdiff2d(48, (4, 4), peclet=1e3, delta=2, nev=4)
    A = p.csr()
    st = O.setup(A, p.part, p.N, p.delta, 4, spd=spd)
    res = O.solve(st, p.b, one_level="ras", coarse="deflated")
    assert res.converged
    x = spla.spsolve(A.tocsc(), p.b)
    assert np.linalg.norm(res.x - x) / np.linalg.norm(x) < 1e-5
    # two-level beats one-level RAS on the same Krylov method
    one = O.fgmres(A, p.b, st.apply_one_level_ras)
    assert res.iterations < one.iterations


# ---------------------------------------------------------------------------
# selection by the threshold tau (Prop. 5.1: eigenvalues above tau^2;
# Section 5.2: singular values above tau)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("tau", [0.3, 0.6])
def test_threshold_selection_satisfies_theorem2(tau):
    # nev large enough that the threshold alone decides: Theorem 5.3 then
    # holds with the prescribed tau (not an effective one)
    p = poisson2d(16, 16, 2, 2)
    A = p.csr()
    st = O.setup(A, p.part, p.N, 1, 64, tau=tau)
    for loc in st.locals:
        k = len(loc.values)
        assert np.all(loc.all_values[:k] > tau * tau)
        assert k == len(loc.all_values) or loc.all_values[k] <= tau * tau
    ovs = [l.ov for l in st.locals]
    kc = O.color_count(ovs)
    lam_s = O.lambda_star(A, ovs)
    nu_eff = max(O.lifting_gevp(O.local_matrix(A, ov), ov)[0][0] for ov in ovs)
    assert 1.0 <= O.condition_number(st) <= O.bound_thm2(kc, nu_eff, lam_s, tau)


def test_threshold_selection_general_path():
    p = convdiff2d(32, (2, 2), peclet=1e2, delta=2, nev=64)
    A = p.csr()
    tau = 0.5
    st = O.setup(A, p.part, p.N, 2, 64, spd=False, tau=tau)
    for loc in st.locals:
        k = len(loc.values)
        assert np.all(loc.all_values[:k] > tau)
        assert k == len(loc.all_values) or loc.all_values[k] <= tau


def test_more_overlap_contributes_fewer_vectors_at_fixed_tau():
    # Section 6 (discussion of Fig. 1): for a fixed tau, more overlap layers
    # decrease the number of vectors each subdomain contributes
    p = poisson2d(48, 48, 3, 3)
    A = p.csr()
    sizes = [O.setup(A, p.part, p.N, d, 200, tau=0.25).n_C for d in (1, 2, 3)]
    assert sizes[0] > sizes[1] > sizes[2] > 0, sizes
