"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks a printed
example, a closed form, a theorem of the paper, an independent brute-force
computation or a special case with a known answer.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
from asm_inputs import SplitMix64, poisson2d, diffusion3d, convdiff2d

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def read_worked_example():
    sec, data = None, {}
    with open(os.path.join(GOLDEN, "worked_example_7x7.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                sec = line[1:-1]
                data[sec] = []
                continue
            data[sec].append(line)
    A = np.array([[float(t) for t in row.split()] for row in data["A"]])
    part = np.array([int(t) - 1 for t in data["partition"][0].split()])
    exp = {}
    for d in (1, 2):
        kv = dict(l.split(" = ") for l in data[f"delta={d}"])
        exp[d] = {k: np.array([int(t) for t in v.split()]) for k, v in kv.items()}
    return A, part, exp


def random_spd(n, seed, density=0.08):
    """Sparse SPD matrix with a random symmetric pattern: a weighted graph
    Laplacian plus a random positive diagonal."""
    r = SplitMix64(seed)
    m = int(density * n * n / 2)
    i = r.integers(0, n - 1, m)
    j = r.integers(0, n - 1, m)
    keep = i != j
    w = 0.1 + r.uniform(m)
    W = sp.coo_matrix((w[keep], (i[keep], j[keep])), shape=(n, n)).tocsr()
    W = W + W.T
    L = sp.diags(np.asarray(W.sum(axis=1)).ravel()) - W
    # tridiagonal backbone keeps the graph connected
    t = sp.diags([-np.ones(n - 1), -np.ones(n - 1)], [-1, 1])
    Lt = sp.diags(-np.asarray(t.sum(axis=1)).ravel()) + t
    A = (L + Lt + sp.diags(0.05 + r.uniform(n))).tocsr()
    A.sort_indices()
    return A


def contiguous_part(n, N):
    return (np.arange(n) * N // n).astype(np.int32)


# ---------------------------------------------------------------------------
# SplitMix64 (published test values)
# ---------------------------------------------------------------------------
def test_splitmix64_published_values():
    # first outputs of SplitMix64 from state 0 and from state 1234567
    assert [int(x) for x in SplitMix64(0).raw(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert int(SplitMix64(1234567).raw(1)[0]) == 6457827717110365317


# ---------------------------------------------------------------------------
# Section 2.1: worked example, brute-force overlap, PoU
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("delta", [1, 2])
def test_worked_example(delta):
    A, part, exp = read_worked_example()
    ovs = O.overlap(sp.csr_matrix(A), part, 2, delta)
    for i in (1, 2):
        np.testing.assert_array_equal(ovs[i - 1].omega + 1, exp[delta][f"omega{i}"])
        np.testing.assert_array_equal(O.pou(ovs[i - 1]), exp[delta][f"D{i}"])


def _bfs_distance_bruteforce(A, sources):
    """Graph distance from a node set by repeated boolean products with the
    dense adjacency of A + A^T (no BFS queue involved)."""
    n = A.shape[0]
    Ad = (A.toarray() != 0)
    adj = (Ad | Ad.T) & ~np.eye(n, dtype=bool)
    dist = np.full(n, -1)
    reach = np.zeros(n, dtype=bool)
    reach[sources] = True
    dist[sources] = 0
    k = 0
    while True:
        k += 1
        nxt = (adj[reach].any(axis=0)) & ~reach
        if not nxt.any():
            break
        dist[nxt] = k
        reach |= nxt
    return dist


@pytest.mark.parametrize("delta", [1, 2, 3])
def test_overlap_matches_bruteforce_distances(delta):
    n = 60
    r = SplitMix64(77)
    m = 90
    i = r.integers(0, n - 1, m); j = r.integers(0, n - 1, m)
    A = sp.coo_matrix((np.ones(m), (i, j)), shape=(n, n)).tocsr() + sp.eye(n)  # nonsymmetric pattern
    part = (r.integers(0, 4, n)).astype(np.int32)
    ovs = O.overlap(A, part, 5, delta)
    for s, ov in enumerate(ovs):
        I = np.nonzero(part == s)[0]
        dist = _bfs_distance_bruteforce(sp.csr_matrix(A), I) if I.size else np.full(n, -1)
        expect = [np.nonzero(dist == k)[0] for k in range(delta + 1)]
        np.testing.assert_array_equal(ov.omega, np.concatenate(expect))
        np.testing.assert_array_equal(np.diff(ov.offsets), [len(e) for e in expect])


def test_partition_of_unity():
    p = poisson2d(20, 12, 3, 2, delta=2)
    ovs = O.overlap(p.csr(), p.part, p.N, 2)
    S = np.zeros((p.n, p.n))
    for ov in ovs:
        R = np.zeros((ov.n, p.n)); R[np.arange(ov.n), ov.omega] = 1
        S += R.T @ np.diag(O.pou(ov)) @ R
    np.testing.assert_array_equal(S, np.eye(p.n))


# ---------------------------------------------------------------------------
# Local matrices: closed-form Laplacian spectra
# ---------------------------------------------------------------------------
def test_local_matrix_2d_laplacian_closed_form():
    p = poisson2d(64, 64, 4, 4)
    ovs = O.overlap(p.csr(), p.part, p.N, 1)
    ov = ovs[5]  # interior 16 x 16 box
    Aii = O.local_matrix(p.csr(), ov)
    ev = np.sort(np.linalg.eigvalsh(Aii[:ov.p, :ov.p]))
    j = np.arange(1, 17)
    ref = np.sort((4 - 2 * np.cos(j[:, None] * np.pi / 17) - 2 * np.cos(j[None, :] * np.pi / 17)).ravel())
    np.testing.assert_allclose(ev, ref, rtol=0, atol=1e-12)


def test_local_matrix_3d_laplacian_closed_form():
    p = diffusion3d(16, (2, 2, 2), contrast=1.0)
    ovs = O.overlap(p.csr(), p.part, p.N, 1)
    ov = ovs[3]
    Aii = O.local_matrix(p.csr(), ov)
    ev = np.sort(np.linalg.eigvalsh(Aii[:ov.p, :ov.p]))
    c = 2 * np.cos(np.arange(1, 9) * np.pi / 9)
    ref = np.sort((6 - c[:, None, None] - c[None, :, None] - c[None, None, :]).ravel())
    np.testing.assert_allclose(ev, ref, rtol=0, atol=1e-12)
    # nnz of the 64^3 configuration: 7 per row minus the boundary faces
    assert diffusion3d(64, contrast=1.0).nnz == 7 * 64 ** 3 - 6 * 64 ** 2


# ---------------------------------------------------------------------------
# Section 3: harmonic projection, local SPSD splitting, lifting spectrum
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("delta", [1, 2, 3])
def test_harmonic_operator_is_aii_orthogonal_projection(delta):
    A = random_spd(80, 5)
    part = contiguous_part(80, 4)
    for ov in O.overlap(A, part, 4, delta):
        Aii = O.local_matrix(A, ov)
        Pi = O.harmonic_operator(Aii, ov.m)
        I = np.eye(ov.n)
        np.testing.assert_allclose(Pi @ Pi, Pi, atol=1e-10)
        np.testing.assert_allclose((I - Pi).T @ Aii @ Pi, 0, atol=1e-9)
        # Pi v is harmonic: A_ii Pi v vanishes on Omega_{1:delta-1}
        v = SplitMix64(3).normal(ov.n)
        np.testing.assert_allclose((Aii @ Pi @ v)[:ov.m], 0, atol=1e-9)
        # Pi leaves Gamma_delta values unchanged
        np.testing.assert_allclose((Pi @ v)[ov.m:], v[ov.m:], atol=1e-12)


@pytest.mark.parametrize("delta", [1, 2, 3])
def test_local_spsd_splitting(delta):
    A = random_spd(72, 11)
    part = contiguous_part(72, 4)
    ovs = O.overlap(A, part, 4, delta)
    Ad = A.toarray()
    total = np.zeros_like(Ad)
    for ov in ovs:
        Aii = O.local_matrix(A, ov)
        Pi = O.harmonic_operator(Aii, ov.m)
        I = np.eye(ov.n)
        At = O.local_spsd_splitting(Aii, ov)
        # eq. local_problem_local_spsd_splitting
        np.testing.assert_allclose((I - Pi).T @ Aii @ (I - Pi), At, atol=1e-9)
        Ati = np.zeros_like(Ad)
        Ati[np.ix_(ov.omega, ov.omega)] = At
        # Lemma 3.1: Atilde_i and A - Atilde_i are SPSD
        assert np.linalg.eigvalsh(Ati).min() > -1e-9
        assert np.linalg.eigvalsh(Ad - Ati).min() > -1e-9
        total += Ati
    # Lemma 3.2: 0 <= u^T sum Atilde_i u <= k_c u^T A u
    kc = O.color_count(ovs)
    ev = sla.eigh(total, Ad, eigvals_only=True)
    assert ev.min() > -1e-9 and ev.max() <= kc + 1e-9


@pytest.mark.parametrize("delta", [1, 2])
def test_lifting_gevp_spectrum_structure(delta):
    # Theorem 3.4: 0 with multiplicity |Gamma_{1:delta}|, 1 with multiplicity
    # dim ker A_{Gamma, I}, everything else > 1
    for A, part, N in ((random_spd(70, 21), contiguous_part(70, 3), 3),
                       (poisson2d(12, 12, 2, 2).csr(), poisson2d(12, 12, 2, 2).part, 4)):
        for ov in O.overlap(A, part, N, delta):
            Aii = O.local_matrix(A, ov)
            lam, U = O.lifting_gevp(Aii, ov)
            nG = ov.n - ov.p
            rank = np.linalg.matrix_rank(Aii[ov.p:, :ov.p], tol=1e-10)
            assert np.sum(np.abs(lam) < 1e-9) == nG
            assert np.sum(np.abs(lam - 1) < 1e-9) == ov.p - rank
            rest = lam[(np.abs(lam) >= 1e-9) & (np.abs(lam - 1) >= 1e-9)]
            assert np.all(rest > 1)
            # eigenvectors are A_ii-orthonormal
            np.testing.assert_allclose(U.T @ Aii @ U, np.eye(ov.n), atol=1e-8)


# ---------------------------------------------------------------------------
# Section 5: eq. gevpsvd and its SVD-like splitting
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("delta", [1, 2])
def test_gevpsvd_structure_and_splitting(delta):
    A = random_spd(90, 31)
    part = contiguous_part(90, 3)
    tau2 = 0.05
    for ov in O.overlap(A, part, 3, delta):
        Aii = O.local_matrix(A, ov)
        mu, W, Pi = O.gevp_svd(Aii, ov)
        assert mu.min() > -1e-10
        assert np.sum(mu > 1e-10) <= ov.g
        np.testing.assert_allclose(W.T @ Aii @ W, np.eye(ov.n), atol=1e-8)
        D = np.diag(O.pou(ov))
        k = int(np.sum(mu > tau2))
        W1, W2 = W[:, :k], W[:, k:]
        X1 = D @ Pi @ W1 @ W1.T @ Aii
        X2 = D @ Pi @ W2 @ W2.T @ Aii
        np.testing.assert_allclose(X1 + X2, D @ Pi, atol=1e-9)          # eq. svdsplitting
        np.testing.assert_allclose(X2.T @ Aii @ X1, 0, atol=1e-9)       # eq. gevpsplitting1
        ev = sla.eigh(0.5 * (X2.T @ Aii @ X2 + (X2.T @ Aii @ X2).T), Aii, eigvals_only=True)
        assert ev.max() <= tau2 + 1e-9                                    # eq. gevpsplitting2


def test_reduced_interface_form_matches_full_gevp():
    """The CUDA path reduces eq. gevpsvd to Gamma_delta.  With X = -B^{-1} C,
    X_p its first |I_i| rows, S = G - C^T B^{-1} C and K = X_p^T A_II X_p, the
    nonzero spectrum of eq. gevpsvd is that of K y = mu S y, and [X_p y; 0]
    spans D Pi W^(1).  With A_ii = L L^T, W = L^{-1} and U = W[Gamma, I], the
    same spectrum is that of the symmetric U A_II U^T z = mu z and X_p y = U^T z
    (what the kernels compute).  Both forms are checked against the dense
    full-size eigenproblem."""
    for delta in (1, 2):
        A = random_spd(90, 41)
        part = contiguous_part(90, 3)
        for ov in O.overlap(A, part, 3, delta):
            Aii = O.local_matrix(A, ov)
            mu, W, Pi = O.gevp_svd(Aii, ov)
            m, p = ov.m, ov.p
            B, C, G = Aii[:m, :m], Aii[:m, m:], Aii[m:, m:]
            X = -np.linalg.solve(B, C)
            Xp = X[:p]
            K = Xp.T @ Aii[:p, :p] @ Xp
            S = G - C.T @ np.linalg.solve(B, C)
            red, Y = sla.eigh(0.5 * (K + K.T), S)
            red = red[::-1]; Y = Y[:, ::-1]
            nz = int(np.sum(mu > 1e-10))
            np.testing.assert_allclose(red[:nz], mu[:nz], rtol=1e-9)
            Linv = np.linalg.inv(np.linalg.cholesky(Aii))
            U = Linv[m:, :p]
            sym = U @ Aii[:p, :p] @ U.T
            ev, Zs = np.linalg.eigh(0.5 * (sym + sym.T))
            ev = ev[::-1]; Zs = Zs[:, ::-1]
            np.testing.assert_allclose(ev[:nz], mu[:nz], rtol=1e-9)
            k = min(3, nz)
            Zfull = (np.diag(O.pou(ov)) @ Pi @ W[:, :k])[:p]
            if k and (mu[k - 1] - mu[k]) / mu[k - 1] > 1e-6:
                P1 = Zfull @ np.linalg.pinv(Zfull)
                for Zred in (Xp @ Y[:, :k], U.T @ Zs[:, :k]):
                    np.testing.assert_allclose(Zred @ np.linalg.pinv(Zred), P1, atol=1e-8)
                # A_ii-normalised w and unit z give coarse vectors of A_II-energy mu
                Zr = U.T @ Zs[:, :k]
                np.testing.assert_allclose(np.einsum("ij,ij->j", Zr, Aii[:p, :p] @ Zr), ev[:k], rtol=1e-8)
                np.testing.assert_allclose(np.einsum("ij,ij->j", Zfull, Aii[:p, :p] @ Zfull), mu[:k], rtol=1e-8)


# ---------------------------------------------------------------------------
# Section 4 / 5: preconditioner properties and bounds
# ---------------------------------------------------------------------------
def test_one_subdomain_is_exact_inverse():
    p = poisson2d(12, 10, 1, 1)
    A = p.csr()
    st = O.setup(A, p.part, 1, 1, 4)
    assert st.n_C == 0   # Gamma is empty: no coarse vectors
    Minv = O.dense_operator(st)
    np.testing.assert_allclose(Minv @ A.toarray(), np.eye(p.n), atol=1e-12)
    res = O.solve(st, p.b)
    assert res.iterations == 1 and res.converged


def test_preconditioner_symmetric_positive_definite():
    p = poisson2d(16, 16, 2, 2, nev=3)
    st = O.setup(p.csr(), p.part, p.N, 1, 3)
    M = O.dense_operator(st)
    scale = np.abs(M).max()
    assert np.abs(M - M.T).max() <= 1e-13 * scale * p.n
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def test_coarse_correction_is_a_orthogonal_projection():
    p = poisson2d(16, 16, 2, 2, nev=3)
    st = O.setup(p.csr(), p.part, p.N, 1, 3)
    Ad = st.A.toarray()
    P = np.column_stack([st.apply_coarse(Ad[:, j]) for j in range(p.n)])
    np.testing.assert_allclose(P @ P, P, atol=1e-10)
    np.testing.assert_allclose(Ad @ P, (Ad @ P).T, atol=1e-10)


def test_full_spectra_give_exact_coarse_space_and_thm1():
    """Keeping every nonzero eigenvector of eq. gevpsvd reproduces the harmonic
    part of eq. coarse_space; with eq. uppergevp on at nu the bound of
    Theorem 4.5 holds."""
    p = poisson2d(12, 12, 2, 2)
    A = p.csr()
    nu = 2.0
    st = O.setup(A, p.part, p.N, 1, nev=10_000, nu=nu)
    cols = []
    for loc in st.locals:
        ov = loc.ov
        Aii = O.local_matrix(A, ov)
        H = np.vstack([-np.linalg.solve(Aii[:ov.m, :ov.m], Aii[:ov.m, ov.m:]), np.eye(ov.g)])
        lam, U = O.lifting_gevp(Aii, ov)
        blk = np.hstack([H, U[:, lam > nu]])[:ov.p]
        c = np.zeros((p.n, blk.shape[1])); c[ov.omega[:ov.p]] = blk
        cols.append(c)
    R0 = np.hstack(cols)
    Zd = st.Z.toarray()
    assert np.linalg.matrix_rank(R0) == np.linalg.matrix_rank(Zd)
    ang = sla.subspace_angles(Zd, R0)
    assert ang.max() < 1e-8
    # Theorem 4.5 with nu_eff = the largest eigenvalue of eq. uppergevp left out
    ovs = [l.ov for l in st.locals]
    kc = O.color_count(ovs)
    nu_eff = max(max([v for v in O.lifting_gevp(O.local_matrix(A, ov), ov)[0] if v <= nu] or [0.0])
                 for ov in ovs)
    assert O.condition_number(st) <= O.bound_thm1(kc, nu_eff)


@pytest.mark.parametrize("nev", [1, 3, 6])
def test_theorem2_bound(nev):
    p = poisson2d(16, 16, 2, 2)
    A = p.csr()
    st = O.setup(A, p.part, p.N, 1, nev)
    ovs = [l.ov for l in st.locals]
    kc = O.color_count(ovs)
    lam_s = O.lambda_star(A, ovs)
    tau = np.sqrt(max(max(l.all_values[nev], 0.0) for l in st.locals))
    nu_eff = max(O.lifting_gevp(O.local_matrix(A, ov), ov)[0][0] for ov in ovs)
    kappa = O.condition_number(st)
    assert 1.0 <= kappa <= O.bound_thm2(kc, nu_eff, lam_s, tau)
    # more coarse vectors never make the bound worse
    assert kc == 4


def test_pcg_matches_direct_solve():
    p = poisson2d(64, 64, 4, 4)
    A = p.csr()
    st = O.setup(A, p.part, p.N, 1, p.nev)
    res = O.solve(st, p.b)
    assert res.converged and res.final_relres <= 1e-8
    x = spla.spsolve(A.tocsc(), p.b)
    kappa_A = 4 * 64 ** 2  # upper estimate of cond(A) for the 2D Laplacian
    assert np.linalg.norm(res.x - x) / np.linalg.norm(x) <= kappa_A * 1e-8
    true = np.linalg.norm(p.b - A @ res.x) / np.linalg.norm(p.b)
    assert true <= 2e-8
    # the two-level method needs fewer iterations than the one-level one
    st1 = O.setup(A, p.part, p.N, 1, 0)
    assert O.solve(st1, p.b).iterations > res.iterations


def test_krylov_without_preconditioner_terminates():
    A = random_spd(30, 9)
    b = SplitMix64(5).normal(30)
    res = O.pcg(A, b, lambda r: r, rtol=1e-12, maxit=200)
    np.testing.assert_allclose(res.x, np.linalg.solve(A.toarray(), b), rtol=1e-8)
    An = (A + sp.diags(np.ones(29), 1) * 0.3).tocsr()
    res = O.fgmres(An, b, lambda r: r, restart=30, rtol=1e-12, maxit=30)
    assert res.iterations <= 30
    np.testing.assert_allclose(res.x, np.linalg.solve(An.toarray(), b), rtol=1e-8)


def test_grid_and_operator_complexity():
    p = poisson2d(32, 32, 2, 2, nev=3)
    st = O.setup(p.csr(), p.part, p.N, 1, 3)
    assert st.n_C == 4 * 3
    assert st.gc() == 1 + 12 / 1024
    assert st.oc() == 1 + np.count_nonzero(st.E) / p.nnz
    # 2 x 2 boxes: every pair of subdomains sharing an edge couples
    # the diagonal pairs (0,3) and (1,2) do not touch: 4 of the 16 blocks vanish
    assert np.count_nonzero(st.E) == 12 * 12 - 4 * 9


# ---------------------------------------------------------------------------
# Nonsymmetric variant (Section 5 of the paper's Section "Extension to
# nonsymmetric matrices")
# ---------------------------------------------------------------------------
def test_nonsymmetric_one_subdomain_and_full_space():
    p = convdiff2d(24, (1, 1), peclet=50.0, delta=2)
    st = O.setup(p.csr(), p.part, 1, 2, 4, spd=False)
    res = O.solve(st, p.b)
    assert res.iterations == 1
    q = convdiff2d(24, (3, 3), peclet=50.0, delta=2)
    A = q.csr()
    st = O.setup(A, q.part, q.N, 2, nev=10_000, spd=False)
    for loc in st.locals:
        ov = loc.ov
        Aii = O.local_matrix(A, ov)
        # singular values of the Boolean D_i never exceed 1
        assert np.linalg.svd(np.diag(O.pou(ov)), compute_uv=False).max() <= 1.0
        H = -np.linalg.solve(Aii[:ov.m, :ov.m], Aii[:ov.m, ov.m:])[:ov.p]
        ang = sla.subspace_angles(loc.basis, H)
        assert ang.max() < 1e-8
    res = O.solve(st, q.b)
    x = spla.spsolve(A.tocsc(), q.b)
    assert res.converged
    assert np.linalg.norm(res.x - x) / np.linalg.norm(x) < 1e-6


def test_nonsymmetric_fgmres_matches_direct():
    p = convdiff2d(48, (4, 4), peclet=1e3, delta=2, nev=4)
    A = p.csr()
    st = O.setup(A, p.part, p.N, 2, 4, spd=False)
    res = O.solve(st, p.b)
    assert res.converged
    true = np.linalg.norm(p.b - A @ res.x) / np.linalg.norm(p.b)
    assert true <= 1e-7
    x = spla.spsolve(A.tocsc(), p.b)
    assert np.linalg.norm(res.x - x) / np.linalg.norm(x) < 1e-5


@pytest.mark.parametrize("delta", [1, 2, 3])
def test_reduced_lifting_form_matches_full_gevp(delta):
    """Eq. uppergevp in the reduced form the CUDA path uses (I_i ordered first,
    A_ii = L L^T, W = L^{-1}, W21 = W[Omega_i minus I_i, I_i]): its eigenvalues
    are 1 + the eigenvalues of W21 A_II W21^T, and the A_ii-normalised
    eigenvector restricted to I_i is sqrt((1 + s) / s) W21^T z for the unit
    eigenvector z of eigenvalue s.  Checked against the full dense pencil
    D_i A_ii D_i u = lambda A_ii u of the oracle."""
    p = diffusion3d(12, (2, 2, 2), contrast=1e3, delta=delta, nev=4)
    A = p.csr()
    ov = O.overlap(A, p.part, p.N, delta)[3]
    Aii = O.local_matrix(A, ov)
    lam, U = O.lifting_gevp(Aii, ov)
    pi = ov.p
    W = np.linalg.inv(np.linalg.cholesky(Aii))
    W21 = W[pi:, :pi]
    s2, Zs = np.linalg.eigh(W21 @ Aii[:pi, :pi] @ W21.T)
    s2, Zs = s2[::-1], Zs[:, ::-1]
    k = 6
    np.testing.assert_allclose(1.0 + s2[:k], lam[:k], rtol=1e-11)
    assert np.all(lam[:k] > 1.0)
    for j in range(k):
        if (lam[j] - lam[j + 1]) / lam[j] < 1e-6:
            continue
        u = np.sqrt((1 + s2[j]) / s2[j]) * (W21.T @ Zs[:, j])
        uo = U[:pi, j]
        assert abs(abs(u @ uo) - np.linalg.norm(u) * np.linalg.norm(uo)) < 1e-10 * np.linalg.norm(uo) ** 2
        np.testing.assert_allclose(np.linalg.norm(u), np.linalg.norm(uo), rtol=1e-10)
