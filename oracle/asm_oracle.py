"""Plain, slow FP64 CPU oracle of the fully algebraic two-level Schwarz method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module.  It
shares no code with the CUDA path in ``paper_2401_03915_gb300``.

Everything follows the paper (Al Daas, Jolivet, Nataf, Tournier, "A robust
two-level Schwarz preconditioner for sparse matrices") in its own notation:

* Section 2.1: overlapping subdomains grown through the sparsity graph of
  A + A^T, ordered [I_i, layer 1, ..., layer delta]; Boolean PoU D_i.
* Section 2.3: A_ii = R_i A R_i^T, one-level ASM (eq. onelevelasm).
* Section 3.2: local harmonic operator Pi_i (eq. HOp).
* Section 3.3: lifting GEVP D_i A_ii D_i u = lambda A_ii u (eq. uppergevp).
* Section 5.1: GEVP Pi_i^T D_i A_ii D_i Pi_i w = lambda^2 A_ii w
  (eq. gevpsvd) and the coarse space of eq. coarse_space_2.
* Section 4.1: coarse operator A_00 = R_0 A R_0^T (the coarse matrix E).
* Remark in Section 4.3: M_2^{-1} = sum_{i=0}^N R_i^T A_ii^{-1} R_i.
* Section 2.3 / Section 6: restricted ASM (eq. onelevelras) and the deflated
  coarse correction that the experiments combine it with (a reading: the
  formula is in the paper's PCHPDDM reference, not in the paper).
* Section 6: the nonsymmetric variant keeps left singular vectors of
  D_i Pi_i (Euclidean) and drops eq. uppergevp.
* Theorems 4.5 / 5.3 (labels th:upper_bound_1, th:upper_bound_2): the
  condition-number bounds.

Each local eigenproblem is solved densely on the full |Omega_i| problem with
LAPACK (scipy.linalg.eigh / svd); nothing is blocked, fused or reduced.
Readings of points the paper leaves open are listed where they are used.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


class OracleError(RuntimeError):
    pass


# ---------------------------------------------------------------------------
# Section 2.1: graph, overlap, partition of unity
# ---------------------------------------------------------------------------
def pattern_graph(A: sp.spmatrix) -> sp.csr_matrix:
    """Sparsity graph of A + A^T (Section 2.1): every stored entry is an edge,
    self loops are dropped.  Returned as a 0/1 CSR adjacency with sorted rows."""
    A = sp.csr_matrix(A)
    B = sp.csr_matrix((np.ones(A.nnz), A.indices, A.indptr), shape=A.shape)
    G = (B + B.T).tocsr()
    G.setdiag(0)
    G.eliminate_zeros()
    G.sort_indices()
    G.data[:] = 1.0
    return G


@dataclass
class Overlap:
    """Omega_{i,1:delta} = [I_i, Gamma_{i,1}, ..., Gamma_{i,delta}] (Section 2.1)."""
    omega: np.ndarray          # global indices in R_i order
    offsets: np.ndarray        # [0, |I|, |I|+|G1|, ..., |Omega|]

    @property
    def p(self) -> int:        # |Omega_{I_i}|
        return int(self.offsets[1])

    @property
    def n(self) -> int:        # |Omega_{i,1:delta}|
        return int(self.offsets[-1])

    @property
    def g(self) -> int:        # |Gamma_{i,delta}|
        return int(self.offsets[-1] - self.offsets[-2])

    @property
    def m(self) -> int:        # |Omega_{i,1:delta-1}|
        return int(self.offsets[-2])


def overlap(A: sp.spmatrix, part: np.ndarray, N: int, delta: int) -> list[Overlap]:
    """Grow each nonoverlapping subdomain by delta layers (Section 2.1).

    Layer k holds the nodes at graph distance exactly k from I_i.  Reading of
    the unspecified order inside a layer (the paper's example has one node per
    layer): ascending global index, and I_i itself ascending."""
    G = pattern_graph(A)
    n = G.shape[0]
    out = []
    for i in range(N):
        I = np.nonzero(part == i)[0]
        seen = np.zeros(n, dtype=bool)
        seen[I] = True
        frontier = I
        pieces = [I]
        for _ in range(delta):
            if frontier.size:
                nb = np.concatenate([G.indices[G.indptr[v]:G.indptr[v + 1]] for v in frontier])
                nb = np.unique(nb)
                layer = nb[~seen[nb]]
            else:
                layer = np.zeros(0, dtype=np.int64)
            seen[layer] = True
            pieces.append(layer)
            frontier = layer
        offsets = np.cumsum([0] + [len(q) for q in pieces])
        out.append(Overlap(np.concatenate(pieces).astype(np.int64), offsets.astype(np.int64)))
    return out


def pou(ov: Overlap) -> np.ndarray:
    """Boolean partition of unity D_i (Section 2.1): 1 on the first |I_i| entries."""
    d = np.zeros(ov.n)
    d[:ov.p] = 1.0
    return d


def local_matrix(A: sp.spmatrix, ov: Overlap) -> np.ndarray:
    """A_ii = R_i A R_i^T as a dense array (Section 2.3)."""
    A = sp.csr_matrix(A)
    return A[ov.omega][:, ov.omega].toarray()


# ---------------------------------------------------------------------------
# Section 3: harmonic operator, local SPSD splitting, lifting GEVP
# ---------------------------------------------------------------------------
def harmonic_operator(Aii: np.ndarray, m: int) -> np.ndarray:
    """Pi_i of eq. HOp: v -> [-B^{-1} C; I] v_Gamma_delta, with
    B = A_{Omega_{1:delta-1}, Omega_{1:delta-1}} and C = A_{Omega_{1:delta-1}, Gamma_delta}."""
    n = Aii.shape[0]
    Pi = np.zeros((n, n))
    if n == m:
        return Pi
    B = Aii[:m, :m]
    C = Aii[:m, m:]
    Pi[:m, m:] = -np.linalg.solve(B, C) if m else np.zeros((0, n - m))
    Pi[m:, m:] = np.eye(n - m)
    return Pi


def local_spsd_splitting(Aii: np.ndarray, ov: Overlap) -> np.ndarray:
    """Atilde_ii from eq. LSPSD restricted to Omega_i, with S from eq. S_G.

    Blocks in the order [I, Gamma_{1:delta-1}, Gamma_delta].  For delta = 1 the
    middle block is empty and I touches Gamma_1 directly; the (3,3) block then
    reads C^T A_II^{-1} C, the same Schur-complement form with an empty
    Gamma_{1:delta-1} (reading)."""
    p, m, n = ov.p, ov.m, ov.n
    At = np.zeros_like(Aii)
    At[:m, :m] = Aii[:m, :m]
    At[:m, m:] = Aii[:m, m:]
    At[m:, :m] = Aii[m:, :m]
    if m > p:
        AII = Aii[:p, :p]
        AIG = Aii[:p, p:m]
        AGG = Aii[p:m, p:m]
        S = AGG - AIG.T @ np.linalg.solve(AII, AIG)          # eq. S_G
        AGd = Aii[p:m, m:]                                      # A_{Gamma_{1:d-1}, Gamma_d}
        At[m:, m:] = AGd.T @ np.linalg.solve(S, AGd)
    else:
        C = Aii[:m, m:]
        At[m:, m:] = C.T @ np.linalg.solve(Aii[:m, :m], C)
    return At


def _scaled_pencil_eigh(lhs: np.ndarray, Aii: np.ndarray):
    """Eigenpairs of lhs u = lambda A_ii u through the congruent pencil
    (S lhs S, S A_ii S) with S = diag(A_ii)^{-1/2}: identical eigenvalues,
    u = S u^; LAPACK's error is then eps * cond(S A_ii S) instead of
    eps * cond(A_ii), which matters for high-contrast coefficients."""
    s = 1.0 / np.sqrt(np.abs(np.diag(Aii)))
    lam, Uh = sla.eigh(s[:, None] * lhs * s[None, :], s[:, None] * Aii * s[None, :])
    return lam, s[:, None] * Uh


def lifting_gevp(Aii: np.ndarray, ov: Overlap):
    """Eigenpairs of D_i A_ii D_i u = lambda A_ii u (eq. uppergevp), eigenvalues
    descending, eigenvectors A_ii-orthonormal."""
    d = pou(ov)
    lam, U = _scaled_pencil_eigh(d[:, None] * Aii * d[None, :], Aii)
    return lam[::-1], U[:, ::-1]


def gevp_svd(Aii: np.ndarray, ov: Overlap):
    """Eigenpairs of Pi^T D A_ii D Pi w = lambda^2 A_ii w (eq. gevpsvd),
    eigenvalues (the lambda^2) descending, eigenvectors A_ii-orthonormal."""
    d = pou(ov)
    Pi = harmonic_operator(Aii, ov.m)
    DPi = d[:, None] * Pi
    lhs = DPi.T @ Aii @ DPi
    lhs = 0.5 * (lhs + lhs.T)
    mu, W = _scaled_pencil_eigh(lhs, Aii)
    return mu[::-1], W[:, ::-1], Pi


def svd_dpi(Aii: np.ndarray, ov: Overlap):
    """Euclidean SVD of D_i Pi_i (Section 5 and Section 6): left singular vectors
    and singular values, descending."""
    d = pou(ov)
    Pi = harmonic_operator(Aii, ov.m)
    U, s, _ = np.linalg.svd(d[:, None] * Pi)
    return s, U, Pi


# ---------------------------------------------------------------------------
# Setup: coarse space (eq. coarse_space_2) and coarse operator (Section 4.1)
# ---------------------------------------------------------------------------
RANK_TOL = 1e-12   # eigen/singular values below RANK_TOL * max are treated as zero


@dataclass
class LocalResult:
    ov: Overlap
    values: np.ndarray          # eq. gevpsvd lambda^2 (SPD) or sigma (general), top ones kept
    all_values: np.ndarray      # the full spectrum, descending
    basis: np.ndarray           # p x k block: rows I_i of R_i^T D_i (...) columns
    lift_values: np.ndarray = field(default_factory=lambda: np.zeros(0))


@dataclass
class OracleSetup:
    A: sp.csr_matrix
    N: int
    delta: int
    spd: bool
    locals: list
    Z: sp.csc_matrix            # n x n_C, columns R_i^T D_i (Pi_i W_i^(1), Z_i)
    E: np.ndarray               # n_C x n_C = Z^T A Z
    factors: list               # per-subdomain dense factorizations of A_ii
    E_factor: object

    @property
    def n_C(self) -> int:
        return self.Z.shape[1]

    def gc(self) -> float:
        """Grid complexity 1 + n_C / n (Section 6)."""
        return 1.0 + self.n_C / self.A.shape[0]

    def oc(self) -> float:
        """Operator complexity 1 + nnz_C / nnz_A (Section 6)."""
        return 1.0 + np.count_nonzero(self.E) / self.A.nnz

    # -- apply --------------------------------------------------------------
    def apply_one_level(self, r: np.ndarray) -> np.ndarray:
        """sum_i R_i^T A_ii^{-1} R_i r (eq. onelevelasm)."""
        z = np.zeros_like(r)
        for loc, f in zip(self.locals, self.factors):
            y = _local_solve(f, r[loc.ov.omega], self.spd)
            np.add.at(z, loc.ov.omega, y)
        return z

    def apply_coarse(self, r: np.ndarray) -> np.ndarray:
        """R_0^T A_00^{-1} R_0 r = Z E^{-1} Z^T r."""
        if self.n_C == 0:
            return np.zeros_like(r)
        c = self.Z.T @ r
        if self.spd:
            y = sla.cho_solve(self.E_factor, c)
        else:
            y = sla.lu_solve(self.E_factor, c)
        return self.Z @ y

    def apply(self, r: np.ndarray) -> np.ndarray:
        """M_2^{-1} r = sum_{i=0}^N R_i^T A_ii^{-1} R_i r (Remark, Section 4.3)."""
        return self.apply_one_level(r) + self.apply_coarse(r)

    def apply_one_level_ras(self, r: np.ndarray) -> np.ndarray:
        """sum_i R_i^T D_i A_ii^{-1} R_i r (eq. onelevelras, Boolean D_i)."""
        z = np.zeros_like(r)
        for loc, f in zip(self.locals, self.factors):
            y = _local_solve(f, r[loc.ov.omega], self.spd)
            np.add.at(z, loc.ov.omega, pou(loc.ov) * y)
        return z

    def apply_variant(self, r: np.ndarray, one_level: str = "asm", coarse: str = "additive") -> np.ndarray:
        """The apply with either one-level part and either coarse correction.

        one_level: "asm" (eq. onelevelasm) or "ras" (eq. onelevelras).
        coarse: "additive" (the Remark of Section 4.3: M_1^{-1} r + Q r) or
        "deflated", the combination the experiments of Section 6 use.  The
        paper takes the deflated form from its PCHPDDM reference without
        printing it; reading: M^{-1} r = Q r + M_1^{-1} (r - A Q r) with
        Q = Z E^{-1} Z^T, so that M^{-1} A Z = Z."""
        one = self.apply_one_level_ras if one_level == "ras" else self.apply_one_level
        if coarse == "deflated":
            q = self.apply_coarse(r)
            return q + one(r - self.A @ q)
        return one(r) + self.apply_coarse(r)


def _local_solve(f, x, spd):
    return sla.cho_solve(f, x) if spd else sla.lu_solve(f, x)


def select_count(values: np.ndarray, nev: int, threshold: float | None = None) -> int:
    """How many of the descending ``values`` enter the coarse space.

    The paper keeps the eigenvalues of eq. gevpsvd above tau^2 (Prop. 5.1),
    or the singular values of D_i Pi_i above tau (Section 5.2).  With
    ``threshold`` (tau^2, or tau) given that rule is applied; ``nev`` caps the
    count either way (reading: a fixed count when no threshold is given), and
    numerically zero values are never kept."""
    if values.size == 0 or nev <= 0:
        return 0
    vmax = max(float(values[0]), 0.0)
    nz = int(np.count_nonzero(values > RANK_TOL * vmax)) if vmax > 0 else 0
    k = min(nev, nz)
    if threshold is not None:
        k = min(k, int(np.count_nonzero(values > threshold)))
    return k


def setup(A: sp.spmatrix, part: np.ndarray, N: int, delta: int, nev: int, spd: bool = True,
          nu: float | None = None, nev_lift: int | None = None,
          subdomains: list | None = None, tau: float | None = None) -> OracleSetup:
    """Build the two-level preconditioner.

    SPD: per subdomain the top ``nev`` eigenvectors of eq. gevpsvd, mapped by
    D_i Pi_i, and, if ``nu`` is given, the eigenvectors of eq. uppergevp with
    lambda > nu (at most ``nev_lift``), mapped by D_i.  General A: the top
    ``nev`` left singular vectors of D_i Pi_i (Section 6).  With ``tau``, only
    eigenvalues above tau^2 (singular values above tau) are kept, at most
    ``nev`` of them (Prop. 5.1, Section 5.2).  The coarse operator
    is E = Z^T A Z, Cholesky-factored (SPD) or LU-factored (general)."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    ovs = overlap(A, part, N, delta)
    locals_, factors = [], []
    rows, cols, vals = [], [], []
    col0 = 0
    idx = range(N) if subdomains is None else subdomains
    for i in idx:
        ov = ovs[i]
        Aii = local_matrix(A, ov)
        d = pou(ov)
        if spd:
            try:
                factors.append(sla.cho_factor(Aii, lower=True))
            except np.linalg.LinAlgError as e:
                raise OracleError(f"A_ii of subdomain {i} is not SPD") from e
            mu, W, Pi = gevp_svd(Aii, ov)
            k = select_count(mu, nev, None if tau is None else tau * tau)
            blocks = [(d[:, None] * (Pi @ W[:, :k]))]
            lift = np.zeros(0)
            if nu is not None:
                lam, U = lifting_gevp(Aii, ov)
                keep = np.nonzero(lam > nu)[0]
                if nev_lift is not None:
                    keep = keep[:nev_lift]
                lift = lam[keep]
                blocks.append(d[:, None] * U[:, keep])
            Bi = np.hstack(blocks)
            vals_i = mu[:k]
        else:
            factors.append(sla.lu_factor(Aii))
            s, U, Pi = svd_dpi(Aii, ov)
            k = select_count(s, nev, tau)
            Bi = d[:, None] * U[:, :k]
            mu, lift, vals_i = s, np.zeros(0), s[:k]
        basis = Bi[:ov.p]
        locals_.append(LocalResult(ov, vals_i, mu, basis, lift))
        kk = basis.shape[1]
        rr, cc = np.meshgrid(ov.omega[:ov.p], np.arange(col0, col0 + kk), indexing="ij")
        rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append(basis.ravel())
        col0 += kk
    if col0:
        Z = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(n, col0))
    else:
        Z = sp.csc_matrix((n, 0))
    E = (Z.T @ (A @ Z)).toarray() if col0 else np.zeros((0, 0))
    E_factor = None
    if col0:
        if spd:
            try:
                E_factor = sla.cho_factor(0.5 * (E + E.T), lower=True)
            except np.linalg.LinAlgError as e:
                raise OracleError("coarse operator E is not SPD (Section 4.1 assumes full rank)") from e
        else:
            E_factor = sla.lu_factor(E)
    return OracleSetup(A, N, delta, spd, locals_, Z, E, factors, E_factor)


# ---------------------------------------------------------------------------
# Krylov solvers (Section 6: relative tolerance 1e-8 on the unpreconditioned
# residual; reading: x0 = 0)
# ---------------------------------------------------------------------------
@dataclass
class SolveResult:
    x: np.ndarray
    iterations: int
    history: list
    converged: bool

    @property
    def final_relres(self) -> float:
        return self.history[-1] if self.history else float("nan")


def pcg(A, b, apply, rtol: float = 1e-8, maxit: int = 1000) -> SolveResult:
    """Preconditioned conjugate gradient (Hestenes-Stiefel), x0 = 0; stops on
    the recursive residual ||r_k|| / ||b|| <= rtol.  One iteration = one SpMV."""
    x = np.zeros_like(b)
    r = b.copy()
    bn = np.linalg.norm(b)
    hist = [1.0]
    if bn == 0:
        return SolveResult(x, 0, hist, True)
    z = apply(r)
    p = z.copy()
    rz = r @ z
    for k in range(1, maxit + 1):
        q = A @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        res = np.linalg.norm(r) / bn
        hist.append(res)
        if res <= rtol:
            return SolveResult(x, k, hist, True)
        z = apply(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return SolveResult(x, maxit, hist, False)


def fgmres(A, b, apply, restart: int = 30, rtol: float = 1e-8, maxit: int = 1000) -> SolveResult:
    """Right-preconditioned flexible GMRES(restart) with classical Gram-Schmidt
    applied twice and Givens rotations; x0 = 0.  Stops when the least-squares
    residual estimate ||r|| / ||b|| <= rtol.  One iteration = one SpMV."""
    n = b.size
    x = np.zeros_like(b)
    bn = np.linalg.norm(b)
    hist = [1.0]
    if bn == 0:
        return SolveResult(x, 0, hist, True)
    total = 0
    while total < maxit:
        r = b - A @ x
        beta = np.linalg.norm(r)
        if beta / bn <= rtol:
            return SolveResult(x, total, hist, True)
        V = np.zeros((restart + 1, n))
        Zs = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart); sn = np.zeros(restart)
        g = np.zeros(restart + 1); g[0] = beta
        V[0] = r / beta
        j_used = 0
        for j in range(restart):
            Zs[j] = apply(V[j])
            w = A @ Zs[j]
            h = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h
            h2 = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h2
            h = h + h2
            hn = np.linalg.norm(w)
            H[:j + 1, j] = h
            H[j + 1, j] = hn
            if hn > 0:
                V[j + 1] = w / hn
            for k in range(j):
                t = cs[k] * H[k, j] + sn[k] * H[k + 1, j]
                H[k + 1, j] = -sn[k] * H[k, j] + cs[k] * H[k + 1, j]
                H[k, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den; sn[j] = H[j + 1, j] / den
            H[j, j] = den; H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            total += 1
            j_used = j + 1
            hist.append(abs(g[j + 1]) / bn)
            if abs(g[j + 1]) / bn <= rtol or total >= maxit:
                break
        y = sla.solve_triangular(H[:j_used, :j_used], g[:j_used])
        x = x + Zs[:j_used].T @ y
        if hist[-1] <= rtol:
            return SolveResult(x, total, hist, True)
    return SolveResult(x, total, hist, False)


def solve(st: OracleSetup, b: np.ndarray, rtol: float = 1e-8, maxit: int = 1000,
          restart: int = 30, one_level: str = "asm", coarse: str = "additive") -> SolveResult:
    """PCG for SPD A with the additive ASM preconditioner (symmetric);
    right-preconditioned FGMRES otherwise, as with RAS or the deflated
    correction, which are not symmetric (Section 6)."""
    if st.spd and one_level == "asm" and coarse == "additive":
        return pcg(st.A, b, st.apply, rtol, maxit)
    return fgmres(st.A, b, lambda r: st.apply_variant(r, one_level, coarse), restart, rtol, maxit)


# ---------------------------------------------------------------------------
# Quantities entering the bounds (Lemma 3.2, Theorems 4.5 and 5.3)
# ---------------------------------------------------------------------------
def color_count(ovs: list[Overlap]) -> int:
    """k_c of Lemma 3.2.  Reading: greedy colouring, in ascending subdomain
    order, of the graph whose edges join overlapping subdomains."""
    N = len(ovs)
    sets = [set(ov.omega.tolist()) for ov in ovs]
    colors = [-1] * N
    for i in range(N):
        used = {colors[j] for j in range(i) if sets[i] & sets[j]}
        c = 0
        while c in used:
            c += 1
        colors[i] = c
    return max(colors) + 1 if N else 0


def lambda_star(A: sp.spmatrix, ovs: list[Overlap]) -> float:
    """Largest eigenvalue of sum_i R_i^T A_ii R_i u = lambda A u (eq. lambda_star); dense."""
    Ad = sp.csr_matrix(A).toarray()
    S = np.zeros_like(Ad)
    for ov in ovs:
        S[np.ix_(ov.omega, ov.omega)] += Ad[np.ix_(ov.omega, ov.omega)]
    return float(sla.eigh(S, Ad, eigvals_only=True)[-1])


def bound_thm1(kc: int, nu: float) -> float:
    """kappa(M_2^{-1} A) <= (k_c + 1)(2 + (2 k_c + 1) k_c nu) (Theorem 4.5)."""
    return (kc + 1) * (2 + (2 * kc + 1) * kc * nu)


def bound_thm2(kc: int, nu: float, lam_star: float, tau: float) -> float:
    """kappa(M_2^{-1} A) <= (k_c+1)(2 + (2k_c+1) nu (k_c + lambda_* (2 tau + tau^2)))
    (Theorem 5.3; the intermediate line of its proof carries a stray factor tau,
    the theorem statement is used)."""
    return (kc + 1) * (2 + (2 * kc + 1) * nu * (kc + lam_star * (2 * tau + tau * tau)))


def dense_operator(st: OracleSetup) -> np.ndarray:
    """M_2^{-1} as a dense matrix, column by column (tiny problems only)."""
    n = st.A.shape[0]
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n); e[j] = 1.0
        M[:, j] = st.apply(e)
    return M


def condition_number(st: OracleSetup) -> float:
    """kappa(M^{-1} A) for SPD A from the eigenvalues of L^T A L, M^{-1} = L L^T."""
    Minv = dense_operator(st)
    Minv = 0.5 * (Minv + Minv.T)
    L = np.linalg.cholesky(Minv)
    ev = np.linalg.eigvalsh(L.T @ st.A.toarray() @ L)
    return float(ev[-1] / ev[0])
