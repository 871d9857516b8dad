"""Seeded synthetic sparse systems shaped like the paper's workloads.

The paper (Section 6) solves finite-element systems whose coefficient fields
come from other papers and are not reproduced there.  The generators below
build finite-difference / Q1 stand-ins with the same structure: 2D and 3D
stencils with a natural box partition, high-contrast diffusion, linear
elasticity and upwind convection-diffusion.  Every random choice comes from
``asm_inputs.rng.SplitMix64`` so the same seed gives the same CSR, partition
and right-hand side on any host.

Returned matrices are CSR with int32 indices, sorted column indices and no
duplicate entries; ``part`` is an int32 array with values 0..N-1.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from .rng import SplitMix64


@dataclass
class Problem:
    name: str
    n: int
    indptr: np.ndarray
    indices: np.ndarray
    data: np.ndarray
    part: np.ndarray
    N: int
    delta: int
    nev: int
    b: np.ndarray
    spd: bool
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def csr(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.data, self.indices, self.indptr), shape=(self.n, self.n))


def _finish(name, A, part, N, delta, nev, b, spd, meta) -> Problem:
    A = sp.csr_matrix(A)
    A.sum_duplicates()
    A.sort_indices()
    return Problem(
        name=name, n=A.shape[0],
        indptr=np.ascontiguousarray(A.indptr, dtype=np.int32),
        indices=np.ascontiguousarray(A.indices, dtype=np.int32),
        data=np.ascontiguousarray(A.data, dtype=np.float64),
        part=np.ascontiguousarray(part, dtype=np.int32), N=int(N), delta=int(delta),
        nev=int(nev), b=np.ascontiguousarray(b, dtype=np.float64), spd=spd, meta=meta)


def _box_part(coords, extents, nparts):
    """Box partition: along each axis, index x of extent m goes to floor(x * k / m)."""
    pid = np.zeros(coords[0].shape, dtype=np.int64)
    stride = 1
    for x, m, k in zip(coords, extents, nparts):
        pid += (x * k // m) * stride
        stride *= k
    return pid.astype(np.int32), stride


def rhs(n: int, seed: int) -> np.ndarray:
    """b ~ N(0, 1) from stream ``seed``."""
    return SplitMix64(seed).normal(n)


# ---------------------------------------------------------------------------
# 2D 5-point Poisson (Dirichlet, unscaled: 4 on the diagonal)
# ---------------------------------------------------------------------------
def poisson2d(nx: int = 64, ny: int = 64, px: int = 4, py: int = 4, delta: int = 1,
              nev: int = 4, seed: int = 0) -> Problem:
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    ix = ix.ravel(); iy = iy.ravel()
    v = ix + nx * iy
    rows = [v]; cols = [v]; vals = [np.full(v.size, 4.0)]
    for dx, dy in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        jx, jy = ix + dx, iy + dy
        ok = (jx >= 0) & (jx < nx) & (jy >= 0) & (jy < ny)
        rows.append(v[ok]); cols.append((jx + nx * jy)[ok]); vals.append(np.full(ok.sum(), -1.0))
    n = nx * ny
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    part, N = _box_part((ix, iy), (nx, ny), (px, py))
    return _finish(f"poisson2d_{nx}x{ny}", A, part, N, delta, nev, rhs(n, seed + 1000), True,
                   {"grid": (nx, ny), "boxes": (px, py), "seed": seed})


# ---------------------------------------------------------------------------
# 3D 7-point high-contrast diffusion
# ---------------------------------------------------------------------------
def contrast_field(m: int, contrast: float, frac: float, seed: int):
    """Voxel coefficient: 1, with seeded full-length 2x2 channels along a random
    axis and boxes of side 2..8 set to ``contrast`` until at least ``frac`` of
    the voxels are high.  Returns (kappa[z, y, x], exact high fraction)."""
    rng = SplitMix64(seed * 7919 + 3)
    high = np.zeros((m, m, m), dtype=bool)
    target = frac * m ** 3
    while high.sum() < target:
        kind = rng.uniform(1)[0]
        if kind < 0.5:
            axis = int(rng.integers(0, 2, 1)[0])
            a, c = (int(t) for t in rng.integers(0, m - 2, 2))
            sl = [slice(a, a + 2), slice(c, c + 2)]
            sl.insert(axis, slice(0, m))
            high[tuple(sl)] = True
        else:
            s = rng.integers(2, min(8, m), 3)
            o = [int(rng.integers(0, m - int(si), 1)[0]) for si in s]
            high[o[0]:o[0] + s[0], o[1]:o[1] + s[1], o[2]:o[2] + s[2]] = True
    kappa = np.where(high, contrast, 1.0)
    return kappa, float(high.mean())


def diffusion3d(m: int = 64, boxes=(8, 8, 8), contrast: float = 1e6, frac: float = 0.10,
                delta: int = 1, nev: int = 16, seed: int = 0) -> Problem:
    """-div(kappa grad u) on an m^3 voxel grid, 7-point finite volumes with the
    harmonic mean of the two voxel coefficients on each interior face and the
    voxel's own coefficient on a Dirichlet boundary face."""
    if contrast == 1.0:
        kappa, hf = np.ones((m, m, m)), 0.0
    else:
        kappa, hf = contrast_field(m, contrast, frac, seed)
    iz, iy, ix = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    ix = ix.ravel(); iy = iy.ravel(); iz = iz.ravel()
    k = kappa.ravel()
    v = ix + m * (iy + m * iz)
    diag = np.zeros(v.size)
    rows, cols, vals = [], [], []
    for dx, dy, dz in ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)):
        jx, jy, jz = ix + dx, iy + dy, iz + dz
        ok = (jx >= 0) & (jx < m) & (jy >= 0) & (jy < m) & (jz >= 0) & (jz < m)
        w = (jx + m * (jy + m * jz))
        kw = np.where(ok, k[np.where(ok, w, 0)], k)
        face = np.where(ok, 2.0 * k * kw / (k + kw), k)
        diag += face
        rows.append(v[ok]); cols.append(w[ok]); vals.append(-face[ok])
    rows.append(v); cols.append(v); vals.append(diag)
    n = m ** 3
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    part, N = _box_part((ix, iy, iz), (m, m, m), boxes)
    return _finish(f"diffusion3d_{m}", A, part, N, delta, nev, rhs(n, seed + 1000), True,
                   {"grid": m, "boxes": tuple(boxes), "contrast": contrast,
                    "high_fraction": hf, "seed": seed})


# ---------------------------------------------------------------------------
# 3D Q1 linear elasticity
# ---------------------------------------------------------------------------
def _q1_element_stiffness(h: float, nu: float) -> np.ndarray:
    """24x24 stiffness of a cube of side h, Young's modulus 1, 2x2x2 Gauss.
    Local node a = i + 2j + 4k at corner (i, j, k); dof = 3a + component."""
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1.0 / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[np.arange(3, 6), np.arange(3, 6)] = mu
    corners = np.array([[i, j, k] for k in (0, 1) for j in (0, 1) for i in (0, 1)], dtype=float)
    s = 2 * corners - 1  # reference coordinates of the corners, in {-1, 1}
    g = 1 / np.sqrt(3.0)
    K = np.zeros((24, 24))
    for gx in (-g, g):
        for gy in (-g, g):
            for gz in (-g, g):
                xi = np.array([gx, gy, gz])
                dN = np.empty((8, 3))
                for a in range(8):
                    f = 1 + s[a] * xi
                    dN[a, 0] = s[a, 0] * f[1] * f[2] / 8
                    dN[a, 1] = f[0] * s[a, 1] * f[2] / 8
                    dN[a, 2] = f[0] * f[1] * s[a, 2] / 8
                dN *= 2.0 / h
                B = np.zeros((6, 24))
                for a in range(8):
                    bx, by, bz = dN[a]
                    B[0, 3 * a] = bx; B[1, 3 * a + 1] = by; B[2, 3 * a + 2] = bz
                    B[3, 3 * a] = by; B[3, 3 * a + 1] = bx
                    B[4, 3 * a + 1] = bz; B[4, 3 * a + 2] = by
                    B[5, 3 * a] = bz; B[5, 3 * a + 2] = bx
                K += B.T @ D @ B * (h / 2) ** 3
    return K


def elasticity3d(ne: int = 32, boxes=(4, 8, 8), nu: float = 0.3, delta: int = 1,
                 nev: int = 24, seed: int = 0) -> Problem:
    """Q1 hexahedra on the unit cube, per-element Young's modulus lognormal(0, 1),
    face x = 0 clamped by identity rows and columns (n stays 3 (ne+1)^3)."""
    nn = ne + 1
    h = 1.0 / ne
    Ke = _q1_element_stiffness(h, nu)
    E = np.exp(SplitMix64(seed * 104729 + 11).normal(ne ** 3))
    ez, ey, ex = np.meshgrid(np.arange(ne), np.arange(ne), np.arange(ne), indexing="ij")
    ex = ex.ravel(); ey = ey.ravel(); ez = ez.ravel()
    corner_nodes = []
    for k in (0, 1):
        for j in (0, 1):
            for i in (0, 1):
                corner_nodes.append((ex + i) + nn * ((ey + j) + nn * (ez + k)))
    nodes = np.stack(corner_nodes, axis=1)  # (nel, 8)
    dofs = (3 * nodes[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 24)
    rows = np.repeat(dofs, 24, axis=1).ravel()
    cols = np.tile(dofs, (1, 24)).ravel()
    vals = (E[:, None] * Ke.ravel()[None, :]).ravel()
    n = 3 * nn ** 3
    A = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    # clamp the face x = 0: identity rows/columns
    nz_, ny_, nx_ = np.meshgrid(np.arange(nn), np.arange(nn), np.arange(nn), indexing="ij")
    nx_ = nx_.ravel(); ny_ = ny_.ravel(); nz_ = nz_.ravel()
    clamped_nodes = np.nonzero(nx_ == 0)[0]
    clamped = (3 * clamped_nodes[:, None] + np.arange(3)[None, :]).ravel()
    keep = np.ones(n); keep[clamped] = 0.0
    Kd = sp.diags(keep)
    A = (Kd @ A @ Kd).tocsr()
    A = A + sp.diags(1.0 - keep)
    A = sp.csr_matrix(A)
    A.eliminate_zeros()
    A = sp.csr_matrix(0.5 * (A + A.T))  # exact symmetry despite summation order
    npart, N = _box_part((nx_, ny_, nz_), (nn, nn, nn), boxes)
    part = np.repeat(npart, 3)
    b = rhs(n, seed + 1000)
    b[clamped] = 0.0
    return _finish(f"elasticity3d_{ne}", A, part, N, delta, nev, b, True,
                   {"elements": ne, "boxes": tuple(boxes), "poisson_ratio": nu, "seed": seed})


# ---------------------------------------------------------------------------
# 2D upwind convection-diffusion (nonsymmetric)
# ---------------------------------------------------------------------------
def convdiff2d(m: int = 512, boxes=(32, 32), peclet: float = 1e3, delta: int = 2,
               nev: int = 16, seed: int = 0) -> Problem:
    """-eps Lap u + v . grad u on the unit square, m x m interior nodes, first-order
    upwind, Dirichlet, everything multiplied by h^2.  v is the rotation field
    (-(y - 1/2), x - 1/2) scaled to max-norm 1 over the grid, eps = 1 / peclet."""
    h = 1.0 / (m + 1)
    eps = 1.0 / peclet
    iy, ix = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    ix = ix.ravel(); iy = iy.ravel()
    x = (ix + 1) * h; y = (iy + 1) * h
    vx = -(y - 0.5); vy = x - 0.5
    scale = max(np.abs(vx).max(), np.abs(vy).max())
    vx /= scale; vy /= scale
    v = ix + m * iy
    diag = 4 * eps + h * (np.abs(vx) + np.abs(vy))
    coef = {(-1, 0): -eps - h * np.maximum(vx, 0), (1, 0): -eps - h * np.maximum(-vx, 0),
            (0, -1): -eps - h * np.maximum(vy, 0), (0, 1): -eps - h * np.maximum(-vy, 0)}
    rows = [v]; cols = [v]; vals = [diag]
    for (dx, dy), c in coef.items():
        jx, jy = ix + dx, iy + dy
        ok = (jx >= 0) & (jx < m) & (jy >= 0) & (jy < m)
        rows.append(v[ok]); cols.append((jx + m * jy)[ok]); vals.append(c[ok])
    n = m * m
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    part, N = _box_part((ix, iy), (m, m), boxes)
    return _finish(f"convdiff2d_{m}", A, part, N, delta, nev, rhs(n, seed + 1000), False,
                   {"grid": m, "boxes": tuple(boxes), "peclet": peclet, "seed": seed})


# ---------------------------------------------------------------------------
# The batched stream of 3D diffusion instances
# ---------------------------------------------------------------------------
def stream_instance(k: int, base_seed: int = 0, nev: int = 16) -> Problem:
    """Instance k of the stream: cube side m ~ U{24..48}, contrast 10^U(2, 6),
    the channel/box field at 10% and boxes from splitting each axis into
    ceil(m / 8) near-equal parts."""
    r = SplitMix64(base_seed * 1_000_003 + 7 * k + 5)
    m = int(r.integers(24, 48, 1)[0])
    contrast = 10.0 ** (2 + 4 * r.uniform(1)[0])
    parts = -(-m // 8)
    p = diffusion3d(m=m, boxes=(parts, parts, parts), contrast=contrast, frac=0.10,
                    delta=1, nev=nev, seed=base_seed * 7907 + k)
    p.name = f"stream_{k}_m{m}"
    p.meta["stream_index"] = k
    return p


# ---------------------------------------------------------------------------
# Named configurations
# ---------------------------------------------------------------------------
def config(name: str, seed: int = 0) -> Problem:
    if name == "c1":
        return poisson2d(64, 64, 4, 4, delta=1, nev=4, seed=seed)
    if name == "c2":
        return diffusion3d(64, (8, 8, 8), 1e6, 0.10, delta=1, nev=16, seed=seed)
    if name == "c3":
        return elasticity3d(32, (4, 8, 8), 0.3, delta=1, nev=24, seed=seed)
    if name == "c4":
        return convdiff2d(512, (32, 32), 1e3, delta=2, nev=16, seed=seed)
    if name == "c2-40":  # the 64^3 recipe on a 40^3 grid (125 boxes of 8^3), for profiler captures
        return diffusion3d(40, (5, 5, 5), 1e6, 0.10, delta=1, nev=16, seed=seed)
    raise KeyError(name)
