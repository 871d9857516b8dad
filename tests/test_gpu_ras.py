"""Restricted one-level part (eq. onelevelras) and the deflated coarse
correction of the Section 6 experiments on the CUDA path, against the oracle
and against their definitions evaluated with the GPU's own Z and E."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from asm_inputs import SplitMix64, poisson2d, diffusion3d, convdiff2d

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


def gpu_Z(P, h, ovs, n):
    blocks, col = P.asm_get_coarse_basis(h, [ov.p for ov in ovs])
    Z = np.zeros((n, col[-1]))
    for i, ov in enumerate(ovs):
        Z[ov.omega[:ov.p], col[i]:col[i + 1]] = blocks[i]
    return Z


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ras_one_level_matches_oracle(P, prec):
    prob = diffusion3d(16, (2, 2, 2), contrast=1e4, nev=6)
    A = prob.csr()
    st = O.setup(A, prob.part, prob.N, 1, 0)
    pre = make(P, A, prob.part, prob.N, 1, 0, precision=prec, coarse=0, one_level=1)
    r = SplitMix64(41).normal(prob.n)
    z = pre.apply(torch.as_tensor(r, device="cuda")).cpu().numpy()
    zr = st.apply_one_level_ras(r)
    if prec == "fp64":
        np.testing.assert_allclose(z, zr, rtol=0, atol=1e-11 * np.abs(zr).max())
    else:
        # the same single-precision local solves as the additive part
        assert np.linalg.norm(z - zr) / np.linalg.norm(zr) < 1e-3
    # every node takes exactly one local solution: z differs from the additive sum
    pre_a = make(P, A, prob.part, prob.N, 1, 0, precision=prec, coarse=0)
    za = pre_a.apply(torch.as_tensor(r, device="cuda")).cpu().numpy()
    assert np.linalg.norm(za - z) > 1e-3 * np.linalg.norm(z)
    pre.close(); pre_a.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("one_level", [0, 1])
def test_deflated_apply_matches_its_definition(P, prec, one_level):
    """z = Q r + M_1^{-1}(r - A Q r) with the GPU's own Z and E (Q solved
    densely on the CPU) and the GPU's own one-level part; and M^{-1} A Z c = Z c."""
    prob = diffusion3d(24, (4, 4, 4), contrast=1e3, nev=8)
    A = prob.csr()
    pre = make(P, A, prob.part, prob.N, 1, 8, precision=prec, one_level=one_level, coarse_mode=1)
    pre1 = make(P, A, prob.part, prob.N, 1, 0, precision=prec, one_level=one_level, coarse=0)
    ovs = O.overlap(A, prob.part, prob.N, 1)
    Z = gpu_Z(P, pre.h, ovs, prob.n)
    E = P.asm_get_coarse_matrix(pre.h)
    Es = 0.5 * (E + E.T)
    r = SplitMix64(8).normal(prob.n)
    q = Z @ np.linalg.solve(Es, Z.T @ r)
    w = r - A @ q
    m1w = pre1.apply(torch.as_tensor(w, device="cuda")).cpu().numpy()
    ref = q + m1w
    z = pre.apply(torch.as_tensor(r, device="cuda")).cpu().numpy()
    tol = 1e-9 if prec == "fp64" else 2e-5
    np.testing.assert_allclose(z, ref, rtol=0, atol=tol * np.abs(ref).max())
    # the deflated preconditioner is the inverse of A on range(Z)
    c = SplitMix64(9).normal(Z.shape[1])
    zc = pre.apply(torch.as_tensor(A @ (Z @ c), device="cuda")).cpu().numpy()
    tol = 1e-8 if prec == "fp64" else 1e-4
    np.testing.assert_allclose(zc, Z @ c, rtol=0, atol=tol * np.abs(Z @ c).max())
    pre.close(); pre1.close()


def test_ras_deflated_fgmres_c1(P):
    prob = poisson2d(64, 64, 4, 4, nev=4)
    A = prob.csr()
    st = O.setup(A, prob.part, prob.N, 1, 4)
    ref = O.solve(st, prob.b, restart=64, one_level="ras", coarse="deflated")
    pre = make(P, A, prob.part, prob.N, 1, 4, one_level=1, coarse_mode=1, **FP64)
    x, info = pre.solve(torch.as_tensor(prob.b, device="cuda"), restart=64)
    xr = x.cpu().numpy()
    rel = np.linalg.norm(prob.b - A @ xr) / np.linalg.norm(prob.b)
    assert info.converged and rel <= 1.5e-8
    # the GPU's coarse space spans the oracle's up to the eigensolver tolerance
    assert abs(info.iterations - ref.iterations) <= max(2, 0.1 * ref.iterations), (info.iterations, ref.iterations)
    np.testing.assert_allclose(xr, ref.x, rtol=0, atol=1e-5 * np.abs(ref.x).max())
    pre.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ras_deflated_general_path(P, prec):
    prob = convdiff2d(64, (4, 4), peclet=1e3, delta=2, nev=6)
    A = prob.csr()
    pre = make(P, A, prob.part, prob.N, 2, 6, spd=False, precision=prec, one_level=1, coarse_mode=1)
    x, info = pre.solve(torch.as_tensor(prob.b, device="cuda"), restart=64)
    rel = np.linalg.norm(prob.b - A @ x.cpu().numpy()) / np.linalg.norm(prob.b)
    assert info.converged and rel <= 1e-7
    if prec == "fp64":
        st = O.setup(A, prob.part, prob.N, 2, 6, spd=False)
        ref = O.solve(st, prob.b, restart=64, one_level="ras", coarse="deflated")
        assert abs(info.iterations - ref.iterations) <= max(2, 0.1 * ref.iterations), (info.iterations, ref.iterations)
    pre.close()


def test_invalid_variant_options(P):
    prob = poisson2d(16, 16, 2, 2, nev=2)
    with pytest.raises(P.AsmError) as e:
        make(P, prob.csr(), prob.part, prob.N, 1, 2, one_level=2)
    assert e.value.name == "INVALID_ARG"
    with pytest.raises(P.AsmError) as e:
        make(P, prob.csr(), prob.part, prob.N, 1, 2, coarse_mode=-1)
    assert e.value.name == "INVALID_ARG"
