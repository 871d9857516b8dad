"""Pins of the warm-start oracle (network, subspace loss, features).

The learned warm start is not in the paper; its oracle is a definition, so
each test checks it against something independent: a closed-form network,
the principal angles of scipy.linalg.subspace_angles, central finite
differences, the eigenvalues of eq. gevpsvd from the full dense pencil,
invariance under diagonal scaling, and closed forms on the 2D Laplacian.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import oracle as O
from oracle import warm_mlp as W
from asm_inputs import SplitMix64, poisson2d, diffusion3d


def rand_params(H, K, seed, scale=1.0):
    r = SplitMix64(seed)
    p = r.normal(W.num_params(H, K)) * scale
    W1, b1, W2, b2, W3, b3 = W.unpack(p, H, K)
    # padding columns of W3 / b3 stay zero, as in the C ABI layout
    Kp = W.padded(K)
    o = W.F * H + H + H * H + H
    w3 = p[o:o + H * Kp].reshape(H, Kp)
    w3[:, K:] = 0
    p[o + H * Kp + K:] = 0
    return p


def test_forward_closed_form():
    """W1 = I, W2 = I, b2 = -1/2, W3 = [I_4 0], b3 = 1/4 gives
    Y = max(max(X, 0) - 1/2, 0)[:, :4] + 1/4."""
    H, K = 16, 4
    Kp = W.padded(K)
    p = np.concatenate([np.eye(16).ravel(), np.zeros(H), np.eye(H).ravel(), -0.5 * np.ones(H),
                        np.eye(H, Kp).ravel(), np.r_[0.25 * np.ones(K), np.zeros(Kp - K)]])
    X = SplitMix64(3).normal(40 * 16).reshape(40, 16)
    Y, _ = W.forward(p, X, H, K)
    np.testing.assert_allclose(Y, np.maximum(np.maximum(X, 0) - 0.5, 0)[:, :K] + 0.25, rtol=0, atol=1e-15)


def test_loss_zero_on_target_span_and_k_on_complement():
    r = SplitMix64(11)
    Q, _ = np.linalg.qr(r.normal(50 * 10).reshape(50, 10))
    Z, Zc = Q[:, :4], Q[:, 4:8]
    R = r.normal(16).reshape(4, 4) + 3 * np.eye(4)
    seg = np.array([0, 50])
    l, _ = W.subspace_loss(Z @ R, Z, seg)
    assert abs(l[0]) < 1e-12
    l, _ = W.subspace_loss(Zc @ R, Z, seg)
    assert abs(l[0] - 4) < 1e-12


def test_loss_is_sum_of_squared_principal_sines():
    r = SplitMix64(12)
    sizes = [30, 45, 17]
    seg = np.cumsum([0] + sizes)
    Y = r.normal(seg[-1] * 5).reshape(-1, 5)
    Z = np.zeros_like(Y)
    for a, b in zip(seg[:-1], seg[1:]):
        Z[a:b] = np.linalg.qr(r.normal((b - a) * 5).reshape(b - a, 5))[0]
    l, _ = W.subspace_loss(Y, Z, seg)
    for i, (a, b) in enumerate(zip(seg[:-1], seg[1:])):
        th = sla.subspace_angles(Y[a:b], Z[a:b])
        assert abs(l[i] - np.sum(np.sin(th) ** 2)) < 1e-10


def test_loss_gradient_in_y_matches_finite_differences():
    r = SplitMix64(13)
    seg = np.array([0, 12, 25])
    Y = r.normal(25 * 3).reshape(25, 3)
    Z = np.zeros_like(Y)
    for a, b in zip(seg[:-1], seg[1:]):
        Z[a:b] = np.linalg.qr(r.normal((b - a) * 3).reshape(b - a, 3))[0]
    _, dY = W.subspace_loss(Y, Z, seg)
    h = 1e-6
    for (i, j) in [(0, 0), (5, 2), (13, 1), (24, 0)]:
        Yp, Ym = Y.copy(), Y.copy()
        Yp[i, j] += h
        Ym[i, j] -= h
        fd = (W.subspace_loss(Yp, Z, seg)[0].sum() - W.subspace_loss(Ym, Z, seg)[0].sum()) / (2 * h)
        assert abs(fd - dY[i, j]) < 1e-7 * max(1.0, abs(fd))


def test_parameter_gradient_matches_central_differences():
    H, K = 16, 3
    p = rand_params(H, K, 21, scale=0.4)
    r = SplitMix64(22)
    seg = np.array([0, 9, 21, 28])
    X = r.normal(28 * 16).reshape(28, 16)
    Z = np.zeros((28, K))
    for a, b in zip(seg[:-1], seg[1:]):
        Z[a:b] = np.linalg.qr(r.normal((b - a) * K).reshape(b - a, K))[0]
    loss, g = W.loss_and_grad(p, X, Z, seg, H, K)
    idx = SplitMix64(23).integers(0, W.num_params(H, K) - 1, 80)
    h = 1e-6
    checked = 0
    for q in idx:
        pp, pm = p.copy(), p.copy()
        pp[q] += h
        pm[q] -= h
        lp = W.loss_and_grad(pp, X, Z, seg, H, K)[0]
        lm = W.loss_and_grad(pm, X, Z, seg, H, K)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[q]) < 1e-6 * max(1.0, abs(fd)), (q, fd, g[q])
        checked += abs(g[q]) > 1e-8
    assert checked > 20
    # padding entries carry no gradient
    Kp = W.padded(K)
    o = W.F * H + H + H * H + H
    assert np.all(g[o:o + H * Kp].reshape(H, Kp)[:, K:] == 0)


def test_reduced_operator_spectrum_is_gevpsvd():
    """The features' K has the nonzero eigenvalues lambda^2 of eq. gevpsvd,
    computed here from the full dense pencil on Omega_i."""
    A = diffusion3d(m=10, boxes=(2, 2, 2), contrast=1e3, frac=0.1, delta=1, nev=4, seed=4)
    Acsr = A.csr()
    for ov in O.overlap(Acsr, A.part, A.N, 1)[:3]:
        K = W.reduced_operator(Acsr, ov)
        ev = np.sort(np.linalg.eigvalsh(0.5 * (K + K.T)))[::-1]
        mu, _, _ = O.gevp_svd(O.local_matrix(Acsr, ov), ov)
        nz = int(np.sum(mu > 1e-8 * mu[0]))
        np.testing.assert_allclose(ev[:nz], mu[:nz], rtol=1e-8)


def test_features_invariant_under_diagonal_scaling():
    """A -> S A S (S > 0 diagonal) leaves A^ and K unchanged, so every feature
    but the two log-diagonal ones stays; those shift by the log of S^2."""
    P = poisson2d(24, 24, 3, 3, delta=1, nev=4)
    A = P.csr()
    s = 10.0 ** SplitMix64(5).uniform(A.shape[0])
    As = (sp.diags(s) @ A @ sp.diags(s)).tocsr()
    ovs = O.overlap(A, P.part, P.N, 1)
    for ov in ovs[:4]:
        f = W.features(A, ov)
        fs = W.features(As, ov)
        np.testing.assert_allclose(fs[:, 2:], f[:, 2:], rtol=1e-9, atol=1e-9)
        la = 2 * np.log10(s[ov.omega[ov.m:]])
        np.testing.assert_allclose(fs[:, 0], f[:, 0] + (la - la.mean()) / 6, atol=1e-12)


def test_features_closed_forms_on_laplacian():
    """5-point Laplacian (diagonal 4, off-diagonals -1): la is constant so
    features 0 and 1 vanish; every coupling is 1/4, so each sum is its count
    times 1/4 and the counts add up to the node's degree; the positional
    features are the stated closed forms; the normalised K-features peak at 1."""
    P = poisson2d(20, 20, 2, 2, delta=1, nev=4)
    A = P.csr()
    deg = np.diff(A.indptr) - 1
    for ov in O.overlap(A, P.part, P.N, 1):
        f = W.features(A, ov)
        g = ov.g
        gam = ov.omega[ov.m:]
        assert np.all(f[:, 0] == 0) and np.all(f[:, 1] == 0)
        for c, s in ((5, 2), (6, 3), (7, 4)):
            np.testing.assert_allclose(f[:, s], f[:, c] * 6 / 4, atol=1e-15)
        np.testing.assert_allclose((f[:, 5] + f[:, 6] + f[:, 7]) * 6, deg[gam], atol=1e-12)
        t = np.arange(g) / (g - 1) - 0.5
        np.testing.assert_allclose(f[:, 13], t, atol=1e-15)
        np.testing.assert_allclose(f[:, 14], np.cos(2 * np.pi * (t + 0.5)), atol=1e-14)
        np.testing.assert_allclose(f[:, 15], np.sin(2 * np.pi * (t + 0.5)), atol=1e-14)
        for c in (8, 10, 12):
            assert abs(np.max(np.abs(f[:, c])) - 1) < 1e-14
        np.testing.assert_allclose(f[:, 9], np.log10(1e-4 + np.abs(f[:, 8])) / 4 + 1, atol=1e-14)
