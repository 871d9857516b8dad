"""Plain FP64 CPU oracle of the learned warm start of the subspace iteration.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module.  It
shares no code with the CUDA path.

The paper has no learned part: it starts its randomized subspace iteration
(Section 5.1) from random vectors.  The warm start replaces the first k of
those vectors by the output of a per-node network, so the definitions below
are this project's, written out plainly:

* features(): 16 inputs per node of Gamma_delta (the outermost overlap layer,
  whose nodes index the rows of the iteration's block), computed from A, the
  overlap of Section 2.1 and the iteration's operator K = U A^_II U^T, where
  A^ = D^{-1/2} A D^{-1/2} (D = diag|A|), A^_ii = L L^T, W = L^{-1} and
  U = W[Gamma_delta, I_i] (the reduced form of eq. gevpsvd, whose nonzero
  eigenvalues are the lambda^2 of eq. gevpsvd).
* forward(): 16 -> H -> H -> K with ReLU after both hidden layers.
* subspace_loss(): L_i = K - tr(G^{-1} A^T A) with G = Y^T Y, A = Z^T Y, the
  sum of squared sines of the principal angles between span(Y_i) and the
  span of orthonormal targets Z_i; a batch's loss is the mean over segments.
* loss_and_grad(): reverse-mode derivative of that mean loss, by hand.

Parameter vector layout (as the C ABI): W1 (16 x H, row-major), b1 (H),
W2 (H x H), b2 (H), W3 (H x Kp), b3 (Kp), Kp = K rounded up to 16.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .asm_oracle import Overlap

F = 16


def padded(K: int) -> int:
    return (K + 15) // 16 * 16


def unpack(params: np.ndarray, H: int, K: int):
    Kp = padded(K)
    p = np.asarray(params, dtype=np.float64)
    o = 0

    def take(r, c):
        nonlocal o
        a = p[o:o + r * c].reshape(r, c)
        o += r * c
        return a

    W1 = take(F, H); b1 = take(1, H)[0]
    W2 = take(H, H); b2 = take(1, H)[0]
    W3 = take(H, Kp); b3 = take(1, Kp)[0]
    assert o == p.size, "parameter vector has the wrong length"
    return W1, b1, W2, b2, W3[:, :K], b3[:K]


def num_params(H: int, K: int) -> int:
    Kp = padded(K)
    return F * H + H + H * H + H + H * Kp + Kp


def forward(params, X, H, K):
    """Network output Y (rows x K) and the hidden activations."""
    W1, b1, W2, b2, W3, b3 = unpack(params, H, K)
    Z1 = X @ W1 + b1
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ W2 + b2
    H2 = np.maximum(Z2, 0.0)
    Y = H2 @ W3 + b3
    return Y, (X, Z1, H1, Z2, H2)


def subspace_loss(Y, Z, seg):
    """Per-segment loss K - tr((Y^T Y)^{-1} Y^T Z Z^T Y) and dL_i/dY."""
    Y = np.asarray(Y, dtype=np.float64)
    Z = np.asarray(Z, dtype=np.float64)
    K = Y.shape[1]
    losses = np.zeros(len(seg) - 1)
    dY = np.zeros_like(Y)
    for i in range(len(seg) - 1):
        a, b = seg[i], seg[i + 1]
        Yi, Zi = Y[a:b], Z[a:b]
        G = Yi.T @ Yi
        A = Zi.T @ Yi
        Gi = np.linalg.inv(G)
        M = A.T @ A
        losses[i] = K - np.trace(Gi @ M)
        # d tr(G^{-1} M) / dY = 2 (Z A G^{-1} - Y G^{-1} M G^{-1})
        dY[a:b] = 2.0 * (Yi @ Gi @ M @ Gi - Zi @ A @ Gi)
    return losses, dY


def loss_and_grad(params, X, Z, seg, H, K):
    """Mean subspace loss over the segments and its gradient with respect to
    the parameter vector (same layout, padding entries zero)."""
    W1, b1, W2, b2, W3, b3 = unpack(params, H, K)
    Y, (X_, Z1, H1, Z2, H2) = forward(params, X, H, K)
    losses, dY = subspace_loss(Y, Z, seg)
    nseg = len(seg) - 1
    dY = dY / nseg
    gW3 = H2.T @ dY
    gb3 = dY.sum(axis=0)
    dH2 = dY @ W3.T
    dZ2 = dH2 * (Z2 > 0)
    gW2 = H1.T @ dZ2
    gb2 = dZ2.sum(axis=0)
    dH1 = dZ2 @ W2.T
    dZ1 = dH1 * (Z1 > 0)
    gW1 = X_.T @ dZ1
    gb1 = dZ1.sum(axis=0)
    Kp = padded(K)
    gW3p = np.zeros((H, Kp)); gW3p[:, :K] = gW3
    gb3p = np.zeros(Kp); gb3p[:K] = gb3
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3p.ravel(), gb3p])
    return float(losses.mean()), g


# ---------------------------------------------------------------------------
# features
# ---------------------------------------------------------------------------
def reduced_operator(A: sp.spmatrix, ov: Overlap):
    """K = U A^_II U^T (g x g) of the scaled local matrix, the operator of the
    subspace iteration for eq. gevpsvd."""
    A = sp.csr_matrix(A)
    d = 1.0 / np.sqrt(np.abs(A.diagonal()))
    Ah = sp.diags(d) @ A @ sp.diags(d)
    Ahii = Ah[ov.omega][:, ov.omega].toarray()
    L = np.linalg.cholesky(Ahii)
    W = np.linalg.inv(L)
    m, p = ov.m, ov.p
    U = W[m:, :p]
    return U @ Ahii[:p, :p] @ U.T


def features(A: sp.spmatrix, ov: Overlap) -> np.ndarray:
    """g x 16 features of the Gamma_delta nodes of one subdomain, in R_i order."""
    A = sp.csr_matrix(A)
    A.sort_indices()
    n_glob = A.shape[0]
    dg = np.abs(A.diagonal())
    la = np.log10(dg)
    m, nloc, g = ov.m, ov.n, ov.g
    if g == 0:
        return np.zeros((0, F))
    local = -np.ones(n_glob, dtype=np.int64)
    local[ov.omega] = np.arange(nloc)
    gam = ov.omega[m:]
    K = reduced_operator(A, ov)
    one = np.full(g, 1.0 / np.sqrt(g))
    t = np.arange(g) / (g - 1 if g > 1 else 1) - 0.5
    K1 = K @ one
    KK1 = K @ K1
    Kt = K @ t

    def normed(y):
        mx = np.max(np.abs(y))
        return y / mx if mx > 0 else np.zeros_like(y)

    y0, y1, y2 = normed(K1), normed(KK1), normed(Kt)
    out = np.zeros((g, F))
    mean_la = la[gam].mean()
    for r, v in enumerate(gam):
        s_in = s_g = s_out = 0.0
        c_in = c_g = c_out = 0
        dmax = None
        for q in range(A.indptr[v], A.indptr[v + 1]):
            u = A.indices[q]
            if u == v:
                continue
            w = abs(A.data[q]) / np.sqrt(dg[v] * dg[u])
            lc = local[u]
            if 0 <= lc < m:
                dmax = la[u] - la[v] if dmax is None else max(dmax, la[u] - la[v])
                s_in += w; c_in += 1
            elif lc >= m:
                s_g += w; c_g += 1
            else:
                s_out += w; c_out += 1
        out[r] = [(la[v] - mean_la) / 6, (0.0 if dmax is None else dmax) / 6, s_in, s_g, s_out, c_in / 6, c_g / 6, c_out / 6,
                  y0[r], np.log10(1e-4 + abs(y0[r])) / 4 + 1, y1[r], np.log10(1e-4 + abs(y1[r])) / 4 + 1,
                  y2[r], t[r], np.cos(2 * np.pi * (t[r] + 0.5)), np.sin(2 * np.pi * (t[r] + 0.5))]
    return out
