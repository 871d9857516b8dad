"""GPU tests of the learned warm start: features and targets against the
oracle, network forward and gradients against the FP64 CPU oracle, and what
the trained network gains over the randomized start of the subspace
iteration."""
import numpy as np
import pytest

import oracle as O
from oracle import warm_mlp as W
from asm_inputs import SplitMix64, poisson2d, diffusion3d, stream_instance

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2401_03915_gb300 as P  # noqa: E402


def dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def setup(prob, precision="fp64", **opts):
    return P.TwoLevelSchwarz(prob.indptr, prob.indices, prob.data, prob.part, prob.N, prob.delta, prob.nev,
                             precision=precision, **opts)


def contrast_case():
    return diffusion3d(m=16, boxes=(2, 2, 2), contrast=1e4, frac=0.1, delta=1, nev=8, seed=2)


@pytest.mark.parametrize("precision,atol", [("fp64", 2e-6), ("fp32", 5e-3)])
@pytest.mark.parametrize("case", ["poisson", "contrast"])
def test_features_match_oracle(case, precision, atol):
    prob = poisson2d(32, 32, 2, 2, delta=1, nev=4) if case == "poisson" else contrast_case()
    S = setup(prob, precision, record_warm=1)
    off, X, T = P.asm_get_warm_data(S.h)
    X = X.cpu().numpy().astype(np.float64)
    A = prob.csr()
    ovs = O.overlap(A, prob.part, prob.N, prob.delta)
    for i, ov in enumerate(ovs):
        assert off[i + 1] - off[i] == ov.g
        f = W.features(A, ov)
        np.testing.assert_allclose(X[off[i]:off[i + 1]], f, rtol=0, atol=atol, err_msg=f"subdomain {i}")
    S.close()


def test_targets_span_oracle_eigenvectors():
    prob = contrast_case()
    S = setup(prob, "fp64", record_warm=1, eig_tol=1e-10)
    off, X, T = P.asm_get_warm_data(S.h)
    T = T.cpu().numpy().astype(np.float64)
    A = prob.csr()
    checked = 0
    for i, ov in enumerate(O.overlap(A, prob.part, prob.N, prob.delta)):
        K = W.reduced_operator(A, ov)
        ev, V = np.linalg.eigh(0.5 * (K + K.T))
        ev, V = ev[::-1], V[:, ::-1]
        Ti = T[off[i]:off[i + 1]]
        # compare the spans of the leading k vectors where the spectrum has a gap
        for k in range(1, prob.nev):
            if (ev[k - 1] - ev[k]) / ev[0] > 1e-3:
                Pt = Ti[:, :k] @ Ti[:, :k].T
                Po = V[:, :k] @ V[:, :k].T
                assert np.max(np.abs(Pt - Po)) < 1e-5, (i, k)
                checked += 1
        # orthonormal targets (FP32 storage)
        np.testing.assert_allclose(Ti.T @ Ti, np.eye(prob.nev), atol=1e-6)
    assert checked > 0
    S.close()


def test_mlp_forward_matches_oracle():
    net = P.WarmStartNet(256, 16, seed=5)
    p = net.params().astype(np.float64)
    X = SplitMix64(6).normal(3000 * 16).reshape(3000, 16)
    Y = net.forward(dev(X, torch.float32)).cpu().numpy()
    Yo, _ = W.forward(p, X, 256, 16)
    # FP16 operands (2^-11 relative), FP32 accumulation over 16 + 256 + 256 terms
    err = np.linalg.norm(Y - Yo) / np.linalg.norm(Yo)
    assert err < 5e-3, err
    net.close()


def test_mlp_gradient_matches_oracle():
    """The GPU backward (FP16 operands, FP32 accumulation) against the FP64
    analytic gradient of the oracle, which the CPU tests pin to central
    finite differences."""
    H, K = 256, 16
    net = P.WarmStartNet(H, K, seed=7)
    p = net.params().astype(np.float64)
    r = SplitMix64(8)
    sizes = r.integers(40, 120, 24)
    seg = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    rows = int(seg[-1])
    X = r.normal(rows * 16).reshape(rows, 16)
    Z = np.zeros((rows, K))
    for a, b in zip(seg[:-1], seg[1:]):
        Z[a:b] = np.linalg.qr(r.normal((b - a) * K).reshape(b - a, K))[0]
    loss, g = net.loss_grad(dev(X, torch.float32), dev(Z, torch.float32), dev(seg, torch.int64))
    lo, go = W.loss_and_grad(p, X, Z, seg, H, K)
    assert abs(loss - lo) < 1e-3 * abs(lo), (loss, lo)
    g = g.astype(np.float64)
    rel = np.linalg.norm(g - go) / np.linalg.norm(go)
    cos = g @ go / (np.linalg.norm(g) * np.linalg.norm(go))
    assert rel < 3e-2 and cos > 0.999, (rel, cos)
    # per layer
    o = 0
    for size in (16 * H, H, H * H, H, H * 16, 16):
        gs, gos = g[o:o + size], go[o:o + size]
        assert np.linalg.norm(gs - gos) <= 5e-2 * np.linalg.norm(gos) + 1e-9
        o += size
    net.close()


def _collect(probs, precision="fp32"):
    Xs, Ts, offs, base = [], [], [0], 0
    for prob in probs:
        S = setup(prob, precision, record_warm=1)
        off, X, T = P.asm_get_warm_data(S.h)
        Xs.append(X)
        Ts.append(T)
        offs.extend((off[1:] + base).tolist())
        base += int(off[-1])
        S.close()
    return torch.cat(Xs), torch.cat(Ts), np.asarray(offs, dtype=np.int64)


def test_training_reduces_loss_and_warm_start_gains():
    """Train on generated 3D high-contrast subdomains (seeds disjoint from the
    held-out ones) and compare, on held-out instances, the subspace loss of the
    predicted start against random starts, and the eigen-residual reached in a
    fixed small number of sweeps with and without the network."""
    train = [stream_instance(k, base_seed=1) for k in range(6)]
    X, T, off = _collect(train)
    net = P.WarmStartNet(256, 16, seed=1)
    seg_all = dev(off, torch.int64)
    loss0, _ = net.loss_grad(X, T, seg_all)
    net.train(X, T, off, steps=400, lr=1e-3, batch=32)
    loss1, _ = net.loss_grad(X, T, seg_all)
    assert loss1 < 0.8 * loss0, (loss0, loss1)

    test = [stream_instance(k, base_seed=0) for k in range(2)]
    Xh, Th, offh = _collect(test)
    segh = dev(offh, torch.int64)
    loss_net, _ = net.loss_grad(Xh, Th, segh)
    Yr = torch.as_tensor(SplitMix64(9).normal(Xh.shape[0] * 16).reshape(-1, 16), dtype=torch.float32, device="cuda")
    loss_rand, _ = W.subspace_loss(Yr.cpu().numpy(), Th.cpu().numpy(), offh)[0].mean(), None
    assert loss_net < 0.9 * loss_rand, (loss_net, loss_rand)

    # the warm start cuts sweeps at the default tolerance and leaves smaller
    # eigen-residuals after a fixed small number of sweeps
    sweeps, resid = {0: [], 1: []}, {0: [], 1: []}
    for prob in test:
        for warm in (0, 1):
            kw = dict(warm_start=warm, warm_net=net.ptr if warm else None)
            S = setup(prob, "fp32", **kw)
            sweeps[warm].append(P.asm_get_eigen_stats(S.h)[1])
            x, info = S.solve(torch.as_tensor(prob.b, device="cuda"))
            A = prob.csr()
            rel = np.linalg.norm(prob.b - A @ x.cpu().numpy()) / np.linalg.norm(prob.b)
            assert info.converged and rel <= 1.5e-8
            S.close()
            S = setup(prob, "fp32", max_sweeps=3, **kw)
            r, _ = P.asm_get_eigen_stats(S.h)
            resid[warm].append(r[:, :8].max(axis=1))
            S.close()
    sw0, sw1 = np.concatenate(sweeps[0]).mean(), np.concatenate(sweeps[1]).mean()
    r0, r1 = np.median(np.concatenate(resid[0])), np.median(np.concatenate(resid[1]))
    print(f"mean sweeps random {sw0:.2f} warm {sw1:.2f}; median residual after 3 sweeps random {r0:.3e} warm {r1:.3e}")
    # measured on GB300: mean sweeps 5.98 -> 5.24, median residual after three
    # sweeps 9.7e-2 -> 2.1e-2; the margins leave room for run-to-run spread
    assert sw1 <= 0.95 * sw0 and r1 <= 0.5 * r0, (sw0, sw1, r0, r1)
    net.close()


def test_learned_start_on_the_batched_stream():
    """The learned start on the 200 held-out instances of the stream, set up
    in batches of 20 (one asm_setup per block-diagonal batch, one PCG per
    instance through asm_solve_segments), arms alternated and the best of two
    passes kept (the apply tuner caches its choice per shape, so a first pass
    would favour whichever arm runs second): it cuts the mean sweep count by at
    least 10% (measured: 5.93 -> 5.18), every instance still reaches 1e-8, and
    setup + solve is not slower.  The wall-clock gain is small (measured 2%):
    a batch's eigen stage lasts as long as its slowest subdomain."""
    import scipy.sparse as sp
    train = [stream_instance(k, base_seed=1) for k in range(12)]
    X, T, off = _collect(train)
    net = P.WarmStartNet(256, 16, seed=1)
    net.train(X, T, off, steps=2000, lr=1e-3, batch=32)
    insts = [stream_instance(k, base_seed=0) for k in range(200)]
    batches = []
    for g0 in range(0, len(insts), 20):
        chunk = insts[g0:g0 + 20]
        A = sp.block_diag([p.csr() for p in chunk], format="csr")
        A.sort_indices()
        parts, o, offs = [], 0, [0]
        for p in chunk:
            parts.append(np.asarray(p.part, dtype=np.int32) + o)
            o += p.N
            offs.append(offs[-1] + p.n)
        b = np.concatenate([p.b for p in chunk])
        batches.append((A, np.concatenate(parts), o, np.asarray(offs, dtype=np.int32),
                        torch.as_tensor(b, device="cuda")))
    times, sweeps = {}, {}
    for warm in (0, 1, 0, 1):   # twice each, best kept
        kw = dict(warm_start=warm, warm_net=net.ptr if warm else None)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        sw = []
        for A, part, N, offs, bt in batches:
            S = P.TwoLevelSchwarz(A.indptr, A.indices, A.data, part, N, 1, 16, precision="fp32", **kw)
            sw.append(P.asm_get_eigen_stats(S.h)[1])
            x = torch.zeros_like(bt)
            infos = P.asm_solve_segments(S.h, bt, x, offs, P.default_solve_opts(rtol=1e-8, max_it=5000))
            assert all(i.converged and i.true_relres <= 1.5e-8 for i in infos)
            S.close()
        t1.record()
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
        times[warm] = min(times.get(warm, 3e38), ms)
        sweeps[warm] = np.concatenate(sw).mean()
    print(f"batched stream (200 instances): random {times[0]:.1f} ms, learned {times[1]:.1f} ms; "
          f"mean sweeps {sweeps[0]:.2f} -> {sweeps[1]:.2f}")
    assert sweeps[1] <= 0.9 * sweeps[0], sweeps
    assert times[1] <= 1.02 * times[0], times
    net.close()
