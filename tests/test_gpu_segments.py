"""asm_solve_segments: several independent SPD problems set up by one
asm_setup on their block-diagonal matrix and solved in one call, one CG
recurrence per problem.  Each segment must reproduce what the oracle does on
its problem alone (iteration count within one, the same solution), reach its
own tolerance, and the call must reject segments that do not split A or the
subdomains."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from asm_inputs import SplitMix64, diffusion3d, poisson2d

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


def problems():
    return [diffusion3d(12, (2, 2, 2), contrast=1e4, nev=4, seed=3),
            poisson2d(40, 24, 4, 3, nev=4, seed=4),
            diffusion3d(16, (2, 2, 2), contrast=1e2, nev=4, seed=5)]


def stacked(probs):
    mats = [p.csr() for p in probs]
    A = sp.block_diag(mats, format="csr")
    A.sort_indices()
    parts, off, offs = [], 0, [0]
    for p in probs:
        parts.append(np.asarray(p.part, dtype=np.int32) + off)
        off += p.N
        offs.append(offs[-1] + p.n)
    return A, np.concatenate(parts), off, np.asarray(offs, dtype=np.int32)


def test_segments_match_each_problem_alone(P):
    probs = problems()
    A, part, N, offs = stacked(probs)
    pre = P.TwoLevelSchwarz(A.indptr, A.indices, A.data, part, N, 1, 4, **FP64)
    b = np.concatenate([p.b for p in probs])
    bt = torch.as_tensor(b, device="cuda")
    x = torch.zeros_like(bt)
    rtol = 1e-10
    infos = P.asm_solve_segments(pre.h, bt, x, offs, P.default_solve_opts(rtol=rtol, max_it=2000), pre.stream)
    xv = x.cpu().numpy()
    for k, p in enumerate(probs):
        seg = slice(offs[k], offs[k + 1])
        Ak = p.csr()
        rel = np.linalg.norm(p.b - Ak @ xv[seg]) / np.linalg.norm(p.b)
        assert infos[k].converged and rel <= 1.5 * rtol, (k, rel)
        np.testing.assert_allclose(infos[k].true_relres, rel, rtol=1e-3)
        st = O.setup(Ak, p.part, p.N, 1, 4)
        ref = O.solve(st, p.b, rtol=rtol)
        assert abs(infos[k].iterations - ref.iterations) <= 1, (k, infos[k].iterations, ref.iterations)
        np.testing.assert_allclose(xv[seg], ref.x, rtol=0, atol=1e-7 * np.abs(ref.x).max())
    # the segments converge at different iterations: each keeps its own count
    assert len({i.iterations for i in infos}) > 1
    pre.close()


def test_zero_segment_and_host_io(P):
    """A segment whose right-hand side is zero stops at once with x = 0; a
    host-built handle takes host vectors."""
    probs = problems()[:2]
    A, part, N, offs = stacked(probs)
    pre = P.TwoLevelSchwarz(A.indptr, A.indices, A.data, part, N, 1, 4, device=False)
    b = np.concatenate([np.zeros(probs[0].n), probs[1].b])
    x = np.full_like(b, 7.0)
    infos = P.asm_solve_segments(pre.h, b, x, offs, P.default_solve_opts(rtol=1e-8, max_it=2000))
    assert infos[0].iterations == 0 and infos[0].converged
    assert np.all(x[:offs[1]] == 0)
    rel = np.linalg.norm(probs[1].b - probs[1].csr() @ x[offs[1]:]) / np.linalg.norm(probs[1].b)
    assert infos[1].converged and rel <= 1.5e-8
    pre.close()


def test_segments_must_split_A_and_the_subdomains(P):
    probs = problems()[:2]
    A, part, N, offs = stacked(probs)
    pre = P.TwoLevelSchwarz(A.indptr, A.indices, A.data, part, N, 1, 4)
    bt = torch.as_tensor(SplitMix64(2).normal(A.shape[0]), device="cuda")
    x = torch.zeros_like(bt)
    # a boundary inside the first problem cuts its couplings and its subdomains
    bad = np.array([0, offs[1] // 2, offs[2]], dtype=np.int32)
    with pytest.raises(P.AsmError):
        P.asm_solve_segments(pre.h, bt, x, bad)
    with pytest.raises(P.AsmError):
        P.asm_solve_segments(pre.h, bt, x, np.array([0, offs[1]], dtype=np.int32))  # does not end at n
    with pytest.raises(P.AsmError):
        P.asm_solve_segments(pre.h, bt, x, np.array([0, offs[2], offs[1]], dtype=np.int32))  # decreasing
    pre.close()
