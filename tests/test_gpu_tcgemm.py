"""The tensor-core tile-product kernel (asm_tile_products, tcgen05 3xTF32)
against FP64 products of the same FP32 inputs.

Bound per element: the split x = hi + lo keeps hi exact and lo to TF32 (a
relative 2^-11 of lo, itself at most 2^-11 |x|); the dropped lo*lo term is at
most 2^-22 |a||b|; so each term a*b carries at most 3 * 2^-22 |a||b|, and
the FP32 accumulation over K terms adds at most K * 2^-24 sum |a||b| (first
order).  The test checks |C - C_ref| <= (3 * 2^-22 + K * 2^-24) (|A| |B|^T)
elementwise, and that the error is far below a single TF32 pass's."""
import numpy as np
import pytest

from asm_inputs import SplitMix64

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

T = 64


@pytest.fixture(scope="module")
def P():
    from paper_2401_03915_gb300 import build
    build.build()
    import paper_2401_03915_gb300 as P
    P.load()
    return P


def tile(buf, off, ld):
    """64 x 64 view of the flat array buf at element offset off, row stride ld."""
    return np.lib.stride_tricks.as_strided(buf[off:], shape=(T, T), strides=(ld * 8, 8))


def reference(j, A, B, C0):
    acc = np.zeros((T, T))
    absacc = np.zeros((T, T))
    for t in range(j["nprod"]):
        a = tile(A, j["a0"] + t * j["a_step"], j["lda"])
        b = tile(B, j["b0"] + t * j["b_step"], j["ldb"])
        if j["flags"] & 1:
            a = a.T
        if j["flags"] & 2:
            b = b.T
        acc += a @ b.T
        absacc += np.abs(a) @ np.abs(b).T
    if j["flags"] & 8:
        acc = -acc
    if j["flags"] & 4:
        acc = acc + tile(C0, j["c_in"], j["ldc_in"])
    return acc, absacc


def run_jobs(P, jobs, A, B, C, inplace_b=False):
    dev = torch.device("cuda")
    At = torch.as_tensor(A.astype(np.float32), device=dev)
    Bt = torch.as_tensor(B.astype(np.float32), device=dev) if not inplace_b else At
    Ct = torch.as_tensor(C.astype(np.float32), device=dev)
    P.asm_tile_products(jobs, At, Bt, Ct, Ct)
    return Ct.cpu().numpy().astype(np.float64)


def make_jobs(rng, njobs, lda, ldb, ldc, rows_a, rows_b, flags_list):
    import paper_2401_03915_gb300 as P
    jobs = np.zeros(njobs, dtype=P.TILE_JOB_DTYPE)
    for k in range(njobs):
        npd = int(rng.integers(1, 5, 1)[0])
        fl = flags_list[k % len(flags_list)]
        jobs[k]["nprod"] = npd
        jobs[k]["flags"] = fl
        jobs[k]["lda"], jobs[k]["ldb"] = lda, ldb
        jobs[k]["ldc_in"] = jobs[k]["ldc_out"] = ldc
        # products walk down (A) or across (B) their matrices
        jobs[k]["a0"] = int(rng.integers(0, 3, 1)[0]) * 4 + int(rng.integers(0, rows_a - T * 5 - 1, 1)[0]) * lda
        jobs[k]["a_step"] = T * lda if k % 2 else T
        jobs[k]["b0"] = int(rng.integers(0, rows_b - T * 5 - 1, 1)[0]) * ldb
        jobs[k]["b_step"] = T if k % 3 else T * ldb
        jobs[k]["c_in"] = jobs[k]["c_out"] = k * T * ldc
    return jobs


def check(C, jobs, A, B, C0, one_pass_factor=True):
    for j in jobs:
        ref, absr = reference(j, A, B, C0)
        out = tile(C.ravel(), j["c_out"], j["ldc_out"])
        K = T * j["nprod"]
        bound = (3 * 2.0 ** -22 + K * 2.0 ** -24) * absr + (np.abs(tile(C0, j["c_in"], j["ldc_in"])) * 2.0 ** -24
                                                          if j["flags"] & 4 else 0)
        err = np.abs(out - ref)
        assert np.all(err <= bound), (int(j["flags"]), float(np.max(err / (bound + 1e-300))))
        if one_pass_factor:
            # a single TF32 pass would leave errors near 2^-11 |a||b|
            assert np.max(err / absr) < 2.0 ** -16


@pytest.mark.parametrize("flags", [0, 1, 2, 3, 4 | 8, 1 | 2 | 4 | 8])
def test_tile_products_all_operand_forms(P, flags):
    rng = SplitMix64(100 + flags)
    lda, ldb, ldc = 400, 388, 72
    ra, rb = 640, 600
    A = rng.normal(ra * lda) * np.exp(rng.normal(ra * lda))
    B = rng.normal(rb * ldb)
    A32, B32 = A.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64)
    njobs = 40
    jobs = make_jobs(rng, njobs, lda, ldb, ldc, ra, rb, [flags])
    C0 = rng.normal(njobs * T * ldc).astype(np.float32).astype(np.float64)
    C = run_jobs(P, jobs, A32, B32, C0)
    check(C.ravel(), jobs, A32, B32, C0)
    # columns beyond the 64 of each output row are untouched
    Cm = C.reshape(njobs * T, ldc)
    np.testing.assert_array_equal(Cm[:, T:], C0.reshape(njobs * T, ldc)[:, T:])


def test_tile_products_in_place_output(P):
    """A job whose output is its own A operand (the panel step L = C Dinv^T)."""
    rng = SplitMix64(7)
    ld = 256
    A = rng.normal(2 * T * ld).astype(np.float32).astype(np.float64)
    jobs = np.zeros(2, dtype=P.TILE_JOB_DTYPE)
    for k in range(2):
        jobs[k]["a0"] = jobs[k]["c_out"] = jobs[k]["c_in"] = k * T * ld
        jobs[k]["b0"] = k * T * ld + 128
        jobs[k]["lda"] = jobs[k]["ldb"] = jobs[k]["ldc_in"] = jobs[k]["ldc_out"] = ld
        jobs[k]["nprod"] = 1
        jobs[k]["flags"] = 0
    refs = [reference(j, A, A, A) for j in jobs]
    dev = torch.device("cuda")
    At = torch.as_tensor(A.astype(np.float32), device=dev)
    P.asm_tile_products(jobs, At, At, None, At)
    out = At.cpu().numpy().astype(np.float64)
    for j, (ref, absr) in zip(jobs, refs):
        err = np.abs(tile(out, j["c_out"], ld) - ref)
        assert np.all(err <= (3 * 2.0 ** -22 + T * 2.0 ** -24) * absr)


def test_tile_products_many_jobs_and_empty(P):
    """More jobs than resident blocks (each block strides over several), and
    an empty batch."""
    rng = SplitMix64(9)
    ld = 128
    A = rng.normal(8 * T * ld).astype(np.float32).astype(np.float64)
    njobs = 2000
    jobs = np.zeros(njobs, dtype=P.TILE_JOB_DTYPE)
    for k in range(njobs):
        jobs[k]["a0"] = (k % 8) * T * ld
        jobs[k]["b0"] = ((k * 3) % 8) * T * ld + 64
        jobs[k]["lda"] = jobs[k]["ldb"] = ld
        jobs[k]["ldc_out"] = T
        jobs[k]["c_out"] = k * T * T
        jobs[k]["nprod"] = 1
        jobs[k]["flags"] = 2
    dev = torch.device("cuda")
    At = torch.as_tensor(A.astype(np.float32), device=dev)
    Ct = torch.full((njobs * T * T,), np.nan, dtype=torch.float32, device=dev)
    P.asm_tile_products(jobs, At, At, None, Ct)
    C = Ct.cpu().numpy().astype(np.float64)
    for k in range(0, njobs, 97):
        ref, absr = reference(jobs[k], A, A, None)
        err = np.abs(tile(C, jobs[k]["c_out"], T) - ref)
        assert np.all(err <= (3 * 2.0 ** -22 + T * 2.0 ** -24) * absr)
    assert np.isfinite(C).all()
    P.asm_tile_products(jobs[:0], At, At, None, Ct)


def test_tile_products_argument_checks(P):
    rng = SplitMix64(1)
    dev = torch.device("cuda")
    A = torch.zeros(T * T, dtype=torch.float32, device=dev)
    jobs = np.zeros(1, dtype=P.TILE_JOB_DTYPE)
    jobs[0]["lda"] = jobs[0]["ldb"] = jobs[0]["ldc_out"] = T
    jobs[0]["nprod"] = 0
    with pytest.raises(P.AsmError):
        P.asm_tile_products(jobs, A, A, None, A)
    jobs[0]["nprod"] = 1
    jobs[0]["a0"] = 2  # not 16-byte aligned
    with pytest.raises(P.AsmError):
        P.asm_tile_products(jobs, A, A, None, A)
    jobs[0]["a0"] = 0
    jobs[0]["flags"] = 4  # C_in without cin
    with pytest.raises(P.AsmError):
        P.asm_tile_products(jobs, A, A, None, A)
    del rng
