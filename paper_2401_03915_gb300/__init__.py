"""Python binding of the sm_103a two-level additive Schwarz library.

Argument marshalling only: every step of the method runs in the CUDA kernels
of ``libasm_gb300.so`` behind the C ABI declared in ``include/asm.h``.  The
functions below keep the C names (``asm_setup``, ``asm_apply``,
``asm_solve``, ...); :class:`TwoLevelSchwarz` wraps a handle for callers
holding NumPy arrays or torch tensors.  There is no CPU fallback: if the
library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

ASM_OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "NOT_SPD", 3: "ZERO_PIVOT", 4: "COARSE_SINGULAR",
          5: "NONFINITE", 6: "NO_CONVERGENCE", 7: "TIMEOUT", 8: "CUDA", 9: "OOM", 10: "UNSUPPORTED"}
PREC_FP64, PREC_FP32, PREC_FP32_H16, PREC_FP32_B16 = 0, 1, 2, 3


class AsmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class asm_csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int32), ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p),
                ("val", C.c_void_p), ("on_device", C.c_int32)]


class asm_options(C.Structure):
    _fields_ = [("spd", C.c_int32), ("local_precision", C.c_int32), ("oversample", C.c_int32),
                ("max_sweeps", C.c_int32), ("eig_tol", C.c_double), ("nu", C.c_double),
                ("nev_lift", C.c_int32), ("coarse", C.c_int32), ("seed", C.c_uint64),
                ("warm_start", C.c_int32), ("filter_degree", C.c_int32), ("record_warm", C.c_int32),
                ("one_level", C.c_int32), ("coarse_mode", C.c_int32),
                ("reserved", C.c_int32 * 1), ("tau", C.c_double), ("warm_net", C.c_void_p)]


class asm_solve_opts(C.Structure):
    _fields_ = [("method", C.c_int32), ("restart", C.c_int32), ("rtol", C.c_double), ("max_it", C.c_int32),
                ("use_x0", C.c_int32), ("check_every", C.c_int32), ("reserved", C.c_int32 * 5)]


class asm_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("final_relres", C.c_double),
                ("true_relres", C.c_double), ("solve_ms", C.c_double)]


class asm_setup_info(C.Structure):
    _fields_ = [("n", C.c_int32), ("N", C.c_int32), ("overlap", C.c_int32), ("nev", C.c_int32),
                ("n_C", C.c_int32), ("nnz_C", C.c_int64), ("gc", C.c_double), ("oc", C.c_double),
                ("sum_ni", C.c_int64), ("max_ni", C.c_int32), ("sweeps_max", C.c_int32),
                ("eig_resid_max", C.c_double), ("stage_ms", C.c_double * 12), ("coarse_levels", C.c_int32),
                ("coarse_fronts", C.c_int32), ("coarse_front_entries", C.c_int64), ("coarse_max_front", C.c_int32),
                ("tile_ctas", C.c_int32), ("local_sym", C.c_int32), ("local_fp16", C.c_int32)]


_lib = None


def lib_path() -> str:
    return _build.lib_path()


def load(path: str | None = None) -> C.CDLL:
    """Load (once) the shared library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2401_03915_gb300.build.build()")
    L = C.CDLL(path)
    vp, i32, pp = C.c_void_p, C.c_int32, C.POINTER(C.c_void_p)
    L.asm_default_options.argtypes = [C.POINTER(asm_options)]
    L.asm_default_solve_opts.argtypes = [C.POINTER(asm_solve_opts)]
    L.asm_setup.argtypes = [C.POINTER(asm_csr), vp, i32, i32, i32, C.POINTER(asm_options), vp, pp]
    L.asm_apply.argtypes = [vp, vp, vp, vp]
    L.asm_spmv.argtypes = [vp, vp, vp, vp]
    L.asm_solve.argtypes = [vp, vp, vp, C.POINTER(asm_solve_opts), C.POINTER(asm_solve_info), vp]
    L.asm_get_info.argtypes = [vp, C.POINTER(asm_setup_info)]
    L.asm_get_overlap.argtypes = [vp, vp, vp, vp]
    L.asm_get_local_values.argtypes = [vp, vp, vp]
    L.asm_get_lift_values.argtypes = [vp, vp, vp]
    L.asm_get_eigen_stats.argtypes = [vp, vp, vp]
    L.asm_get_coarse_basis.argtypes = [vp, vp, vp]
    L.asm_get_coarse_matrix.argtypes = [vp, vp]
    L.asm_kernel_launches.restype = C.c_uint64
    L.asm_kernel_launches.argtypes = []
    L.asm_time_apply.argtypes = [vp, vp, vp, i32, vp, C.POINTER(C.c_double)]
    L.asm_time_apply.restype = C.c_int
    L.asm_csr_spmv.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp]
    L.asm_csr_spmv.restype = C.c_int
    L.asm_time_spmv.argtypes = [vp, vp, vp, i32, vp, C.POINTER(C.c_double)]
    L.asm_time_spmv.restype = C.c_int
    L.asm_spmv_dot_noalloc.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp]
    L.asm_spmv_dot_noalloc.restype = C.c_int
    i64, f32 = C.c_int64, C.c_float
    L.asm_tile_products.argtypes = [vp, i64, vp, vp, vp, vp, vp]
    L.asm_tile_products.restype = C.c_int
    L.asm_solve_segments.argtypes = [vp, vp, vp, i32, vp, C.POINTER(asm_solve_opts), vp, vp]
    L.asm_solve_segments.restype = C.c_int
    L.asm_mlp_create.argtypes = [i32, i32, C.c_uint64, pp]
    L.asm_mlp_destroy.argtypes = [vp]
    L.asm_mlp_destroy.restype = None
    L.asm_mlp_num_params.argtypes = [vp]
    L.asm_mlp_num_params.restype = i64
    L.asm_mlp_get_params.argtypes = [vp, vp]
    L.asm_mlp_set_params.argtypes = [vp, vp]
    L.asm_mlp_forward.argtypes = [vp, vp, i32, vp, vp]
    L.asm_mlp_loss_grad.argtypes = [vp, vp, i32, vp, vp, i32, C.POINTER(C.c_double), vp, vp]
    L.asm_mlp_train_step.argtypes = [vp, vp, i32, vp, vp, i32, f32, C.POINTER(C.c_double), vp]
    L.asm_get_warm_data.argtypes = [vp, vp, vp, vp, vp]
    L.asm_destroy.argtypes = [vp]
    L.asm_destroy.restype = None
    L.asm_last_error.restype = C.c_char_p
    L.asm_stage_name.restype = C.c_char_p
    L.asm_stage_name.argtypes = [i32]
    for f in ("asm_setup", "asm_apply", "asm_spmv", "asm_solve", "asm_get_info", "asm_get_overlap",
              "asm_get_local_values", "asm_get_lift_values", "asm_get_eigen_stats", "asm_get_coarse_basis", "asm_get_coarse_matrix", "asm_mlp_create",
              "asm_mlp_get_params", "asm_mlp_set_params", "asm_mlp_forward", "asm_mlp_loss_grad",
              "asm_mlp_train_step", "asm_get_warm_data"):
        getattr(L, f).restype = C.c_int
    _lib = L
    return L


def _check(status: int) -> None:
    if status != ASM_OK:
        raise AsmError(status, load().asm_last_error().decode())


def _ptr(a) -> int:
    """Address of a torch tensor (device or host) or a NumPy array."""
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _stream(stream) -> int:
    if stream is None:
        return 0
    return getattr(stream, "cuda_stream", stream)


def default_options(**kw) -> asm_options:
    o = asm_options()
    load().asm_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def default_solve_opts(**kw) -> asm_solve_opts:
    o = asm_solve_opts()
    load().asm_default_solve_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


# ---------------------------------------------------------------------------
# C-named entry points
# ---------------------------------------------------------------------------
def asm_setup(row_ptr, col_idx, val, part, N: int, overlap: int, nev: int, opt: asm_options | None = None,
              stream=None, on_device: bool | None = None) -> int:
    """Build the preconditioner; returns the opaque handle (an int)."""
    if on_device is None:
        on_device = hasattr(row_ptr, "is_cuda") and row_ptr.is_cuda
    n = len(row_ptr) - 1
    nnz = int(row_ptr[-1]) if not on_device else int(val.numel())
    A = asm_csr(n, nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(val), 1 if on_device else 0)
    h = C.c_void_p()
    _check(load().asm_setup(C.byref(A), _ptr(part), N, overlap, nev, C.byref(opt) if opt else None,
                            _stream(stream), C.byref(h)))
    return h.value


def asm_apply(h: int, r, z, stream=None) -> None:
    _check(load().asm_apply(h, _ptr(r), _ptr(z), _stream(stream)))


def asm_spmv(h: int, x, y, stream=None) -> None:
    _check(load().asm_spmv(h, _ptr(x), _ptr(y), _stream(stream)))


def asm_solve(h: int, b, x, opts: asm_solve_opts | None = None, stream=None,
              raise_on_no_convergence: bool = True) -> asm_solve_info:
    info = asm_solve_info()
    st = load().asm_solve(h, _ptr(b), _ptr(x), C.byref(opts) if opts else None, C.byref(info), _stream(stream))
    if st == 6 and not raise_on_no_convergence:
        return info
    _check(st)
    return info


def asm_solve_segments(h: int, b, x, seg_off, opts: asm_solve_opts | None = None, stream=None,
                       raise_on_no_convergence: bool = True):
    """PCG on the independent systems of the row segments [seg_off[k],
    seg_off[k+1]) of a block-diagonal handle, each to its own tolerance
    (asm_solve_segments); returns one asm_solve_info per segment."""
    off = np.ascontiguousarray(np.asarray(seg_off, dtype=np.int32))
    nseg = len(off) - 1
    infos = (asm_solve_info * max(nseg, 1))()
    st = load().asm_solve_segments(h, _ptr(b), _ptr(x), nseg, off.ctypes.data, C.byref(opts) if opts else None,
                                   infos, _stream(stream))
    if not (st == 6 and not raise_on_no_convergence):
        _check(st)
    return [infos[k] for k in range(nseg)]


def asm_get_info(h: int) -> asm_setup_info:
    inf = asm_setup_info()
    _check(load().asm_get_info(h, C.byref(inf)))
    return inf


def asm_get_overlap(h: int):
    """(sub_offsets[N+1], layer_offsets[N, overlap+2], omega[sum n_i]) as NumPy arrays."""
    inf = asm_get_info(h)
    sub = np.zeros(inf.N + 1, dtype=np.int32)
    lay = np.zeros((inf.N, inf.overlap + 2), dtype=np.int32)
    om = np.zeros(inf.sum_ni, dtype=np.int32)
    _check(load().asm_get_overlap(h, sub.ctypes.data, lay.ctypes.data, om.ctypes.data))
    return sub, lay, om


def asm_get_local_values(h: int):
    inf = asm_get_info(h)
    vals = np.zeros((inf.N, max(inf.nev, 1)), dtype=np.float64)
    cnt = np.zeros(inf.N, dtype=np.int32)
    _check(load().asm_get_local_values(h, vals.ctypes.data if inf.nev else None, cnt.ctypes.data))
    return vals[:, :inf.nev], cnt


def asm_get_lift_values(h: int, nev_lift: int):
    """Kept eigenvalues of eq. uppergevp per subdomain (N x nev_lift, descending) and counts."""
    inf = asm_get_info(h)
    vals = np.zeros((inf.N, max(nev_lift, 1)), dtype=np.float64)
    cnt = np.zeros(inf.N, dtype=np.int32)
    _check(load().asm_get_lift_values(h, vals.ctypes.data if nev_lift else None, cnt.ctypes.data))
    return vals[:, :nev_lift], cnt


def asm_get_eigen_stats(h: int):
    """(residuals [N, nev], sweeps [N]) of the subspace iteration."""
    inf = asm_get_info(h)
    res = np.zeros((inf.N, max(inf.nev, 1)), dtype=np.float64)
    sw = np.zeros(inf.N, dtype=np.int32)
    _check(load().asm_get_eigen_stats(h, res.ctypes.data if inf.nev else None, sw.ctypes.data))
    return res[:, :inf.nev], sw


def asm_get_coarse_basis(h: int, p_sizes):
    """List of per-subdomain blocks Z_i (|I_i| x count_i) and the column offsets."""
    inf = asm_get_info(h)
    col = np.zeros(inf.N + 1, dtype=np.int32)
    _check(load().asm_get_coarse_basis(h, None, col.ctypes.data))
    counts = np.diff(col)
    tot = int(np.sum(np.asarray(p_sizes, dtype=np.int64) * counts))
    Z = np.zeros(max(tot, 1), dtype=np.float64)
    _check(load().asm_get_coarse_basis(h, Z.ctypes.data, None))
    out, o = [], 0
    for p, k in zip(p_sizes, counts):
        out.append(Z[o:o + p * k].reshape(p, k))
        o += p * k
    return out, col


def asm_get_coarse_matrix(h: int) -> np.ndarray:
    inf = asm_get_info(h)
    E = np.zeros((inf.n_C, inf.n_C), dtype=np.float64)
    if inf.n_C:
        _check(load().asm_get_coarse_matrix(h, E.ctypes.data))
    return E


def asm_kernel_launches() -> int:
    return int(load().asm_kernel_launches())


def asm_time_apply(h: int, r, z, iters: int = 10, stream=None) -> dict:
    ms = (C.c_double * 6)()
    _check(load().asm_time_apply(h, _ptr(r), _ptr(z), iters, _stream(stream), ms))
    return {"tile_pass": ms[0], "local": ms[1], "coarse": ms[2], "pull": ms[3], "sequential": ms[4],
            "apply": ms[5]}


def asm_csr_spmv(row_ptr, col_idx, val, x, y, stream=None) -> None:
    """y = A x for a CSR matrix held in CUDA tensors (int32 indices, float64
    values and vectors), with the library's SpMV kernel; no handle."""
    import torch
    for name, t, dt in (("row_ptr", row_ptr, torch.int32), ("col_idx", col_idx, torch.int32),
                        ("val", val, torch.float64), ("x", x, torch.float64), ("y", y, torch.float64)):
        if not isinstance(t, torch.Tensor) or t.dtype != dt or not t.is_cuda or not t.is_contiguous():
            raise TypeError(f"{name} must be a contiguous CUDA tensor of {dt}")
    n = int(x.numel())
    if row_ptr.numel() != n + 1 or y.numel() != n or col_idx.numel() != val.numel():
        raise ValueError("sizes: row_ptr n + 1, y n, col_idx and val alike")
    _check(load().asm_csr_spmv(n, int(val.numel()), _ptr(row_ptr), _ptr(col_idx), _ptr(val), _ptr(x), _ptr(y),
                               _stream(stream)))


TILE_AT, TILE_BT, TILE_BETA, TILE_NEG = 1, 2, 4, 8
# mirrors asm_tile_job (include/asm.h)
TILE_JOB_DTYPE = [("a0", "<i8"), ("b0", "<i8"), ("a_step", "<i8"), ("b_step", "<i8"), ("c_in", "<i8"),
                  ("c_out", "<i8"), ("lda", "<i4"), ("ldb", "<i4"), ("ldc_in", "<i4"), ("ldc_out", "<i4"),
                  ("nprod", "<i4"), ("flags", "<i4"), ("sub", "<i4"), ("unused", "<i4")]


def asm_tile_products(jobs, a, b, cin, cout, stream=None) -> None:
    """Batched 64 x 64 tile products on the tensor cores (asm_tile_products):
    jobs is a NumPy array of TILE_JOB_DTYPE records; a, b, cin (or None) and
    cout contiguous float32 CUDA tensors, offsets in elements."""
    import numpy as np
    import torch
    jobs = np.ascontiguousarray(np.asarray(jobs, dtype=TILE_JOB_DTYPE))
    for name, t in (("a", a), ("b", b), ("cin", cin), ("cout", cout)):
        if t is None and name == "cin":
            continue
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
            raise TypeError(f"{name} must be a contiguous CUDA tensor of float32")
    _check(load().asm_tile_products(jobs.ctypes.data, len(jobs), _ptr(a), _ptr(b),
                                    _ptr(cin) if cin is not None else None, _ptr(cout), _stream(stream)))


def asm_time_spmv(h: int, p, q, iters: int = 100, stream=None) -> float:
    """Mean ms of the PCG loop's fused q = A p, p.q launch on the handle's matrix."""
    ms = (C.c_double * 1)()
    _check(load().asm_time_spmv(h, _ptr(p), _ptr(q), iters, _stream(stream), ms))
    return ms[0]


def asm_spmv_dot_noalloc(row_ptr, col_idx, val, x, y, xty, stream=None) -> None:
    """y = A x and xty[0] = x^T y without any device allocation (contiguous CUDA
    tensors: int32 row_ptr (n + 1) and col_idx, float64 val, x, y, xty; y must
    not overlap x)."""
    import torch
    n = int(x.numel())
    for name, t, dt in (("row_ptr", row_ptr, torch.int32), ("col_idx", col_idx, torch.int32), ("val", val, torch.float64),
                        ("x", x, torch.float64), ("y", y, torch.float64), ("xty", xty, torch.float64)):
        if not isinstance(t, torch.Tensor) or t.dtype != dt or not t.is_cuda or not t.is_contiguous():
            raise TypeError(f"{name} must be a contiguous CUDA tensor of {dt}")
    if row_ptr.numel() != n + 1 or y.numel() != n or xty.numel() < 1 or col_idx.numel() != val.numel():
        raise ValueError("sizes: row_ptr n + 1, y n, xty >= 1, col_idx and val alike")
    _check(load().asm_spmv_dot_noalloc(n, _ptr(row_ptr), _ptr(col_idx), _ptr(val), _ptr(x), _ptr(y), _ptr(xty),
                                       _stream(stream)))


def asm_destroy(h: int) -> None:
    if h:
        load().asm_destroy(h)


# ---------------------------------------------------------------------------
# Learned warm start
# ---------------------------------------------------------------------------
WARM_FEATURES = 16


def asm_mlp_create(hidden: int = 256, outputs: int = 16, seed: int = 0) -> int:
    net = C.c_void_p()
    _check(load().asm_mlp_create(hidden, outputs, seed, C.byref(net)))
    return net.value


def asm_mlp_destroy(net: int) -> None:
    if net:
        load().asm_mlp_destroy(net)


def asm_mlp_num_params(net: int) -> int:
    return int(load().asm_mlp_num_params(net))


def asm_mlp_get_params(net: int) -> np.ndarray:
    p = np.zeros(asm_mlp_num_params(net), dtype=np.float32)
    _check(load().asm_mlp_get_params(net, p.ctypes.data))
    return p


def asm_mlp_set_params(net: int, params) -> None:
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.size != asm_mlp_num_params(net):
        raise ValueError("parameter vector has the wrong length")
    _check(load().asm_mlp_set_params(net, p.ctypes.data))


def asm_mlp_forward(net: int, X, Y, stream=None) -> None:
    """Y (rows x outputs) = network(X (rows x 16)); device float32 tensors."""
    _check(load().asm_mlp_forward(net, _ptr(X), int(X.shape[0]), _ptr(Y), _stream(stream)))


def asm_mlp_loss_grad(net: int, X, T, seg, stream=None):
    """(mean loss, gradient as a float32 NumPy vector); X, T float32 and seg
    int64 (nseg+1, seg[0] = 0) device tensors."""
    loss = C.c_double()
    g = np.zeros(asm_mlp_num_params(net), dtype=np.float32)
    _check(load().asm_mlp_loss_grad(net, _ptr(X), int(X.shape[0]), _ptr(T), _ptr(seg), int(seg.shape[0]) - 1,
                                    C.byref(loss), g.ctypes.data, _stream(stream)))
    return loss.value, g


def asm_mlp_train_step(net: int, X, T, seg, lr: float, stream=None, want_loss: bool = True):
    loss = C.c_double()
    _check(load().asm_mlp_train_step(net, _ptr(X), int(X.shape[0]), _ptr(T), _ptr(seg), int(seg.shape[0]) - 1,
                                     lr, C.byref(loss) if want_loss else None, _stream(stream)))
    return loss.value if want_loss else None


def asm_get_warm_data(h: int, stream=None):
    """(row offsets [N+1] NumPy int64, features [rows x 16], targets [rows x nev])
    of a handle set up with record_warm=1; the arrays are device tensors."""
    import torch
    inf = asm_get_info(h)
    off = np.zeros(inf.N + 1, dtype=np.int64)
    _check(load().asm_get_warm_data(h, off.ctypes.data, None, None, _stream(stream)))
    rows = int(off[-1])
    X = torch.empty((rows, WARM_FEATURES), dtype=torch.float32, device="cuda")
    T = torch.empty((rows, inf.nev), dtype=torch.float32, device="cuda")
    _check(load().asm_get_warm_data(h, None, _ptr(X), _ptr(T), _stream(stream)))
    return off, X, T


class WarmStartNet:
    """Owns one warm-start network (C ABI ``asm_mlp_*``)."""

    def __init__(self, hidden: int = 256, outputs: int = 16, seed: int = 0):
        self.hidden, self.outputs = hidden, outputs
        self.ptr = asm_mlp_create(hidden, outputs, seed)

    def params(self) -> np.ndarray:
        return asm_mlp_get_params(self.ptr)

    def set_params(self, p) -> None:
        asm_mlp_set_params(self.ptr, p)

    def forward(self, X):
        import torch
        Y = torch.empty((X.shape[0], self.outputs), dtype=torch.float32, device=X.device)
        asm_mlp_forward(self.ptr, X, Y)
        return Y

    def loss_grad(self, X, T, seg):
        return asm_mlp_loss_grad(self.ptr, X, T, seg)

    def train(self, X, T, offsets, steps: int, lr: float = 1e-3, batch: int = 64, seed: int = 0,
              log_every: int = 0) -> list[float]:
        """Adam on minibatches of `batch` consecutive subdomains (the batch
        order reshuffled every epoch).  X, T: device tensors of all rows;
        offsets: NumPy int64 row offsets of the subdomains.  Returns the loss of
        every `log_every`-th step (none if 0)."""
        import torch
        nseg = len(offsets) - 1
        starts = list(range(0, nseg, batch))
        batches = []
        for s0 in starts:
            s1 = min(nseg, s0 + batch)
            r0, r1 = int(offsets[s0]), int(offsets[s1])
            seg = torch.as_tensor(offsets[s0:s1 + 1] - r0, dtype=torch.int64, device=X.device)
            batches.append((X[r0:r1].contiguous(), T[r0:r1].contiguous(), seg))
        rng = np.random.default_rng(seed)
        order, losses = [], []
        for step in range(steps):
            if not order:
                order = list(rng.permutation(len(batches)))
            Xb, Tb, sb = batches[order.pop()]
            want = log_every > 0 and step % log_every == 0
            l = asm_mlp_train_step(self.ptr, Xb, Tb, sb, lr, want_loss=want)
            if want:
                losses.append(l)
        return losses

    def close(self):
        if getattr(self, "ptr", None):
            asm_mlp_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stage_names() -> list[str]:
    L = load()
    return [L.asm_stage_name(i).decode() for i in range(12)]


# ---------------------------------------------------------------------------
# Convenience wrapper
# ---------------------------------------------------------------------------
class TwoLevelSchwarz:
    """Owns one handle.  ``A`` is anything with ``indptr``, ``indices`` and
    ``data`` (scipy CSR / asm_inputs.Problem style) or a tuple of arrays."""

    def __init__(self, indptr, indices, data, part, N: int, overlap: int, nev: int, *, spd: bool = True,
                 precision: str = "fp64", device: bool = True, stream=None, **opts):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        prec = {"fp64": PREC_FP64, "fp32": PREC_FP32, "fp32h": PREC_FP32_H16, "fp32b": PREC_FP32_B16}[precision]
        o = default_options(spd=1 if spd else 0, local_precision=prec, **opts)
        self.device = device
        self.n = len(indptr) - 1
        if device:
            dev = torch.device("cuda")
            self._rp = torch.as_tensor(np.asarray(indptr, dtype=np.int32), device=dev)
            self._ci = torch.as_tensor(np.asarray(indices, dtype=np.int32), device=dev)
            self._va = torch.as_tensor(np.asarray(data, dtype=np.float64), device=dev)
            self._pa = torch.as_tensor(np.asarray(part, dtype=np.int32), device=dev)
            self.h = asm_setup(self._rp, self._ci, self._va, self._pa, N, overlap, nev, o, stream, True)
        else:
            self._rp = np.ascontiguousarray(indptr, dtype=np.int32)
            self._ci = np.ascontiguousarray(indices, dtype=np.int32)
            self._va = np.ascontiguousarray(data, dtype=np.float64)
            self._pa = np.ascontiguousarray(part, dtype=np.int32)
            self.h = asm_setup(self._rp, self._ci, self._va, self._pa, N, overlap, nev, o, stream, False)
        self.stream = stream

    @property
    def info(self) -> asm_setup_info:
        return asm_get_info(self.h)

    def apply(self, r, z=None):
        import torch
        if z is None:
            z = torch.empty_like(r)
        asm_apply(self.h, r, z, self.stream)
        return z

    def solve(self, b, x=None, **kw):
        if x is None:
            if self.device:
                import torch
                x = torch.zeros_like(b)
            else:
                x = np.zeros_like(b)
        info = asm_solve(self.h, b, x, default_solve_opts(**kw), self.stream,
                         raise_on_no_convergence=kw.get("max_it", None) is None)
        return x, info

    def close(self):
        if getattr(self, "h", None):
            asm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
