// C ABI of the library: argument checks, stage orchestration, error mapping.
#include <algorithm>
#include <cstring>
#include <new>

#include "handle.cuh"
#include "tcgemm.cuh"

using namespace asmgpu;

struct asm_handle {
  Handle h;
};

namespace {
thread_local std::string g_last_error;

asm_status set_error(asm_status s, const std::string& m) {
  g_last_error = m;
  return s;
}

const char* kStageNames[12] = {"overlap", "gather", "sweep", "pack", "eigen", "coarse_assembly",
                               "coarse_factor", "setup_total", "", "", "", ""};

void init_pool() {
  static bool done = false;
  if (done) return;
  done = true;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = 64ull << 30;  // keep up to 64 GiB cached between setups
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
}

template <typename F>
asm_status guarded(F&& f) {
  try {
    f();
    return ASM_OK;
  } catch (const AsmError& e) {
    return set_error(e.status, e.msg);
  } catch (const std::bad_alloc&) {
    return set_error(ASM_ERR_OOM, "host allocation failed");
  } catch (...) {
    return set_error(ASM_ERR_CUDA, "unexpected internal error");
  }
}

void free_handle_memory(Handle& h) {
  cudaDeviceSynchronize();
  h.mem.stream = nullptr;
  h.mem.release();
  if (h.kr.hpin) { cudaFreeHost(h.kr.hpin); h.kr.hpin = nullptr; }
  if (h.events)
    for (auto& e : h.ev) cudaEventDestroy(e);
  h.events = false;
  if (h.side) { cudaStreamDestroy(h.side); h.side = nullptr; }
  if (h.ev_fork) { cudaEventDestroy(h.ev_fork); h.ev_fork = nullptr; }
  if (h.ev_join) { cudaEventDestroy(h.ev_join); h.ev_join = nullptr; }
  cudaGetLastError();
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
    cudaGetLastError();
    return 0.f;
  }
  return ms;
}
}  // namespace

namespace asmgpu {
asm_status set_last_error(asm_status s, const std::string& msg) { return set_error(s, msg); }

void check_device_error(Handle& h, cudaStream_t s, const char* stage) {
  int32_t e = 0;
  CK(cudaMemcpyAsync(&e, h.dn.err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (!e) return;
  CK(cudaMemsetAsync(h.dn.err, 0, sizeof(int32_t), s));
  std::string st(stage);
  if (e & DERR_NONFINITE) fail(ASM_ERR_NONFINITE, st + ": non-finite value");
  if (e & DERR_NOT_SPD) fail(ASM_ERR_NOT_SPD, st + ": a local pivot is not positive (A is not SPD)");
  if (e & DERR_ZERO_PIVOT) fail(ASM_ERR_ZERO_PIVOT, st + ": zero local pivot");
  if (e & DERR_COARSE) fail(ASM_ERR_COARSE_SINGULAR, st + ": coarse matrix E is not SPD / singular");
  if (e & DERR_CAPACITY) fail(ASM_ERR_UNSUPPORTED, st + ": capacity exceeded");
  if (e & DERR_TIMEOUT) fail(ASM_ERR_TIMEOUT, st + ": a bounded device wait gave up");
}
}  // namespace asmgpu

extern "C" {

void asm_default_options(asm_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->spd = 1;
  o->local_precision = ASM_PREC_FP64;
  o->oversample = 8;
  o->max_sweeps = 0;  // 0: 40
  o->eig_tol = 0;     // 0: 1e-8 (FP64) / 4e-3 (FP32)
  o->nu = 0;
  o->nev_lift = 0;
  o->coarse = 1;
  o->seed = 0;
  o->warm_start = 0;
  o->filter_degree = 0;  // 0: 4
}

void asm_default_solve_opts(asm_solve_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->method = 0;
  o->restart = 0;  // automatic
  o->rtol = 1e-8;
  o->max_it = 1000;
  o->use_x0 = 0;
  o->check_every = 8;
}

const char* asm_last_error(void) { return g_last_error.c_str(); }

const char* asm_stage_name(int32_t stage) {
  if (stage < 0 || stage >= 12) return "";
  return kStageNames[stage];
}

asm_status asm_setup(const asm_csr* A, const int32_t* part, int32_t N, int32_t overlap, int32_t nev,
                     const asm_options* opt, void* stream, asm_handle** out) {
  if (out) *out = nullptr;
  if (!A || !part || !out) return set_error(ASM_ERR_INVALID_ARG, "null argument");
  if (A->n <= 0 || A->nnz < 0 || !A->row_ptr || !A->col_idx || (A->nnz > 0 && !A->val))
    return set_error(ASM_ERR_INVALID_ARG, "CSR arrays missing or n <= 0");
  if (N < 1 || N > A->n) return set_error(ASM_ERR_INVALID_ARG, "N must be in 1..n");
  if (N >= 131072) return set_error(ASM_ERR_UNSUPPORTED, "more than 131071 subdomains");
  if (overlap < 1 || overlap > 64) return set_error(ASM_ERR_INVALID_ARG, "overlap must be in 1..64");
  if (nev < 0 || nev > 120) return set_error(ASM_ERR_INVALID_ARG, "nev must be in 0..120");
  asm_options o;
  if (opt) o = *opt; else asm_default_options(&o);
  if (o.local_precision != ASM_PREC_FP64 && o.local_precision != ASM_PREC_FP32 &&
      o.local_precision != ASM_PREC_FP32_H16 && o.local_precision != ASM_PREC_FP32_B16)
    return set_error(ASM_ERR_INVALID_ARG,
                     "local_precision must be ASM_PREC_FP64, ASM_PREC_FP32, ASM_PREC_FP32_H16 or ASM_PREC_FP32_B16");
  if (o.oversample < 0 || o.oversample > 64) return set_error(ASM_ERR_INVALID_ARG, "oversample must be in 0..64");
  if (o.warm_start && (!o.warm_net || !o.spd))
    return set_error(ASM_ERR_INVALID_ARG, "warm_start needs warm_net and the SPD method");
  if (o.one_level != 0 && o.one_level != 1) return set_error(ASM_ERR_INVALID_ARG, "one_level must be 0 or 1");
  if (!(o.tau >= 0) || !std::isfinite(o.tau)) return set_error(ASM_ERR_INVALID_ARG, "tau must be finite and >= 0");
  if (o.coarse_mode != 0 && o.coarse_mode != 1) return set_error(ASM_ERR_INVALID_ARG, "coarse_mode must be 0 or 1");
  if (!(o.nu == 0 || o.nu >= 1) || !std::isfinite(o.nu))
    return set_error(ASM_ERR_INVALID_ARG, "nu must be 0 (off) or >= 1 (eigenvalues of eq. uppergevp are >= 1)");
  if (o.nu > 0 && !o.spd) return set_error(ASM_ERR_INVALID_ARG, "nu (eq. uppergevp) needs the SPD method");
  if (o.nev_lift < 0 || o.nev_lift > 120) return set_error(ASM_ERR_INVALID_ARG, "nev_lift must be in 0..120");
  if (o.nu > 0 && nev + (o.nev_lift > 0 ? o.nev_lift : nev) > 128)
    return set_error(ASM_ERR_UNSUPPORTED, "nev + nev_lift exceeds 128");
  asm_handle* H = new (std::nothrow) asm_handle();
  if (!H) return set_error(ASM_ERR_OOM, "host allocation failed");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  asm_status st = guarded([&] {
    init_pool();
    Handle& h = H->h;
    h.n = A->n; h.nnz = A->nnz; h.N = N; h.delta = overlap; h.nev = nev; h.opt = o;
    h.host_io = A->on_device == 0;
    h.fp32 = o.local_precision != ASM_PREC_FP64;
    h.s16 = o.local_precision == ASM_PREC_FP32_H16 && o.spd;
    h.b16eig = o.local_precision == ASM_PREC_FP32_B16 && o.spd;
    h.lift = o.nu > 0 && o.spd && o.coarse;
    h.nev_lift = h.lift ? (o.nev_lift > 0 ? o.nev_lift : nev) : 0;
    if (h.lift && h.nev_lift == 0) h.lift = false;
    {
      int dev = 0, sms = 0;
      CK(cudaGetDevice(&dev));
      CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      if (sms > 0) h.num_sms = sms;
    }
    h.mem.stream = s;
    for (auto& e : h.ev) CK(cudaEventCreate(&e));
    h.events = true;
    {
      // the coarse part of the apply is a chain of short FP64 kernels: at the
      // highest priority they take SM slots as soon as the tile passes free them
      int least = 0, greatest = 0;
      CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
      CK(cudaStreamCreateWithPriority(&h.side, cudaStreamNonBlocking, greatest));
    }
    CK(cudaEventCreateWithFlags(&h.ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h.ev_join, cudaEventDisableTiming));
    CK(cudaEventRecord(h.ev[0], s));
    h.row_ptr = h.mem.alloc<int32_t>(h.n + 1);
    h.col_idx = h.mem.alloc<int32_t>(h.nnz);
    h.val = h.mem.alloc<double>(h.nnz);
    h.part = h.mem.alloc<int32_t>(h.n);
    if (h.host_io) {
      // host arrays: validate row_ptr before trusting nnz
      if (A->row_ptr[0] != 0 || A->row_ptr[A->n] != A->nnz)
        fail(ASM_ERR_INVALID_ARG, "row_ptr[0] must be 0 and row_ptr[n] must equal nnz");
    }
    CK(cudaMemcpyAsync(h.row_ptr, A->row_ptr, sizeof(int32_t) * (h.n + 1), cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(h.col_idx, A->col_idx, sizeof(int32_t) * h.nnz, cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(h.val, A->val, sizeof(double) * h.nnz, cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(h.part, part, sizeof(int32_t) * h.n, cudaMemcpyDefault, s));
    h.dn.err = h.mem.alloc<int32_t>(1);
    CK(cudaMemsetAsync(h.dn.err, 0, sizeof(int32_t), s));
    build_overlap(h, s);
    CK(cudaEventRecord(h.ev[1], s));
    build_local(h, s);
    build_eigen(h, s);
    CK(cudaEventRecord(h.ev[6], s));
    CK(cudaEventRecord(h.ev[7], s));
    build_coarse(h, s);
    CK(cudaEventRecord(h.ev[8], s));
    if (h.opt.coarse_mode == 1 && h.co.n_C > 0) {
      h.defl_q = h.mem.alloc<double>(h.n);
      h.defl_w = h.mem.alloc<double>(h.n);
    }
    tune_apply(h, s);
    CK(cudaStreamSynchronize(s));
    // info
    asm_setup_info& inf = h.info;
    std::memset(&inf, 0, sizeof(inf));
    inf.n = h.n; inf.N = h.N; inf.overlap = h.delta; inf.nev = h.nev;
    inf.n_C = h.co.n_C;
    inf.nnz_C = h.co.nnz_C;
    inf.gc = 1.0 + (double)h.co.n_C / h.n;
    inf.oc = 1.0 + (double)h.co.nnz_C / std::max(1, h.nnz);
    inf.sum_ni = h.ov.sum_n;
    inf.max_ni = h.ov.max_n;
    int smax = 0;
    for (int v : h.co.h_sweeps) smax = std::max(smax, v);
    inf.sweeps_max = smax;
    if (h.co.n_C > 0 && h.co.resid) {
      std::vector<double> res((size_t)h.N * h.nev);
      CK(cudaMemcpy(res.data(), h.co.resid, sizeof(double) * res.size(), cudaMemcpyDeviceToHost));
      double m = 0;
      for (double v : res) m = std::max(m, v);
      inf.eig_resid_max = m;
    }
    inf.stage_ms[0] = elapsed(h.ev[0], h.ev[1]);
    inf.stage_ms[1] = elapsed(h.ev[2], h.ev[3]);
    inf.stage_ms[2] = elapsed(h.ev[3], h.ev[4]);
    inf.stage_ms[3] = elapsed(h.ev[4], h.ev[5]);
    inf.stage_ms[4] = elapsed(h.ev[5], h.ev[6]);
    inf.stage_ms[5] = h.co.n_C > 0 ? elapsed(h.ev[6], h.ev[7]) : 0.f;
    inf.stage_ms[6] = h.co.n_C > 0 ? elapsed(h.ev[7], h.ev[8]) : 0.f;
    inf.stage_ms[7] = elapsed(h.ev[0], h.ev[8]);
    inf.coarse_levels = h.nd.nlevels;
    inf.coarse_fronts = h.nd.nfronts;
    inf.coarse_front_entries = h.nd.n_mat;
    inf.coarse_max_front = h.nd.max_m;
    inf.tile_ctas = h.tile_ctas;
    for (int8_t v : h.dn.h_sym) inf.local_sym += v ? 1 : 0;
    for (int8_t v : h.dn.h_s16) inf.local_fp16 += v ? 1 : 0;
  });
  if (st != ASM_OK) {
    free_handle_memory(H->h);
    delete H;
    return st;
  }
  *out = H;
  return ASM_OK;
}

asm_status asm_apply(asm_handle* H, const double* r, double* z, void* stream) {
  if (!H || !r || !z) return set_error(ASM_ERR_INVALID_ARG, "null argument");
  if (r == z) return set_error(ASM_ERR_INVALID_ARG, "r and z must not alias");
  return guarded([&] {
    apply_preconditioner(H->h, r, z, static_cast<cudaStream_t>(stream));
    CK_LAUNCH("apply");
    check_device_error(H->h, static_cast<cudaStream_t>(stream), "apply");
  });
}

asm_status asm_spmv(asm_handle* H, const double* x, double* y, void* stream) {
  if (!H || !x || !y) return set_error(ASM_ERR_INVALID_ARG, "null argument");
  return guarded([&] { spmv(H->h, x, y, static_cast<cudaStream_t>(stream)); });
}

asm_status asm_solve(asm_handle* H, const double* b, double* x, const asm_solve_opts* o, asm_solve_info* info,
                     void* stream) {
  asm_solve_info dummy;
  if (!info) info = &dummy;
  std::memset(info, 0, sizeof(*info));
  if (!H || !b || !x) return set_error(ASM_ERR_INVALID_ARG, "null argument");
  asm_solve_opts so;
  if (o) so = *o; else asm_default_solve_opts(&so);
  if (!(so.rtol > 0) || so.max_it < 1) return set_error(ASM_ERR_INVALID_ARG, "rtol must be > 0 and max_it >= 1");
  Handle& h = H->h;
  // automatic restart length: GMRES without restart (up to 512 vectors) for
  // the restricted or deflated apply, as the Section 6 experiments; 30 otherwise
  const bool auto_restart = so.restart <= 0;
  if (auto_restart)
    so.restart = (h.opt.one_level == 1 || (h.opt.coarse_mode == 1 && h.co.n_C > 0)) ? 512 : 30;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bool conv = false;
  asm_status st = guarded([&] {
    const double* db = b;
    double* dx = x;
    if (h.host_io) {
      if (!h.kr.bx) h.kr.bx = h.mem.alloc<double>(2LL * h.n);
      db = h.kr.bx;
      dx = h.kr.bx + h.n;
      CK(cudaMemcpyAsync(h.kr.bx, b, sizeof(double) * h.n, cudaMemcpyHostToDevice, s));
      if (so.use_x0) CK(cudaMemcpyAsync(dx, x, sizeof(double) * h.n, cudaMemcpyHostToDevice, s));
    }
    // PCG needs a symmetric preconditioner: the additive ASM with the additive
    // coarse correction; the restricted or deflated forms go to FGMRES
    const bool symmetric = h.opt.spd && h.opt.one_level == 0 && (h.opt.coarse_mode == 0 || h.co.n_C == 0);
    int method = so.method ? so.method : (symmetric ? 1 : 2);
    if (method == 1) solve_pcg(h, db, dx, so, *info, s);
    else solve_fgmres(h, db, dx, so, *info, s, auto_restart);
    check_device_error(h, s, "solve");
    if (h.host_io) {
      CK(cudaMemcpyAsync(x, dx, sizeof(double) * h.n, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    }
    conv = info->converged != 0;
  });
  if (st != ASM_OK) return st;
  if (!conv) return set_error(ASM_ERR_NO_CONVERGENCE, "Krylov iteration did not reach rtol");
  return ASM_OK;
}

uint64_t asm_kernel_launches(void) { return (uint64_t)total_kernel_launches(); }

asm_status asm_time_apply(asm_handle* H, const double* r, double* z, int32_t iters, void* stream, double* ms) {
  if (!H || !r || !z || !ms || iters < 1) return set_error(ASM_ERR_INVALID_ARG, "null argument or iters < 1");
  return guarded([&] { time_apply(H->h, r, z, iters, static_cast<cudaStream_t>(stream), ms); });
}

asm_status asm_csr_spmv(int32_t n, int32_t nnz, const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                        const double* x, double* y, void* stream) {
  if (n < 0 || nnz < 0 || (n > 0 && (!row_ptr || !col_idx || !val || !x || !y)))
    return set_error(ASM_ERR_INVALID_ARG, "asm_csr_spmv: null pointer or negative size");
  if (n > 0 && x == y) return set_error(ASM_ERR_INVALID_ARG, "asm_csr_spmv: x and y must not alias");
  return guarded([&] { csr_spmv(n, nnz, row_ptr, col_idx, val, x, y, static_cast<cudaStream_t>(stream)); });
}

asm_status asm_time_spmv(asm_handle* H, const double* p, double* q, int32_t iters, void* stream, double* ms) {
  if (!H || !p || !q || !ms || iters < 1) return set_error(ASM_ERR_INVALID_ARG, "null argument or iters < 1");
  if (p == q) return set_error(ASM_ERR_INVALID_ARG, "p and q must not alias");
  return guarded([&] { time_pcg_spmv(H->h, p, q, iters, static_cast<cudaStream_t>(stream), ms); });
}

asm_status asm_solve_segments(asm_handle* H, const double* b, double* x, int32_t nseg, const int32_t* seg_off,
                              const asm_solve_opts* o, asm_solve_info* info, void* stream) {
  if (!H || !b || !x || !seg_off || !info) return set_error(ASM_ERR_INVALID_ARG, "null argument");
  if (nseg < 1 || nseg > 65535) return set_error(ASM_ERR_INVALID_ARG, "nseg must be in 1 .. 65535");
  Handle& h = H->h;
  if (seg_off[0] != 0 || seg_off[nseg] != h.n)
    return set_error(ASM_ERR_INVALID_ARG, "seg_off must start at 0 and end at n");
  for (int k = 0; k < nseg; ++k)
    if (seg_off[k + 1] < seg_off[k]) return set_error(ASM_ERR_INVALID_ARG, "seg_off must be non-decreasing");
  asm_solve_opts so;
  if (o) so = *o; else asm_default_solve_opts(&so);
  if (!(so.rtol > 0) || so.max_it < 1) return set_error(ASM_ERR_INVALID_ARG, "rtol must be > 0 and max_it >= 1");
  const bool symmetric = h.opt.spd && h.opt.one_level == 0 && (h.opt.coarse_mode == 0 || h.co.n_C == 0);
  if (!symmetric || (so.method != 0 && so.method != 1))
    return set_error(ASM_ERR_UNSUPPORTED, "asm_solve_segments: PCG with the additive SPD preconditioner only");
  std::memset(info, 0, sizeof(asm_solve_info) * nseg);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bool conv = true;
  asm_status st = guarded([&] {
    const double* db = b;
    double* dx = x;
    if (h.host_io) {
      if (!h.kr.bx) h.kr.bx = h.mem.alloc<double>(2LL * h.n);
      db = h.kr.bx;
      dx = h.kr.bx + h.n;
      CK(cudaMemcpyAsync(h.kr.bx, b, sizeof(double) * h.n, cudaMemcpyHostToDevice, s));
    }
    solve_pcg_segments(h, db, dx, nseg, seg_off, so, info, s);
    check_device_error(h, s, "segmented solve");
    if (h.host_io) {
      CK(cudaMemcpyAsync(x, dx, sizeof(double) * h.n, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    }
    for (int k = 0; k < nseg; ++k) conv = conv && info[k].converged != 0;
  });
  if (st != ASM_OK) return st;
  return conv ? ASM_OK : set_error(ASM_ERR_NO_CONVERGENCE, "asm_solve_segments: max_it reached on a segment");
}

asm_status asm_tile_products(const asm_tile_job* jobs, int64_t njobs, const float* a, const float* b,
                             const float* cin, float* cout, void* stream) {
  static_assert(sizeof(asm_tile_job) == sizeof(TcJob), "asm_tile_job must mirror TcJob");
  if (njobs < 0 || (njobs > 0 && (!jobs || !a || !b || !cout)))
    return set_error(ASM_ERR_INVALID_ARG, "asm_tile_products: null pointer or negative count");
  for (int64_t k = 0; k < njobs; ++k) {
    const asm_tile_job& j = jobs[k];
    const bool beta = (j.flags & ASM_TILE_BETA) != 0;
    if (j.nprod < 1 || (j.flags & ~15) || (beta && !cin))
      return set_error(ASM_ERR_INVALID_ARG, "asm_tile_products: nprod < 1, unknown flag or missing C_in");
    const int64_t al[] = {j.a0, j.b0, j.a_step, j.b_step, j.c_in, j.c_out, j.lda, j.ldb, j.ldc_in, j.ldc_out};
    for (int64_t v : al)
      if (v % 4 != 0) return set_error(ASM_ERR_INVALID_ARG, "asm_tile_products: offsets and strides must be multiples of 4");
    if (j.lda < 64 || j.ldb < 64 || j.ldc_out < 64 || (beta && j.ldc_in < 64))
      return set_error(ASM_ERR_INVALID_ARG, "asm_tile_products: a row stride below 64");
  }
  return guarded([&] {
    if (njobs == 0) return;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TcJob* d = nullptr;
    int32_t* err = nullptr;
    CK(cudaMallocAsync(&d, sizeof(TcJob) * njobs, s));
    CK(cudaMallocAsync(&err, sizeof(int32_t), s));
    CK(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
    CK(cudaMemcpyAsync(d, jobs, sizeof(TcJob) * njobs, cudaMemcpyHostToDevice, s));
    int dev = 0, sms = 152;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    tc_tiles(d, njobs, a, b, cin, cout, nullptr, err, sms, s);
    int32_t e = 0;
    CK(cudaMemcpyAsync(&e, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaFreeAsync(d, s));
    CK(cudaFreeAsync(err, s));
    CK(cudaStreamSynchronize(s));
    if (e & DERR_TIMEOUT) fail(ASM_ERR_TIMEOUT, "asm_tile_products: a bounded device wait gave up");
  });
}

asm_status asm_get_info(const asm_handle* H, asm_setup_info* info) {
  if (!H || !info) return set_error(ASM_ERR_INVALID_ARG, "null argument");
  *info = H->h.info;
  return ASM_OK;
}

asm_status asm_get_overlap(const asm_handle* H, int32_t* sub_offsets, int32_t* layer_offsets, int32_t* omega) {
  if (!H) return set_error(ASM_ERR_INVALID_ARG, "null argument");
  const Handle& h = H->h;
  return guarded([&] {
    if (sub_offsets) std::memcpy(sub_offsets, h.ov.h_sub_off.data(), sizeof(int32_t) * (h.N + 1));
    if (layer_offsets)
      std::memcpy(layer_offsets, h.ov.h_lay_off.data(), sizeof(int32_t) * h.ov.h_lay_off.size());
    if (omega) CK(cudaMemcpy(omega, h.ov.omega, sizeof(int32_t) * h.ov.sum_n, cudaMemcpyDeviceToHost));
  });
}

asm_status asm_get_local_values(const asm_handle* H, double* values, int32_t* counts) {
  if (!H) return set_error(ASM_ERR_INVALID_ARG, "null argument");
  const Handle& h = H->h;
  return guarded([&] {
    if (values) {
      if (h.co.values) CK(cudaMemcpy(values, h.co.values, sizeof(double) * h.N * h.nev, cudaMemcpyDeviceToHost));
      else std::memset(values, 0, sizeof(double) * h.N * h.nev);
    }
    if (counts) {
      for (int i = 0; i < h.N; ++i) counts[i] = i < (int)h.co.h_count_g.size() ? h.co.h_count_g[i] : 0;
    }
  });
}

asm_status asm_get_lift_values(const asm_handle* H, double* values, int32_t* counts) {
  if (!H) return set_error(ASM_ERR_INVALID_ARG, "null argument");
  const Handle& h = H->h;
  return guarded([&] {
    const int nl = std::max(h.nev_lift, 1);
    if (values) {
      if (h.co.lift_values)
        CK(cudaMemcpy(values, h.co.lift_values, sizeof(double) * h.N * h.nev_lift, cudaMemcpyDeviceToHost));
      else std::memset(values, 0, sizeof(double) * h.N * nl);
    }
    if (counts)
      for (int i = 0; i < h.N; ++i) counts[i] = i < (int)h.co.h_lift_count.size() ? h.co.h_lift_count[i] : 0;
  });
}

asm_status asm_get_eigen_stats(const asm_handle* H, double* resid, int32_t* sweeps) {
  if (!H) return set_error(ASM_ERR_INVALID_ARG, "null argument");
  const Handle& h = H->h;
  return guarded([&] {
    if (resid) {
      if (h.co.resid) CK(cudaMemcpy(resid, h.co.resid, sizeof(double) * h.N * h.nev, cudaMemcpyDeviceToHost));
      else std::memset(resid, 0, sizeof(double) * h.N * h.nev);
    }
    if (sweeps)
      for (int i = 0; i < h.N; ++i) sweeps[i] = i < (int)h.co.h_sweeps.size() ? h.co.h_sweeps[i] : 0;
  });
}

asm_status asm_get_coarse_basis(const asm_handle* H, double* Z, int32_t* col_offsets) {
  if (!H) return set_error(ASM_ERR_INVALID_ARG, "null argument");
  const Handle& h = H->h;
  return guarded([&] {
    if (col_offsets) {
      for (int i = 0; i <= h.N; ++i) col_offsets[i] = i < (int)h.co.h_col_off.size() ? h.co.h_col_off[i] : 0;
    }
    if (Z && h.co.n_C > 0) {
      // compact p_i x nev blocks to p_i x count_i
      int64_t tot = h.co.h_z_off.back();
      std::vector<double> buf(tot);
      CK(cudaMemcpy(buf.data(), h.co.Z, sizeof(double) * tot, cudaMemcpyDeviceToHost));
      int64_t o = 0;
      for (int i = 0; i < h.N; ++i) {
        int k = h.co.h_count[i], p = h.h_p[i];
        for (int r = 0; r < p; ++r)
          for (int j = 0; j < k; ++j) Z[o++] = buf[h.co.h_z_off[i] + (int64_t)r * h.co.zld + j];
      }
    }
  });
}

asm_status asm_get_coarse_matrix(const asm_handle* H, double* E) {
  if (!H || !E) return set_error(ASM_ERR_INVALID_ARG, "null argument");
  const Handle& h = H->h;
  return guarded([&] {
    const int nC = h.co.n_C;
    if (nC == 0) return;
    const int ld = (int)round_up(nC, 64);
    CK(cudaMemcpy2D(E, sizeof(double) * nC, h.co.E_copy, sizeof(double) * ld, sizeof(double) * nC, nC,
                    cudaMemcpyDeviceToHost));
  });
}

asm_status asm_get_warm_data(const asm_handle* H, int64_t* row_offsets, float* X, float* T, void* stream) {
  if (!H) return set_error(ASM_ERR_INVALID_ARG, "null argument");
  const Handle& h = H->h;
  if (!h.wfeat || (T && !h.wtgt))
    return set_error(ASM_ERR_INVALID_ARG, "nothing recorded: set up with record_warm = 1 (SPD)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return guarded([&] {
    if (row_offsets) std::memcpy(row_offsets, h.h_wseg.data(), sizeof(int64_t) * (h.N + 1));
    if (X) CK(cudaMemcpyAsync(X, h.wfeat, sizeof(float) * h.warm_rows * WARM_FEATURES, cudaMemcpyDeviceToDevice, s));
    if (T) CK(cudaMemcpyAsync(T, h.wtgt, sizeof(float) * h.warm_rows * h.nev, cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
  });
}

void asm_destroy(asm_handle* H) {
  if (!H) return;
  free_handle_memory(H->h);
  delete H;
}

}  // extern "C"
