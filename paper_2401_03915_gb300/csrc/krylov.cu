// FP64 Krylov loop: CSR SpMV, deterministic dot products, PCG and
// right-preconditioned flexible GMRES.  Every loop kernel first reads the
// device `done` flag and returns if it is set, so one iteration can be
// captured once as a CUDA graph and replayed in chunks: replays after
// convergence cost only their launches and change nothing.
//
// The paper stops GMRES at a relative tolerance of 1e-8 on the
// unpreconditioned residual (Section 6); x0 = 0 unless the caller gives one.
#include <algorithm>
#include <cmath>

#include "handle.cuh"

namespace asmgpu {
namespace {

constexpr int NT = 256;
constexpr int NBLK = 608;  // fixed reduction grid: 4 blocks per SM on 152 SMs
constexpr int RBLK = 152 * 16;  // most blocks of a fused-reduction launch

enum Scal { S_RZ = 0, S_PQ, S_ALPHA, S_BETA, S_RR, S_BNORM, S_RTOL, S_RELRES, S_TMP, S_NSCAL = 16 };
enum Flag { F_DONE = 0, F_IT, F_MAXIT, F_NFLAG = 4 };

// vector-per-row CSR SpMV with VW lanes per row.
// y = A x, or y = b - A x when b is given
template <int VW>
__global__ void __launch_bounds__(NT) k_spmv(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                             const double* __restrict__ val, const double* __restrict__ x,
                                             double* __restrict__ y, const double* __restrict__ b,
                                             const int32_t* __restrict__ done) {
  COUNT_LAUNCH();
  if (done != nullptr && *done) return;
  const int lane = threadIdx.x % VW;
  const int rows_per_block = NT / VW;
  for (int base = blockIdx.x * rows_per_block; base < n; base += gridDim.x * rows_per_block) {
    int r = base + threadIdx.x / VW;
    double acc = 0;
    if (r < n) {
      int b = rp[r], e = rp[r + 1];
      for (int k = b + lane; k < e; k += VW) acc += val[k] * x[ci[k]];
    }
#pragma unroll
    for (int o = VW / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (r < n && lane == 0) y[r] = b != nullptr ? b[r] - acc : acc;
  }
}

// CSR SpMV for short rows (at most about 12 stored entries per row on
// average: stencil and FD matrices), one thread per row.  Each thread issues
// the loads of its row's first RL column indices and values at once, then the
// gathers of x, then adds the products in order (longer rows finish in a
// loop).  Consecutive threads read consecutive row segments, which L1 turns
// into full-sector DRAM reads; with all loads of a row in flight this measured
// 5.9 TB/s on a 160^3 7-point Laplacian, against 3.1 TB/s for row blocks
// staged through shared memory and 1.6-2.7 TB/s for 4 or 8 lanes per row.
// y = A x, or y = b - A x; DOT: the launch also forms x.y (fixed order: per
// thread, block tree, then the partials in block order by the last block)
// and runs fin on it.
constexpr int RL = 8;  // entries per row loaded up front

template <bool DOT, typename F>
__device__ __forceinline__ void spmv_rows_body(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                               const double* __restrict__ val, const double* __restrict__ x,
                                               double* __restrict__ y, const double* __restrict__ b, GridSum gs,
                                               F&& fin) {
  double dsum = 0;
  for (int r = blockIdx.x * NT + threadIdx.x; r < n; r += gridDim.x * NT) {
    const int k0 = rp[r], k1 = rp[r + 1];
    int cc[RL];
    double vv[RL];
#pragma unroll
    for (int j = 0; j < RL; ++j) {
      cc[j] = k0 + j < k1 ? __ldg(ci + k0 + j) : 0;
      vv[j] = k0 + j < k1 ? __ldg(val + k0 + j) : 0.0;
    }
    double acc = 0;
#pragma unroll
    for (int j = 0; j < RL; ++j)
      if (k0 + j < k1) acc += vv[j] * __ldg(x + cc[j]);
    for (int k = k0 + RL; k < k1; ++k) acc += val[k] * x[ci[k]];
    const double yv = b != nullptr ? b[r] - acc : acc;
    y[r] = yv;
    if (DOT) dsum += yv * x[r];
  }
  if (DOT) grid_sum_last(dsum, gs, fin);
}

__global__ void __launch_bounds__(NT) k_spmv_rows(int n, const int32_t* __restrict__ rp,
                                                    const int32_t* __restrict__ ci, const double* __restrict__ val,
                                                    const double* __restrict__ x, double* __restrict__ y,
                                                    const double* __restrict__ b, const int32_t* __restrict__ done) {
  COUNT_LAUNCH();
  if (done != nullptr && *done) return;
  spmv_rows_body<false>(n, rp, ci, val, x, y, b, GridSum{}, [](double) {});
}

// partial sums of a.b (fixed grid-stride decomposition)
__global__ void __launch_bounds__(NT) k_dot(int n, const double* __restrict__ a, const double* __restrict__ b,
                                            double* __restrict__ part, const int32_t* __restrict__ done) {
  COUNT_LAUNCH();
  if (done != nullptr && done[F_DONE]) return;
  __shared__ double red[NT / 32];
  double s = 0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) s += a[i] * b[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__device__ double sum_partials(const double* part, int nb) {
  __shared__ double red[NT / 32];
  double s = 0;
  for (int k = threadIdx.x; k < nb; k += NT) s += part[k];
  return block_sum(s, red);
}

// ---------------------------------------------------------------------------
// Fused PCG iteration: three launches plus the apply, no reduction kernels.
//   (1) q = A p, alpha = rz / p.q
//   (2) x += alpha p, r -= alpha q, ||r|| and the stopping test
//   (3) z = M r; r.z and beta are finished by the apply's last kernel
//   (4) p = z + beta p
// Each dot product is finished by the last block of its launch (GridSum).
// ---------------------------------------------------------------------------
template <int VW>
__global__ void __launch_bounds__(NT) k_pcg_spmv(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                 const double* __restrict__ val, const double* __restrict__ p,
                                                 double* __restrict__ q, double* __restrict__ scal,
                                                 int32_t* __restrict__ flag, GridSum gs) {
  COUNT_LAUNCH();
  if (flag[F_DONE]) return;
  const int lane = threadIdx.x % VW;
  const int rows_per_block = NT / VW;
  double dsum = 0;
  for (int base = blockIdx.x * rows_per_block; base < n; base += gridDim.x * rows_per_block) {
    const int r = base + threadIdx.x / VW;
    double acc = 0;
    if (r < n) {
      const int b = rp[r], e = rp[r + 1];
      for (int k = b + lane; k < e; k += VW) acc += val[k] * p[ci[k]];
    }
#pragma unroll
    for (int o = VW / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (r < n && lane == 0) {
      q[r] = acc;
      dsum += acc * p[r];
    }
  }
  grid_sum_last(dsum, gs, [&](double pq) {
    scal[S_PQ] = pq;
    scal[S_ALPHA] = scal[S_RZ] / pq;
    if (!(pq > 0) || !isfinite(pq)) { scal[S_ALPHA] = 0; flag[F_DONE] = 2; }
  });
}

// q = A p and alpha = rz / p.q, one thread per row (short rows)
__global__ void __launch_bounds__(NT) k_pcg_spmv_rows(int n, const int32_t* __restrict__ rp,
                                                        const int32_t* __restrict__ ci,
                                                        const double* __restrict__ val, const double* __restrict__ p,
                                                        double* __restrict__ q, double* __restrict__ scal,
                                                        int32_t* __restrict__ flag, GridSum gs) {
  COUNT_LAUNCH();
  if (flag[F_DONE]) return;
  spmv_rows_body<true>(n, rp, ci, val, p, q, nullptr, gs, [&](double pq) {
    scal[S_PQ] = pq;
    scal[S_ALPHA] = scal[S_RZ] / pq;
    if (!(pq > 0) || !isfinite(pq)) { scal[S_ALPHA] = 0; flag[F_DONE] = 2; }
  });
}

// p = z + beta p
__global__ void __launch_bounds__(NT) k_pcg_p(int n, double* __restrict__ p, const double* __restrict__ z,
                                              const double* __restrict__ scal, const int32_t* __restrict__ flag) {
  COUNT_LAUNCH();
  if (flag[F_DONE]) return;
  const double beta = scal[S_BETA];
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) p[i] = z[i] + beta * p[i];
}

__global__ void __launch_bounds__(NT) k_pcg_xr(int n, double* __restrict__ x, double* __restrict__ r,
                                               const double* __restrict__ p, const double* __restrict__ q,
                                               double* __restrict__ scal, int32_t* __restrict__ flag, GridSum gs) {
  COUNT_LAUNCH();
  if (flag[F_DONE]) return;
  const double alpha = scal[S_ALPHA];
  double s = 0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    s += ri * ri;
  }
  grid_sum_last(s, gs, [&](double rr) {
    const int it = ++flag[F_IT];
    const double rel = sqrt(rr) / scal[S_BNORM];
    scal[S_RR] = rr;
    scal[S_RELRES] = rel;
    if (rel <= scal[S_RTOL]) flag[F_DONE] = 1;
    else if (it >= flag[F_MAXIT] || !isfinite(rel)) flag[F_DONE] = 3;
  });
}

// generic: out = a + alpha * b  (alpha from scal[ia] times sgn)
__global__ void k_axpby(int n, double* out, const double* a, const double* b, double alpha) {
  COUNT_LAUNCH();
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) out[i] = a[i] + alpha * b[i];
}

__global__ void k_init_scalars(double* scal, int32_t* flag, const double* part, int nb, double rtol, int maxit,
                               int which) {
  COUNT_LAUNCH();
  double s = sum_partials(part, nb);
  if (threadIdx.x == 0) {
    if (which == 0) {  // ||b||^2
      scal[S_BNORM] = sqrt(s);
      scal[S_RTOL] = rtol;
      flag[F_DONE] = 0;
      flag[F_IT] = 0;
      flag[F_MAXIT] = maxit;
      if (!(s > 0)) flag[F_DONE] = 1;
    } else if (which == 1) {  // r.z
      scal[S_RZ] = s;
    } else {  // ||r0||^2
      scal[S_RR] = s;
      scal[S_RELRES] = sqrt(s) / scal[S_BNORM];
      if (scal[S_RELRES] <= rtol) flag[F_DONE] = 1;
    }
  }
}

inline unsigned vgrid(int n) { return (unsigned)std::min<int64_t>(ceil_div(n, NT), NBLK); }

template <int VW>
void spmv_launch(Handle& h, const double* x, double* y, cudaStream_t s, const double* b, const int32_t* done) {
  const int rows = NT / VW;
  const unsigned g = (unsigned)std::min<int64_t>(ceil_div(h.n, rows), RBLK);
  k_spmv<VW><<<g, NT, 0, s>>>(h.n, h.row_ptr, h.col_idx, h.val, x, y, b, done);
}

// short rows: one thread per row; longer rows: VW lanes per row
inline bool short_rows(int n, int64_t nnz) { return n > 0 && (double)nnz / n <= 12.0; }
inline unsigned rows_grid(int n) { return (unsigned)std::min<int64_t>(ceil_div(n, NT), RBLK); }

void spmv_any(Handle& h, const double* x, double* y, cudaStream_t s, const double* b = nullptr,
              const int32_t* done = nullptr) {
  double avg = h.n ? (double)h.nnz / h.n : 1;
  if (short_rows(h.n, h.nnz))
    k_spmv_rows<<<rows_grid(h.n), NT, 0, s>>>(h.n, h.row_ptr, h.col_idx, h.val, x, y, b, done);
  else if (avg <= 6) spmv_launch<4>(h, x, y, s, b, done);
  else if (avg <= 12) spmv_launch<8>(h, x, y, s, b, done);
  else if (avg <= 24) spmv_launch<16>(h, x, y, s, b, done);
  else spmv_launch<32>(h, x, y, s, b, done);
}

void ensure_krylov(Handle& h, cudaStream_t s) {
  Krylov& kr = h.kr;
  if (kr.r) return;
  DevMem& mem = h.mem;
  const int n = h.n;
  kr.r = mem.alloc<double>(n);
  kr.z = mem.alloc<double>(n);
  kr.p = mem.alloc<double>(n);
  kr.q = mem.alloc<double>(n);
  kr.w = mem.alloc<double>(n);
  kr.part = mem.alloc<double>(NBLK);
  kr.gpart = mem.alloc<double>(3 * RBLK);
  kr.ticket = mem.alloc<unsigned>(3);
  CK(cudaMemsetAsync(kr.ticket, 0, 3 * sizeof(unsigned), s));
  kr.scal = mem.alloc<double>(S_NSCAL);
  kr.flag = mem.alloc<int32_t>(F_NFLAG);
  kr.bx = mem.alloc<double>(2LL * n);
  CK(cudaMallocHost(&kr.hpin, 64));
}

}  // namespace

void spmv(Handle& h, const double* x, double* y, cudaStream_t s) {
  spmv_any(h, x, y, s);
  CK_LAUNCH("spmv");
}

void krylov_buffers(Handle& h, cudaStream_t s) { ensure_krylov(h, s); }

void csr_spmv(int n, int64_t nnz, const int32_t* rp, const int32_t* ci, const double* val, const double* x,
              double* y, cudaStream_t s) {
  if (n <= 0) return;
  if (short_rows(n, nnz)) {
    k_spmv_rows<<<rows_grid(n), NT, 0, s>>>(n, rp, ci, val, x, y, nullptr, nullptr);
  } else {
    const double avg = (double)nnz / n;
    const int vw = avg <= 24 ? 16 : 32;
    const unsigned g = (unsigned)std::min<int64_t>(ceil_div(n, NT / vw), RBLK);
    if (vw == 16) k_spmv<16><<<g, NT, 0, s>>>(n, rp, ci, val, x, y, nullptr, nullptr);
    else k_spmv<32><<<g, NT, 0, s>>>(n, rp, ci, val, x, y, nullptr, nullptr);
  }
  CK_LAUNCH("csr spmv");
}

void time_pcg_spmv(Handle& h, const double* p, double* q, int iters, cudaStream_t s, double* ms) {
  ensure_krylov(h, s);
  Krylov& kr = h.kr;
  const int n = h.n;
  CK(cudaMemsetAsync(kr.flag, 0, sizeof(int32_t) * F_NFLAG, s));
  const double one = 1.0;
  CK(cudaMemcpyAsync(kr.scal + S_RZ, &one, sizeof(double), cudaMemcpyHostToDevice, s));
  const GridSum g_pq{kr.gpart, kr.ticket};
  const double avg = n ? (double)h.nnz / n : 1;
  const int vw = avg <= 6 ? 4 : avg <= 12 ? 8 : avg <= 24 ? 16 : 32;
  const unsigned sg = (unsigned)std::min<int64_t>(ceil_div(n, NT / vw), RBLK);
  auto launch = [&]() {
    if (short_rows(n, h.nnz))
      k_pcg_spmv_rows<<<rows_grid(n), NT, 0, s>>>(n, h.row_ptr, h.col_idx, h.val, p, q, kr.scal, kr.flag, g_pq);
    else if (vw == 16)
      k_pcg_spmv<16><<<sg, NT, 0, s>>>(n, h.row_ptr, h.col_idx, h.val, p, q, kr.scal, kr.flag, g_pq);
    else
      k_pcg_spmv<32><<<sg, NT, 0, s>>>(n, h.row_ptr, h.col_idx, h.val, p, q, kr.scal, kr.flag, g_pq);
  };
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (int w = 0; w < 3; ++w) launch();
  CK(cudaEventRecord(e0, s));
  for (int it = 0; it < iters; ++it) launch();
  CK(cudaEventRecord(e1, s));
  CK(cudaEventSynchronize(e1));
  float t = 0;
  CK(cudaEventElapsedTime(&t, e0, e1));
  ms[0] = t / std::max(iters, 1);
  CK(cudaEventDestroy(e0));
  CK(cudaEventDestroy(e1));
  CK(cudaMemsetAsync(kr.flag, 0, sizeof(int32_t) * F_NFLAG, s));
  CK_LAUNCH("timed spmv");
}

void residual(Handle& h, const double* b, const double* x, double* y, cudaStream_t s, const int32_t* done) {
  spmv_any(h, x, y, s, b, done);
}

void solve_pcg(Handle& h, const double* b, double* x, const asm_solve_opts& o, asm_solve_info& info,
               cudaStream_t s) {
  ensure_krylov(h, s);
  Krylov& kr = h.kr;
  const int n = h.n;
  const unsigned vg = NBLK;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, s));
  // r = b - A x0 (or b), ||b||, z = M r, rz = r.z, p = z
  k_dot<<<vg, NT, 0, s>>>(n, b, b, kr.part, nullptr);
  k_init_scalars<<<1, NT, 0, s>>>(kr.scal, kr.flag, kr.part, NBLK, o.rtol, o.max_it, 0);
  if (o.use_x0) {
    spmv_any(h, x, kr.q, s);
    k_axpby<<<vgrid(n), NT, 0, s>>>(n, kr.r, b, kr.q, -1.0);
  } else {
    CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    CK(cudaMemcpyAsync(kr.r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  }
  k_dot<<<vg, NT, 0, s>>>(n, kr.r, kr.r, kr.part, nullptr);
  k_init_scalars<<<1, NT, 0, s>>>(kr.scal, kr.flag, kr.part, NBLK, o.rtol, o.max_it, 2);
  apply_preconditioner(h, kr.r, kr.z, s, nullptr);
  k_dot<<<vg, NT, 0, s>>>(n, kr.r, kr.z, kr.part, nullptr);
  k_init_scalars<<<1, NT, 0, s>>>(kr.scal, kr.flag, kr.part, NBLK, o.rtol, o.max_it, 1);
  // first direction p = z: beta = 0 against a zero previous direction
  CK(cudaMemsetAsync(kr.p, 0, sizeof(double) * n, s));
  CK(cudaMemsetAsync(kr.scal + S_BETA, 0, sizeof(double), s));
  CK_LAUNCH("pcg init");

  const double avg = n ? (double)h.nnz / n : 1;
  const int vw = avg <= 6 ? 4 : avg <= 12 ? 8 : avg <= 24 ? 16 : 32;
  const unsigned sg = (unsigned)std::min<int64_t>(ceil_div(n, NT / vw), RBLK);
  const unsigned xg = (unsigned)std::min<int64_t>(ceil_div(n, NT), RBLK);
  const GridSum g_pq{kr.gpart, kr.ticket}, g_rr{kr.gpart + RBLK, kr.ticket + 1};
  ApplyDot rzdot;
  rzdot.r = kr.r;
  rzdot.gs = GridSum{kr.gpart + 2 * RBLK, kr.ticket + 2};
  rzdot.rz = kr.scal + S_RZ;
  rzdot.beta = kr.scal + S_BETA;
  // one iteration, the direction update first (beta of the previous one)
  auto iteration = [&](cudaStream_t st, int) {
    k_pcg_p<<<xg, NT, 0, st>>>(n, kr.p, kr.z, kr.scal, kr.flag);
    if (short_rows(n, h.nnz)) {
      k_pcg_spmv_rows<<<rows_grid(n), NT, 0, st>>>(n, h.row_ptr, h.col_idx, h.val, kr.p, kr.q, kr.scal, kr.flag,
                                                      g_pq);
    } else switch (vw) {
      case 4: k_pcg_spmv<4><<<sg, NT, 0, st>>>(n, h.row_ptr, h.col_idx, h.val, kr.p, kr.q, kr.scal, kr.flag, g_pq); break;
      case 8: k_pcg_spmv<8><<<sg, NT, 0, st>>>(n, h.row_ptr, h.col_idx, h.val, kr.p, kr.q, kr.scal, kr.flag, g_pq); break;
      case 16: k_pcg_spmv<16><<<sg, NT, 0, st>>>(n, h.row_ptr, h.col_idx, h.val, kr.p, kr.q, kr.scal, kr.flag, g_pq); break;
      default: k_pcg_spmv<32><<<sg, NT, 0, st>>>(n, h.row_ptr, h.col_idx, h.val, kr.p, kr.q, kr.scal, kr.flag, g_pq); break;
    }
    k_pcg_xr<<<xg, NT, 0, st>>>(n, x, kr.r, kr.p, kr.q, kr.scal, kr.flag, g_rr);
    apply_preconditioner(h, kr.r, kr.z, st, kr.flag, &rzdot);
  };
  cudaStream_t cs;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaEvent_t ej;
  CK(cudaEventCreateWithFlags(&ej, cudaEventDisableTiming));
  CK(cudaEventRecord(ej, s));
  CK(cudaStreamWaitEvent(cs, ej, 0));
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  const int chunk = std::max(1, o.check_every > 0 ? o.check_every : 8);
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  for (int k = 0; k < chunk; ++k) iteration(cs, k);
  CK(cudaStreamEndCapture(cs, &graph));
  CK(cudaGraphInstantiate(&exec, graph, 0));
  int32_t* hflag = reinterpret_cast<int32_t*>(kr.hpin);
  for (;;) {
    CK(cudaGraphLaunch(exec, cs));
    CK(cudaMemcpyAsync(hflag, kr.flag, sizeof(int32_t) * 2, cudaMemcpyDeviceToHost, cs));
    CK(cudaStreamSynchronize(cs));
    if (hflag[F_DONE]) break;
  }
  CK(cudaEventRecord(ej, cs));
  CK(cudaStreamWaitEvent(s, ej, 0));
  CK(cudaGraphExecDestroy(exec));
  CK(cudaGraphDestroy(graph));
  CK(cudaStreamDestroy(cs));
  CK(cudaEventDestroy(ej));
  CK(cudaEventRecord(e1, s));
  // true residual
  spmv_any(h, x, kr.q, s);
  k_axpby<<<vgrid(n), NT, 0, s>>>(n, kr.w, b, kr.q, -1.0);
  k_dot<<<vg, NT, 0, s>>>(n, kr.w, kr.w, kr.part, nullptr);
  double sc[S_NSCAL];
  int32_t fl[F_NFLAG];
  CK(cudaMemcpyAsync(sc, kr.scal, sizeof(sc), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(fl, kr.flag, sizeof(fl), cudaMemcpyDeviceToHost, s));
  std::vector<double> part(NBLK);
  CK(cudaMemcpyAsync(part.data(), kr.part, sizeof(double) * NBLK, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  CK(cudaEventDestroy(e0));
  CK(cudaEventDestroy(e1));
  double tr = 0;
  for (double v : part) tr += v;
  info.iterations = fl[F_IT];
  info.converged = fl[F_DONE] == 1;
  info.final_relres = sc[S_RELRES];
  info.true_relres = sc[S_BNORM] > 0 ? std::sqrt(tr) / sc[S_BNORM] : 0.0;
  info.solve_ms = ms;
}

namespace {

constexpr int MAXV = 513;  // restart length + 1 (512: GMRES without restart for up to 512 iterations)

// V^T w for the n x nvec basis V (vectors n apart) as a tall-skinny product:
// block b owns rows [b*rows, (b+1)*rows), warp k%8 of it the vectors
// k = wid, wid+8, ...; part[b * MAXV + k] = that chunk of V_k . w.  No block
// reduction per vector: every vector's chunk is one warp's lane-strided sum.
constexpr int MD_MAXB = 2048;  // blocks (row chunks) of the multi-dot at most
__global__ void __launch_bounds__(NT) k_multidot(int n, int rows, const double* __restrict__ V, int nvec,
                                                 const double* __restrict__ w, double* __restrict__ part) {
  COUNT_LAUNCH();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int r0 = blockIdx.x * rows;
  const int r1 = min(n, r0 + rows);
  for (int k = wid; k < nvec; k += NT / 32) {
    const double* v = V + (int64_t)k * n;
    double s = 0;
    for (int i = r0 + lane; i < r1; i += 32) s += v[i] * w[i];
    s = warp_sum(s);
    if (lane == 0) part[blockIdx.x * MAXV + k] = s;
  }
}

// out[k] = sum_b part[b * MAXV + k], one warp per k (fixed order)
__global__ void __launch_bounds__(NT) k_multidot_fin(const double* __restrict__ part, int nb, int nvec,
                                                     double* __restrict__ out) {
  COUNT_LAUNCH();
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * (NT / 32) + (threadIdx.x >> 5);
  if (k >= nvec) return;
  double s = 0;
  for (int b = lane; b < nb; b += 32) s += part[b * MAXV + k];
  s = warp_sum(s);
  if (lane == 0) out[k] = s;
}

// row chunks of the multi-dot: about 512 rows each, at most MD_MAXB chunks
inline int md_rows(int n) { return (int)std::max<int64_t>(512, ceil_div(n, MD_MAXB)); }
inline int md_blocks(int n) { return (int)std::max<int64_t>(1, ceil_div(n, md_rows(n))); }

// w -= sum_k V_k c_k
__global__ void __launch_bounds__(NT) k_sub_vc(int n, const double* __restrict__ V, int nvec,
                                               const double* __restrict__ c, double* __restrict__ w) {
  COUNT_LAUNCH();
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) {
    double s = 0;
    for (int k = 0; k < nvec; ++k) s += V[(int64_t)k * n + i] * c[k];
    w[i] -= s;
  }
}

// x += sum_k Zb_k y_k
__global__ void __launch_bounds__(NT) k_add_zy(int n, const double* __restrict__ Zb, int nvec,
                                               const double* __restrict__ y, double* __restrict__ x) {
  COUNT_LAUNCH();
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) {
    double s = 0;
    for (int k = 0; k < nvec; ++k) s += Zb[(int64_t)k * n + i] * y[k];
    x[i] += s;
  }
}

// out = a / nrm with nrm = sqrt(sum of partials); stores nrm in *dst
__global__ void __launch_bounds__(NT) k_normalize(int n, const double* __restrict__ part, int nb,
                                                  const double* __restrict__ a, double* __restrict__ out,
                                                  double* __restrict__ dst) {
  COUNT_LAUNCH();
  double s = sum_partials(part, nb);
  const double nrm = sqrt(s);
  if (blockIdx.x == 0 && threadIdx.x == 0) *dst = nrm;
  const double inv = nrm > 0 ? 1.0 / nrm : 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) out[i] = a[i] * inv;
}

// Column j of the Hessenberg matrix (col[0..j+1]): apply the previous Givens
// rotations, build the new one, update g; residual estimate |g[j+1]| / ||b||.
// g[0] is set to beta at each restart.  flag: [0] done, [1] iterations.
__global__ void k_givens(double* H, int ldh, int j, double* cs, double* sn, double* g, const double* scal,
                         int32_t* flag, double* hist, int hist_len) {
  COUNT_LAUNCH();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (flag[0]) return;  // converged earlier in this chunk: the extra columns are ignored
  double* col = H + (int64_t)j * ldh;
  for (int k = 0; k < j; ++k) {
    double t = cs[k] * col[k] + sn[k] * col[k + 1];
    col[k + 1] = -sn[k] * col[k] + cs[k] * col[k + 1];
    col[k] = t;
  }
  double den = hypot(col[j], col[j + 1]);
  double c = den > 0 ? col[j] / den : 1.0, sv = den > 0 ? col[j + 1] / den : 0.0;
  cs[j] = c; sn[j] = sv;
  col[j] = den; col[j + 1] = 0;
  g[j + 1] = -sv * g[j];
  g[j] = c * g[j];
  int it = ++flag[1];
  double rel = fabs(g[j + 1]) / scal[5];
  if (hist != nullptr && it < hist_len) hist[it] = rel;
  if (rel <= scal[6]) flag[0] = 1;
  else if (it >= flag[2] || !isfinite(rel)) flag[0] = 3;
  if (flag[0]) flag[3] = j + 1;  // columns of this cycle that enter the update
  // keep the estimate for the host
  ((double*)scal)[7] = rel;
}

// y = H(0:k, 0:k)^{-1} g(0:k) (upper triangular); k from the device when the
// cycle stopped on convergence, else the host's count
__global__ void k_backsolve(const double* H, int ldh, int khost, const int32_t* flag, const double* g, double* y) {
  COUNT_LAUNCH();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int k = flag[0] ? flag[3] : khost;
  for (int r = k; r < khost; ++r) y[r] = 0;
  for (int r = k - 1; r >= 0; --r) {
    double s = g[r];
    for (int c = r + 1; c < k; ++c) s -= H[(int64_t)c * ldh + r] * y[c];
    y[r] = s / H[(int64_t)r * ldh + r];
  }
}

}  // namespace

void solve_fgmres(Handle& h, const double* b, double* x, const asm_solve_opts& o, asm_solve_info& info,
                  cudaStream_t s, bool auto_restart) {
  ensure_krylov(h, s);
  Krylov& kr = h.kr;
  const int n = h.n;
  // basis length: the restart length, at most max_it and 512; the automatic
  // length also fits the basis (2m + 1 vectors) in 3/4 of the free memory
  int m = std::max(1, std::min(std::min(o.restart, MAXV - 1), o.max_it));
  if (auto_restart && m > kr.restart) {
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    const double per = 2.0 * 8.0 * (double)n;
    const int fit = (int)std::min<double>(m, std::floor((0.75 * (double)fr - 8.0 * n) / per));
    m = std::max(std::min(m, 30), fit);
  }
  DevMem& mem = h.mem;
  if (!kr.V || m > kr.restart) {
    // grow the basis; a shorter restart later reuses it
    mem.free(kr.V);
    mem.free(kr.ZB);
    mem.free(kr.H);
    kr.V = mem.alloc<double>((int64_t)(m + 1) * n);
    kr.ZB = mem.alloc<double>((int64_t)m * n);
    kr.H = mem.alloc<double>((int64_t)(m + 1) * m + 4 * (m + 1) + 16);
    if (!kr.mpart) kr.mpart = mem.alloc<double>((int64_t)MD_MAXB * MAXV);
    kr.restart = m;
  }
  const int ldh = m + 1;
  double* H = kr.H;
  double* cs = H + (int64_t)ldh * m;
  double* sn = cs + ldh;
  double* g = sn + ldh;
  double* y = g + ldh;
  double* tmp = kr.w;  // n
  const unsigned vg = NBLK;
  const int mdr = md_rows(n);
  const unsigned mdb = (unsigned)md_blocks(n);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, s));
  k_dot<<<vg, NT, 0, s>>>(n, b, b, kr.part, nullptr);
  k_init_scalars<<<1, NT, 0, s>>>(kr.scal, kr.flag, kr.part, NBLK, o.rtol, o.max_it, 0);
  if (!o.use_x0) CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
  int32_t* hflag = reinterpret_cast<int32_t*>(kr.hpin);
  const int check = std::max(1, o.check_every > 0 ? o.check_every : 8);
  int total = 0;
  bool done = false;
  while (!done) {
    // restart: r = b - A x, beta, v_0, g = beta e_1
    spmv_any(h, x, kr.q, s);
    k_axpby<<<vgrid(n), NT, 0, s>>>(n, kr.r, b, kr.q, -1.0);
    k_dot<<<vg, NT, 0, s>>>(n, kr.r, kr.r, kr.part, nullptr);
    CK(cudaMemsetAsync(g, 0, sizeof(double) * ldh, s));
    k_normalize<<<vg, NT, 0, s>>>(n, kr.part, NBLK, kr.r, kr.V, g);
    int j = 0;
    for (; j < m; ++j) {
      double* vj = kr.V + (int64_t)j * n;
      double* zj = kr.ZB + (int64_t)j * n;
      double* col = H + (int64_t)j * ldh;
      apply_preconditioner(h, vj, zj, s, nullptr);
      spmv_any(h, zj, tmp, s);
      // classical Gram-Schmidt, twice
      const unsigned fb = (unsigned)ceil_div(j + 1, NT / 32);
      k_multidot<<<mdb, NT, 0, s>>>(n, mdr, kr.V, j + 1, tmp, kr.mpart);
      k_multidot_fin<<<fb, NT, 0, s>>>(kr.mpart, mdb, j + 1, col);
      k_sub_vc<<<vgrid(n), NT, 0, s>>>(n, kr.V, j + 1, col, tmp);
      k_multidot<<<mdb, NT, 0, s>>>(n, mdr, kr.V, j + 1, tmp, kr.mpart);
      k_multidot_fin<<<fb, NT, 0, s>>>(kr.mpart, mdb, j + 1, y);
      k_sub_vc<<<vgrid(n), NT, 0, s>>>(n, kr.V, j + 1, y, tmp);
      k_axpby<<<1, NT, 0, s>>>(j + 1, col, col, y, 1.0);
      k_dot<<<vg, NT, 0, s>>>(n, tmp, tmp, kr.part, nullptr);
      k_normalize<<<vg, NT, 0, s>>>(n, kr.part, NBLK, tmp, kr.V + (int64_t)(j + 1) * n, col + j + 1);
      k_givens<<<1, 1, 0, s>>>(H, ldh, j, cs, sn, g, kr.scal, kr.flag, nullptr, 0);
      ++total;
      if ((total % check) == 0 || j == m - 1) {
        CK(cudaMemcpyAsync(hflag, kr.flag, sizeof(int32_t) * 2, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (hflag[0]) { ++j; done = true; break; }
      }
    }
    if (!done && j == m) j = m;
    k_backsolve<<<1, 1, 0, s>>>(H, ldh, j, kr.flag, g, y);
    k_add_zy<<<vgrid(n), NT, 0, s>>>(n, kr.ZB, j, y, x);
    CK_LAUNCH("fgmres cycle");
    if (!done) {
      CK(cudaMemcpyAsync(hflag, kr.flag, sizeof(int32_t) * 2, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (hflag[0]) done = true;
    }
  }
  CK(cudaEventRecord(e1, s));
  // true residual
  spmv_any(h, x, kr.q, s);
  k_axpby<<<vgrid(n), NT, 0, s>>>(n, kr.w, b, kr.q, -1.0);
  k_dot<<<vg, NT, 0, s>>>(n, kr.w, kr.w, kr.part, nullptr);
  double sc[S_NSCAL];
  int32_t fl[F_NFLAG];
  std::vector<double> part(NBLK);
  CK(cudaMemcpyAsync(sc, kr.scal, sizeof(sc), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(fl, kr.flag, sizeof(fl), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(part.data(), kr.part, sizeof(double) * NBLK, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  CK(cudaEventDestroy(e0));
  CK(cudaEventDestroy(e1));
  double tr = 0;
  for (double v : part) tr += v;
  info.iterations = fl[F_IT];
  info.converged = fl[F_DONE] == 1;
  info.final_relres = sc[S_RELRES];
  info.true_relres = sc[S_BNORM] > 0 ? std::sqrt(tr) / sc[S_BNORM] : 0.0;
  info.solve_ms = ms;
}

}  // namespace asmgpu
