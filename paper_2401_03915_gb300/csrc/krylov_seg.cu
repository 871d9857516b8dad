// PCG on independent systems that share one handle: A (and with it every
// R_i, A_ii^{-1} and the coarse correction) is block diagonal over contiguous
// row segments, so each segment is its own SPD system A_s x_s = b_s, and CG
// runs one recurrence per segment (its own alpha, beta and stopping test,
// ||b_s - A_s x_s|| / ||b_s|| <= rtol) while the SpMV and the two-level apply
// are launched once for all segments.  This is how a stream of problems of
// uneven sizes is set up in one pass (their subdomains in the same launches)
// and solved without one problem's spectrum slowing another's convergence:
// a single CG on the block-diagonal system would need to resolve the
// outlying eigenvalues of every segment at once.
//
// Segment reductions are deterministic: a 2D grid (chunks x segments) writes
// per-chunk partial sums in a fixed order, one block then combines them per
// segment in a fixed order.
#include <cmath>

#include "handle.cuh"

namespace asmgpu {
namespace {

constexpr int NT = 256;
constexpr int FT = 1024;  // threads of the single-block finalisers

// per-segment scalars, stride SC
enum { C_BN = 0, C_RZ, C_ALPHA, C_BETA, C_RELRES, C_TRUE, SC };

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
  return t;
}

// part[s * cb + chunk] = the chunk's share of a_s . b_s
__global__ void __launch_bounds__(NT) k_seg_dot(const int32_t* __restrict__ off, const double* __restrict__ a,
                                               const double* __restrict__ b, double* __restrict__ part, int cb,
                                               const int32_t* __restrict__ gflag) {
  COUNT_LAUNCH();
  __shared__ double red[NT / 32];
  if (gflag && *gflag) return;
  const int sg = blockIdx.y;
  const int r0 = off[sg], r1 = off[sg + 1];
  double v = 0;
  for (int r = r0 + blockIdx.x * NT + threadIdx.x; r < r1; r += cb * NT) v += a[r] * b[r];
  v = block_sum(v, red);
  if (threadIdx.x == 0) part[(int64_t)sg * cb + blockIdx.x] = v;
}

__device__ __forceinline__ double seg_total(const double* __restrict__ part, int s, int cb) {
  double t = 0;
  for (int k = 0; k < cb; ++k) t += part[(int64_t)s * cb + k];
  return t;
}

// setup of the scalars: what = 0: ||b_s||; 1: rz_s = r.z, beta 0; relres from
// the r.r partials of what = 2
__global__ void __launch_bounds__(FT) k_seg_init(int nseg, int what, const double* __restrict__ part, int cb,
                                                 double* __restrict__ sc, int32_t* __restrict__ done,
                                                 int32_t* __restrict__ its, int32_t* __restrict__ gflag,
                                                 int32_t* __restrict__ counter, double rtol) {
  COUNT_LAUNCH();
  __shared__ int all;
  if (threadIdx.x == 0) all = 1;
  __syncthreads();
  for (int s = threadIdx.x; s < nseg; s += FT) {
    const double t = seg_total(part, s, cb);
    double* c = sc + (int64_t)s * SC;
    if (what == 0) {
      c[C_BN] = sqrt(t);
    } else if (what == 2) {
      c[C_RELRES] = c[C_BN] > 0 ? sqrt(t) / c[C_BN] : 0.0;
      done[s] = (c[C_BN] == 0 || c[C_RELRES] <= rtol) ? 1 : 0;
      its[s] = 0;
      if (!done[s]) atomicAnd(&all, 0);
    } else {
      c[C_RZ] = t;
      c[C_BETA] = 0;
      c[C_ALPHA] = 0;
    }
  }
  __syncthreads();
  if (what == 2 && threadIdx.x == 0) {
    *gflag = all ? 1 : 0;
    *counter = 0;
  }
}

// alpha_s = rz_s / p_s.q_s (0 for converged segments); a non-positive p.q
// means A or M is not SPD on that segment
__global__ void __launch_bounds__(FT) k_seg_alpha(int nseg, const double* __restrict__ part, int cb,
                                                  double* __restrict__ sc, const int32_t* __restrict__ done,
                                                  const int32_t* __restrict__ gflag, int32_t* __restrict__ err) {
  COUNT_LAUNCH();
  if (*gflag) return;
  for (int s = threadIdx.x; s < nseg; s += FT) {
    double* c = sc + (int64_t)s * SC;
    const double pq = seg_total(part, s, cb);
    if (done[s]) {
      c[C_ALPHA] = 0;
    } else if (!(pq > 0) || !isfinite(pq)) {
      c[C_ALPHA] = 0;
      atomicOr(err, DERR_NOT_SPD);
    } else {
      c[C_ALPHA] = c[C_RZ] / pq;
    }
  }
}

// relres_s from r.r; newly converged segments record the iteration
__global__ void __launch_bounds__(FT) k_seg_check(int nseg, const double* __restrict__ part, int cb,
                                                  double* __restrict__ sc, int32_t* __restrict__ done,
                                                  int32_t* __restrict__ its, const int32_t* __restrict__ gflag,
                                                  const int32_t* __restrict__ counter, double rtol) {
  COUNT_LAUNCH();
  if (*gflag) return;
  for (int s = threadIdx.x; s < nseg; s += FT) {
    if (done[s]) continue;
    double* c = sc + (int64_t)s * SC;
    c[C_RELRES] = sqrt(seg_total(part, s, cb)) / c[C_BN];
    its[s] = *counter + 1;
    if (c[C_RELRES] <= rtol) done[s] = 1;
  }
}

// beta_s = rz_new / rz_s, the iteration counter, the all-done / cap flag
__global__ void __launch_bounds__(FT) k_seg_beta(int nseg, const double* __restrict__ part, int cb,
                                                 double* __restrict__ sc, const int32_t* __restrict__ done,
                                                 int32_t* __restrict__ gflag, int32_t* __restrict__ counter,
                                                 int max_it) {
  COUNT_LAUNCH();
  __shared__ int all;
  if (*gflag) return;
  if (threadIdx.x == 0) all = 1;
  __syncthreads();
  for (int s = threadIdx.x; s < nseg; s += FT) {
    double* c = sc + (int64_t)s * SC;
    if (done[s]) continue;
    atomicAnd(&all, 0);
    const double rz = seg_total(part, s, cb);
    c[C_BETA] = c[C_RZ] != 0 ? rz / c[C_RZ] : 0.0;
    c[C_RZ] = rz;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int it = *counter + 1;
    *counter = it;
    if (all) *gflag = 1;
    else if (it >= max_it) *gflag = 2;
  }
}

// p_s = z_s + beta_s p_s
__global__ void __launch_bounds__(NT) k_seg_p(const int32_t* __restrict__ off, double* __restrict__ p,
                                             const double* __restrict__ z, const double* __restrict__ sc, int cb,
                                             const int32_t* __restrict__ done, const int32_t* __restrict__ gflag) {
  COUNT_LAUNCH();
  if (*gflag) return;
  const int sg = blockIdx.y;
  if (done[sg]) return;
  const double beta = sc[(int64_t)sg * SC + C_BETA];
  const int r0 = off[sg], r1 = off[sg + 1];
  for (int r = r0 + blockIdx.x * NT + threadIdx.x; r < r1; r += cb * NT) p[r] = z[r] + beta * p[r];
}

// x_s += alpha_s p_s, r_s -= alpha_s q_s
__global__ void __launch_bounds__(NT) k_seg_xr(const int32_t* __restrict__ off, double* __restrict__ x,
                                              double* __restrict__ r, const double* __restrict__ p,
                                              const double* __restrict__ q, const double* __restrict__ sc, int cb,
                                              const int32_t* __restrict__ gflag) {
  COUNT_LAUNCH();
  if (*gflag) return;
  const int sg = blockIdx.y;
  const double alpha = sc[(int64_t)sg * SC + C_ALPHA];
  if (alpha == 0) return;
  const int r0 = off[sg], r1 = off[sg + 1];
  for (int k = r0 + blockIdx.x * NT + threadIdx.x; k < r1; k += cb * NT) {
    x[k] += alpha * p[k];
    r[k] -= alpha * q[k];
  }
}

__global__ void k_seg_sub(int n, double* __restrict__ w, const double* __restrict__ b, const double* __restrict__ q) {
  COUNT_LAUNCH();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    w[k] = b[k] - q[k];
}

// 1 in bad[0] if an entry of A couples two segments, in bad[1] if a
// subdomain's rows lie in more than one segment (seg_of[v]: segment of row v)
__global__ void k_seg_validate(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                               const int32_t* __restrict__ part, const int32_t* __restrict__ seg_of,
                               int32_t* __restrict__ sub_seg, int32_t* __restrict__ bad) {
  COUNT_LAUNCH();
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int sv = seg_of[v];
    for (int e = rp[v]; e < rp[v + 1]; ++e)
      if (seg_of[ci[e]] != sv) atomicOr(bad, 1);
    const int old = atomicCAS(&sub_seg[part[v]], -1, sv);
    if (old != -1 && old != sv) atomicOr(bad + 1, 1);
  }
}

__global__ void k_seg_of(int nseg, const int32_t* __restrict__ off, int32_t* __restrict__ seg_of) {
  COUNT_LAUNCH();
  const int sg = blockIdx.y;
  for (int r = off[sg] + blockIdx.x * blockDim.x + threadIdx.x; r < off[sg + 1]; r += gridDim.x * blockDim.x)
    seg_of[r] = sg;
}

}  // namespace

void solve_pcg_segments(Handle& h, const double* b, double* x, int nseg, const int32_t* h_off,
                        const asm_solve_opts& o, asm_solve_info* info, cudaStream_t s) {
  krylov_buffers(h, s);
  const int n = h.n;
  int maxlen = 0;
  for (int k = 0; k < nseg; ++k) maxlen = std::max(maxlen, h_off[k + 1] - h_off[k]);
  const int cb = (int)std::max<int64_t>(1, std::min<int64_t>(64, ceil_div(maxlen, 4 * NT)));
  // scratch, stream-ordered (freed at the end of the call)
  int32_t *d_off = nullptr, *ints = nullptr;
  double *part = nullptr, *sc = nullptr, *vec = nullptr;
  const int64_t nints = 2LL * nseg + 4 + (int64_t)n + h.N;
  CK(cudaMallocAsync(&d_off, sizeof(int32_t) * (nseg + 1), s));
  CK(cudaMallocAsync(&ints, sizeof(int32_t) * nints, s));
  CK(cudaMallocAsync(&part, sizeof(double) * (int64_t)nseg * cb, s));
  CK(cudaMallocAsync(&sc, sizeof(double) * (int64_t)nseg * SC, s));
  CK(cudaMallocAsync(&vec, sizeof(double) * 5 * (int64_t)n, s));
  int32_t* done = ints;
  int32_t* its = ints + nseg;
  int32_t* gflag = ints + 2 * nseg;
  int32_t* counter = gflag + 1;
  int32_t* bad = gflag + 2;  // 2 entries
  int32_t* seg_of = gflag + 4;
  int32_t* sub_seg = seg_of + n;
  double *r = vec, *z = vec + n, *p = vec + 2 * (int64_t)n, *q = vec + 3 * (int64_t)n, *w = vec + 4 * (int64_t)n;
  auto release = [&]() {
    cudaFreeAsync(d_off, s);
    cudaFreeAsync(ints, s);
    cudaFreeAsync(part, s);
    cudaFreeAsync(sc, s);
    cudaFreeAsync(vec, s);
  };
  CK(cudaMemcpyAsync(d_off, h_off, sizeof(int32_t) * (nseg + 1), cudaMemcpyHostToDevice, s));
  // the segments must split A and the subdomains: checked on the device
  CK(cudaMemsetAsync(bad, 0, sizeof(int32_t) * 2, s));
  CK(cudaMemsetAsync(sub_seg, 0xFF, sizeof(int32_t) * h.N, s));
  const dim3 gseg((unsigned)cb, (unsigned)nseg);
  k_seg_of<<<gseg, NT, 0, s>>>(nseg, d_off, seg_of);
  const unsigned vg = (unsigned)std::min<int64_t>(ceil_div(std::max(n, 1), NT), 152 * 16);
  k_seg_validate<<<vg, NT, 0, s>>>(n, h.row_ptr, h.col_idx, h.part, seg_of, sub_seg, bad);
  int32_t hb[2] = {0, 0};
  CK(cudaMemcpyAsync(hb, bad, sizeof(hb), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hb[0] || hb[1]) {
    release();
    fail(ASM_ERR_INVALID_ARG, hb[0] ? "asm_solve_segments: an entry of A couples two segments"
                                    : "asm_solve_segments: a subdomain has rows in two segments");
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, s));
  // x0 = 0: r = b, ||b_s||, z = M r, rz_s, p = 0, beta = 0
  CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
  CK(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(p, 0, sizeof(double) * n, s));
  k_seg_dot<<<gseg, NT, 0, s>>>(d_off, b, b, part, cb, nullptr);
  k_seg_init<<<1, FT, 0, s>>>(nseg, 0, part, cb, sc, done, its, gflag, counter, o.rtol);
  k_seg_init<<<1, FT, 0, s>>>(nseg, 2, part, cb, sc, done, its, gflag, counter, o.rtol);  // r = b
  apply_preconditioner(h, r, z, s, nullptr);
  k_seg_dot<<<gseg, NT, 0, s>>>(d_off, r, z, part, cb, nullptr);
  k_seg_init<<<1, FT, 0, s>>>(nseg, 1, part, cb, sc, done, its, gflag, counter, o.rtol);
  CK_LAUNCH("segmented pcg init");
  auto iteration = [&](cudaStream_t st) {
    k_seg_p<<<gseg, NT, 0, st>>>(d_off, p, z, sc, cb, done, gflag);
    spmv(h, p, q, st);
    k_seg_dot<<<gseg, NT, 0, st>>>(d_off, p, q, part, cb, gflag);
    k_seg_alpha<<<1, FT, 0, st>>>(nseg, part, cb, sc, done, gflag, h.dn.err);
    k_seg_xr<<<gseg, NT, 0, st>>>(d_off, x, r, p, q, sc, cb, gflag);
    k_seg_dot<<<gseg, NT, 0, st>>>(d_off, r, r, part, cb, gflag);
    k_seg_check<<<1, FT, 0, st>>>(nseg, part, cb, sc, done, its, gflag, counter, o.rtol);
    apply_preconditioner(h, r, z, st, gflag);
    k_seg_dot<<<gseg, NT, 0, st>>>(d_off, r, z, part, cb, gflag);
    k_seg_beta<<<1, FT, 0, st>>>(nseg, part, cb, sc, done, gflag, counter, o.max_it);
  };
  // chunks of iterations captured as one CUDA graph, replayed until every
  // segment has converged or the cap is reached
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
  for (int k = 0; k < chunk; ++k) iteration(cs);
  CK(cudaStreamEndCapture(cs, &graph));
  CK(cudaGraphInstantiate(&exec, graph, 0));
  int32_t* hflag = reinterpret_cast<int32_t*>(h.kr.hpin);
  for (;;) {
    CK(cudaGraphLaunch(exec, cs));
    CK(cudaMemcpyAsync(hflag, gflag, sizeof(int32_t), cudaMemcpyDeviceToHost, cs));
    CK(cudaStreamSynchronize(cs));
    if (hflag[0]) break;
  }
  CK(cudaEventRecord(ej, cs));
  CK(cudaStreamWaitEvent(s, ej, 0));
  CK(cudaGraphExecDestroy(exec));
  CK(cudaGraphDestroy(graph));
  CK(cudaStreamDestroy(cs));
  CK(cudaEventDestroy(ej));
  CK(cudaEventRecord(e1, s));
  // true residuals
  spmv(h, x, q, s);
  k_seg_sub<<<vg, NT, 0, s>>>(n, w, b, q);
  k_seg_dot<<<gseg, NT, 0, s>>>(d_off, w, w, part, cb, nullptr);
  std::vector<double> hsc((size_t)nseg * SC), hpart((size_t)nseg * cb);
  std::vector<int32_t> hdone(nseg), hits(nseg);
  CK(cudaMemcpyAsync(hsc.data(), sc, sizeof(double) * hsc.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hpart.data(), part, sizeof(double) * hpart.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hdone.data(), done, sizeof(int32_t) * nseg, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hits.data(), its, sizeof(int32_t) * nseg, cudaMemcpyDeviceToHost, s));
  release();
  CK(cudaStreamSynchronize(s));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  CK(cudaEventDestroy(e0));
  CK(cudaEventDestroy(e1));
  for (int k = 0; k < nseg; ++k) {
    double t = 0;
    for (int c = 0; c < cb; ++c) t += hpart[(size_t)k * cb + c];
    const double bn = hsc[(size_t)k * SC + C_BN];
    info[k].iterations = hits[k];
    info[k].converged = hdone[k];
    info[k].final_relres = hsc[(size_t)k * SC + C_RELRES];
    info[k].true_relres = bn > 0 ? std::sqrt(t) / bn : 0.0;
    info[k].solve_ms = ms;
  }
}

}  // namespace asmgpu
