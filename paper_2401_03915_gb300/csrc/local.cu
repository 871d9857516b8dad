// Local dense stage: gather A_ii out of CSR A (Section 2.3), invert it in
// place by a blocked Gauss-Jordan sweep, and pack the inverse into the tiles
// the apply streams.
//
// What is gathered is the symmetrically scaled A^_ii = D^{-1/2} A_ii D^{-1/2},
// D = diag(A): A_ii^{-1} = D^{-1/2} A^_ii^{-1} D^{-1/2}, and the scaling maps
// the local eigenproblem onto itself (same eigenvalues, vectors scaled by
// D^{1/2} on Gamma and the coarse vectors by D^{-1/2} on I_i).  It removes
// the coefficient contrast from the conditioning of the single-precision
// sweep; the apply and the eigen stage undo it.
//
// The sweep eliminates the unknowns of Omega_{i,1:delta-1} first.  At that
// midpoint the working matrix holds
//     [ B^{-1}         B^{-1} C          ]
//     [ -C^T B^{-1}    G - C^T B^{-1} C  ]      (general A: -A_{Gamma,Omega'} B^{-1})
// with B = A_{Omega_{1:delta-1}}, C = A_{Omega_{1:delta-1}, Gamma_delta} and
// G = A_{Gamma_delta, Gamma_delta}: the block -B^{-1} C of the harmonic
// operator Pi_i (eq. HOp) and the Schur complement S = G - C^T B^{-1} C.
// Their first |I_i| rows X_p = -(B^{-1}C)[:p] and S are copied out; the sweep
// then continues over Gamma_delta and leaves A_ii^{-1}, whose trailing block
// is S^{-1}.
#include <algorithm>

#include "handle.cuh"

namespace asmgpu {
namespace {

constexpr int NT = 256;
constexpr int KB = 32;  // pivot block of the sweep

template <typename T>
__global__ void k_gather(const int32_t* __restrict__ omega, int64_t m, const int32_t* __restrict__ pos_sub,
                         const int32_t* __restrict__ sub_off, const int32_t* __restrict__ rp,
                         const int32_t* __restrict__ ci, const double* __restrict__ val,
                         const double* __restrict__ ds, const int64_t* __restrict__ ent_off,
                         const int32_t* __restrict__ lcol, const int64_t* __restrict__ work_off,
                         const int32_t* __restrict__ np, T* work) {
  COUNT_LAUNCH();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
    int v = omega[k], i = pos_sub[k];
    int a = (int)(k - sub_off[i]);
    T* row = work + work_off[i] + (int64_t)a * np[i];
    int64_t e0 = ent_off[k];
    int b = rp[v], e = rp[v + 1];
    const double sv = ds[v];
    for (int t = 0; t < e - b; ++t) {
      int lc = lcol[e0 + t];
      if (lc >= 0) row[lc] = (T)(val[b + t] * sv * ds[ci[b + t]]);
    }
  }
}

template <typename T>
__device__ __forceinline__ bool pivot_ok(T piv, bool spd) {
  return isfinite((double)piv) && (spd ? piv > T(0) : piv != T(0));
}

// One block per subdomain; the matrix lives in global memory (L2-resident
// for the active tiles), pivot block and panel chunks in shared memory.
template <typename T, bool SPD>
__global__ void __launch_bounds__(NT) k_sweep(T* __restrict__ work, const int64_t* __restrict__ work_off,
                                              const int32_t* __restrict__ np_arr, const int32_t* __restrict__ n_arr,
                                              const int32_t* __restrict__ m_arr, const int32_t* __restrict__ p_arr,
                                              T* __restrict__ XpT, const int64_t* __restrict__ xs_off,
                                              T* __restrict__ Sout, const int64_t* __restrict__ s_off,
                                              int32_t* err) {
  COUNT_LAUNCH();
  __shared__ T P[KB][KB + 1];
  __shared__ T bufA[64][KB + 1];
  __shared__ T bufB[KB][64 + 1];
  __shared__ int bad;
  const int i = blockIdx.x;
  const int n = n_arr[i], m = m_arr[i], p = p_arr[i], ld = np_arr[i];
  T* M = work + work_off[i];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  if (tid == 0) bad = 0;
  int k0 = 0;
  while (k0 < n) {
    const int lim = k0 < m ? m : n;
    const int kb = min(KB, lim - k0);
    const int k1 = k0 + kb;
    // ---- 1. invert the pivot block in shared memory (unblocked Gauss-Jordan)
    __syncthreads();
    for (int idx = tid; idx < kb * kb; idx += NT) {
      int r = idx / kb, c = idx % kb;
      P[r][c] = M[(int64_t)(k0 + r) * ld + k0 + c];
    }
    __syncthreads();
    for (int t = 0; t < kb; ++t) {
      T piv = P[t][t];
      if (!pivot_ok(piv, SPD)) {
        if (tid == 0) bad = 1;
      }
      __syncthreads();
      if (bad) break;
      T inv = T(1) / piv;
      for (int idx = tid; idx < kb * kb; idx += NT) {
        int r = idx / kb, c = idx % kb;
        if (r != t && c != t) P[r][c] -= P[r][t] * P[t][c] * inv;
      }
      __syncthreads();
      if (tid < kb && tid != t) P[t][tid] *= inv;
      if (tid >= 32 && tid - 32 < kb && tid - 32 != t) P[tid - 32][t] *= -inv;
      __syncthreads();
      if (tid == 0) P[t][t] = inv;
      __syncthreads();
    }
    if (bad) {
      if (tid == 0) atomicOr(err, SPD ? DERR_NOT_SPD : DERR_ZERO_PIVOT);
      return;
    }
    // ---- 2. row panel M_KJ <- P M_KJ (columns outside K)
    for (int c0 = 0; c0 < n; c0 += 64) {
      const int cw = min(64, n - c0);
      for (int idx = tid; idx < kb * 64; idx += NT) {
        int t = idx >> 6, c = idx & 63;
        bufB[t][c] = c < cw ? M[(int64_t)(k0 + t) * ld + c0 + c] : T(0);
      }
      __syncthreads();
      for (int idx = tid; idx < kb * 64; idx += NT) {
        int t = idx >> 6, c = idx & 63;
        int gc = c0 + c;
        if (c < cw && (gc < k0 || gc >= k1)) {
          T acc = 0;
          for (int u = 0; u < kb; ++u) acc += P[t][u] * bufB[u][c];
          M[(int64_t)(k0 + t) * ld + gc] = acc;
        }
      }
      __syncthreads();
    }
    // ---- 3. rank-kb update of the rest: M_JJ -= M_JK M_KJ (new row panel)
    for (int r0 = 0; r0 < n; r0 += 64) {
      const int rw = min(64, n - r0);
      for (int idx = tid; idx < 64 * KB; idx += NT) {
        int r = idx / KB, t = idx % KB;
        bufA[r][t] = (r < rw && t < kb) ? M[(int64_t)(r0 + r) * ld + k0 + t] : T(0);
      }
      for (int c0 = 0; c0 < n; c0 += 64) {
        const int cw = min(64, n - c0);
        __syncthreads();
        for (int idx = tid; idx < KB * 64; idx += NT) {
          int t = idx >> 6, c = idx & 63;
          bufB[t][c] = (t < kb && c < cw) ? M[(int64_t)(k0 + t) * ld + c0 + c] : T(0);
        }
        __syncthreads();
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = 0;
        for (int t = 0; t < kb; ++t) {
          T av[4], bv[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) av[a] = bufA[ty + 16 * a][t];
#pragma unroll
          for (int b = 0; b < 4; ++b) bv[b] = bufB[t][tx + 16 * b];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          int r = ty + 16 * a, gr = r0 + r;
          if (r >= rw || (gr >= k0 && gr < k1)) continue;
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            int c = tx + 16 * b, gc = c0 + c;
            if (c >= cw || (gc >= k0 && gc < k1)) continue;
            M[(int64_t)gr * ld + gc] -= acc[a][b];
          }
        }
      }
      __syncthreads();
    }
    // ---- 4. column panel M_JK <- -M_JK P (rows outside K)
    for (int r0 = 0; r0 < n; r0 += 64) {
      const int rw = min(64, n - r0);
      __syncthreads();
      for (int idx = tid; idx < 64 * KB; idx += NT) {
        int r = idx / KB, t = idx % KB;
        bufA[r][t] = (r < rw && t < kb) ? M[(int64_t)(r0 + r) * ld + k0 + t] : T(0);
      }
      __syncthreads();
      for (int idx = tid; idx < 64 * KB; idx += NT) {
        int r = idx / KB, t = idx % KB;
        int gr = r0 + r;
        if (r < rw && t < kb && (gr < k0 || gr >= k1)) {
          T acc = 0;
          for (int u = 0; u < kb; ++u) acc += bufA[r][u] * P[u][t];
          M[(int64_t)gr * ld + k0 + t] = -acc;
        }
      }
    }
    __syncthreads();
    // ---- 5. pivot block <- its inverse
    for (int idx = tid; idx < kb * kb; idx += NT) {
      int r = idx / kb, c = idx % kb;
      M[(int64_t)(k0 + r) * ld + k0 + c] = P[r][c];
    }
    __syncthreads();
    // ---- midpoint snapshot: X_p^T = -(B^{-1}C)[:p]^T and S
    if (k1 == m && m < n) {
      const int g = n - m;
      T* X = XpT + xs_off[i];
      for (int r0 = 0; r0 < p; r0 += 64) {
        for (int q0 = 0; q0 < g; q0 += KB) {
          __syncthreads();
          for (int idx = tid; idx < 64 * KB; idx += NT) {
            int r = idx / KB, q = idx % KB;
            bufA[r][q] = (r0 + r < p && q0 + q < g) ? M[(int64_t)(r0 + r) * ld + m + q0 + q] : T(0);
          }
          __syncthreads();
          for (int idx = tid; idx < 64 * KB; idx += NT) {
            int q = idx >> 6, r = idx & 63;
            if (r0 + r < p && q0 + q < g) X[(int64_t)(q0 + q) * p + r0 + r] = -bufA[r][q];
          }
        }
      }
      T* Sg = Sout + s_off[i];
      for (int64_t idx = tid; idx < (int64_t)g * g; idx += NT) {
        int a = (int)(idx / g), b = (int)(idx % g);
        Sg[idx] = M[(int64_t)(m + a) * ld + m + b];
      }
      __syncthreads();
    }
    k0 = k1;
  }
}

// Copy A_ii^{-1} into TILE x TILE tiles: SPD keeps the lower tiles (I >= J),
// the general path keeps all of them.  One block per tile.
template <typename T>
__global__ void __launch_bounds__(NT) k_pack(const T* __restrict__ work, const int64_t* __restrict__ work_off,
                                             const int32_t* __restrict__ np, const int32_t* __restrict__ n_arr,
                                             const int4* __restrict__ desc, int64_t ntiles, T* __restrict__ tiles) {
  COUNT_LAUNCH();
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int4 d = desc[t];
    int i = d.x, I = d.y, J = d.z;
    int n = n_arr[i], ld = np[i];
    const T* M = work + work_off[i];
    T* out = tiles + t * (TILE * TILE);
    for (int idx = threadIdx.x; idx < TILE * TILE; idx += NT) {
      int r = idx / TILE, c = idx % TILE;
      int gr = I * TILE + r, gc = J * TILE + c;
      out[idx] = (gr < n && gc < n) ? M[(int64_t)gr * ld + gc] : T(0);
    }
  }
}

template <typename T>
void run_local(Handle& h, cudaStream_t s) {
  const int N = h.N;
  Dense& dn = h.dn;
  Overlap& ov = h.ov;
  DevMem& mem = h.mem;
  const bool spd = h.opt.spd != 0;
  // -- sizes and offsets
  dn.h_np.resize(N); dn.h_work_off.resize(N); dn.h_xs_off.resize(N); dn.h_s_off.resize(N);
  dn.h_nt.resize(N); dn.h_tile_off.resize(N + 1); dn.h_part_off.resize(N + 1);
  int64_t w = 0, xs = 0, ss = 0, tl = 0, pt = 0;
  std::vector<int4> desc;
  for (int i = 0; i < N; ++i) {
    int ni = h.h_n[i];
    int np = (int)round_up(ni, TILE);
    int nt = np / TILE;
    dn.h_np[i] = np;
    dn.h_nt[i] = nt;
    dn.h_work_off[i] = w;
    w += (int64_t)np * np;
    dn.h_xs_off[i] = xs;
    xs += (int64_t)h.h_g[i] * h.h_p[i];
    dn.h_s_off[i] = ss;
    ss += (int64_t)h.h_g[i] * h.h_g[i];
    dn.h_tile_off[i] = tl;
    for (int I = 0; I < nt; ++I)
      for (int J = 0; J < (spd ? I + 1 : nt); ++J) desc.push_back(make_int4(i, I, J, 0));
    tl = (int64_t)desc.size();
    dn.h_part_off[i] = pt;
    pt += (int64_t)nt * nt * TILE;
  }
  dn.h_tile_off[N] = tl;
  dn.h_part_off[N] = pt;
  dn.n_work = w; dn.n_xs = xs; dn.n_s = ss; dn.n_tiles = tl; dn.n_part = pt;
  dn.np = mem.alloc<int32_t>(N);
  dn.nt = mem.alloc<int32_t>(N);
  dn.work_off = mem.alloc<int64_t>(N);
  dn.xs_off = mem.alloc<int64_t>(N);
  dn.s_off = mem.alloc<int64_t>(N);
  dn.tile_off = mem.alloc<int64_t>(N + 1);
  dn.part_off = mem.alloc<int64_t>(N + 1);
  dn.tile_desc = mem.alloc<int4>(tl);
  int32_t* d_n = mem.alloc<int32_t>(N);
  int32_t* d_m = mem.alloc<int32_t>(N);
  int32_t* d_p = mem.alloc<int32_t>(N);
  CK(cudaMemcpyAsync(dn.np, dn.h_np.data(), 4 * N, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dn.nt, dn.h_nt.data(), 4 * N, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dn.work_off, dn.h_work_off.data(), 8 * N, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dn.xs_off, dn.h_xs_off.data(), 8 * N, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dn.s_off, dn.h_s_off.data(), 8 * N, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dn.tile_off, dn.h_tile_off.data(), 8 * (N + 1), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dn.part_off, dn.h_part_off.data(), 8 * (N + 1), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dn.tile_desc, desc.data(), sizeof(int4) * tl, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_n, h.h_n.data(), 4 * N, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_m, h.h_m.data(), 4 * N, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_p, h.h_p.data(), 4 * N, cudaMemcpyHostToDevice, s));
  T* work = mem.alloc<T>(w);
  dn.work = work;
  dn.XpT = mem.alloc<T>(xs);
  dn.S = mem.alloc<T>(ss);
  dn.tiles = mem.alloc<T>(tl * TILE * TILE);
  dn.partials = mem.alloc<T>(pt);
  dn.ypos = mem.alloc<double>(ov.sum_n);
  h.dev_n = d_n; h.dev_m = d_m; h.dev_p = d_p;
  // -- gather A_ii
  CK(cudaMemsetAsync(work, 0, sizeof(T) * w, s));
  if (h.events) CK(cudaEventRecord(h.ev[2], s));
  unsigned gg = (unsigned)std::min<int64_t>(ceil_div(ov.sum_n, NT), 152 * 16);
  k_gather<T><<<gg, NT, 0, s>>>(ov.omega, ov.sum_n, ov.pos_sub, ov.sub_off, h.row_ptr, h.col_idx, h.val,
                                h.dscale, ov.ent_off,
                                ov.lcol, dn.work_off, dn.np, work);
  CK_LAUNCH("gather A_ii");
  if (h.events) CK(cudaEventRecord(h.ev[3], s));
  // -- sweep
  if (spd)
    k_sweep<T, true><<<N, NT, 0, s>>>(work, dn.work_off, dn.np, d_n, d_m, d_p, (T*)dn.XpT, dn.xs_off,
                                      (T*)dn.S, dn.s_off, dn.err);
  else
    k_sweep<T, false><<<N, NT, 0, s>>>(work, dn.work_off, dn.np, d_n, d_m, d_p, (T*)dn.XpT, dn.xs_off,
                                       (T*)dn.S, dn.s_off, dn.err);
  CK_LAUNCH("local sweep");
  if (h.events) CK(cudaEventRecord(h.ev[4], s));
  // -- pack the apply tiles
  unsigned gp = (unsigned)std::min<int64_t>(std::max<int64_t>(tl, 1), 152 * 8);
  k_pack<T><<<gp, NT, 0, s>>>(work, dn.work_off, dn.np, d_n, dn.tile_desc, tl, (T*)dn.tiles);
  CK_LAUNCH("pack tiles");
  if (h.events) CK(cudaEventRecord(h.ev[5], s));
}

}  // namespace

void build_local(Handle& h, cudaStream_t s) {
  if (h.fp32) run_local<float>(h, s); else run_local<double>(h, s);
  check_device_error(h, s, "local inverse");
}

}  // namespace asmgpu
