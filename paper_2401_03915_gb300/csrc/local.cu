// Local dense stage: gather A_ii out of CSR A (Section 2.3), factor it, and
// pack the result into the tiles the apply streams.
//
// SPD A: blocked Cholesky and triangular inverse W = L^{-1} (FP64: k_chol_trtri;
// single precision: factor_spd_levels, tensor-core tile jobs by levels); the apply
// multiplies by W^T W and the eigen stage reads the block
// W[Gamma_delta, I_i].  General A: blocked Gauss-Jordan sweep (k_sweep).
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
//     [ B^{-1}                 B^{-1} C                  ]
//     [ -A_{Gamma,Omega'} B^{-1}   G - A_{Gamma,Omega'} B^{-1} C ]
// with B = A_{Omega_{1:delta-1}}, C = A_{Omega_{1:delta-1}, Gamma_delta} and
// G = A_{Gamma_delta, Gamma_delta}: the block -B^{-1} C of the harmonic
// operator Pi_i (eq. HOp).  Its first |I_i| rows X_p = -(B^{-1}C)[:p] are
// copied out; the sweep then continues over Gamma_delta and leaves A_ii^{-1}.
#include <algorithm>
#include <mutex>

#include <cuda_fp16.h>

#include "handle.cuh"
#include "tcgemm.cuh"

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
      __syncthreads();
    }
    k0 = k1;
  }
}

// SPD local factor in FP64: blocked Cholesky A^_ii = L L^T (right-looking)
// followed by the blocked triangular inverse W = L^{-1}, both in place in the
// lower triangle, one block per subdomain, 64 x 64 blocks.  The apply
// multiplies by W^T W = A^_ii^{-1}: symmetric positive definite for any
// rounding of W, and accurate to about cond(A^_ii) * eps (an explicitly
// inverted A^_ii^{-1} would only be accurate to cond^2 * eps).  Dinv receives
// the inverses of the diagonal blocks of L (which are the diagonal blocks of
// W).  The single-precision factor runs the same steps by levels of tile
// products on the tensor cores (factor_spd_levels below).
// 64 x 64 x 64 block products acc (+)= Am * (btrans ? Bm^T : Bm) from shared
// memory ([64][65] layout) on CUDA-core FMAs, thread (tx, ty) owning rows
// ty + 16a, columns tx + 16b.
template <typename T>
struct BlockAcc {
  T v[4][4];
};

template <typename T>
__device__ __forceinline__ void acc_zero(BlockAcc<T>& acc) {
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc.v[a][b] = T(0);
}

__device__ __forceinline__ void acc_mma(BlockAcc<double>& acc, const double (*Am)[TILE + 1],
                                        const double (*Bm)[TILE + 1], bool btrans) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int q = 0; q < TILE; ++q) {
    double av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = Am[ty + 16 * a][q];
#pragma unroll
    for (int b = 0; b < 4; ++b) bv[b] = btrans ? Bm[tx + 16 * b][q] : Bm[q][tx + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc.v[a][b] += av[a] * bv[b];
  }
}

// f(row, col, value) for every element of the thread's share of the block
template <typename F>
__device__ __forceinline__ void acc_for_each(const BlockAcc<double>& acc, F&& f) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) f(ty + 16 * a, tx + 16 * b, acc.v[a][b]);
}
template <typename T>
__global__ void __launch_bounds__(NT) k_chol_trtri(T* __restrict__ work, const int64_t* __restrict__ work_off,
                                                   const int32_t* __restrict__ np_arr,
                                                   const int32_t* __restrict__ n_arr, T* __restrict__ dinv_all,
                                                   const int64_t* __restrict__ dinv_off, int32_t* err,
                                                   int8_t* __restrict__ sym, double sym_max_ratio) {
  COUNT_LAUNCH();
  extern __shared__ unsigned char smraw[];
  T (*Dm)[TILE + 1] = reinterpret_cast<T (*)[TILE + 1]>(smraw);
  T (*Xm)[TILE + 1] = Dm + TILE;
  T (*Ym)[TILE + 1] = Xm + TILE;
  __shared__ int bad;
  __shared__ double piv_min, piv_max;
  const int i = blockIdx.x;
  const int n = n_arr[i], ld = np_arr[i];
  T* M = work + work_off[i];
  T* Dinv = dinv_all + dinv_off[i];
  const int nt = (n + TILE - 1) / TILE;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  auto blk = [&](int rb, int cb) { return M + (int64_t)rb * TILE * ld + cb * TILE; };
  auto load = [&](T (*S)[TILE + 1], int rb, int cb) {
    const T* B = blk(rb, cb);
    const int rw = min(TILE, n - rb * TILE), cw = min(TILE, n - cb * TILE);
    for (int idx = tid; idx < TILE * TILE; idx += NT) {
      int r = idx / TILE, c = idx % TILE;
      S[r][c] = (r < rw && c < cw) ? B[(int64_t)r * ld + c] : T(0);
    }
  };
  if (tid == 0) { bad = 0; piv_min = 3.0e300; piv_max = 0; }
  // ---------------- phase 1: Cholesky
  for (int kb = 0; kb < nt; ++kb) {
    const int kw = min(TILE, n - kb * TILE);
    __syncthreads();
    {
      const T* B = blk(kb, kb);
      for (int idx = tid; idx < TILE * TILE; idx += NT) {
        int r = idx / TILE, c = idx % TILE;
        T v = (r < kw && c < kw) ? B[(int64_t)max(r, c) * ld + min(r, c)] : (r == c ? T(1) : T(0));
        Dm[r][c] = v;
      }
    }
    __syncthreads();
    for (int j = 0; j < TILE; ++j) {
      if (tid == 0) {
        T d = Dm[j][j];
        if (!(d > T(0)) || !isfinite((double)d)) { bad = 1; d = T(1); }
        if (j < kw) { piv_min = fmin(piv_min, (double)d); piv_max = fmax(piv_max, (double)d); }
        Dm[j][j] = sqrt(d);
      }
      __syncthreads();
      if (bad) break;
      for (int r = j + 1 + tid; r < TILE; r += NT) Dm[r][j] /= Dm[j][j];
      __syncthreads();
      for (int idx = tid; idx < TILE * TILE; idx += NT) {
        int r = idx / TILE, c = idx % TILE;
        if (c > j && r >= c) Dm[r][c] -= Dm[r][j] * Dm[c][j];
      }
      __syncthreads();
    }
    if (bad) {
      if (tid == 0) atomicOr(err, DERR_NOT_SPD);
      return;
    }
    // inverse of the lower diagonal block (column c by thread c)
    if (tid < TILE) {
      const int c = tid;
      for (int r = 0; r < c; ++r) Xm[r][c] = 0;
      for (int r = c; r < TILE; ++r) {
        T v = r == c ? T(1) : T(0);
        for (int t = c; t < r; ++t) v -= Dm[r][t] * Xm[t][c];
        Xm[r][c] = v / Dm[r][r];
      }
    }
    __syncthreads();
    {
      T* B = blk(kb, kb);
      T* Dv = Dinv + (int64_t)kb * TILE * TILE;
      for (int idx = tid; idx < TILE * TILE; idx += NT) {
        int r = idx / TILE, c = idx % TILE;
        if (r < kw && c < kw && c <= r) B[(int64_t)r * ld + c] = Dm[r][c];
        Dv[idx] = Xm[r][c];
      }
    }
    // panel: L_rk = A_rk Dinv^T
    for (int rb = kb + 1; rb < nt; ++rb) {
      __syncthreads();
      load(Ym, rb, kb);
      __syncthreads();
      BlockAcc<T> acc;
      acc_zero(acc);
      acc_mma(acc, Ym, Xm, true);
      const int rw = min(TILE, n - rb * TILE);
      T* B = blk(rb, kb);
      acc_for_each(acc, [&](int r, int c, T v) {
        if (r < rw && c < kw) B[(int64_t)r * ld + c] = v;
      });
    }
    // trailing update: A_rc -= L_rk L_ck^T, c <= r
    for (int rb = kb + 1; rb < nt; ++rb) {
      __syncthreads();
      load(Ym, rb, kb);
      for (int cb = kb + 1; cb <= rb; ++cb) {
        __syncthreads();
        load(Dm, cb, kb);
        __syncthreads();
        BlockAcc<T> acc;
        acc_zero(acc);
        acc_mma(acc, Ym, Dm, true);
        const int rw = min(TILE, n - rb * TILE), cw = min(TILE, n - cb * TILE);
        T* B = blk(rb, cb);
        acc_for_each(acc, [&](int r, int c, T v) {
          if (r < rw && c < cw && (cb < rb || c <= r)) B[(int64_t)r * ld + c] -= v;
        });
      }
    }
  }
  // ---------------- phase 2: W = L^{-1}, block column by block column
  for (int jb = 0; jb < nt; ++jb) {
    const int jw = min(TILE, n - jb * TILE);
    __syncthreads();
    {
      T* B = blk(jb, jb);
      const T* Dv = Dinv + (int64_t)jb * TILE * TILE;
      for (int idx = tid; idx < TILE * TILE; idx += NT) {
        int r = idx / TILE, c = idx % TILE;
        if (r < jw && c < jw) B[(int64_t)r * ld + c] = c <= r ? Dv[idx] : T(0);
      }
    }
    for (int ib = jb + 1; ib < nt; ++ib) {
      BlockAcc<T> acc;
      acc_zero(acc);
      for (int kb = jb; kb < ib; ++kb) {
        __syncthreads();
        load(Ym, ib, kb);   // L_ik (kb >= jb: not yet overwritten)
        load(Xm, kb, jb);   // W_kj (kb < ib: already computed)
        __syncthreads();
        acc_mma(acc, Ym, Xm, false);
      }
      __syncthreads();
      // W_ij = -Dinv_i acc
      acc_for_each(acc, [&](int r, int c, T v) { Xm[r][c] = v; });
      {
        const T* Dv = Dinv + (int64_t)ib * TILE * TILE;
        for (int idx = tid; idx < TILE * TILE; idx += NT) Ym[idx / TILE][idx % TILE] = Dv[idx];
      }
      __syncthreads();
      BlockAcc<T> w;
      acc_zero(w);
      acc_mma(w, Ym, Xm, false);
      const int rw = min(TILE, n - ib * TILE);
      T* B = blk(ib, jb);
      acc_for_each(w, [&](int r, int c, T v) {
        if (r < rw && c < jw) B[(int64_t)r * ld + c] = -v;
      });
    }
  }
  // The pivot ratio max/min of the Cholesky bounds cond(A^_ii) from below
  // (a positive ratio asks for the explicit-inverse decision; FP64 passes 0).
  if (tid == 0) sym[i] = (sym_max_ratio > 0 && piv_max <= sym_max_ratio * piv_min) ? 1 : 0;
}

// ---------------------------------------------------------------------------
// Single-precision SPD factor by levels.  Level kb of the Cholesky:
//   (1) C_rk = A_rk - sum_{j<kb} L_rj L_kj^T for every row block r >= kb
//       (tile jobs, one per (subdomain, r));
//   (2) the 64 x 64 diagonal block: C_kk = L_kk L_kk^T and Dinv_kk = L_kk^{-1}
//       (k_diag_chol, one block per subdomain);
//   (3) L_rk = C_rk Dinv_kk^T for r > kb (tile jobs).
// Then W = L^{-1} by row levels i: T_ij = sum_{k=j}^{i-1} L_ik W_kj for every
// j < i, W_ij = -Dinv_i T_ij (W_jj = Dinv_j), and for the subdomains that get
// the explicit inverse, S_IJ = sum_{K >= I} W_KI^T W_KJ.  Every step but (2)
// is a batch of 64 x 64 tile products on the tensor cores (tcgemm.cu).  L_kk
// itself is never read again: the diagonal tile of the working matrix
// receives W_kk = Dinv_kk (lower triangle, zero above and in the padding).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_diag_chol(int kb, const int32_t* __restrict__ subs, float* __restrict__ work,
                                                  const int64_t* __restrict__ work_off,
                                                  const int32_t* __restrict__ np_arr, const int32_t* __restrict__ n_arr,
                                                  float* __restrict__ dinv_all, const int64_t* __restrict__ dinv_off,
                                                  double* __restrict__ piv_lo, double* __restrict__ piv_hi,
                                                  int32_t* err) {
  COUNT_LAUNCH();
  __shared__ float Dm[TILE][TILE + 1];
  __shared__ float Xm[TILE][TILE + 1];
  __shared__ int bad;
  __shared__ double pmin, pmax;
  const int i = subs[blockIdx.x];
  const int n = n_arr[i], ld = np_arr[i];
  const int kw = min(TILE, n - kb * TILE);
  float* B = work + work_off[i] + (int64_t)kb * TILE * ld + kb * TILE;
  const int tid = threadIdx.x;
  if (tid == 0) {
    bad = 0;
    pmin = kb == 0 ? 3.0e300 : piv_lo[i];
    pmax = kb == 0 ? 0.0 : piv_hi[i];
  }
  for (int idx = tid; idx < TILE * TILE; idx += NT) {
    const int r = idx / TILE, c = idx % TILE;
    Dm[r][c] = (r < kw && c < kw) ? B[(int64_t)max(r, c) * ld + min(r, c)] : (r == c ? 1.f : 0.f);
  }
  __syncthreads();
  // outer-product form with the unscaled pivot column (one barrier per
  // column): a_rc -= a_rj a_cj / a_jj for r >= c > j, the columns scaled by
  // 1 / sqrt(a_jj) at the end; a non-positive pivot is flagged and taken as 1
  for (int j = 0; j < TILE; ++j) {
    float d = Dm[j][j];
    const bool ok = d > 0.f && isfinite(d);
    if (!ok) d = 1.f;
    if (tid == 0) {
      if (!ok) bad = 1;
      if (j < kw) { pmin = fmin(pmin, (double)d); pmax = fmax(pmax, (double)d); }
    }
    const float inv = 1.f / d;
    const int m = TILE - 1 - j;  // trailing size
    for (int idx = tid; idx < m * m; idx += NT) {
      const int r = j + 1 + idx / m, c = j + 1 + idx % m;
      if (r >= c) Dm[r][c] -= Dm[r][j] * (Dm[c][j] * inv);
    }
    __syncthreads();
  }
  for (int idx = tid; idx < TILE * TILE; idx += NT) {
    const int r = idx / TILE, c = idx % TILE;
    if (r > c) {
      float d = Dm[c][c];
      if (!(d > 0.f && isfinite(d))) d = 1.f;
      Xm[r][c] = Dm[r][c] / sqrtf(d);
    }
  }
  __syncthreads();
  for (int idx = tid; idx < TILE * TILE; idx += NT) {
    const int r = idx / TILE, c = idx % TILE;
    if (r > c) Dm[r][c] = Xm[r][c];
    else if (r == c) {
      float d = Dm[r][r];
      if (!(d > 0.f && isfinite(d))) d = 1.f;
      Dm[r][r] = sqrtf(d);
    }
  }
  __syncthreads();
  // inverse of the lower diagonal block (column c by thread c)
  if (tid < TILE) {
    const int c = tid;
    for (int r = 0; r < c; ++r) Xm[r][c] = 0.f;
    for (int r = c; r < TILE; ++r) {
      float v = r == c ? 1.f : 0.f;
      for (int t = c; t < r; ++t) v -= Dm[r][t] * Xm[t][c];
      Xm[r][c] = v / Dm[r][r];
    }
  }
  __syncthreads();
  float* Dv = dinv_all + dinv_off[i] + (int64_t)kb * TILE * TILE;
  for (int idx = tid; idx < TILE * TILE; idx += NT) {
    const int r = idx / TILE, c = idx % TILE;
    Dv[idx] = Xm[r][c];
    B[(int64_t)r * ld + c] = (r < kw && c < kw && c <= r) ? Xm[r][c] : 0.f;
  }
  if (tid == 0) {
    if (bad) atomicOr(err, DERR_NOT_SPD);
    piv_lo[i] = pmin;
    piv_hi[i] = pmax;
  }
}

// The pivot ratio max/min of the Cholesky bounds cond(A^_ii) from below;
// within ratio the subdomain gets the explicit inverse S = W^T W; past it, it
// keeps the two-pass W^T W form, which stays SPD whatever the rounding (an
// explicit FP32 inverse would not).
__global__ void k_sym_decide(int N, const double* __restrict__ piv_lo, const double* __restrict__ piv_hi,
                             double ratio, int8_t* __restrict__ sym) {
  COUNT_LAUNCH();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) sym[i] = (ratio > 0 && piv_hi[i] <= ratio * piv_lo[i]) ? 1 : 0;
}

// The job descriptors are written straight into a pinned host buffer that
// persists across setups (grown as needed), then copied in one transfer.
std::mutex g_jobs_mutex;
TcJob* g_jobs_pin = nullptr;
size_t g_jobs_cap = 0;

void factor_spd_levels(Handle& h, float* work, const int32_t* d_n, double ratio, cudaStream_t s) {
  const int N = h.N;
  Dense& dn = h.dn;
  DevMem& mem = h.mem;
  const int64_t T2 = (int64_t)TILE * TILE;
  int ntmax = 0;
  size_t bound = 0;  // at most nt^2 updates + panels, nt^2 inverse jobs, nt (nt + 1) / 2 W^T W jobs
  for (int i = 0; i < N; ++i) {
    ntmax = std::max(ntmax, dn.h_nt[i]);
    bound += 3 * (size_t)dn.h_nt[i] * dn.h_nt[i] + 2 * (size_t)dn.h_nt[i] + 1;
  }
  std::lock_guard<std::mutex> jobs_lock(g_jobs_mutex);
  if (bound > g_jobs_cap) {
    if (g_jobs_pin) CK(cudaFreeHost(g_jobs_pin));
    g_jobs_pin = nullptr;
    CK(cudaMallocHost(&g_jobs_pin, sizeof(TcJob) * bound));
    g_jobs_cap = bound;
  }
  struct PinnedJobs {
    TcJob* p;
    size_t n, cap;
    size_t size() const { return n; }
    void push_back(const TcJob& J) {
      if (n >= cap) fail(ASM_ERR_CUDA, "tile job bound exceeded");
      p[n++] = J;
    }
    bool empty() const { return n == 0; }
    const TcJob* data() const { return p; }
  };
  // one launch of tile jobs: [first, first + count) of the job array and the
  // bases it reads and writes (0 work, 1 dinv, 2 scratch, 3 apply tiles)
  struct Step {
    int kind;  // 0 tile jobs, 1 diagonal blocks of level kb, 2 explicit-inverse decision
    int64_t first, count;
    int a, b, c, kb;
  };
  PinnedJobs jobs{g_jobs_pin, 0, g_jobs_cap};
  std::vector<int32_t> subs;
  std::vector<Step> steps;
  auto tile_at = [&](int i, int r, int c) { return dn.h_work_off[i] + (int64_t)r * TILE * dn.h_np[i] + c * TILE; };
  auto job = [&](int64_t a0, int64_t a_step, int lda, int64_t b0, int64_t b_step, int ldb, int64_t c0, int ldc,
                 int nprod, int flags, int sub) {
    TcJob J{};
    J.a0 = a0; J.a_step = a_step; J.lda = lda;
    J.b0 = b0; J.b_step = b_step; J.ldb = ldb;
    J.c_in = c0; J.c_out = c0; J.ldc_in = ldc; J.ldc_out = ldc;
    J.nprod = nprod; J.flags = flags; J.sub = sub;
    jobs.push_back(J);
  };
  auto close = [&](int64_t first, int a, int b, int c) {
    if ((int64_t)jobs.size() > first) steps.push_back({0, first, (int64_t)jobs.size() - first, a, b, c, 0});
  };
  // Cholesky levels
  for (int kb = 0; kb < ntmax; ++kb) {
    int64_t f = (int64_t)jobs.size();
    if (kb > 0) {
      for (int i = 0; i < N; ++i) {
        const int nt = dn.h_nt[i], ld = dn.h_np[i];
        if (nt <= kb) continue;
        for (int r = kb; r < nt; ++r)
          job(tile_at(i, r, 0), TILE, ld, tile_at(i, kb, 0), TILE, ld, tile_at(i, r, kb), ld, kb,
              TCF_NEG | TCF_BETA, i);
      }
      close(f, 0, 0, 0);
    }
    const int64_t s0 = (int64_t)subs.size();
    for (int i = 0; i < N; ++i)
      if (dn.h_nt[i] > kb) subs.push_back(i);
    steps.push_back({1, s0, (int64_t)subs.size() - s0, 0, 0, 0, kb});
    f = (int64_t)jobs.size();
    for (int i = 0; i < N; ++i) {
      const int nt = dn.h_nt[i], ld = dn.h_np[i];
      for (int r = kb + 1; r < nt; ++r)
        job(tile_at(i, r, kb), 0, ld, dn.h_s_off[i] + kb * T2, 0, TILE, tile_at(i, r, kb), ld, 1, 0, i);
    }
    close(f, 0, 1, 0);
  }
  // the pivots are known: the explicit-inverse decision (read by the W^T W jobs)
  steps.push_back({2, 0, 0, 0, 0, 0, 0});
  // triangular inverse by row levels; T_ij in the scratch, then W_ij
  int64_t scratch_tiles = 0;
  for (int il = 1; il < ntmax; ++il) {
    const int64_t f = (int64_t)jobs.size();
    int64_t q = 0;
    for (int i = 0; i < N; ++i) {
      const int ld = dn.h_np[i];
      if (dn.h_nt[i] <= il) continue;
      for (int j = 0; j < il; ++j, ++q)
        job(tile_at(i, il, j), TILE, ld, tile_at(i, j, j), (int64_t)TILE * ld, ld, q * T2, TILE, il - j, TCF_BT, i);
    }
    close(f, 0, 0, 2);
    scratch_tiles = std::max(scratch_tiles, q);
    const int64_t g = (int64_t)jobs.size();
    q = 0;
    for (int i = 0; i < N; ++i) {
      const int ld = dn.h_np[i];
      if (dn.h_nt[i] <= il) continue;
      for (int j = 0; j < il; ++j, ++q) {
        TcJob J{};
        J.a0 = dn.h_s_off[i] + il * T2; J.lda = TILE;
        J.b0 = q * T2; J.ldb = TILE;
        J.c_out = tile_at(i, il, j); J.ldc_out = ld; J.ldc_in = ld;
        J.nprod = 1; J.flags = TCF_BT | TCF_NEG; J.sub = i;
        jobs.push_back(J);
      }
    }
    close(g, 1, 2, 0);
  }
  // S = W^T W for the explicit-inverse subdomains, into the apply tiles
  {
    const int64_t f = (int64_t)jobs.size();
    for (int i = 0; i < N; ++i) {
      const int nt = dn.h_nt[i], ld = dn.h_np[i];
      for (int I = 0; I < nt; ++I)
        for (int J = 0; J <= I; ++J) {
          TcJob Jb{};
          Jb.a0 = tile_at(i, I, I); Jb.a_step = (int64_t)TILE * ld; Jb.lda = ld;
          Jb.b0 = tile_at(i, I, J); Jb.b_step = (int64_t)TILE * ld; Jb.ldb = ld;
          Jb.c_out = (dn.h_tile_off[i] + (int64_t)I * (I + 1) / 2 + J) * T2; Jb.ldc_out = TILE; Jb.ldc_in = TILE;
          Jb.nprod = nt - I; Jb.flags = TCF_AT | TCF_BT | TCF_SYMONLY; Jb.sub = i;
          jobs.push_back(Jb);
        }
    }
    close(f, 0, 0, 3);
  }
  TcJob* d_jobs = mem.alloc<TcJob>(std::max<size_t>(jobs.size(), 1));
  int32_t* d_subs = mem.alloc<int32_t>(std::max<size_t>(subs.size(), 1));
  float* scratch = mem.alloc<float>(std::max<int64_t>(scratch_tiles, 1) * T2);
  double* piv = mem.alloc<double>(2 * N);
  if (!jobs.empty()) CK(cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(TcJob) * jobs.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_subs, subs.data(), sizeof(int32_t) * subs.size(), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));  // the pinned buffer is reused by the next setup
  float* bases[4] = {work, (float*)dn.dinv, scratch, (float*)dn.tiles};
  for (const Step& st : steps) {
    if (st.kind == 1) {
      k_diag_chol<<<(unsigned)st.count, NT, 0, s>>>(st.kb, d_subs + st.first, work, dn.work_off, dn.np, d_n,
                                                    (float*)dn.dinv, dn.dinv_off, piv, piv + N, dn.err);
      CK_LAUNCH("diagonal blocks of the local Cholesky");
    } else if (st.kind == 2) {
      k_sym_decide<<<(unsigned)ceil_div(N, 256), 256, 0, s>>>(N, piv, piv + N, ratio, dn.sym);
      CK_LAUNCH("explicit-inverse decision");
    } else {
      tc_tiles(d_jobs + st.first, st.count, bases[st.a], bases[st.b], bases[st.c], bases[st.c], dn.sym, dn.err,
               h.num_sms, s);
    }
  }
}

// ---------------------------------------------------------------------------
// FP16 storage of the explicit inverses.  Rounding S_i to FP16 perturbs it
// by dS with ||dS||_2 <= ||dS||_inf <= 2^-11 ||S_i||_inf + n_i 2^-25 (normal
// and subnormal range), and lambda_min(S_i) = 1 / lambda_max(A^_ii) >=
// 1 / ||A^_ii||_inf; so (S_i + dS) A^_ii = I + dS A^_ii has its eigenvalues
// within 1 -+ ||dS|| ||A^_ii||_inf.  A subdomain is stored in FP16 when that
// bound is at most 1/4 (then also |S_ij| <= 512 / ||A^_ii||_inf: no overflow).
// All reductions run in a fixed order (the decision is reproducible).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// rmax[boff[i] + I] = max over the rows r of row block I of sum_j |S_rj|, from
// the stored lower tiles: rows of (I, J <= I) and columns of (K > I, I).
__global__ void __launch_bounds__(NT) k_s_rowsum(const float* __restrict__ tiles, const int64_t* __restrict__ tile_off,
                                                 const int32_t* __restrict__ nt_arr, const int2* __restrict__ items,
                                                 int nitems, const int64_t* __restrict__ boff,
                                                 float* __restrict__ rmax) {
  COUNT_LAUNCH();
  __shared__ float racc[TILE];
  __shared__ float part[NT / TILE][TILE];
  __shared__ float red[2];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int2 w = items[it];
    const int i = w.x, I = w.y, nt = nt_arr[i];
    const float* base = tiles + tile_off[i] * (int64_t)(TILE * TILE);
    if (tid < TILE) racc[tid] = 0.f;
    __syncthreads();
    for (int J = 0; J <= I; ++J) {
      const float* T0 = base + ((int64_t)I * (I + 1) / 2 + J) * (TILE * TILE);
      for (int r = wid; r < TILE; r += NT / 32) {
        float v = fabsf(T0[r * TILE + lane]) + fabsf(T0[r * TILE + lane + 32]);
        v = warp_sum(v);
        if (lane == 0) racc[r] += v;
      }
    }
    __syncthreads();
    for (int K = I + 1; K < nt; ++K) {
      const float* T0 = base + ((int64_t)K * (K + 1) / 2 + I) * (TILE * TILE);
      const int c = tid % TILE, g = tid / TILE;
      float v = 0.f;
      for (int k = g * (TILE * TILE / NT); k < (g + 1) * (TILE * TILE / NT); ++k) v += fabsf(T0[k * TILE + c]);
      part[g][c] = v;
      __syncthreads();
      if (tid < TILE) {
        float sm = racc[tid];
        for (int q = 0; q < NT / TILE; ++q) sm += part[q][tid];
        racc[tid] = sm;
      }
      __syncthreads();
    }
    if (tid < TILE) {
      const float m = warp_max_f(racc[tid]);
      if (lane == 0) red[wid] = m;
    }
    __syncthreads();
    if (tid == 0) rmax[boff[i] + I] = fmaxf(red[0], red[1]);
    __syncthreads();
  }
}

// amax[i] = ||A^_ii||_inf for the explicit-inverse subdomains (0 elsewhere)
__global__ void __launch_bounds__(NT) k_a_rowsum(const int32_t* __restrict__ sub_off, const int32_t* __restrict__ n_arr,
                                                 const int32_t* __restrict__ omega, const int64_t* __restrict__ ent_off,
                                                 const int32_t* __restrict__ lcol, const int32_t* __restrict__ rp,
                                                 const int32_t* __restrict__ ci, const double* __restrict__ val,
                                                 const double* __restrict__ ds, const int8_t* __restrict__ sym,
                                                 double* __restrict__ amax) {
  COUNT_LAUNCH();
  __shared__ double red[NT / 32];
  const int i = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  double m = 0;
  if (sym[i]) {
    const int n = n_arr[i], b0 = sub_off[i];
    for (int a = tid; a < n; a += NT) {
      const int v = omega[b0 + a];
      const double sv = ds[v];
      const int64_t e0 = ent_off[b0 + a];
      const int b = rp[v], e = rp[v + 1];
      double acc = 0;
      for (int q = 0; q < e - b; ++q)
        if (lcol[e0 + q] >= 0) acc += fabs(val[b + q] * sv * ds[ci[b + q]]);
      m = fmax(m, acc);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) red[wid] = m;
  __syncthreads();
  if (tid == 0) {
    double t = red[0];
    for (int q = 1; q < NT / 32; ++q) t = fmax(t, red[q]);
    amax[i] = t;
  }
}

__global__ void k_decide_s16(int N, const int8_t* __restrict__ sym, const int32_t* __restrict__ nt_arr,
                             const int32_t* __restrict__ n_arr, const int64_t* __restrict__ boff,
                             const float* __restrict__ rmax, const double* __restrict__ amax,
                             int8_t* __restrict__ s16) {
  COUNT_LAUNCH();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int8_t ok = 0;
  if (sym[i]) {
    double ms = 0;
    for (int I = 0; I < nt_arr[i]; ++I) ms = fmax(ms, (double)rmax[boff[i] + I]);
    const double bound = (ldexp(ms, -11) + n_arr[i] * ldexp(1.0, -25)) * amax[i];
    ok = isfinite(bound) && bound <= 0.25;
  }
  s16[i] = ok;
}

// Biases of the float-float tile pass (explicit-inverse subdomains): with
// the apply's input scaled to max |x| < 1, every partial sum over a row, or
// over a column segment of a tile, of row block I is at most rmax[I]; the
// bias is the power of two at or above 4 (1.001 rmax + n_i 2^-24), the
// factors covering the FP32 summation of rmax and FP16 rounding of the tiles.
__global__ void k_sym_bias(int64_t nitems, const int2* __restrict__ items, const int64_t* __restrict__ boff,
                           const int32_t* __restrict__ n_arr, const float* __restrict__ rmax,
                           float* __restrict__ bias) {
  COUNT_LAUNCH();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nitems; k += (int64_t)gridDim.x * blockDim.x) {
    const int2 w = items[k];
    const int64_t b = boff[w.x] + w.y;
    const float m = 4.f * (1.001f * rmax[b] + (float)n_arr[w.x] * 0x1.0p-24f);
    bias[b] = __uint_as_float((__float_as_uint(m) + 0x7fffffu) & 0x7f800000u);
  }
}

// in place: the FP32 tile becomes FP16 in the first half of its slot
__global__ void __launch_bounds__(NT) k_tiles_to_half(float* __restrict__ tiles, const int4* __restrict__ desc,
                                                      int64_t ntiles, const int8_t* __restrict__ s16) {
  COUNT_LAUNCH();
  constexpr int PER = TILE * TILE / NT;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    if (!s16[desc[t].x]) continue;  // the same for the whole block
    float* src = tiles + t * (TILE * TILE);
    float v[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) v[k] = src[threadIdx.x + k * NT];
    __syncthreads();  // the whole tile is read before any of it is overwritten
    __half* dst = reinterpret_cast<__half*>(src);
#pragma unroll
    for (int k = 0; k < PER; ++k) dst[threadIdx.x + k * NT] = __float2half_rn(v[k]);
    __syncthreads();
  }
}

// Copy A_ii^{-1} into TILE x TILE tiles: SPD keeps the lower tiles (I >= J),
// the general path keeps all of them.  One block per tile.
template <typename T>
__global__ void __launch_bounds__(NT) k_pack(const T* __restrict__ work, const int64_t* __restrict__ work_off,
                                             const int32_t* __restrict__ np, const int32_t* __restrict__ n_arr,
                                             const int4* __restrict__ desc, int64_t ntiles,
                                             const int8_t* __restrict__ sym, T* __restrict__ tiles) {
  COUNT_LAUNCH();
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int4 d = desc[t];
    int i = d.x, I = d.y, J = d.z;
    if (sym != nullptr && sym[i]) continue;  // tiles of S already written
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
  dn.h_nt.resize(N); dn.h_tile_off.resize(N + 1);
  std::vector<int64_t> h_pad_off(N + 1);
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
    dn.h_s_off[i] = ss;
    if (spd) {
      ss += (int64_t)nt * TILE * TILE;  // inverses of the diagonal blocks of L
    } else {
      xs += (int64_t)h.h_g[i] * h.h_p[i];
    }
    dn.h_tile_off[i] = tl;
    for (int I = 0; I < nt; ++I)
      for (int J = 0; J < (spd ? I + 1 : nt); ++J) desc.push_back(make_int4(i, I, J, 0));
    tl = (int64_t)desc.size();
    h_pad_off[i] = pt;
    pt += (int64_t)nt * TILE;
  }
  dn.h_tile_off[N] = tl;
  h_pad_off[N] = pt;
  dn.n_work = w; dn.n_xs = xs; dn.n_s = ss; dn.n_tiles = tl; dn.n_pad = pt;
  dn.np = mem.alloc<int32_t>(N);
  dn.nt = mem.alloc<int32_t>(N);
  dn.work_off = mem.alloc<int64_t>(N);
  dn.xs_off = mem.alloc<int64_t>(N);
  dn.s_off = mem.alloc<int64_t>(N);
  dn.tile_off = mem.alloc<int64_t>(N + 1);
  dn.pad_off = mem.alloc<int64_t>(N + 1);
  dn.sym = mem.alloc<int8_t>(N);
  CK(cudaMemsetAsync(dn.sym, 0, N, s));
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
  CK(cudaMemcpyAsync(dn.pad_off, h_pad_off.data(), 8 * (N + 1), cudaMemcpyHostToDevice, s));

  CK(cudaMemcpyAsync(dn.tile_desc, desc.data(), sizeof(int4) * tl, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_n, h.h_n.data(), 4 * N, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_m, h.h_m.data(), 4 * N, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_p, h.h_p.data(), 4 * N, cudaMemcpyHostToDevice, s));
  T* work = mem.alloc<T>(w);
  dn.work = work;
  dn.XpT = mem.alloc<T>(std::max<int64_t>(xs, 1));
  dn.dinv = mem.alloc<T>(std::max<int64_t>(ss, 1));
  dn.dinv_off = dn.s_off;
  dn.tiles = mem.alloc<T>(tl * TILE * TILE);
  // single precision: the apply's vectors are float-float pairs
  dn.xpad = mem.alloc<T>(pt * (sizeof(T) == 4 ? 2 : 1));
  dn.tpad = mem.alloc<T>(pt * (sizeof(T) == 4 ? 2 : 1));
  if (sizeof(T) == 4) dn.xunscale = mem.alloc<double>(N);
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
  // -- local factor
  if (spd) {
    if constexpr (sizeof(T) == 4) {
      // single precision: subdomains whose Cholesky pivots span at most three
      // decades get the explicit inverse (one pass in the apply)
      factor_spd_levels(h, work, d_n, 1e3, s);
    } else {
      const size_t sm3 = sizeof(T) * 3 * TILE * (TILE + 1);
      CK(cudaFuncSetAttribute(k_chol_trtri<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
      k_chol_trtri<T><<<N, NT, sm3, s>>>(work, dn.work_off, dn.np, d_n, (T*)dn.dinv, dn.dinv_off, dn.err, dn.sym,
                                         0.0);
    }
  } else {
    k_sweep<T, false><<<N, NT, 0, s>>>(work, dn.work_off, dn.np, d_n, d_m, d_p, (T*)dn.XpT, dn.xs_off,
                                       (T*)dn.S, dn.s_off, dn.err);
  }
  CK_LAUNCH("local factor");
  if (h.events) CK(cudaEventRecord(h.ev[4], s));
  // -- pack the apply tiles
  unsigned gp = (unsigned)std::min<int64_t>(std::max<int64_t>(tl, 1), 152 * 8);
  k_pack<T><<<gp, NT, 0, s>>>(work, dn.work_off, dn.np, d_n, dn.tile_desc, tl, spd ? dn.sym : nullptr,
                              (T*)dn.tiles);
  CK_LAUNCH("pack tiles");
  if (h.events) CK(cudaEventRecord(h.ev[5], s));
  // apply work items, longest first.  Row pass: every row block (SPD: row I
  // has I+1 tiles; general: nt).  Column pass: the column blocks (nt-J
  // tiles) of the subdomains kept in the two-pass form; the explicit-inverse
  // subdomains instead add their column contributions per row block.
  dn.h_sym.assign(N, 0);
  if (spd) {
    CK(cudaMemcpyAsync(dn.h_sym.data(), dn.sym, N, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  std::vector<std::pair<int, int2>> ri, ci;
  std::vector<int2> si;
  for (int i = 0; i < N; ++i) {
    const int nt = dn.h_nt[i];
    for (int b = 0; b < nt; ++b) {
      ri.push_back({spd ? b + 1 : nt, make_int2(i, b)});
      if (spd && !dn.h_sym[i]) ci.push_back({nt - b, make_int2(i, b)});
      if (spd && dn.h_sym[i]) si.push_back(make_int2(i, b));
    }
  }
  auto longest_first = [](const std::pair<int, int2>& a, const std::pair<int, int2>& b) { return a.first > b.first; };
  std::stable_sort(ri.begin(), ri.end(), longest_first);
  std::stable_sort(ci.begin(), ci.end(), longest_first);
  std::vector<int2> rv, cv;
  for (auto& e : ri) rv.push_back(e.second);
  for (auto& e : ci) cv.push_back(e.second);
  dn.n_row_items = (int)rv.size();
  dn.n_col_items = (int)cv.size();
  dn.n_sym_items = (int)si.size();
  dn.row_items = mem.alloc<int2>(std::max(dn.n_row_items, 1));
  dn.col_items = mem.alloc<int2>(std::max(dn.n_col_items, 1));
  dn.sym_items = mem.alloc<int2>(std::max(dn.n_sym_items, 1));
  CK(cudaMemcpyAsync(dn.row_items, rv.data(), sizeof(int2) * rv.size(), cudaMemcpyHostToDevice, s));
  if (!cv.empty()) CK(cudaMemcpyAsync(dn.col_items, cv.data(), sizeof(int2) * cv.size(), cudaMemcpyHostToDevice, s));
  if (!si.empty()) CK(cudaMemcpyAsync(dn.sym_items, si.data(), sizeof(int2) * si.size(), cudaMemcpyHostToDevice, s));
  if (spd && !si.empty()) dn.slots = mem.alloc<T>(tl * TILE * (sizeof(T) == 4 ? 2 : 1));
  if constexpr (sizeof(T) == 4) {
    if (spd && !si.empty()) {
      // row-block bounds of the explicit inverses: the tile pass's biases and
      // the FP16-storage decision
      std::vector<int64_t> bo(N);
      int64_t nb = 0;
      for (int i = 0; i < N; ++i) { bo[i] = nb; nb += dn.h_nt[i]; }
      dn.boff = mem.alloc<int64_t>(N);
      float* rmax = mem.alloc<float>(std::max<int64_t>(nb, 1));
      dn.sym_bias = mem.alloc<float>(std::max<int64_t>(nb, 1));
      CK(cudaMemcpyAsync(dn.boff, bo.data(), 8 * N, cudaMemcpyHostToDevice, s));
      const unsigned gs = (unsigned)std::min<int64_t>((int64_t)si.size(), 152 * 8);
      k_s_rowsum<<<gs, NT, 0, s>>>((const float*)dn.tiles, dn.tile_off, dn.nt, dn.sym_items, (int)si.size(), dn.boff,
                                   rmax);
      k_sym_bias<<<(unsigned)std::min<int64_t>(ceil_div((int64_t)si.size(), NT), 152 * 4), NT, 0, s>>>(
          (int64_t)si.size(), dn.sym_items, dn.boff, d_n, rmax, dn.sym_bias);
      CK_LAUNCH("row-block bounds of the explicit inverses");
      if (h.s16) {
        const int64_t* boff = dn.boff;
        double* amax = mem.alloc<double>(N);
        dn.s16 = mem.alloc<int8_t>(N);
        k_a_rowsum<<<N, NT, 0, s>>>(ov.sub_off, d_n, ov.omega, ov.ent_off, ov.lcol, h.row_ptr, h.col_idx, h.val,
                                    h.dscale, dn.sym, amax);
        k_decide_s16<<<(unsigned)ceil_div(N, NT), NT, 0, s>>>(N, dn.sym, dn.nt, d_n, boff, rmax, amax, dn.s16);
        k_tiles_to_half<<<gp, NT, 0, s>>>((float*)dn.tiles, dn.tile_desc, tl, dn.s16);
        CK_LAUNCH("FP16 storage of the explicit inverses");
        dn.h_s16.assign(N, 0);
        CK(cudaMemcpyAsync(dn.h_s16.data(), dn.s16, N, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        std::vector<int2> rh, rf;
        for (const int2& e : rv) (dn.h_s16[e.x] ? rh : rf).push_back(e);
        dn.n_row_items_h = (int)rh.size();
        dn.n_row_items_f = (int)rf.size();
        if (!rh.empty()) {
          dn.row_items_h = mem.alloc<int2>(rh.size());
          dn.row_items_f = mem.alloc<int2>(std::max<size_t>(rf.size(), 1));
          CK(cudaMemcpyAsync(dn.row_items_h, rh.data(), sizeof(int2) * rh.size(), cudaMemcpyHostToDevice, s));
          if (!rf.empty())
            CK(cudaMemcpyAsync(dn.row_items_f, rf.data(), sizeof(int2) * rf.size(), cudaMemcpyHostToDevice, s));
          CK(cudaStreamSynchronize(s));
        }
      }
    }
    // descriptors of the single-precision tile passes' work items
    std::vector<int64_t> bo(N);
    for (int i = 0, nb = 0; i < N; ++i) { bo[i] = nb; nb += dn.h_nt[i]; }
    auto make_desc = [&](const int2* dev_items, int count, bool col) -> TileItem* {
      if (count <= 0) return nullptr;
      std::vector<int2> it(count);
      CK(cudaMemcpyAsync(it.data(), dev_items, sizeof(int2) * count, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      std::vector<TileItem> d(count);
      for (int k = 0; k < count; ++k) {
        const int i = it[k].x, B = it[k].y, nt = dn.h_nt[i];
        TileItem& e = d[k];
        e.i = i;
        e.B = B;
        e.cnt = col ? nt - B : (spd ? B + 1 : nt);
        e.symi = (!col && spd && dn.h_sym[i]) ? 1 : 0;
        e.pad = h_pad_off[i];
        e.tile0 = dn.h_tile_off[i] + (col ? 0 : (spd ? (int64_t)B * (B + 1) / 2 : (int64_t)B * nt));
        e.bias0 = e.symi ? bo[i] : 0;
        e.slot0 = dn.h_tile_off[i] + (int64_t)B * (B + 1) / 2;
        e.n = h.h_n[i];
        e.sub_off = ov.h_sub_off[i];
        e.nt = nt;
        e.unused = 0;
      }
      TileItem* out = mem.alloc<TileItem>(count);
      CK(cudaMemcpyAsync(out, d.data(), sizeof(TileItem) * count, cudaMemcpyHostToDevice, s));
      CK(cudaStreamSynchronize(s));
      return out;
    };
    dn.row_desc = make_desc(dn.row_items, dn.n_row_items, false);
    dn.col_desc = make_desc(dn.col_items, dn.n_col_items, true);
    dn.row_desc_h = make_desc(dn.row_items_h, dn.n_row_items_h, false);
    dn.row_desc_f = make_desc(dn.row_items_f, dn.n_row_items_f, false);
  }
}

}  // namespace

void build_local(Handle& h, cudaStream_t s) {
  if (h.fp32) run_local<float>(h, s); else run_local<double>(h, s);
  check_device_error(h, s, "local inverse");
}

}  // namespace asmgpu
