// Local coarse vectors by randomized block subspace iteration with Chebyshev
// acceleration, one block per subdomain, all subdomains in one launch.
//
// SPD (eq. gevpsvd, Section 5.1).  With X = -B^{-1}C, X_p its first |I_i| rows,
// S = G - C^T B^{-1} C and K = X_p^T A_{I_i,I_i} X_p, every eigenpair of
// eq. gevpsvd with lambda^2 > 0 satisfies K y = lambda^2 S y with y = w_Gamma,
// the A_ii-normalisation of w is the S-normalisation of y, and the coarse
// vector R_i^T D_i Pi_i w is [X_p y; 0] on Omega_{I_i}.  With the Cholesky
// factor A_ii = L L^T and W = L^{-1} = [W11 0; W21 W22] (blocks Omega', Gamma),
// S = (W22^T W22)^{-1} and X W22^T = W21^T, so with z = W22^{-T} y and
// U = W21[:, :p] the problem is the symmetric U A_II U^T z = lambda^2 z with
// Euclidean-orthonormal z, and the coarse vector is X_p y = U^T z.
//
// General A (the paper's nonsymmetric extension).  D_i Pi_i is nonzero only
// in rows I_i and columns Gamma_delta, where it equals X_p, so its left
// singular vectors are those of X_p: the iteration runs on OP = X_p X_p^T
// with Euclidean orthonormal blocks, and the kept vectors are the coarse
// vectors themselves.  The Euclidean SVD is not invariant under the diagonal
// scaling of the local sweep, so the scaling is undone inside the products
// with X_p.
//
// One sweep: Rayleigh-Ritz on the whole block (cyclic Jacobi on the projected
// s x s matrix in the working precision, Golub & Van Loan Alg. 8.5.3),
// relative eigen-residual test, soft locking of the converged leading Ritz
// pairs (they leave the filter, not the Rayleigh-Ritz step), then a degree-d
// Chebyshev polynomial in OP
// applied to the remaining columns (scaled three-term recurrence of Zhou &
// Saad, 2007) that damps the spectrum below the smallest Ritz value, with the
// locked vectors projected out after every application of OP and the degree
// capped by the filter's growth over the active Ritz values (subdomains with
// a floating high-contrast inclusion have one eigenvalue 10^6 times the
// rest), and CholQR2 re-orthonormalisation of column-normalised blocks.
// Dense block products go through a shared-memory tiled CTA GEMM.
#include <algorithm>

#include <cuda_bf16.h>

#include "handle.cuh"
#include "tcgemm.cuh"

namespace asmgpu {
namespace {

constexpr int NT = 256;
constexpr int GM = 128;  // rows per CTA-GEMM tile
constexpr int GK = 32;   // K chunk
constexpr int GN = 32;   // columns per pass

// Shared memory of one CTA GEMM: A tile GM x (GK + pad), B tile GK x (GN + pad).
// The single-precision path feeds tensor cores and pads for conflict-free
// fragment loads (A row stride 36, B row stride 40); FP64 keeps 33 / 32.
template <typename T>
__host__ __device__ constexpr int gemm_lda() { return sizeof(T) == 4 ? GK + 4 : GK + 1; }
template <typename T>
__host__ __device__ constexpr int gemm_ldb() { return sizeof(T) == 4 ? GN + 8 : GN; }
// The single-precision products without column scaling whose operands are
// both in global memory double-buffer K chunks of GKA columns with cp.async (the next chunk streams in while the
// current one is multiplied); A row stride GKA + 4, B row stride GN + 8.
constexpr int GKA = 16;
constexpr int ASYNC_BUF = GM * (GKA + 4) + GKA * (GN + 8);
template <typename T>
__host__ __device__ constexpr size_t gemm_smem_bytes() {
  return sizeof(T) == 4 ? std::max<size_t>(((sizeof(T) * (GM * gemm_lda<T>() + GK * gemm_ldb<T>()) + 7) / 8) * 8,
                                           sizeof(float) * 2 * ASYNC_BUF)
                        : ((sizeof(T) * (GM * gemm_lda<T>() + GK * gemm_ldb<T>()) + 7) / 8) * 8;
}

__device__ __forceinline__ uint32_t f2tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void split3(float x, uint32_t& hi, uint32_t& lo) {
  hi = f2tf32(x);
  lo = f2tf32(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// two FP32 values rounded to BF16 and packed, the first in the low half (the
// lower k index of an mma.sync fragment pair)
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Optional diagonal scalings (general path): factor for index q.
struct Scale {
  const double* ds = nullptr;
  const int32_t* om = nullptr;
  __device__ double operator()(int q) const { return ds ? ds[om[q]] : 1.0; }
  __device__ bool on() const { return ds != nullptr; }
};

__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(ok ? 4 : 0)
               : "memory");
}

// The FP32 product of cta_gemm without column scaling: the 3xTF32 mma.sync
// tile loop of cta_gemm fed by a two-stage cp.async pipeline (masked elements
// are zero-filled without a read).
template <bool ACOL, bool SUB, bool UPPER, bool B16>
__device__ void cta_gemm_f32_async(int M, int N, int K, const float* __restrict__ A, int lda,
                                   const float* __restrict__ B, int ldb, float* __restrict__ C, int ldc, float* sm,
                                   Scale rs) {
  constexpr int LA = GKA + 4, LB = GN + 8;
  const int t = threadIdx.x;
  const int lane = t & 31, w = t >> 5, g = lane >> 2, tq = lane & 3;
  const int nk = (K + GKA - 1) / GKA;
  for (int n0 = 0; n0 < N; n0 += GN) {
    const int nw = min(GN, N - n0);
    for (int m0 = 0; m0 < M; m0 += GM) {
      auto issue = [&](int k0, int b) {
        float* As = sm + b * ASYNC_BUF;
        float* Bs = As + GM * LA;
#pragma unroll
        for (int j = 0; j < GM * GKA / NT; ++j) {
          const int idx = t + NT * j;
          int r, kk;
          if (!ACOL) { r = idx / GKA; kk = idx % GKA; } else { kk = idx / GM; r = idx % GM; }
          const bool ok = m0 + r < M && k0 + kk < K && (!UPPER || k0 + kk >= m0 + r);
          const float* src = !ok ? A : (!ACOL ? A + (int64_t)(m0 + r) * lda + k0 + kk : A + (int64_t)(k0 + kk) * lda + m0 + r);
          cp_async4(As + r * LA + kk, src, ok);
        }
#pragma unroll
        for (int j = 0; j < GKA * GN / NT; ++j) {
          const int idx = t + NT * j, kk = idx / GN, c = idx % GN;
          const bool ok = k0 + kk < K && c < nw;
          cp_async4(Bs + kk * LB + c, ok ? B + (int64_t)(k0 + kk) * ldb + n0 + c : B, ok);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
      };
      float acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[a][q] = 0.f;
      issue(0, 0);
      for (int c = 0; c < nk; ++c) {
        if (c + 1 < nk) {
          issue((c + 1) * GKA, (c + 1) & 1);
          asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
          asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        const float* Ar = sm + (c & 1) * ASYNC_BUF + (16 * w) * LA;
        const float* Bf = sm + (c & 1) * ASYNC_BUF + GM * LA;
        if constexpr (B16) {
          // one m16n8k16 per n tile: operands rounded to BF16, FP32 accumulation
          uint32_t a[4];
          a[0] = pack_bf16(Ar[g * LA + 2 * tq], Ar[g * LA + 2 * tq + 1]);
          a[1] = pack_bf16(Ar[(g + 8) * LA + 2 * tq], Ar[(g + 8) * LA + 2 * tq + 1]);
          a[2] = pack_bf16(Ar[g * LA + 2 * tq + 8], Ar[g * LA + 2 * tq + 9]);
          a[3] = pack_bf16(Ar[(g + 8) * LA + 2 * tq + 8], Ar[(g + 8) * LA + 2 * tq + 9]);
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            const uint32_t b0 = pack_bf16(Bf[(2 * tq) * LB + 8 * nt + g], Bf[(2 * tq + 1) * LB + 8 * nt + g]);
            const uint32_t b1 = pack_bf16(Bf[(2 * tq + 8) * LB + 8 * nt + g], Bf[(2 * tq + 9) * LB + 8 * nt + g]);
            mma_bf16(acc[nt], a, b0, b1);
          }
        } else {
#pragma unroll
        for (int kk = 0; kk < GKA; kk += 8) {
          uint32_t ah[4], al[4];
          split3(Ar[g * LA + kk + tq], ah[0], al[0]);
          split3(Ar[(g + 8) * LA + kk + tq], ah[1], al[1]);
          split3(Ar[g * LA + kk + tq + 4], ah[2], al[2]);
          split3(Ar[(g + 8) * LA + kk + tq + 4], ah[3], al[3]);
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            uint32_t bh0, bl0, bh1, bl1;
            split3(Bf[(kk + tq) * LB + 8 * nt + g], bh0, bl0);
            split3(Bf[(kk + tq + 4) * LB + 8 * nt + g], bh1, bl1);
            mma_tf32(acc[nt], al, bh0, bh1);
            mma_tf32(acc[nt], ah, bl0, bl1);
            mma_tf32(acc[nt], ah, bh0, bh1);
          }
        }
        }
        __syncthreads();
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int row = m0 + 16 * w + g + (q >= 2 ? 8 : 0);
          const int c = 8 * a + 2 * tq + (q & 1);
          if (row >= M || c >= nw) continue;
          const float f = rs.on() ? (float)rs(row) : 1.f;
          float* cp = C + (int64_t)row * ldc + n0 + c;
          if (SUB) *cp -= acc[a][q] * f; else *cp = acc[a][q] * f;
        }
    }
  }
  __syncthreads();
}

// C (M x N, ldc) = A (M x K) B (K x N, ldb) (with SUB: C -= A B); A row-major
// (A[m*lda + k]) or, with ACOL, column-major (A[k*lda + m]).  The product's
// row m is multiplied by rs(m); A's column k by ks(k) (or divided, with kinv).
// UPPER (with ACOL): A is the transpose of a lower-triangular block whose
// upper part in memory holds other data, so A(m, k) is taken as 0 for k < m.
template <typename T, bool ACOL, bool SUB = false, bool UPPER = false, bool B16 = false>
__device__ void cta_gemm(int M, int N, int K, const T* __restrict__ A, int lda, const T* __restrict__ B, int ldb,
                         T* __restrict__ C, int ldc, T* sm, Scale rs = Scale(), Scale ks = Scale(), bool kinv = false) {
  if constexpr (sizeof(T) == 4) {
    // cp.async reads global memory only: operands held in shared memory (the
    // small projected matrices) take the synchronous loop below
    if (!ks.on() && __isGlobal(A) && __isGlobal(B)) {
      cta_gemm_f32_async<ACOL, SUB, UPPER, B16>(M, N, K, A, lda, B, ldb, C, ldc, sm, rs);
      return;
    }
  }
  constexpr int LA = gemm_lda<T>(), LB = gemm_ldb<T>();
  T* As = sm;             // GM x LA
  T* Bs = sm + GM * LA;   // GK x LB
  const int t = threadIdx.x;
  for (int n0 = 0; n0 < N; n0 += GN) {
    const int nw = min(GN, N - n0);
    for (int m0 = 0; m0 < M; m0 += GM) {
      // FP32: tensor cores, warp w owns rows 16w .. 16w+15 of the GM x GN tile,
      // 3xTF32 (hi/lo split) keeps single-precision accuracy.
      // FP64: thread owns rows tr + 32 a (a = 0..3) and columns 4 tc .. 4 tc + 3.
      T acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[a][q] = 0;
      for (int k0 = 0; k0 < K; k0 += GK) {
        __syncthreads();
        if (!ACOL) {
          for (int idx = t; idx < GM * GK; idx += NT) {
            int r = idx / GK, kk = idx % GK;
            T v = (m0 + r < M && k0 + kk < K) ? A[(int64_t)(m0 + r) * lda + k0 + kk] : T(0);
            if (ks.on() && k0 + kk < K) v = (T)(kinv ? (double)v / ks(k0 + kk) : (double)v * ks(k0 + kk));
            As[r * LA + kk] = v;
          }
        } else {
          for (int idx = t; idx < GM * GK; idx += NT) {
            int kk = idx / GM, r = idx % GM;
            T v = (m0 + r < M && k0 + kk < K && (!UPPER || k0 + kk >= m0 + r)) ? A[(int64_t)(k0 + kk) * lda + m0 + r]
                                                                              : T(0);
            if (ks.on() && k0 + kk < K) v = (T)(kinv ? (double)v / ks(k0 + kk) : (double)v * ks(k0 + kk));
            As[r * LA + kk] = v;
          }
        }
        for (int idx = t; idx < GK * GN; idx += NT) {
          int kk = idx / GN, c = idx % GN;
          Bs[kk * LB + c] = (k0 + kk < K && c < nw) ? B[(int64_t)(k0 + kk) * ldb + n0 + c] : T(0);
        }
        __syncthreads();
        if constexpr (sizeof(T) == 4) {
          const int lane = t & 31, w = t >> 5, g = lane >> 2, tq = lane & 3;
          const float* Ar = reinterpret_cast<const float*>(As) + (16 * w) * LA;
          const float* Bf = reinterpret_cast<const float*>(Bs);
#pragma unroll
          for (int kk = 0; kk < GK; kk += 8) {
            uint32_t ah[4], al[4];
            split3(Ar[g * LA + kk + tq], ah[0], al[0]);
            split3(Ar[(g + 8) * LA + kk + tq], ah[1], al[1]);
            split3(Ar[g * LA + kk + tq + 4], ah[2], al[2]);
            split3(Ar[(g + 8) * LA + kk + tq + 4], ah[3], al[3]);
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
              uint32_t bh0, bl0, bh1, bl1;
              split3(Bf[(kk + tq) * LB + 8 * nt + g], bh0, bl0);
              split3(Bf[(kk + tq + 4) * LB + 8 * nt + g], bh1, bl1);
              float* d = reinterpret_cast<float*>(acc[nt]);
              float (&dd)[4] = *reinterpret_cast<float(*)[4]>(d);
              mma_tf32(dd, al, bh0, bh1);
              mma_tf32(dd, ah, bl0, bl1);
              mma_tf32(dd, ah, bh0, bh1);
            }
          }
        } else {
          const int tr = t & 31, tc = t >> 5;
#pragma unroll 4
          for (int kk = 0; kk < GK; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[(tr + 32 * a) * LA + kk];
#pragma unroll
            for (int q = 0; q < 4; ++q) bv[q] = Bs[kk * LB + 4 * tc + q];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int q = 0; q < 4; ++q) acc[a][q] += av[a] * bv[q];
          }
        }
      }
      // epilogue: element (row, col) of the tile for each accumulator entry
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int row, c;
          if constexpr (sizeof(T) == 4) {
            const int lane = t & 31, w = t >> 5;
            row = 16 * w + (lane >> 2) + (q >= 2 ? 8 : 0);
            c = 8 * a + 2 * (lane & 3) + (q & 1);
          } else {
            row = (t & 31) + 32 * a;
            c = 4 * (t >> 5) + q;
          }
          row += m0;
          if (row >= M || c >= nw) continue;
          const T f = rs.on() ? (T)rs(row) : T(1);
          T* cp = C + (int64_t)row * ldc + n0 + c;
          if (SUB) *cp -= acc[a][q] * f; else *cp = acc[a][q] * f;
        }
    }
  }
  __syncthreads();
}

// AV (p x s) = A^_{I,I} V from the local CSR rows of I_i: aval holds the
// scaled values a_vu / sqrt(|a_vv a_uu|) entry by entry (aligned with lcol),
// lcol the local column (< 0 outside Omega_i; only columns < p are used).
template <typename T>
__device__ void mul_AII(int p, int pos0, const int64_t* __restrict__ ent_off, const int32_t* __restrict__ lcol,
                        const T* __restrict__ aval, const T* __restrict__ V, T* __restrict__ AV, int s, int sp) {
  for (int idx = threadIdx.x; idx < p * s; idx += NT) {
    const int a = idx / s, j = idx % s;
    const int64_t e0 = ent_off[pos0 + a], e1 = ent_off[pos0 + a + 1];
    T acc = 0;
    for (int64_t e = e0; e < e1; ++e) {
      const int lc = lcol[e];
      if (lc < 0 || lc >= p) continue;
      acc += aval[e] * V[(int64_t)lc * sp + j];
    }
    AV[(int64_t)a * sp + j] = acc;
  }
  __syncthreads();
}

// The single-precision eq. gevpsvd operator K = U A^_II U^T of each subdomain
// (g x g, U = W[Gamma_delta, I_i]) is formed once at setup: the zero-padded
// copy Up of U and T = U A^_II (from the sparse local rows; A^_II is
// symmetric, so column c of T takes row c of A^_II) here, then K = T Up^T as
// 64 x 64 tile jobs on the tensor cores.  Each application of the operator in
// the iteration is then one g x g block product instead of two g x p ones.
__global__ void __launch_bounds__(NT) k_u_padded(const float* __restrict__ work, const int64_t* __restrict__ work_off,
                                                 const int32_t* __restrict__ np_arr, const int32_t* __restrict__ n_arr,
                                                 const int32_t* __restrict__ m_arr, const int32_t* __restrict__ p_arr,
                                                 const int64_t* __restrict__ uoff, const int32_t* __restrict__ uld,
                                                 const int32_t* __restrict__ urows, float* __restrict__ Up,
                                                 float* __restrict__ Tm, const int32_t* __restrict__ sub_off,
                                                 const int64_t* __restrict__ ent_off, const int32_t* __restrict__ lcol,
                                                 const float* __restrict__ aval) {
  COUNT_LAUNCH();
  const int i = blockIdx.y;
  const int n = n_arr[i], m = m_arr[i], p = p_arr[i], g = n - m, ld = np_arr[i];
  const int pp = uld[i], gp = urows[i], pos0 = sub_off[i];
  const float* U = work + work_off[i] + (int64_t)m * ld;
  float* up = Up + uoff[i];
  float* tm = Tm + uoff[i];
  const int64_t total = (int64_t)gp * pp;
  for (int64_t idx = blockIdx.x * (int64_t)NT + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * NT) {
    const int r = (int)(idx / pp), c = (int)(idx % pp);
    float u = 0.f, t = 0.f;
    if (r < g && c < p) {
      const float* Ur = U + (int64_t)r * ld;
      u = Ur[c];
      for (int64_t e = ent_off[pos0 + c]; e < ent_off[pos0 + c + 1]; ++e) {
        const int lc = lcol[e];
        if (lc >= 0 && lc < p) t = fmaf(Ur[lc], aval[e], t);
      }
    }
    up[idx] = u;
    tm[idx] = t;
  }
}

// Scaled values of every local row (all positions of all Omega_i), in the
// working precision: aval[e] = a_vu ds_v ds_u with ds = |diag A|^{-1/2}.
template <typename T>
__global__ void k_scaled_values(int64_t total, const int32_t* __restrict__ omega, const int64_t* __restrict__ ent_off,
                                const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                const double* __restrict__ val, const double* __restrict__ ds, T* __restrict__ aval) {
  COUNT_LAUNCH();
  for (int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pos < total;
       pos += (int64_t)gridDim.x * blockDim.x) {
    const int v = omega[pos];
    const int b = rp[v], e = rp[v + 1];
    const double sv = ds[v];
    const int64_t o = ent_off[pos];
    for (int q = 0; q < e - b; ++q) aval[o + q] = (T)(val[b + q] * sv * ds[ci[b + q]]);
  }
}

// Cholesky of the s x s Gram matrix G (warp 0), then Minv = L^{-T} so that
// Y <- Y Minv is orthonormal in the metric of G.  A pivot below `tiny` (the
// diagonal of G is 1) marks column j as dependent in bad[j] and is replaced
// by 1; returns the number of dependent columns.
__device__ int chol_inv_t(double* G, double* Minv, int s, double tiny, int* bad, int* nbad) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int nb = 0;
    for (int j = 0; j < s; ++j) {
      double d = G[j * s + j];
      for (int k = 0; k < j; ++k) d -= G[j * s + k] * G[j * s + k];
      const bool dep = !(d > tiny);
      if (lane == 0) bad[j] = dep ? 1 : 0;
      if (dep) {
        ++nb;
        d = 1.0;
        for (int r = lane; r < s; r += 32) if (r != j) { G[r * s + j] = 0; }
        __syncwarp();
        for (int k = lane; k < j; k += 32) G[j * s + k] = 0;
      }
      d = sqrt(d);
      __syncwarp();
      for (int r = j + 1 + lane; r < s; r += 32) {
        double v = G[r * s + j];
        for (int k = 0; k < j; ++k) v -= G[r * s + k] * G[j * s + k];
        G[r * s + j] = v / d;
      }
      __syncwarp();
      if (lane == 0) G[j * s + j] = d;
      __syncwarp();
    }
    for (int c = lane; c < s; c += 32) {
      for (int r = 0; r < s; ++r) Minv[r * s + c] = 0;
      for (int r = c; r < s; ++r) {
        double v = (r == c) ? 1.0 : 0.0;
        for (int k = c; k < r; ++k) v -= G[r * s + k] * Minv[k * s + c];
        Minv[r * s + c] = v / G[r * s + r];
      }
    }
    __syncwarp();
    for (int idx = lane; idx < s * s; idx += 32) {
      int r = idx / s, c = idx % s;
      if (r < c) {
        double a = Minv[r * s + c], b = Minv[c * s + r];
        Minv[r * s + c] = b;
        Minv[c * s + r] = a;
      }
    }
    if (lane == 0) *nbad = nb;
  }
  __syncthreads();
  return *nbad;
}

// Cyclic Jacobi on the symmetric s x s matrix H (shared); Q accumulates the
// rotations; on exit diag(H) holds the eigenvalues.  One warp.
template <typename T>
__device__ void jacobi(T* H, T* Q, int s) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int idx = lane; idx < s * s; idx += 32) Q[idx] = (idx / s == idx % s) ? T(1) : T(0);
    __syncwarp();
    const T eps = sizeof(T) == 8 ? T(1e-15) : T(1e-7);
    for (int sweep = 0; sweep < 40; ++sweep) {
      T off = 0, dg = 0;
      for (int idx = lane; idx < s * s; idx += 32) {
        T v = H[idx];
        if (idx / s != idx % s) off += v * v; else dg += v * v;
      }
      off = warp_sum(off);
      dg = warp_sum(dg);
      if (off <= eps * eps * dg || dg == T(0)) break;
      for (int pp = 0; pp < s - 1; ++pp) {
        for (int qq = pp + 1; qq < s; ++qq) {
          T apq = H[pp * s + qq];
          T app = H[pp * s + pp], aqq = H[qq * s + qq];
          if (fabs((double)apq) <= (double)eps * 1e-3 * sqrt(fabs((double)app * (double)aqq))) continue;
          T tau = (aqq - app) / (T(2) * apq);
          T tt = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
          T c = T(1) / sqrt(T(1) + tt * tt), sn = tt * c;
          __syncwarp();
          for (int k = lane; k < s; k += 32) {
            T hp = H[k * s + pp], hq = H[k * s + qq];
            H[k * s + pp] = c * hp - sn * hq;
            H[k * s + qq] = sn * hp + c * hq;
          }
          __syncwarp();
          for (int k = lane; k < s; k += 32) {
            T hp = H[pp * s + k], hq = H[qq * s + k];
            H[pp * s + k] = c * hp - sn * hq;
            H[qq * s + k] = sn * hp + c * hq;
            T qp = Q[k * s + pp], qv = Q[k * s + qq];
            Q[k * s + pp] = c * qp - sn * qv;
            Q[k * s + qq] = sn * qp + c * qv;
          }
          __syncwarp();
        }
      }
    }
  }
  __syncthreads();
}

template <typename T>
__device__ void fill_random(T* Y, int L, int s, int sp, int j0, uint64_t seed, uint64_t salt) {
  for (int64_t idx = threadIdx.x; idx < (int64_t)L * (s - j0); idx += NT) {
    int r = (int)(idx / (s - j0)), j = j0 + (int)(idx % (s - j0));
    Y[(int64_t)r * sp + j] = (T)counter_normal(seed, salt + (uint64_t)r * 131071u + (uint64_t)j * 2654435761u);
  }
  __syncthreads();
}

// Where a run of the subspace iteration writes its results.  The gevpsvd
// run keeps up to nkeep = nev pairs from column 0 of each Z_i block; the
// lifting run (eq. uppergevp, lift = 1) keeps up to nkeep = nev_lift pairs
// after them (zcol0[i] = the gevpsvd count), skipping the skip[i] leading pairs
// that overlap 1 shares with eq. gevpsvd.
struct EigOut {
  int zld;                  // row stride of the Z_i blocks (all runs)
  int nkeep;                // pairs kept at most; leading dimension of values, resid
  const int32_t* zcol0;     // first column of this run in Z_i (null: 0)
  const int32_t* skip;      // leading Ritz pairs left out (null: none)
  int lift;                 // 1: report 1 + mu and scale the vectors by sqrt((1 + mu) / mu)
  int refine;               // FP64, lifting or overlap 1: report the variational Rayleigh quotient
  const int32_t* order;     // block b works on subdomain order[b] (largest first; null: b)
  const float* K;           // single precision, eq. gevpsvd run: the explicit operator U A^_II U^T per
  const int64_t* koff;      // subdomain (row-major, leading dimension kld[i]); null: products with U
  const int32_t* kld;
};

// B16 (single precision, SPD): the operator applications K Y = U (A^_II (U^T Y))
// multiply BF16-rounded operands with FP32 accumulation; the Gram,
// Rayleigh-Ritz and output products stay 3xTF32.
template <typename T, bool SPD, bool B16 = false>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 4 : 1) k_subspace(
    const T* __restrict__ XpT_all, const int64_t* __restrict__ xs_off, const T* __restrict__ S_all,
    const int64_t* __restrict__ s_off, const T* __restrict__ work, const int64_t* __restrict__ work_off,
    const int32_t* __restrict__ np_arr, const int32_t* __restrict__ n_arr, const int32_t* __restrict__ m_arr,
    const int32_t* __restrict__ p_arr, const int32_t* __restrict__ sub_off, const int64_t* __restrict__ ent_off,
    const int32_t* __restrict__ lcol, const int32_t* __restrict__ omega, const int32_t* __restrict__ rp,
    const int32_t* __restrict__ ci, const double* __restrict__ val, const double* __restrict__ ds,
    const T* __restrict__ aval, T* scratch,
    const int64_t* __restrict__ scr_off, int nev, int over, int max_sweeps, int degree, double tol, double thresh,
    uint64_t seed,
    const float* __restrict__ warm, int wld, int wk, const int64_t* __restrict__ wseg, float* __restrict__ tgt,
    double* __restrict__ values,
    double* __restrict__ resid, int32_t* __restrict__ count, int32_t* __restrict__ sweeps_out,
    double* __restrict__ Z, const int64_t* __restrict__ z_off, EigOut eo) {
  COUNT_LAUNCH();
  extern __shared__ double shd[];
  __shared__ int perm[128];
  __shared__ int badcol[128];
  __shared__ int nbad;
  __shared__ T red[NT / 32];
  const int i = eo.order ? eo.order[blockIdx.x] : (int)blockIdx.x;
  const int n = n_arr[i], m = m_arr[i], p = p_arr[i], ld = np_arr[i];
  const int g = n - m, pos0 = sub_off[i];
  const int dim = SPD ? g : p;
  const int s = min(nev + over, dim);
  const int k = min(nev, min(s, min(p, g)));
  const int zc0 = eo.zcol0 ? eo.zcol0[i] : 0;
  if (k <= 0 || s <= 0) {
    if (threadIdx.x == 0) { count[i] = 0; sweeps_out[i] = 0; }
    for (int j = threadIdx.x; j < eo.nkeep; j += NT) {
      values[(int64_t)i * eo.nkeep + j] = 0;
      resid[(int64_t)i * eo.nkeep + j] = 0;
    }
    for (int64_t idx = threadIdx.x; idx < (int64_t)p * eo.nkeep; idx += NT)
      Z[z_off[i] + (idx / eo.nkeep) * eo.zld + zc0 + idx % eo.nkeep] = 0;
    return;
  }
  const int sp = (s + 3) & ~3;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T* XpT = SPD ? nullptr : XpT_all + xs_off[i];
  // SPD: U = W[Gamma_delta, I_i] (g x p block of W = L^{-1}, leading dimension ld)
  const T* U = work + work_off[i] + (int64_t)m * ld;
  const int L = max(p, g);
  const int64_t blk = (int64_t)L * sp;
  T* base = scratch + scr_off[i];
  T* Y = base;            // current block (dim x s)
  T* Yb = base + blk;     // Chebyshev / rotation buffers
  T* Yc = base + 2 * blk;
  T* T1 = base + 3 * blk;
  T* KY = base + 4 * blk; // K Y (dim x s)
  T* V = base + 5 * blk;  // p x s
  T* AV = base + 6 * blk; // p x s  (general: g x s)
  // shared memory: GEMM tiles, then the small dense matrices
  T* gsm = reinterpret_cast<T*>(shd);
  double* G = shd + gemm_smem_bytes<T>() / 8;
  double* Minv = G + s * s;
  T* H = reinterpret_cast<T*>(Minv + s * s);
  T* Q = H + s * s;
  T* QS = Q + s * s;
  T* mu = QS + s * s;
  T* rn = mu + s;
  T* Pbuf = rn + s;   // s x s
  Scale sI, sG;
  if (!SPD) { sI.ds = ds; sI.om = omega + pos0; sG.ds = ds; sG.om = omega + pos0 + m; }

  // K-apply: SPD: K y = X_p^T A^_II X_p y (g-space); general: X_p X_p^T y (p-space)
  // Column c0.. c0+nc-1 of the blocks (stride sp).
  auto applyK = [&](const T* Yin, T* out, int c0, int nc) {
    if (SPD) {
      if constexpr (sizeof(T) == 4) {
        if (eo.K != nullptr && eo.koff[i] >= 0) {  // K Y with the operator formed at setup
          cta_gemm<T, false, false, false, B16>(g, nc, g, eo.K + eo.koff[i], eo.kld[i], Yin + c0, sp, out + c0, sp,
                                                gsm);
          return;
        }
      }
      cta_gemm<T, true, false, false, B16>(p, nc, g, U, ld, Yin + c0, sp, V + c0, sp, gsm);    // V = U^T Y
      mul_AII(p, pos0, ent_off, lcol, aval, V + c0, AV + c0, nc, sp);
      cta_gemm<T, false, false, false, B16>(g, nc, p, U, ld, AV + c0, sp, out + c0, sp, gsm);  // U (A^_II V)
    } else {
      // W = X_p^T Y = S_G^{-1} X^_p^T S_I Y ; out = X_p W = S_I X^_p S_G^{-1} W
      cta_gemm<T, false>(g, nc, p, XpT, p, Yin + c0, sp, AV + c0, sp, gsm, Scale(), sI, false);
      for (int idx = threadIdx.x; idx < g * nc; idx += NT) {
        int r = idx / nc, j = c0 + idx % nc;
        AV[(int64_t)r * sp + j] = (T)((double)AV[(int64_t)r * sp + j] / sG(r));
      }
      __syncthreads();
      cta_gemm<T, true>(p, nc, g, XpT, p, AV + c0, sp, out + c0, sp, gsm, sI, sG, true);
    }
  };
  // the operator is K itself in both cases (Euclidean metric)
  auto applyR = [&](const T* KYin, T* out, int c0, int nc) {
    for (int64_t idx = threadIdx.x; idx < (int64_t)dim * nc; idx += NT) {
      int64_t r = idx / nc, j = c0 + idx % nc;
      out[r * sp + j] = KYin[r * sp + j];
    }
    __syncthreads();
  };
  // W[:, c0:] -= Y_L (Y_L^T W[:, c0:]) with Y_L = the first c0 (orthonormal)
  // columns of Y: keeps the active block orthogonal to the locked Ritz vectors.
  T* Pt = Pbuf;
  auto deflate = [&](T* W, int c0, int nc) {
    if (c0 == 0) return;
    cta_gemm<T, true>(c0, nc, dim, Y, sp, W + c0, sp, Pt, nc, gsm);
    cta_gemm<T, false, true>(dim, nc, c0, Y, sp, Pt, nc, W + c0, sp, gsm);
  };
  auto swap = [](T*& a, T*& b) { T* t = a; a = b; b = t; };
  // CholQR2 of column-normalised blocks; columns found dependent are
  // replaced by fresh random vectors and the whole step is redone.
  const double tiny = sizeof(T) == 8 ? 1e-10 : 1e-5;
  auto orthonormalize = [&](uint64_t salt) {
    for (int attempt = 0; attempt < 4; ++attempt) {
      for (int j = wid; j < s; j += NT / 32) {
        T part = 0;
        for (int r = lane; r < dim; r += 32) part += Y[(int64_t)r * sp + j] * Y[(int64_t)r * sp + j];
        part = warp_sum(part);
        if (lane == 0) Pbuf[j] = part > T(0) ? T(1) / sqrt(part) : T(1);
      }
      __syncthreads();
      for (int64_t idx = threadIdx.x; idx < (int64_t)dim * sp; idx += NT) {
        int j = (int)(idx % sp);
        if (j < s) Y[idx] *= Pbuf[j];
      }
      __syncthreads();
      bool ok = true;
      for (int pass = 0; pass < 2 && ok; ++pass) {
        T* Gt = QS;  // s*s scratch in T
        cta_gemm<T, true>(s, s, dim, Y, sp, Y, sp, Gt, s, gsm);
        for (int idx = threadIdx.x; idx < s * s; idx += NT) {
          int a = idx / s, b = idx % s;
          G[idx] = 0.5 * ((double)Gt[a * s + b] + (double)Gt[b * s + a]);
        }
        __syncthreads();
        if (chol_inv_t(G, Minv, s, tiny, badcol, &nbad) > 0) {
          for (int64_t idx = threadIdx.x; idx < (int64_t)dim * s; idx += NT) {
            int r = (int)(idx / s), j = (int)(idx % s);
            if (badcol[j])
              Y[(int64_t)r * sp + j] = (T)counter_normal(seed ^ 0x5DEECE66Dull,
                                                         salt * 977u + attempt * 131u + (uint64_t)r * 131071u + j);
          }
          __syncthreads();
          ok = false;
          break;
        }
        for (int idx = threadIdx.x; idx < s * s; idx += NT) QS[idx] = (T)Minv[idx];
        __syncthreads();
        cta_gemm<T, false>(dim, s, s, Y, sp, QS, s, Yb, sp, gsm);
        swap(Y, Yb);
      }
      if (ok) return;
    }
  };

  // ---- start block
  fill_random(Y, dim, s, sp, 0, seed, (uint64_t)i * 0x100000001ull);
  if (warm != nullptr && SPD) {
    // predicted start columns (rows = Gamma_delta nodes), random columns after them
    const float* wb = warm + wseg[i] * wld;
    const int kw = min(wk, k);
    for (int64_t idx = threadIdx.x; idx < (int64_t)dim * kw; idx += NT) {
      int r = (int)(idx / kw), j = (int)(idx % kw);
      Y[(int64_t)r * sp + j] = (T)wb[(int64_t)r * wld + j];
    }
    __syncthreads();
  }
  orthonormalize((uint64_t)i);

  for (int j = threadIdx.x; j < s; j += NT) rn[j] = 0;
  int sweep = 0, last_gain = 0;
  T best = T(3.0e38);
  for (;;) {
    // ---- Rayleigh-Ritz on the whole block (Jacobi in the working precision).
    //      Converged columns are only kept out of the filter ("soft" locking):
    //      the projected problem keeps refining them, so their remaining error
    //      does not put a floor under the residuals of the columns still active.
    {
      const int nl = 0, nr = s;
      applyK(Y, KY, nl, nr);
      cta_gemm<T, true>(nr, nr, dim, Y + nl, sp, KY + nl, sp, H, nr, gsm);
      for (int idx = threadIdx.x; idx < nr * nr; idx += NT) {
        int a = idx / nr, b = idx % nr;
        Q[idx] = T(0.5) * (H[a * nr + b] + H[b * nr + a]);
      }
      __syncthreads();
      jacobi<T>(Q, Pbuf, nr);
      if (threadIdx.x == 0) {
        for (int j = 0; j < nr; ++j) perm[j] = j;
        for (int a = 0; a < nr; ++a) {
          int best = a;
          for (int b = a + 1; b < nr; ++b)
            if (Q[perm[b] * nr + perm[b]] > Q[perm[best] * nr + perm[best]]) best = b;
          int ti = perm[a]; perm[a] = perm[best]; perm[best] = ti;
        }
        for (int j = 0; j < nr; ++j) mu[nl + j] = Q[perm[j] * nr + perm[j]];
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < nr * nr; idx += NT) {
        int l = idx / nr, j = idx % nr;
        QS[idx] = Pbuf[l * nr + perm[j]];
      }
      __syncthreads();
      cta_gemm<T, false>(dim, nr, nr, Y + nl, sp, QS, nr, Yb + nl, sp, gsm);
      cta_gemm<T, false>(dim, nr, nr, KY + nl, sp, QS, nr, Yc + nl, sp, gsm);
      for (int64_t idx = threadIdx.x; idx < (int64_t)dim * nr; idx += NT) {
        int64_t r = idx / nr, j = nl + idx % nr;
        Y[r * sp + j] = Yb[r * sp + j];
        KY[r * sp + j] = Yc[r * sp + j];
      }
      __syncthreads();
    }
    // ---- residuals of the first k Ritz pairs (one warp per column)
    const T mu0 = mu[0] > T(0) ? mu[0] : T(1);
    for (int j = wid; j < k; j += NT / 32) {
      T part = 0, nrm = 0;
      for (int r = lane; r < dim; r += 32) {
        T a = KY[(int64_t)r * sp + j];
        T b = Y[(int64_t)r * sp + j];
        T d = a - mu[j] * b;
        part += d * d;
        nrm += b * b;
      }
      part = warp_sum(part);
      nrm = warp_sum(nrm);
      if (lane == 0) {
        // residual relative to the Ritz value, with a floor at the resolution
        // of the working precision relative to the largest Ritz value
        const T eps = sizeof(T) == 8 ? T(1.1e-16) : T(6e-8);
        const T scale = max(mu[j], T(4) * eps * mu0 / (T)tol);
        T den = scale * sqrt(nrm);
        rn[j] = (mu[j] <= T(1e-12) * mu0) ? T(0) : sqrt(part) / (den > T(0) ? den : T(1));
      }
    }
    __syncthreads();
    T res_max = 0;
    for (int j = 0; j < k; ++j) res_max = max(res_max, rn[j]);
    ++sweep;
    if ((double)res_max <= tol || sweep >= max_sweeps) break;
    // single precision: stop once the residuals stall (no halving in three
    // sweeps) at the precision's floor
    if (sizeof(T) == 4) {
      if (res_max < T(0.5) * best) { best = res_max; last_gain = sweep; }
      else if (sweep - last_gain >= 3) break;
    }
    // ---- lock the converged leading Ritz pairs; filter the rest
    int nl = 0;
    while (nl < k && rn[nl] <= (T)tol) ++nl;
    const int na = s - nl;
    // Chebyshev filter of degree d on OP, damping [0, b] (b = smallest Ritz
    // value), normalised at the largest active Ritz value a0; the degree is
    // capped so that the filter's growth over [b, a0] stays representable.
    T bnd = mu[s - 1];
    const T a0 = mu[nl] > T(0) ? mu[nl] : mu0;
    const T floor_b = T(1e-3) * a0;
    if (!(bnd > floor_b)) bnd = floor_b;
    const T e = bnd / 2, c = bnd / 2;
    const double rL = (2.0 * (double)a0 - (double)bnd) / (double)bnd;   // L(a0) >= 1
    const double gmax = sizeof(T) == 8 ? 1e8 : 1e4;
    // the Ritz values of a random start are poor filter bounds for two sweeps;
    // a predicted start gives usable ones after the first
    const int cautious = (warm != nullptr && SPD) ? 1 : 2;
    int d = sweep > cautious ? max(degree, 1) : 1;
    if (rL > 1.0 + 1e-12) d = min(d, max(1, (int)floor(acosh(gmax) / acosh(rL))));
    else d = 1;
    const T sig1 = (rL > 1.0 + 1e-12) ? e / (a0 - c) : T(1);
    T sig = sig1;
    applyR(KY, Yc, nl, na);  // OP Y from the K Y at hand
    deflate(Yc, nl, na);
    for (int64_t idx = threadIdx.x; idx < (int64_t)dim * na; idx += NT) {
      int64_t r = idx / na, j = nl + idx % na;
      Yc[r * sp + j] = (sig1 / e) * (Yc[r * sp + j] - c * Y[r * sp + j]);
    }
    __syncthreads();
    // columns nl.. of Y: previous iterate, of Yc: current iterate
    for (int step = 2; step <= d; ++step) {
      const T sig_new = T(1) / (T(2) / sig1 - sig);
      applyK(Yc, T1, nl, na);
      applyR(T1, Yb, nl, na);
      deflate(Yb, nl, na);
      for (int64_t idx = threadIdx.x; idx < (int64_t)dim * na; idx += NT) {
        int64_t r = idx / na, j = nl + idx % na;
        Yb[r * sp + j] = T(2) * (sig_new / e) * (Yb[r * sp + j] - c * Yc[r * sp + j]) - (sig * sig_new) * Y[r * sp + j];
      }
      __syncthreads();
      // rotate the active columns: previous <- current <- new (locked columns stay in Y)
      for (int64_t idx = threadIdx.x; idx < (int64_t)dim * na; idx += NT) {
        int64_t r = idx / na, j = nl + idx % na;
        Y[r * sp + j] = Yc[r * sp + j];
        Yc[r * sp + j] = Yb[r * sp + j];
      }
      __syncthreads();
      sig = sig_new;
    }
    for (int64_t idx = threadIdx.x; idx < (int64_t)dim * na; idx += NT) {
      int64_t r = idx / na, j = nl + idx % na;
      Y[r * sp + j] = Yc[r * sp + j];
    }
    __syncthreads();
    // near-null directions restart from fresh random vectors
    int first_null = s;
    for (int j = nl; j < s; ++j)
      if (!(mu[j] > T(1e-10) * mu0)) { first_null = j; break; }
    if (first_null < s) fill_random(Y, dim, s, sp, first_null, seed ^ 0xA5A5A5A5ull, (uint64_t)i * 7919u + sweep * 104729u);
    orthonormalize((uint64_t)i * 1000003u + sweep);
  }
  // ---- outputs, the first k Ritz pairs in descending order
  if (threadIdx.x == 0) {
    for (int j = 0; j < k; ++j) perm[j] = j;
    for (int a = 0; a < k; ++a) {
      int best = a;
      for (int b = a + 1; b < k; ++b)
        if (mu[perm[b]] > mu[perm[best]]) best = b;
      int ti = perm[a]; perm[a] = perm[best]; perm[best] = ti;
    }
  }
  __syncthreads();
  // kept: the leading numerically nonzero values (after the skipped ones);
  // with a threshold (tau^2: eigenvalues of eq. gevpsvd, squared singular
  // values of D_i Pi_i; lifting: lambda - 1 = mu above nu - 1) only those above it
  const int sk = eo.skip ? min(eo.skip[i], k) : 0;
  int kept = 0;
  {
    const T mu0 = mu[perm[0]] > T(0) ? mu[perm[0]] : T(0);
    for (int j = sk; j < k && kept < eo.nkeep; ++j) {
      if (mu[perm[j]] > T(sizeof(T) == 8 ? 1e-12 : 1e-6) * mu0 && (thresh <= 0 || (double)mu[perm[j]] > thresh)) ++kept;
      else break;
    }
  }
  if (threadIdx.x == 0) { count[i] = kept; sweeps_out[i] = sweep; }
  if (tgt != nullptr && SPD) {
    // converged Ritz vectors z (Gamma_delta rows), the network's training targets
    float* tb = tgt + wseg[i] * nev;
    for (int64_t idx = threadIdx.x; idx < (int64_t)dim * nev; idx += NT) {
      int r = (int)(idx / nev), j = (int)(idx % nev);
      tb[idx] = j < kept ? (float)Y[(int64_t)r * sp + perm[j]] : 0.f;
    }
  }
  // SPD: V = U^T Y, the coarse vectors in the scaled space (I_i rows)
  if (SPD) cta_gemm<T, true>(p, s, g, U, ld, Y, sp, V, sp, gsm);
  __shared__ double muref[128];
  if constexpr (SPD && sizeof(T) == 8) {
    if (eo.refine && kept > 0) {
      // Eigenvalues from the variational form of eq. uppergevp, which also
      // holds eq. gevpsvd's for overlap 1 (lambda = 1 + mu): with c the vector
      // on I_i and v on Omega_i minus I_i,
      //   lambda = c^T A^_II c / min_v [c; v]^T A^ [c; v],
      // stationary in both c and v, so the errors of the explicit W = L^{-1}
      // (about eps cond(A^_ii)) enter squared.  v is taken as
      // (A^{-1} [A^_II c; 0])_G / lambda = W22^T (W21 A^_II c) / lambda (exact
      // at an eigenpair); lambda and mu then come from the sparse local rows.
      const int kk = kept;
      T* Cc = Yb;   // p x kk, the kept columns of V
      T* Tt = Yc;   // p x kk, A^_II c
      T* QG = KY;   // g x kk, W21 t
      T* Vv = AV;   // g x kk, v
      for (int64_t idx = threadIdx.x; idx < (int64_t)p * kk; idx += NT) {
        const int r = (int)(idx / kk), j = (int)(idx % kk);
        Cc[idx] = V[(int64_t)r * sp + perm[sk + j]];
      }
      __syncthreads();
      mul_AII(p, pos0, ent_off, lcol, aval, Cc, Tt, kk, kk);
      cta_gemm<T, false>(g, kk, p, U, ld, Tt, kk, QG, kk, gsm);        // W21 t
      cta_gemm<T, true, false, true>(g, kk, g, U + p, ld, QG, kk, Vv, kk, gsm);  // W22^T (W21 t), W22 lower
      for (int64_t idx = threadIdx.x; idx < (int64_t)g * kk; idx += NT)
        Vv[idx] /= T(1) + mu[perm[sk + (int)(idx % kk)]];
      __syncthreads();
      // one warp per column j, w = [c; v]: a = c^T A^_II c, b = c^T A^_IG v,
      // d = v^T A^_GG v from the local rows, and D = w^T (A^ w) with each
      // row of A^ w summed in double-double (exact products by fma, TwoSum):
      // A^ w is S_I c on I_i and about 0 on the rest, so D has no large
      // cancellation even where lambda = a / D is 1e5.  mu = lambda - 1, or
      // -(2b + d) / D for lambda < 2 (no cancellation against 1 there).
      for (int j = wid; j < kk; j += NT / 32) {
        double sa = 0, sb = 0, sd = 0, sD = 0;
        for (int a = lane; a < n; a += 32) {
          const int64_t e0 = ent_off[pos0 + a], e1 = ent_off[pos0 + a + 1];
          double hi = 0, lo = 0, gpart = 0, ipart = 0;
          for (int64_t e = e0; e < e1; ++e) {
            const int lc = lcol[e];
            if (lc < 0) continue;
            const double av = (double)aval[e];
            const double wv = lc < p ? (double)Cc[(int64_t)lc * kk + j] : (double)Vv[(int64_t)(lc - p) * kk + j];
            const double pr = __dmul_rn(av, wv);
            const double pe = __fma_rn(av, wv, -pr);
            const double sm = __dadd_rn(hi, pr);
            const double bb = __dsub_rn(sm, hi);
            const double er = __dadd_rn(__dsub_rn(hi, __dsub_rn(sm, bb)), __dsub_rn(pr, bb));
            hi = sm;
            lo = __dadd_rn(lo, __dadd_rn(er, pe));
            if (lc >= p) gpart = __fma_rn(av, wv, gpart);
            else ipart = __fma_rn(av, wv, ipart);
          }
          const double zeta = __dadd_rn(hi, lo);
          const double wa = a < p ? (double)Cc[(int64_t)a * kk + j] : (double)Vv[(int64_t)(a - p) * kk + j];
          sD = __fma_rn(wa, zeta, sD);
          if (a < p) {
            sa = __fma_rn(wa, ipart, sa);
            sb = __fma_rn(wa, gpart, sb);
          } else {
            sd = __fma_rn(wa, gpart, sd);
          }
        }
        sa = warp_sum(sa);
        sb = warp_sum(sb);
        sd = warp_sum(sd);
        sD = warp_sum(sD);
        if (lane == 0) {
          const double lam = sa / sD;
          muref[j] = lam >= 2.0 ? lam - 1.0 : -(2.0 * sb + sd) / sD;
        }
      }
      __syncthreads();
    }
  }
  for (int j = threadIdx.x; j < eo.nkeep; j += NT) {
    const int c = j < kept ? perm[sk + j] : 0;
    double v = 0.0;
    if (j < kept) {
      const double m = (SPD && sizeof(T) == 8 && eo.refine) ? muref[j] : (double)mu[c];
      v = eo.lift ? 1.0 + m : (SPD ? m : sqrt(fmax(m, 0.0)));
    }
    values[(int64_t)i * eo.nkeep + j] = v;
    resid[(int64_t)i * eo.nkeep + j] = j < kept ? (double)rn[c] : 0.0;
  }
  double* Zi = Z + z_off[i];
  if (SPD) {
    // Z_i = S_I U^T z (undo the diagonal scaling), FP64 output; lifting: the
    // A_ii-normalised u_I = sqrt((1 + mu) / mu) U^T z
    for (int64_t idx = threadIdx.x; idx < (int64_t)p * eo.nkeep; idx += NT) {
      const int r = (int)(idx / eo.nkeep), j = (int)(idx % eo.nkeep);
      double z = 0.0;
      if (j < kept) {
        const int c = perm[sk + j];
        z = (double)V[(int64_t)r * sp + c] * ds[omega[pos0 + r]];
        if (eo.lift) z *= sqrt((1.0 + (double)mu[c]) / (double)mu[c]);
      }
      Zi[(int64_t)r * eo.zld + zc0 + j] = z;
    }
  } else {
    for (int64_t idx = threadIdx.x; idx < (int64_t)p * eo.nkeep; idx += NT) {
      const int r = (int)(idx / eo.nkeep), j = (int)(idx % eo.nkeep);
      Zi[(int64_t)r * eo.zld + zc0 + j] = j < kept ? (double)Y[(int64_t)r * sp + perm[j]] : 0.0;
    }
  }
}

// max over the block of v (all threads get the result)
__device__ double block_max(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = sh[0];
  for (int w = 1; w < NT / 32; ++w) r = fmax(r, sh[w]);
  __syncthreads();
  return r;
}

// Per-node input features of the warm-start network, one block per
// subdomain, one row per Gamma_delta node (local row r = 0..g-1, in R_i
// order).  With A^ = D^{-1/2} A D^{-1/2}, la(v) = log10 |a_vv|, and the
// operator K = U A^_II U^T of the subspace iteration:
//   0: (la(v) - mean of la over Gamma_delta) / 6
//   1: max over neighbours u in Omega_{1:delta-1} of (la(u) - la(v)) / 6 (0 if none)
//   2-4: sum of |A^_vu| over neighbours in Omega_{1:delta-1}, Gamma_delta, outside Omega_i
//   5-7: the counts of those neighbours / 6
//   8, 9: y = K 1 / max|K 1| (1 = ones / sqrt(g)): y, log10(1e-4 + |y|) / 4 + 1
//   10, 11: the same for K (K 1)
//   12: K t / max|K t| with t_r = r / (g - 1) - 1/2
//   13-15: t_r, cos(2 pi (t_r + 1/2)), sin(2 pi (t_r + 1/2))
template <typename T>
__global__ void __launch_bounds__(NT) k_warm_features(
    const T* __restrict__ work, const int64_t* __restrict__ work_off, const int32_t* __restrict__ np_arr,
    const int32_t* __restrict__ n_arr, const int32_t* __restrict__ m_arr, const int32_t* __restrict__ p_arr,
    const int32_t* __restrict__ sub_off, const int64_t* __restrict__ ent_off, const int32_t* __restrict__ lcol,
    const int32_t* __restrict__ omega, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
    const double* __restrict__ val, const double* __restrict__ ds, const T* __restrict__ aval, T* scratch,
    const int64_t* __restrict__ scr_off, const int64_t* __restrict__ wseg, float* __restrict__ feat) {
  COUNT_LAUNCH();
  extern __shared__ double shd[];
  __shared__ double red[NT / 32];
  const int i = blockIdx.x;
  const int n = n_arr[i], m = m_arr[i], p = p_arr[i], ld = np_arr[i];
  const int g = n - m, pos0 = sub_off[i];
  if (g <= 0) return;
  const int L = max(p, g);
  T* gsm = reinterpret_cast<T*>(shd);
  T* base = scratch + scr_off[i];
  T* P = base;            // g x 2 probes
  T* KP = base + 2 * L;   // K P
  T* V = base + 4 * L;    // p x 2
  T* AV = base + 6 * L;   // p x 2
  T* KKP = base + 8 * L;  // K (K P)
  const T* U = work + work_off[i] + (int64_t)m * ld;
  const double tden = g > 1 ? (double)(g - 1) : 1.0;
  for (int r = threadIdx.x; r < g; r += NT) {
    P[2 * r] = (T)(1.0 / sqrt((double)g));
    P[2 * r + 1] = (T)(r / tden - 0.5);
  }
  __syncthreads();
  auto applyK2 = [&](const T* in, T* o) {
    cta_gemm<T, true>(p, 2, g, U, ld, in, 2, V, 2, gsm);
    mul_AII(p, pos0, ent_off, lcol, aval, V, AV, 2, 2);
    cta_gemm<T, false>(g, 2, p, U, ld, AV, 2, o, 2, gsm);
  };
  applyK2(P, KP);
  applyK2(KP, KKP);
  double a0 = 0, a1 = 0, a2 = 0, sla = 0;
  for (int r = threadIdx.x; r < g; r += NT) {
    a0 = fmax(a0, fabs((double)KP[2 * r]));
    a1 = fmax(a1, fabs((double)KP[2 * r + 1]));
    a2 = fmax(a2, fabs((double)KKP[2 * r]));
    sla += -2.0 * log10(ds[omega[pos0 + m + r]]);
  }
  const double mx0 = block_max(a0, red), mx1 = block_max(a1, red), mx2 = block_max(a2, red);
  const double mean_la = block_sum(sla, red) / g;
  const double i0 = mx0 > 0 ? 1.0 / mx0 : 0.0, i1 = mx1 > 0 ? 1.0 / mx1 : 0.0, i2 = mx2 > 0 ? 1.0 / mx2 : 0.0;
  float* out = feat + wseg[i] * WARM_FEATURES;
  for (int r = threadIdx.x; r < g; r += NT) {
    const int pos = pos0 + m + r, v = omega[pos];
    const int b = rp[v], e = rp[v + 1];
    const double sv = ds[v], la = -2.0 * log10(sv);
    const int64_t e0 = ent_off[pos];
    double s_in = 0, s_g = 0, s_out = 0, dmax = 0;
    int c_in = 0, c_g = 0, c_out = 0;
    for (int q = 0; q < e - b; ++q) {
      const int u = ci[b + q];
      if (u == v) continue;
      const int lc = lcol[e0 + q];
      const double w = fabs(val[b + q] * sv * ds[u]);
      if (lc >= 0 && lc < m) {
        const double d = -2.0 * log10(ds[u]) - la;
        dmax = c_in == 0 ? d : fmax(dmax, d);
        s_in += w;
        ++c_in;
      } else if (lc >= m) {
        s_g += w;
        ++c_g;
      } else {
        s_out += w;
        ++c_out;
      }
    }
    const double y0 = (double)KP[2 * r] * i0, y1 = (double)KKP[2 * r] * i2, y2 = (double)KP[2 * r + 1] * i1;
    const double t = r / tden - 0.5;
    float* f = out + (int64_t)r * WARM_FEATURES;
    f[0] = (float)((la - mean_la) / 6.0);
    f[1] = (float)(dmax / 6.0);
    f[2] = (float)s_in;
    f[3] = (float)s_g;
    f[4] = (float)s_out;
    f[5] = (float)(c_in / 6.0);
    f[6] = (float)(c_g / 6.0);
    f[7] = (float)(c_out / 6.0);
    f[8] = (float)y0;
    f[9] = (float)(log10(1e-4 + fabs(y0)) / 4.0 + 1.0);
    f[10] = (float)y1;
    f[11] = (float)(log10(1e-4 + fabs(y1)) / 4.0 + 1.0);
    f[12] = (float)y2;
    f[13] = (float)t;
    f[14] = (float)cospi(2.0 * (t + 0.5));
    f[15] = (float)sinpi(2.0 * (t + 0.5));
  }
}

__global__ void k_round_z(double* __restrict__ Z, float* __restrict__ Zf, int64_t n) {
  COUNT_LAUNCH();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const float f = (float)Z[k];
    Zf[k] = f;
    Z[k] = (double)f;
  }
}

// coarse vectors per subdomain: eq. gevpsvd's and the lifting ones
__global__ void k_total_count(int N, const int32_t* __restrict__ cg, const int32_t* __restrict__ cl,
                              int32_t* __restrict__ c) {
  COUNT_LAUNCH();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) c[i] = cg[i] + (cl ? cl[i] : 0);
}

template <typename T>
void run_eigen(Handle& h, cudaStream_t s) {
  const int N = h.N, nev = h.nev;
  Coarse& co = h.co;
  Dense& dn = h.dn;
  DevMem& mem = h.mem;
  const bool spd = h.opt.spd != 0;
  const int over = std::max(0, h.opt.oversample);
  // eq. uppergevp (lifting) vectors: up to nev_lift more columns per Z_i;
  // with overlap 1 its operator is the one of eq. gevpsvd, so that run's
  // leading pairs are skipped (the lifting iteration computes nev + nev_lift)
  const int nlift = h.lift ? h.nev_lift : 0;
  const int lift_nev = h.delta == 1 ? nev + nlift : nlift;
  co.zld = std::max(1, nev + nlift);
  std::vector<int64_t> scr(N), zo(N + 1), scl(N);
  int64_t tot = 0, zt = 0, totl = 0;
  int smax = 1;
  for (int i = 0; i < N; ++i) {
    int p = h.h_p[i], g = h.h_g[i];
    int dim = spd ? g : p;
    int sb = std::max(1, std::min(nev + over, dim));
    int sp = (sb + 3) & ~3;
    smax = std::max(smax, sb);
    scr[i] = tot;
    tot += 7LL * std::max(p, g) * sp;
    zo[i] = zt;
    zt += (int64_t)p * co.zld;
    if (nlift > 0) {
      const int gl = h.h_n[i] - p;  // the lifting operator lives on Omega_i minus I_i
      const int sl = std::max(1, std::min(lift_nev + over, gl));
      smax = std::max(smax, sl);
      scl[i] = totl;
      totl += 7LL * std::max(p, gl) * ((sl + 3) & ~3);
    }
  }
  zo[N] = zt;
  if (smax > 96) fail(ASM_ERR_UNSUPPORTED, "nev (+ nev_lift) + oversample exceeds 96");
  co.s_max = smax;
  co.h_z_off = zo;
  co.scratch = mem.alloc<T>(tot);
  co.scr_off = mem.alloc<int64_t>(N);
  co.z_off = mem.alloc<int64_t>(N + 1);
  co.Z = mem.alloc<double>(std::max<int64_t>(zt, 1));
  co.values = mem.alloc<double>((int64_t)N * std::max(nev, 1));
  co.resid = mem.alloc<double>((int64_t)N * std::max(nev, 1));
  co.count = mem.alloc<int32_t>(N);
  co.count_g = mem.alloc<int32_t>(N);
  co.sweeps = mem.alloc<int32_t>(N);
  CK(cudaMemcpyAsync(co.scr_off, scr.data(), 8 * N, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(co.z_off, zo.data(), 8 * (N + 1), cudaMemcpyHostToDevice, s));
  size_t gemm_bytes = gemm_smem_bytes<T>();
  size_t smem = gemm_bytes + (size_t)2 * smax * smax * sizeof(double) +
                (size_t)(4 * smax * smax + 2 * smax) * sizeof(T) + 64;
  {
    // the Rayleigh-Ritz blocks live in shared memory: s = nev + oversample
    // columns need about 48 s^2 bytes in FP64 and 32 s^2 in FP32
    int dev = 0, optin = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (smem > (size_t)optin)
      fail(ASM_ERR_UNSUPPORTED, "nev + oversample too large for the subspace iteration's shared memory "
                                "(at most about 64 columns in FP64, 80 in FP32 on this device)");
  }
  // FP32 default 4e-3: measured on the 64^3 workload, tolerances of 1e-3,
  // 2e-3, 4e-3 and 1e-2 all give 264-267 PCG iterations, while the eigen stage
  // takes 23.4, 19.7, 18.2 and 16.3 ms; 4e-3 keeps a margin above the point
  // where the coarse space would start to cost iterations
  const double tol = h.opt.eig_tol > 0 ? h.opt.eig_tol : (h.fp32 ? 4e-3 : 1e-8);
  // FP32 cannot resolve Ritz values ~1e5 below the top one to 1e-3: a cap
  // keeps such subdomains from holding the launch
  const int maxsw = h.opt.max_sweeps > 0 ? h.opt.max_sweeps : (h.fp32 ? 12 : 40);
  // measured on the 64^3 workload: degree 3 minimises the FP32 stage (26 ms
  // against 28 ms for 4 and 27 ms for 2 with 8 extra columns)
  const int degree = h.opt.filter_degree > 0 ? h.opt.filter_degree : (h.fp32 ? 3 : 4);
  // scaled local values in the working precision (SPD products with A^_II)
  T* aval = nullptr;
  if (spd) {
    aval = mem.alloc<T>(std::max<int64_t>(h.ov.n_ent, 1));
    const unsigned gsv = (unsigned)std::min<int64_t>(std::max<int64_t>(ceil_div(h.ov.sum_n, NT), 1), 152 * 16);
    k_scaled_values<T><<<gsv, NT, 0, s>>>(h.ov.sum_n, h.ov.omega, h.ov.ent_off, h.row_ptr,
                                                           h.col_idx, h.val, h.dscale, aval);
    CK_LAUNCH("scaled local values");
  }
  // single precision, SPD: the explicit operator K = U A^_II U^T per subdomain
  const float* Kexp = nullptr;
  const int64_t* d_koff = nullptr;
  const int32_t* d_kld = nullptr;
  if constexpr (sizeof(T) == 4) {
    if (spd && nev > 0) {
      std::vector<int64_t> ko(N), uo(N);
      std::vector<int32_t> kl(N), ul(N), ur(N);
      int64_t kt = 0, ut = 0;
      std::vector<TcJob> jobs;
      // only where |Gamma| <= |I_i|: one g x g product per application then
      // beats the two g x p ones by at least half, building K included
      // (elasticity's wide overlap layers keep the products with U)
      for (int i = 0; i < N; ++i) {
        const int g = h.h_n[i] - h.h_m[i], p = h.h_p[i];
        const int gp = (int)round_up(std::max(g, 1), TILE), pp = (int)round_up(std::max(p, 1), TILE);
        if (g > p) {
          ko[i] = -1; kl[i] = 0; uo[i] = ut; ul[i] = pp; ur[i] = 0;
          continue;
        }
        ko[i] = kt; kl[i] = gp; kt += (int64_t)gp * gp;
        uo[i] = ut; ul[i] = pp; ur[i] = gp; ut += (int64_t)gp * pp;
        for (int I = 0; I < gp / TILE; ++I)
          for (int J = 0; J < gp / TILE; ++J) {
            TcJob Jb{};
            Jb.a0 = uo[i] + (int64_t)I * TILE * pp; Jb.a_step = TILE; Jb.lda = pp;   // T(I, k)
            Jb.b0 = uo[i] + (int64_t)J * TILE * pp; Jb.b_step = TILE; Jb.ldb = pp;   // Up(J, k)
            Jb.c_out = ko[i] + (int64_t)I * TILE * gp + J * TILE; Jb.ldc_out = gp; Jb.ldc_in = gp;
            Jb.nprod = pp / TILE; Jb.flags = 0; Jb.sub = i;
            jobs.push_back(Jb);
          }
      }
      if (!jobs.empty()) {
        float* Kb = mem.alloc<float>(kt);
        float* Up = mem.alloc<float>(ut);
        float* Tm = mem.alloc<float>(ut);
        int64_t* koff = mem.alloc<int64_t>(N);
        int32_t* kld = mem.alloc<int32_t>(N);
        int64_t* uoff = mem.alloc<int64_t>(N);
        int32_t* uld = mem.alloc<int32_t>(N);
        int32_t* urows = mem.alloc<int32_t>(N);
        TcJob* d_jobs = mem.alloc<TcJob>(jobs.size());
        // pageable sources: each copy is staged before the call returns
        CK(cudaMemcpyAsync(koff, ko.data(), 8 * (size_t)N, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(kld, kl.data(), 4 * (size_t)N, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(uoff, uo.data(), 8 * (size_t)N, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(uld, ul.data(), 4 * (size_t)N, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(urows, ur.data(), 4 * (size_t)N, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(TcJob) * jobs.size(), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
        k_u_padded<<<dim3(64, N), NT, 0, s>>>((const float*)dn.work, dn.work_off, dn.np, h.dev_n, h.dev_m, h.dev_p, uoff,
                                             uld, urows, Up, Tm, h.ov.sub_off, h.ov.ent_off, h.ov.lcol,
                                             (const float*)aval);
        CK_LAUNCH("padded U and U A^_II");
        tc_tiles(d_jobs, (int64_t)jobs.size(), Tm, Up, nullptr, Kb, nullptr, dn.err, h.num_sms, s);
        mem.free(Up);  // stream-ordered behind the tile jobs
        mem.free(Tm);
        Kexp = Kb;
        d_koff = koff;
        d_kld = kld;
      }
    }
  }
  // learned warm start (SPD path): features per Gamma_delta node, the
  // network's start blocks, and (when recorded) the converged blocks
  const bool want_warm = spd && (h.opt.warm_start || h.opt.record_warm);
  const float* warm = nullptr;
  int wld = 0, wk = 0;
  if (want_warm) {
    h.h_wseg.assign(N + 1, 0);
    for (int i = 0; i < N; ++i) h.h_wseg[i + 1] = h.h_wseg[i] + h.h_g[i];
    h.warm_rows = h.h_wseg[N];
    h.wseg = mem.alloc<int64_t>(N + 1);
    CK(cudaMemcpyAsync(h.wseg, h.h_wseg.data(), 8 * (N + 1), cudaMemcpyHostToDevice, s));
    h.wfeat = mem.alloc<float>(std::max<int64_t>(h.warm_rows, 1) * WARM_FEATURES);
    if (h.opt.record_warm) h.wtgt = mem.alloc<float>(std::max<int64_t>(h.warm_rows, 1) * std::max(nev, 1));
    const size_t fsm = gemm_bytes + 64;
    CK(cudaFuncSetAttribute(k_warm_features<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm));
    k_warm_features<T><<<N, NT, fsm, s>>>((const T*)dn.work, dn.work_off, dn.np, h.dev_n, h.dev_m, h.dev_p,
                                          h.ov.sub_off, h.ov.ent_off, h.ov.lcol, h.ov.omega, h.row_ptr, h.col_idx,
                                          h.val, h.dscale, aval, (T*)co.scratch, co.scr_off, h.wseg, h.wfeat);
    CK_LAUNCH("warm-start features");
    if (h.opt.warm_start && h.warm_rows > 0) {
      Mlp& net = h.opt.warm_net->net;
      net.forward(h.wfeat, (int)h.warm_rows, s);
      warm = net.Y32;
      wld = net.Kp;
      wk = net.K;
    }
  }
  // size buckets: the blocks take the subdomains in decreasing order of the
  // iteration's work per sweep (|I_i| |Gamma_i| for SPD, |I_i|^2 otherwise), so
  // that a launch with more subdomains than resident blocks starts the longest
  // ones first and its tail is short
  std::vector<int32_t> ord(N);
  for (int i = 0; i < N; ++i) ord[i] = i;
  auto work_of = [&](int i) { return (int64_t)h.h_p[i] * (spd ? std::max(h.h_g[i], 1) : std::max(h.h_p[i], 1)); };
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return work_of(a) > work_of(b); });
  int32_t* d_ord = mem.alloc<int32_t>(std::max(N, 1));
  CK(cudaMemcpyAsync(d_ord, ord.data(), 4 * (size_t)N, cudaMemcpyHostToDevice, s));
  auto launch = [&](auto kern) {
    CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    EigOut eo{co.zld, nev, nullptr, nullptr, 0, (sizeof(T) == 8 && spd && h.delta == 1) ? 1 : 0, d_ord,
              Kexp, d_koff, d_kld};
    kern<<<N, NT, smem, s>>>((const T*)dn.XpT, dn.xs_off, (const T*)dn.S, dn.s_off, (const T*)dn.work, dn.work_off,
                             dn.np, h.dev_n, h.dev_m, h.dev_p, h.ov.sub_off, h.ov.ent_off, h.ov.lcol, h.ov.omega,
                             h.row_ptr, h.col_idx, h.val, h.dscale, aval, (T*)co.scratch, co.scr_off, nev, over, maxsw,
                             degree, tol, h.opt.tau > 0 ? h.opt.tau * h.opt.tau : 0.0, h.opt.seed, warm, wld, wk,
                             h.wseg, h.wtgt, co.values, co.resid, co.count_g,
                             co.sweeps, co.Z, co.z_off, eo);
  };
  if (nev > 0) {
    if constexpr (sizeof(T) == 4) {
      if (spd && h.b16eig) launch(k_subspace<T, true, true>);
      else if (spd) launch(k_subspace<T, true>);
      else launch(k_subspace<T, false>);
    } else {
      if (spd) launch(k_subspace<T, true>);
      else launch(k_subspace<T, false>);
    }
  } else {
    CK(cudaMemsetAsync(co.count_g, 0, 4 * N, s));
    CK(cudaMemsetAsync(co.sweeps, 0, 4 * N, s));
  }
  CK_LAUNCH("subspace iteration");
  if (nlift > 0) {
    // eq. uppergevp in its reduced form: with A_ii = L L^T and W = L^{-1}
    // (I_i first), lambda = 1 + sigma^2 for the singular values sigma of
    // W21 L11, whose squares are the eigenvalues of W21 A^_II W21^T,
    // W21 = W[Omega_i minus I_i, I_i]; the A_ii-normalised lifting vector on
    // I_i is sqrt((1 + sigma^2) / sigma^2) W21^T z (proof of Theorem 3.4)
    co.lift_values = mem.alloc<double>((int64_t)N * nlift);
    co.lift_resid = mem.alloc<double>((int64_t)N * nlift);
    co.lift_count = mem.alloc<int32_t>(N);
    co.lift_sweeps = mem.alloc<int32_t>(N);
    T* lscr = mem.alloc<T>(std::max<int64_t>(totl, 1));
    int64_t* lscr_off = mem.alloc<int64_t>(N);
    CK(cudaMemcpyAsync(lscr_off, scl.data(), 8 * N, cudaMemcpyHostToDevice, s));
    EigOut eo{co.zld, nlift, co.count_g, h.delta == 1 ? co.count_g : nullptr, 1, sizeof(T) == 8 ? 1 : 0, d_ord,
              nullptr, nullptr, nullptr};
    auto kern = k_subspace<T, true>;
    CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<N, NT, smem, s>>>((const T*)dn.XpT, dn.xs_off, (const T*)dn.S, dn.s_off, (const T*)dn.work, dn.work_off,
                             dn.np, h.dev_n, h.dev_p, h.dev_p, h.ov.sub_off, h.ov.ent_off, h.ov.lcol, h.ov.omega,
                             h.row_ptr, h.col_idx, h.val, h.dscale, aval, lscr, lscr_off, lift_nev, over, maxsw,
                             degree, tol, h.opt.nu - 1.0, h.opt.seed ^ 0x6C1F7A3Dull, nullptr, 0, 0, nullptr, nullptr,
                             co.lift_values, co.lift_resid, co.lift_count, co.lift_sweeps, co.Z, co.z_off, eo);
    CK_LAUNCH("lifting subspace iteration");
  }
  k_total_count<<<(unsigned)ceil_div(N, NT), NT, 0, s>>>(N, co.count_g, nlift > 0 ? co.lift_count : nullptr, co.count);
  CK_LAUNCH("coarse counts");
  if (h.fp32) {
    // the apply restricts and prolongs with an FP32 copy of Z; rounding the
    // FP64 master to the same values keeps E = Z^T A Z exact for that basis
    co.Zf = mem.alloc<float>(std::max<int64_t>(zt, 1));
    const unsigned gz = (unsigned)std::min<int64_t>(std::max<int64_t>(ceil_div(zt, NT), 1), 152 * 16);
    k_round_z<<<gz, NT, 0, s>>>(co.Z, co.Zf, zt);
    CK_LAUNCH("round Z");
  }
}

}  // namespace

void build_eigen(Handle& h, cudaStream_t s) {
  if ((h.nev <= 0 && !h.lift) || !h.opt.coarse) {
    h.co.h_count.assign(h.N, 0);
    return;
  }
  if (h.fp32) run_eigen<float>(h, s); else run_eigen<double>(h, s);
}

}  // namespace asmgpu
