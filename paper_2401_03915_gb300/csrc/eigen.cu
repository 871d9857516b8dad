// Local coarse vectors by randomized block subspace iteration, one block per
// subdomain, all subdomains in one launch.
//
// SPD (eq. gevpsvd, Section 5.1).  With X = -B^{-1}C, X_p its first |I_i| rows,
// S = G - C^T B^{-1} C and K = X_p^T A_{I_i,I_i} X_p, every eigenpair of
// eq. gevpsvd with lambda^2 > 0 satisfies K y = lambda^2 S y with y = w_Gamma,
// the A_ii-normalisation of w is the S-normalisation of y, and the coarse
// vector R_i^T D_i Pi_i w is [X_p y; 0] on Omega_{I_i}.  The iteration runs on
// S^{-1} K (S^{-1} is the trailing block of A_ii^{-1} left by the sweep) with
// S-orthonormal blocks and Rayleigh-Ritz on Y^T K Y.
//
// General A (Section 5 of the paper's nonsymmetric extension).  D_i Pi_i is
// nonzero only in rows I_i and columns Gamma_delta, where it equals X_p, so
// its left singular vectors are those of X_p: the iteration runs on
// X_p X_p^T with Euclidean orthonormal blocks, and the kept vectors are the
// coarse vectors themselves.  The Euclidean SVD is not invariant under the
// diagonal scaling of the local sweep, so here the scaling is undone inside
// the products with X_p.
//
// Each sweep: power step, CholQR2 re-orthonormalisation (Gram in FP64),
// Rayleigh-Ritz with a cyclic Jacobi eigensolver (Golub & Van Loan, Alg.
// 8.5.3) of the small projected matrix, and a relative eigen-residual test.
#include <algorithm>

#include "handle.cuh"

namespace asmgpu {
namespace {

constexpr int NT = 256;
constexpr int NW = NT / 32;
constexpr int JC = 16;  // column chunk held in registers

struct SubdomainView {
  int n, m, p, g, ld;
  const void* XpT;
  const void* S;
  const void* R;  // S^{-1}: trailing block of A_ii^{-1} (ld = padded size)
  int64_t ent0;   // first entry of row 0 of Omega_i in the local CSR
  int pos0;       // omega position of row 0
};

// Diagonal scalings of the general path: X_p = S_I X^_p S_G^{-1}, where X^_p
// comes from the scaled sweep and S = D^{-1/2}.  Null pointers: no scaling.
struct XScale {
  const double* ds = nullptr;
  const int32_t* omI = nullptr;   // omega of I_i
  const int32_t* omG = nullptr;   // omega of Gamma_delta
  __device__ double sI(int r) const { return ds ? ds[omI[r]] : 1.0; }
  __device__ double sG(int k) const { return ds ? ds[omG[k]] : 1.0; }
};

// V (p x s) = X_p Y (Y: g x s); XpT is g x p row-major.
template <typename T>
__device__ void mul_Xp(const T* __restrict__ XpT, int p, int g, const T* __restrict__ Y, T* __restrict__ V, int s,
                       int ncols, XScale sc = XScale()) {
  for (int r = threadIdx.x; r < p; r += NT) {
    for (int j0 = 0; j0 < ncols; j0 += JC) {
      T acc[JC];
#pragma unroll
      for (int q = 0; q < JC; ++q) acc[q] = 0;
      for (int k = 0; k < g; ++k) {
        T x = XpT[(int64_t)k * p + r];
        if (sc.ds) x = (T)((double)x / sc.sG(k));
        const T* y = Y + (int64_t)k * s + j0;
#pragma unroll
        for (int q = 0; q < JC; ++q)
          if (j0 + q < ncols) acc[q] += x * y[q];
      }
      const T f = (T)sc.sI(r);
#pragma unroll
      for (int q = 0; q < JC; ++q)
        if (j0 + q < ncols) V[(int64_t)r * s + j0 + q] = acc[q] * f;
    }
  }
}

// W (g x s) = X_p^T V (V: p x s): one warp per output row.
template <typename T>
__device__ void mul_XpT(const T* __restrict__ XpT, int p, int g, const T* __restrict__ V, T* __restrict__ W, int s,
                        XScale sc = XScale()) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = wid; k < g; k += NW) {
    const T* xr = XpT + (int64_t)k * p;
    for (int j0 = 0; j0 < s; j0 += JC) {
      T acc[JC];
#pragma unroll
      for (int q = 0; q < JC; ++q) acc[q] = 0;
      for (int r = lane; r < p; r += 32) {
        T x = xr[r];
        if (sc.ds) x = (T)((double)x * sc.sI(r));
        const T* v = V + (int64_t)r * s + j0;
#pragma unroll
        for (int q = 0; q < JC; ++q)
          if (j0 + q < s) acc[q] += x * v[q];
      }
      const T f = (T)(1.0 / sc.sG(k));
#pragma unroll
      for (int q = 0; q < JC; ++q) {
        T t = warp_sum(acc[q]);
        if (lane == 0 && j0 + q < s) W[(int64_t)k * s + j0 + q] = t * f;
      }
    }
  }
}

// AV (p x s) = A_{I,I} V, from the local CSR (columns < p).
template <typename T>
__device__ void mul_AII(const SubdomainView& sv, const int32_t* __restrict__ omega, const int32_t* __restrict__ rp,
                        const int32_t* __restrict__ ci, const double* __restrict__ val,
                        const double* __restrict__ ds, const int64_t* __restrict__ ent_off,
                        const int32_t* __restrict__ lcol, const T* __restrict__ V, T* __restrict__ AV, int s) {
  for (int a = threadIdx.x; a < sv.p; a += NT) {
    int v = omega[sv.pos0 + a];
    int b = rp[v], e = rp[v + 1];
    const double sv_ = ds[v];
    int64_t e0 = ent_off[sv.pos0 + a];
    for (int j0 = 0; j0 < s; j0 += JC) {
      T acc[JC];
#pragma unroll
      for (int q = 0; q < JC; ++q) acc[q] = 0;
      for (int t = 0; t < e - b; ++t) {
        int lc = lcol[e0 + t];
        if (lc < 0 || lc >= sv.p) continue;
        T w = (T)(val[b + t] * sv_ * ds[ci[b + t]]);
        const T* vr = V + (int64_t)lc * s + j0;
#pragma unroll
        for (int q = 0; q < JC; ++q)
          if (j0 + q < s) acc[q] += w * vr[q];
      }
#pragma unroll
      for (int q = 0; q < JC; ++q)
        if (j0 + q < s) AV[(int64_t)a * s + j0 + q] = acc[q];
    }
  }
}

// W (g x s) = Mat Y for a symmetric g x g Mat with leading dimension ld
// (read by columns so that consecutive threads read consecutive addresses).
template <typename T>
__device__ void mul_sym(const T* __restrict__ Mat, int ld, int g, const T* __restrict__ Y, T* __restrict__ W, int s) {
  for (int k = threadIdx.x; k < g; k += NT) {
    for (int j0 = 0; j0 < s; j0 += JC) {
      T acc[JC];
#pragma unroll
      for (int q = 0; q < JC; ++q) acc[q] = 0;
      for (int t = 0; t < g; ++t) {
        T mv = Mat[(int64_t)t * ld + k];
        const T* y = Y + (int64_t)t * s + j0;
#pragma unroll
        for (int q = 0; q < JC; ++q)
          if (j0 + q < s) acc[q] += mv * y[q];
      }
#pragma unroll
      for (int q = 0; q < JC; ++q)
        if (j0 + q < s) W[(int64_t)k * s + j0 + q] = acc[q];
    }
  }
}

// G (s x s, FP64, shared) = A^T B over L rows.
template <typename T>
__device__ void gram(const T* __restrict__ A, const T* __restrict__ B, int L, int s, double* G) {
  const int npair = s * s;
  for (int idx = threadIdx.x; idx < npair; idx += NT) {
    int t = idx / s, u = idx % s;
    double acc = 0;
    for (int r = 0; r < L; ++r) acc += (double)A[(int64_t)r * s + t] * (double)B[(int64_t)r * s + u];
    G[idx] = acc;
  }
  __syncthreads();
}

// OUT (L x s) = IN (L x s) * Mat (s x s, shared, FP64 or T), rows in parallel.
template <typename T, typename MT>
__device__ void right_mul(const T* __restrict__ IN, T* __restrict__ OUT, int L, int s, const MT* Mat) {
  for (int r = threadIdx.x; r < L; r += NT) {
    const T* in = IN + (int64_t)r * s;
    for (int j0 = 0; j0 < s; j0 += JC) {
      MT acc[JC];
#pragma unroll
      for (int q = 0; q < JC; ++q) acc[q] = 0;
      for (int l = 0; l < s; ++l) {
        MT x = (MT)in[l];
#pragma unroll
        for (int q = 0; q < JC; ++q)
          if (j0 + q < s) acc[q] += x * Mat[l * s + j0 + q];
      }
#pragma unroll
      for (int q = 0; q < JC; ++q)
        if (j0 + q < s) OUT[(int64_t)r * s + j0 + q] = (T)acc[q];
    }
  }
  __syncthreads();
}

// Cholesky of the s x s Gram matrix G (warp 0), then Minv = L^{-T} so that
// Y <- Y Minv is orthonormal in the metric of G.  Returns false if a pivot
// is not positive (dependent block).
__device__ bool chol_inv_t(double* G, double* Minv, int s, int* flag) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int ok = 1;
    for (int j = 0; j < s; ++j) {
      double d = G[j * s + j];
      for (int k = 0; k < j; ++k) d -= G[j * s + k] * G[j * s + k];
      if (!(d > 0)) { ok = 0; d = 1e-300; }
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
    // lower-triangular inverse, column by column (lane = column)
    for (int c = lane; c < s; c += 32) {
      for (int r = 0; r < s; ++r) Minv[r * s + c] = 0;
      for (int r = c; r < s; ++r) {
        double v = (r == c) ? 1.0 : 0.0;
        for (int k = c; k < r; ++k) v -= G[r * s + k] * Minv[k * s + c];  // Minv holds L^{-1} temporarily as [r][c]
        Minv[r * s + c] = v / G[r * s + r];
      }
    }
    __syncwarp();
    // transpose in place: Minv[l][j] = Linv[j][l]
    for (int idx = lane; idx < s * s; idx += 32) {
      int r = idx / s, c = idx % s;
      if (r < c) {
        double a = Minv[r * s + c], b = Minv[c * s + r];
        Minv[r * s + c] = b;
        Minv[c * s + r] = a;
      }
    }
    if (lane == 0) *flag = ok;
  }
  __syncthreads();
  return *flag != 0;
}

// Cyclic Jacobi on the symmetric s x s matrix H (shared); Q accumulates the
// rotations; on exit diag(H) holds the eigenvalues.  One warp.
template <typename T>
__device__ void jacobi(T* H, T* Q, int s) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  for (int idx = lane; idx < s * s; idx += 32) Q[idx] = (idx / s == idx % s) ? T(1) : T(0);
  __syncwarp();
  const T eps = sizeof(T) == 8 ? T(1e-15) : T(1e-7);
  for (int sweep = 0; sweep < 40; ++sweep) {
    T off = 0, dg = 0;
    for (int idx = lane; idx < s * s; idx += 32) {
      int r = idx / s, c = idx % s;
      T v = H[idx];
      if (r != c) off += v * v; else dg += v * v;
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
        T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
        T c = T(1) / sqrt(T(1) + t * t), sn = t * c;
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

// Sort eigenvalues (diag H) descending and permute Q's columns into QS (T).
template <typename T>
__device__ void sort_desc(const T* H, const T* Q, T* QS, T* mu, int* perm, int s) {
  if (threadIdx.x == 0) {
    for (int j = 0; j < s; ++j) { perm[j] = j; mu[j] = H[j * s + j]; }
    for (int a = 0; a < s; ++a) {
      int best = a;
      for (int b = a + 1; b < s; ++b)
        if (mu[b] > mu[best]) best = b;
      T tv = mu[a]; mu[a] = mu[best]; mu[best] = tv;
      int ti = perm[a]; perm[a] = perm[best]; perm[best] = ti;
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < s * s; idx += NT) {
    int l = idx / s, j = idx % s;
    QS[idx] = Q[l * s + perm[j]];
  }
  __syncthreads();
}

template <typename T>
__device__ void fill_random(T* Y, int L, int s, int j0, uint64_t seed, uint64_t salt) {
  for (int64_t idx = threadIdx.x; idx < (int64_t)L * (s - j0); idx += NT) {
    int r = (int)(idx / (s - j0)), j = j0 + (int)(idx % (s - j0));
    Y[(int64_t)r * s + j] = (T)counter_normal(seed, salt + (uint64_t)r * 131071u + (uint64_t)j * 2654435761u);
  }
  __syncthreads();
}

template <typename T, bool SPD>
__global__ void __launch_bounds__(NT) k_subspace(
    const T* __restrict__ XpT_all, const int64_t* __restrict__ xs_off, const T* __restrict__ S_all,
    const int64_t* __restrict__ s_off, const T* __restrict__ work, const int64_t* __restrict__ work_off,
    const int32_t* __restrict__ np_arr, const int32_t* __restrict__ n_arr, const int32_t* __restrict__ m_arr,
    const int32_t* __restrict__ p_arr, const int32_t* __restrict__ sub_off, const int64_t* __restrict__ ent_off,
    const int32_t* __restrict__ lcol, const int32_t* __restrict__ omega, const int32_t* __restrict__ rp,
    const int32_t* __restrict__ ci, const double* __restrict__ val, const double* __restrict__ ds, T* scratch, const int64_t* __restrict__ scr_off, int nev, int over,
    int max_sweeps, double tol, uint64_t seed, const float* __restrict__ warm, const int64_t* __restrict__ warm_off,
    double* __restrict__ values, double* __restrict__ resid, int32_t* __restrict__ count,
    int32_t* __restrict__ sweeps_out, double* __restrict__ Z, const int64_t* __restrict__ z_off) {
  COUNT_LAUNCH();
  extern __shared__ double shd[];
  __shared__ int flag;
  __shared__ int perm[128];
  const int i = blockIdx.x;
  SubdomainView sv;
  sv.n = n_arr[i]; sv.m = m_arr[i]; sv.p = p_arr[i]; sv.g = sv.n - sv.m; sv.ld = np_arr[i];
  sv.pos0 = sub_off[i];
  const int p = sv.p, g = sv.g;
  // dimension of the operator's space and usable block width
  const int dim = SPD ? g : p;
  const int rank_cap = min(p, g);
  const int s = min(nev + over, dim);
  const int k = min(nev, min(s, rank_cap));
  if (k <= 0 || s <= 0) {
    if (threadIdx.x == 0) { count[i] = 0; sweeps_out[i] = 0; }
    for (int j = threadIdx.x; j < nev; j += NT) { values[(int64_t)i * nev + j] = 0; resid[(int64_t)i * nev + j] = 0; }
    return;
  }
  const T* XpT = XpT_all + xs_off[i];
  const T* Smat = S_all + s_off[i];
  const T* R = work + work_off[i] + (int64_t)sv.m * sv.ld + sv.m;
  XScale xs;
  if (!SPD) { xs.ds = ds; xs.omI = omega + sv.pos0; xs.omG = omega + sv.pos0 + sv.m; }
  const int L = max(p, g);
  T* base = scratch + scr_off[i];
  T* Y = base;                       // dim x s
  T* MY = base + (int64_t)L * s;     // S Y (SPD) / unused
  T* KY = base + 2 * (int64_t)L * s; // K Y (SPD) / X_p^T Y (general, g x s)
  T* V = base + 3 * (int64_t)L * s;  // p x s
  T* AV = base + 4 * (int64_t)L * s; // p x s
  T* TMP = base + 5 * (int64_t)L * s;
  double* G = shd;                   // s*s
  double* Minv = G + s * s;          // s*s
  T* H = (T*)(Minv + s * s);         // s*s
  T* Q = H + s * s;                  // s*s
  T* QS = Q + s * s;                 // s*s
  T* mu = QS + s * s;                // s
  T* rn = mu + s;                    // s: residual norms

  // ---- start block
  fill_random(Y, dim, s, 0, seed, (uint64_t)i * 0x100000001ull);
  if (warm != nullptr && SPD) {
    const float* wb = warm + warm_off[i];
    for (int64_t idx = threadIdx.x; idx < (int64_t)dim * k; idx += NT) {
      int r = (int)(idx / k), j = (int)(idx % k);
      Y[(int64_t)r * s + j] = (T)wb[idx];
    }
    __syncthreads();
  }
  auto orthonormalize = [&](T*& Yb, T*& MYb) {
    for (int pass = 0; pass < 2; ++pass) {
      if (SPD) gram(Yb, MYb, dim, s, G); else gram(Yb, Yb, dim, s, G);
      chol_inv_t(G, Minv, s, &flag);
      right_mul(Yb, TMP, dim, s, Minv);
      { T* t = Yb; Yb = TMP; TMP = t; }
      if (SPD) {
        right_mul(MYb, TMP, dim, s, Minv);
        T* t = MYb; MYb = TMP; TMP = t;
      }
    }
  };
  if (SPD) { mul_sym(Smat, g, g, Y, MY, s); __syncthreads(); }
  orthonormalize(Y, MY);

  int sweep = 0;
  T res_max = 0;
  for (;;) {
    // ---- K Y (SPD) or X_p^T Y (general)
    if (SPD) {
      mul_Xp(XpT, p, g, Y, V, s, s); __syncthreads();
      mul_AII(sv, omega, rp, ci, val, ds, ent_off, lcol, V, AV, s); __syncthreads();
      mul_XpT(XpT, p, g, AV, KY, s); __syncthreads();
      // H = Y^T K Y
      for (int idx = threadIdx.x; idx < s * s; idx += NT) {
        int t = idx / s, u = idx % s;
        T acc = 0;
        for (int r = 0; r < g; ++r) acc += Y[(int64_t)r * s + t] * KY[(int64_t)r * s + u];
        H[idx] = acc;
      }
    } else {
      mul_XpT(XpT, p, g, Y, KY, s, xs); __syncthreads();
      for (int idx = threadIdx.x; idx < s * s; idx += NT) {
        int t = idx / s, u = idx % s;
        T acc = 0;
        for (int r = 0; r < g; ++r) acc += KY[(int64_t)r * s + t] * KY[(int64_t)r * s + u];
        H[idx] = acc;
      }
    }
    __syncthreads();
    // symmetrise
    for (int idx = threadIdx.x; idx < s * s; idx += NT) {
      int t = idx / s, u = idx % s;
      if (t < u) { T a = T(0.5) * (H[t * s + u] + H[u * s + t]); H[t * s + u] = a; H[u * s + t] = a; }
    }
    __syncthreads();
    jacobi(H, Q, s);
    __syncthreads();
    sort_desc(H, Q, QS, mu, perm, s);
    // ---- rotate to Ritz vectors
    right_mul(Y, TMP, dim, s, QS); { T* t = Y; Y = TMP; TMP = t; }
    right_mul(KY, TMP, g, s, QS); { T* t = KY; KY = TMP; TMP = t; }
    if (SPD) { right_mul(MY, TMP, dim, s, QS); T* t = MY; MY = TMP; TMP = t; }
    // ---- residuals of the first k Ritz pairs
    T mu0 = mu[0] > T(0) ? mu[0] : T(1);
    if (!SPD) { mul_Xp(XpT, p, g, KY, V, s, s, xs); __syncthreads(); }   // X_p X_p^T y
    for (int j = 0; j < k; ++j) {
      T part = 0, nrm = 0;
      for (int r = threadIdx.x; r < dim; r += NT) {
        T a, b;
        if (SPD) { a = KY[(int64_t)r * s + j]; b = MY[(int64_t)r * s + j]; }
        else { a = V[(int64_t)r * s + j]; b = Y[(int64_t)r * s + j]; }
        T d = a - mu[j] * b;
        part += d * d;
        nrm += b * b;
      }
      __shared__ T red[NW];
      part = block_sum(part, red);
      nrm = block_sum(nrm, red);
      if (threadIdx.x == 0) {
        T den = (mu[j] > T(0) ? mu[j] : mu0) * sqrt(nrm);
        rn[j] = (mu[j] <= T(1e-12) * mu0) ? T(0) : sqrt(part) / (den > T(0) ? den : T(1));
      }
    }
    __syncthreads();
    res_max = 0;
    for (int j = 0; j < k; ++j) res_max = max(res_max, rn[j]);
    ++sweep;
    if ((double)res_max <= tol || sweep >= max_sweeps) break;
    // ---- power step, columns scaled by the Ritz values; near-null columns restart randomly
    if (SPD) { mul_sym(R, sv.ld, g, KY, Y, s); }
    else { for (int64_t idx = threadIdx.x; idx < (int64_t)p * s; idx += NT) Y[idx] = V[idx]; }
    __syncthreads();
    for (int64_t idx = threadIdx.x; idx < (int64_t)dim * s; idx += NT) {
      int j = (int)(idx % s);
      T sc = mu[j] > T(1e-10) * mu0 ? T(1) / mu[j] : T(0);
      Y[idx] *= sc;
    }
    __syncthreads();
    int first_null = s;
    for (int j = 0; j < s; ++j)
      if (!(mu[j] > T(1e-10) * mu0)) { first_null = j; break; }
    if (first_null < s) fill_random(Y, dim, s, first_null, seed ^ 0xA5A5A5A5ull, (uint64_t)i * 7919u + sweep * 104729u);
    if (SPD) { mul_sym(Smat, g, g, Y, MY, s); __syncthreads(); }
    orthonormalize(Y, MY);
  }
  // ---- outputs
  int kept = 0;
  T mu0 = mu[0] > T(0) ? mu[0] : T(0);
  for (int j = 0; j < k; ++j)
    if (mu[j] > T(sizeof(T) == 8 ? 1e-12 : 1e-6) * mu0) kept = j + 1;
  if (threadIdx.x == 0) { count[i] = kept; sweeps_out[i] = sweep; }
  for (int j = threadIdx.x; j < nev; j += NT) {
    double v = j < kept ? (SPD ? (double)mu[j] : sqrt(fmax((double)mu[j], 0.0))) : 0.0;
    values[(int64_t)i * nev + j] = v;
    resid[(int64_t)i * nev + j] = j < kept ? (double)rn[j] : 0.0;
  }
  double* Zi = Z + z_off[i];
  if (SPD) {
    // Z_i = X_p y, FP64 output (p x nev, columns >= kept zero)
    mul_Xp(XpT, p, g, Y, V, s, kept);
    __syncthreads();
    for (int64_t idx = threadIdx.x; idx < (int64_t)p * nev; idx += NT) {
      int r = (int)(idx / nev), j = (int)(idx % nev);
      Zi[idx] = j < kept ? (double)V[(int64_t)r * s + j] * ds[omega[sv.pos0 + r]] : 0.0;
    }
  } else {
    for (int64_t idx = threadIdx.x; idx < (int64_t)p * nev; idx += NT) {
      int r = (int)(idx / nev), j = (int)(idx % nev);
      Zi[idx] = j < kept ? (double)Y[(int64_t)r * s + j] : 0.0;
    }
  }
}

template <typename T>
void run_eigen(Handle& h, cudaStream_t s) {
  const int N = h.N, nev = h.nev;
  Coarse& co = h.co;
  Dense& dn = h.dn;
  DevMem& mem = h.mem;
  const bool spd = h.opt.spd != 0;
  const int over = std::max(0, h.opt.oversample);
  std::vector<int64_t> scr(N), zo(N + 1);
  int64_t tot = 0, zt = 0;
  int smax = 1;
  for (int i = 0; i < N; ++i) {
    int p = h.h_p[i], g = h.h_g[i];
    int dim = spd ? g : p;
    int sb = std::min(nev + over, dim);
    smax = std::max(smax, sb);
    scr[i] = tot;
    tot += 6LL * std::max(p, g) * std::max(sb, 1);
    zo[i] = zt;
    zt += (int64_t)p * nev;
  }
  zo[N] = zt;
  if (smax > 128) fail(ASM_ERR_UNSUPPORTED, "nev + oversample exceeds 128");
  co.s_max = smax;
  co.h_z_off = zo;
  co.scratch = mem.alloc<T>(tot);
  co.scr_off = mem.alloc<int64_t>(N);
  co.z_off = mem.alloc<int64_t>(N + 1);
  co.Z = mem.alloc<double>(std::max<int64_t>(zt, 1));
  co.values = mem.alloc<double>((int64_t)N * std::max(nev, 1));
  co.resid = mem.alloc<double>((int64_t)N * std::max(nev, 1));
  co.count = mem.alloc<int32_t>(N);
  co.sweeps = mem.alloc<int32_t>(N);
  CK(cudaMemcpyAsync(co.scr_off, scr.data(), 8 * N, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(co.z_off, zo.data(), 8 * (N + 1), cudaMemcpyHostToDevice, s));
  size_t smem = (size_t)2 * smax * smax * sizeof(double) + (size_t)(3 * smax * smax + 2 * smax) * sizeof(T) + 64;
  const double tol = h.opt.eig_tol > 0 ? h.opt.eig_tol : (h.fp32 ? 1e-3 : 1e-8);
  const int maxsw = h.opt.max_sweeps > 0 ? h.opt.max_sweeps : 60;
  if (spd) {
    CK(cudaFuncSetAttribute(k_subspace<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_subspace<T, true><<<N, NT, smem, s>>>(
        (const T*)dn.XpT, dn.xs_off, (const T*)dn.S, dn.s_off, (const T*)dn.work, dn.work_off, dn.np, h.dev_n,
        h.dev_m, h.dev_p, h.ov.sub_off, h.ov.ent_off, h.ov.lcol, h.ov.omega, h.row_ptr, h.col_idx, h.val, h.dscale, (T*)co.scratch,
        co.scr_off, nev, over, maxsw, tol, h.opt.seed, h.warm, h.warm_off, co.values, co.resid, co.count,
        co.sweeps, co.Z, co.z_off);
  } else {
    CK(cudaFuncSetAttribute(k_subspace<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_subspace<T, false><<<N, NT, smem, s>>>(
        (const T*)dn.XpT, dn.xs_off, (const T*)dn.S, dn.s_off, (const T*)dn.work, dn.work_off, dn.np, h.dev_n,
        h.dev_m, h.dev_p, h.ov.sub_off, h.ov.ent_off, h.ov.lcol, h.ov.omega, h.row_ptr, h.col_idx, h.val, h.dscale, (T*)co.scratch,
        co.scr_off, nev, over, maxsw, tol, h.opt.seed, nullptr, nullptr, co.values, co.resid, co.count,
        co.sweeps, co.Z, co.z_off);
  }
  CK_LAUNCH("subspace iteration");
}

}  // namespace

void build_eigen(Handle& h, cudaStream_t s) {
  if (h.nev <= 0 || !h.opt.coarse) {
    h.co.h_count.assign(h.N, 0);
    return;
  }
  if (h.fp32) run_eigen<float>(h, s); else run_eigen<double>(h, s);
}

}  // namespace asmgpu
