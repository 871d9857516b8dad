// Warm-start network for the subspace iteration: a per-node MLP
//     features (F) -> H -> H -> K,  ReLU hidden layers,
// FP16 operands with FP32 accumulation on the tensor cores (mma.sync
// m16n8k16), FP32 master weights, Adam.  Row v of the output is row v of the
// start block Y_0 (the coordinates z of the eigen iteration on Gamma_delta).
//
// Training loss per subdomain (rotation invariant, so eigenvector signs and
// rotations inside clusters do not matter):  L_i = K - tr(G^{-1} A^T A) with
// G = Y^T Y and A = Z^T Y, Z the orthonormal top-K eigenvectors the method
// computes; L_i = sum of sin^2 of the principal angles between span(Y) and
// span(Z).  Gradient: dL/dY = 2 Y G^{-1} A^T A G^{-1} - 2 Z A G^{-1}.
#include <cuda_fp16.h>

#include <algorithm>
#include <new>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "mlp.cuh"

namespace asmgpu {
namespace {

constexpr int GT = 128;      // threads of the GEMM block (4 warps)
constexpr int TM = 64, TN = 64, TK = 16;

__device__ __forceinline__ uint32_t pack2(half a, half b) {
  __half2 v = __halves2half2(a, b);
  return *reinterpret_cast<uint32_t*>(&v);
}

// C (M x N) = op(A) (M x K) op(B) (K x N), FP16 inputs, FP32 accumulation.
// ATRANS: A(m, k) = A[k * lda + m], else A[m * lda + k].
// BTRANS: B(k, n) = B[n * ldb + k], else B[k * ldb + n].
// Epilogue: v = acc (+ bias[n]); if mask: v *= (mask[m * ldm + n] > 0);
// C32[m * ldc + n] = v (fp32, optional); C16 = relu ? max(v, 0) : v (fp16, optional).
// Split K: blockIdx.z handles k in [z * kchunk, (z + 1) * kchunk) and writes
// its partial to C32 + z * M * ldc (bias, mask and C16 unused then).
template <bool ATRANS, bool BTRANS>
__global__ void __launch_bounds__(GT) k_hgemm(int M, int N, int K, const half* __restrict__ A, int lda,
                                              const half* __restrict__ B, int ldb, const float* __restrict__ bias,
                                              const half* __restrict__ mask, int ldm, int relu,
                                              float* __restrict__ C32, int ldc, half* __restrict__ C16, int ldc16,
                                              int kchunk) {
  COUNT_LAUNCH();
  __shared__ half As[TM][TK + 8];
  __shared__ half Bs[TK][TN + 8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, tig = lane & 3;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int kbeg = kchunk > 0 ? blockIdx.z * kchunk : 0;
  const int kend = kchunk > 0 ? min(K, kbeg + kchunk) : K;
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  for (int k0 = kbeg; k0 < kend; k0 += TK) {
    __syncthreads();
    for (int idx = tid; idx < TM * TK; idx += GT) {
      int r = ATRANS ? idx % TM : idx / TK, k = ATRANS ? idx / TM : idx % TK;
      int gm = m0 + r, gk = k0 + k;
      half v = __float2half(0.f);
      if (gm < M && gk < kend) v = ATRANS ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk];
      As[r][k] = v;
    }
    for (int idx = tid; idx < TK * TN; idx += GT) {
      int k = BTRANS ? idx % TK : idx / TN, c = BTRANS ? idx / TK : idx % TN;
      int gk = k0 + k, gn = n0 + c;
      half v = __float2half(0.f);
      if (gk < kend && gn < N) v = BTRANS ? B[(int64_t)gn * ldb + gk] : B[(int64_t)gk * ldb + gn];
      Bs[k][c] = v;
    }
    __syncthreads();
    uint32_t af[2][4], bf[4][2];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
      const int r = wm + mi * 16 + g, c = 2 * tig;
      af[mi][0] = pack2(As[r][c], As[r][c + 1]);
      af[mi][1] = pack2(As[r + 8][c], As[r + 8][c + 1]);
      af[mi][2] = pack2(As[r][c + 8], As[r][c + 9]);
      af[mi][3] = pack2(As[r + 8][c + 8], As[r + 8][c + 9]);
    }
#pragma unroll
    for (int ni = 0; ni < 4; ++ni) {
      const int n = wn + ni * 8 + g, k = 2 * tig;
      bf[ni][0] = pack2(Bs[k][n], Bs[k + 1][n]);
      bf[ni][1] = pack2(Bs[k + 8][n], Bs[k + 9][n]);
    }
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        float* d = acc[mi][ni];
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(af[mi][0]), "r"(af[mi][1]), "r"(af[mi][2]), "r"(af[mi][3]), "r"(bf[ni][0]), "r"(bf[ni][1]));
      }
  }
  // epilogue
  float* Cz = (kchunk > 0 && C32) ? C32 + (int64_t)blockIdx.z * M * ldc : C32;
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + wm + mi * 16 + g + (q >= 2 ? 8 : 0);
        const int n = n0 + wn + ni * 8 + 2 * tig + (q & 1);
        if (m >= M || n >= N) continue;
        float v = acc[mi][ni][q];
        if (kchunk > 0) {
          Cz[(int64_t)m * ldc + n] = v;
          continue;
        }
        if (bias) v += bias[n];
        if (mask && !(__half2float(mask[(int64_t)m * ldm + n]) > 0.f)) v = 0.f;
        if (C32) C32[(int64_t)m * ldc + n] = v;
        if (C16) C16[(int64_t)m * ldc16 + n] = __float2half(relu ? fmaxf(v, 0.f) : v);
      }
}

// out[i] = scale * sum_z part[z * count + i] (fixed order)
__global__ void k_sum_splits(const float* __restrict__ part, int nz, int64_t count, float scale,
                             float* __restrict__ out) {
  COUNT_LAUNCH();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < nz; ++z) s += part[(int64_t)z * count + i];
    out[i] = s * scale;
  }
}

// db[n] = scale * sum_m dY[m][n] (block per column, fixed order)
__global__ void k_col_sum(const half* __restrict__ dY, int M, int ld, float scale, float* __restrict__ db) {
  COUNT_LAUNCH();
  __shared__ float red[8];
  const int n = blockIdx.x;
  float s = 0.f;
  for (int m = threadIdx.x; m < M; m += blockDim.x) s += __half2float(dY[(int64_t)m * ld + n]);
  s = block_sum(s, red);
  if (threadIdx.x == 0) db[n] = s * scale;
}

__global__ void k_to_half(const float* __restrict__ x, int64_t n, half* __restrict__ y) {
  COUNT_LAUNCH();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2half(x[i]);
}

// rows x F fp32 features into rows x Fp fp16 (zero padded)
__global__ void k_pack_features(const float* __restrict__ X, int rows, int F, int Fp, half* __restrict__ X16) {
  COUNT_LAUNCH();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)rows * Fp;
       i += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(i / Fp), c = (int)(i % Fp);
    X16[i] = __float2half(c < F ? X[(int64_t)r * F + c] : 0.f);
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m1,
                       float* __restrict__ m2, int64_t n, float lr, float b1, float b2, float eps, int step) {
  COUNT_LAUNCH();
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float g = gr[i];
    float a = b1 * m1[i] + (1.f - b1) * g;
    float b = b2 * m2[i] + (1.f - b2) * g * g;
    m1[i] = a;
    m2[i] = b;
    p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
  }
}

// Subspace loss and its gradient, one block per segment (subdomain) with
// rows r0..r1-1.  Y (ld) and Z (ldz): FP32, first K columns used.
// loss[seg] = K - tr(G^{-1} M) with G = Y^T Y (+ a ridge of 1e-8 tr(G)/K),
// A = Z^T Y, M = A^T A;  dY16 = 2 (Y G^{-1} M G^{-1} - Z A G^{-1}) (the
// gradient of loss[seg]), zero in the padding columns K..ld16-1.
// Dynamic shared memory: 7 K x K doubles.
__global__ void __launch_bounds__(256) k_subspace_loss(const float* __restrict__ Y, int ld, const float* __restrict__ Z,
                                                       int ldz, const int64_t* __restrict__ seg, int K,
                                                       half* __restrict__ dY, int ld16, float* __restrict__ dY32,
                                                       double* __restrict__ loss) {
  COUNT_LAUNCH();
  extern __shared__ double sm[];
  const int KK = K * K;
  double *G = sm, *Am = sm + KK, *Lc = sm + 2 * KK, *Li = sm + 3 * KK, *Gi = sm + 4 * KK, *B1 = sm + 5 * KK,
         *B2 = sm + 6 * KK;
  const int i = blockIdx.x;
  const int64_t r0 = seg[i], r1 = seg[i + 1];
  for (int idx = threadIdx.x; idx < 2 * KK; idx += blockDim.x) {
    const int e = idx % KK, t = e / K, u = e % K;
    double s = 0;
    if (idx < KK)
      for (int64_t r = r0; r < r1; ++r) s += (double)Y[r * ld + t] * (double)Y[r * ld + u];
    else
      for (int64_t r = r0; r < r1; ++r) s += (double)Z[r * ldz + t] * (double)Y[r * ld + u];
    if (idx < KK) G[e] = s; else Am[e] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0;
    for (int t = 0; t < K; ++t) tr += G[t * K + t];
    const double ridge = 1e-8 * tr / K + 1e-30;
    for (int a = 0; a < K; ++a)
      for (int b = 0; b <= a; ++b) {
        double v = G[a * K + b] + (a == b ? ridge : 0.0);
        for (int c = 0; c < b; ++c) v -= Lc[a * K + c] * Lc[b * K + c];
        Lc[a * K + b] = a == b ? sqrt(fmax(v, 1e-300)) : v / Lc[b * K + b];
      }
    for (int c = 0; c < K; ++c)
      for (int a = 0; a < K; ++a) {
        if (a < c) { Li[a * K + c] = 0; continue; }
        double v = a == c ? 1.0 : 0.0;
        for (int q = c; q < a; ++q) v -= Lc[a * K + q] * Li[q * K + c];
        Li[a * K + c] = v / Lc[a * K + a];
      }
  }
  __syncthreads();
  // Gi = Li^T Li ; Lc <- M = A^T A
  for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) {
    const int a = idx / K, b = idx % K;
    double v = 0, w = 0;
    for (int q = 0; q < K; ++q) {
      v += Li[q * K + a] * Li[q * K + b];
      w += Am[q * K + a] * Am[q * K + b];
    }
    Gi[idx] = v;
    Lc[idx] = w;
  }
  __syncthreads();
  // Li <- T = Gi M ; B2 = A Gi
  for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) {
    const int a = idx / K, b = idx % K;
    double v = 0, w = 0;
    for (int q = 0; q < K; ++q) {
      v += Gi[a * K + q] * Lc[q * K + b];
      w += Am[a * K + q] * Gi[q * K + b];
    }
    Li[idx] = v;
    B2[idx] = w;
  }
  __syncthreads();
  // B1 = T Gi
  for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) {
    const int a = idx / K, b = idx % K;
    double v = 0;
    for (int q = 0; q < K; ++q) v += Li[a * K + q] * Gi[q * K + b];
    B1[idx] = v;
  }
  if (threadIdx.x == 0) {
    double trT = 0;
    for (int a = 0; a < K; ++a) trT += Li[a * K + a];
    loss[i] = K - trT;
  }
  __syncthreads();
  for (int64_t idx = threadIdx.x; idx < (r1 - r0) * ld16; idx += blockDim.x) {
    const int64_t r = r0 + idx / ld16;
    const int c = (int)(idx % ld16);
    double v = 0;
    if (c < K)
      for (int q = 0; q < K; ++q) v += (double)Y[r * ld + q] * B1[q * K + c] - (double)Z[r * ldz + q] * B2[q * K + c];
    v *= 2.0;
    dY[r * ld16 + c] = __float2half((float)v);
    if (dY32 && c < K) dY32[r * K + c] = (float)v;
  }
}

inline dim3 ggrid(int M, int N, int z = 1) { return dim3((unsigned)ceil_div(N, TN), (unsigned)ceil_div(M, TM), z); }

}  // namespace

// ---------------------------------------------------------------------------
Mlp::Mlp(int F_, int H_, int K_, uint64_t seed) : F(F_), H(H_), K(K_) {
  Fp = (int)round_up(F, 16);
  Kp = (int)round_up(K, 16);
  off_W1 = 0;
  off_b1 = off_W1 + (int64_t)Fp * H;
  off_W2 = off_b1 + H;
  off_b2 = off_W2 + (int64_t)H * H;
  off_W3 = off_b2 + H;
  off_b3 = off_W3 + (int64_t)H * Kp;
  nparams = off_b3 + Kp;
  // He-style initialisation from the counter-based generator (host side)
  std::vector<float> p(nparams, 0.f);
  auto fill = [&](int64_t off, int rows, int cols, int fan_in, int valid_rows, int valid_cols) {
    const double sd = std::sqrt(2.0 / fan_in);
    for (int r = 0; r < rows; ++r)
      for (int c = 0; c < cols; ++c) {
        uint64_t k = (uint64_t)(off + (int64_t)r * cols + c);
        uint64_t z = seed + (2 * k + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        uint64_t z2 = seed + (2 * k + 2) * 0x9E3779B97F4A7C15ull;
        z2 = (z2 ^ (z2 >> 30)) * 0xBF58476D1CE4E5B9ull;
        z2 = (z2 ^ (z2 >> 27)) * 0x94D049BB133111EBull;
        z2 ^= z2 >> 31;
        double u1 = (double)(z >> 11) * 0x1.0p-53, u2 = (double)(z2 >> 11) * 0x1.0p-53;
        double nrm = std::sqrt(-2.0 * std::log1p(-u1)) * std::cos(6.283185307179586 * u2);
        p[off + (int64_t)r * cols + c] = (r < valid_rows && c < valid_cols) ? (float)(sd * nrm) : 0.f;
      }
  };
  fill(off_W1, Fp, H, F, F, H);
  fill(off_W2, H, H, H, H, H);
  fill(off_W3, H, Kp, H, H, K);
  CK(cudaMalloc(&params, sizeof(float) * nparams));
  CK(cudaMalloc(&grads, sizeof(float) * nparams));
  CK(cudaMalloc(&m1, sizeof(float) * nparams));
  CK(cudaMalloc(&m2, sizeof(float) * nparams));
  CK(cudaMalloc(&params16, sizeof(half) * nparams));
  CK(cudaMemcpy(params, p.data(), sizeof(float) * nparams, cudaMemcpyHostToDevice));
  CK(cudaMemset(m1, 0, sizeof(float) * nparams));
  CK(cudaMemset(m2, 0, sizeof(float) * nparams));
  sync_half(nullptr);
}

Mlp::~Mlp() {
  cudaFree(params); cudaFree(grads); cudaFree(m1); cudaFree(m2); cudaFree(params16);
  release_work();
}

void Mlp::release_work() {
  for (void* q : work) cudaFree(q);
  work.clear();
  cap = 0;
}

void Mlp::sync_half(cudaStream_t s) {
  k_to_half<<<256, 256, 0, s>>>(params, nparams, params16);
  CK_LAUNCH("mlp weights to fp16");
}

void Mlp::ensure(int rows) {
  if (rows <= cap) return;
  release_work();
  cap = (int)round_up(std::max(rows, 1024), 1024);
  auto al = [&](size_t bytes) { void* q = nullptr; CK(cudaMalloc(&q, bytes)); work.push_back(q); return q; };
  X16 = (half*)al(sizeof(half) * (size_t)cap * Fp);
  H1 = (half*)al(sizeof(half) * (size_t)cap * H);
  H2 = (half*)al(sizeof(half) * (size_t)cap * H);
  Y32 = (float*)al(sizeof(float) * (size_t)cap * Kp);
  dY16 = (half*)al(sizeof(half) * (size_t)cap * Kp);
  dH2 = (half*)al(sizeof(half) * (size_t)cap * H);
  dH1 = (half*)al(sizeof(half) * (size_t)cap * H);
  const int nz = 64;  // split-K partials of the weight gradients (see weight_grad)
  const int64_t wmax = std::max<int64_t>({(int64_t)H * H, (int64_t)Fp * H, (int64_t)H * Kp});
  part = (float*)al(sizeof(float) * (size_t)nz * (size_t)wmax);
}

void Mlp::forward(const float* X, int rows, cudaStream_t s) {
  ensure(rows);
  k_pack_features<<<256, 256, 0, s>>>(X, rows, F, Fp, X16);
  const half* P = params16;
  k_hgemm<false, false><<<ggrid(rows, H), GT, 0, s>>>(rows, H, Fp, X16, Fp, P + off_W1, H, params + off_b1,
                                                      nullptr, 0, 1, nullptr, 0, H1, H, 0);
  k_hgemm<false, false><<<ggrid(rows, H), GT, 0, s>>>(rows, H, H, H1, H, P + off_W2, H, params + off_b2, nullptr,
                                                      0, 1, nullptr, 0, H2, H, 0);
  k_hgemm<false, false><<<ggrid(rows, Kp), GT, 0, s>>>(rows, Kp, H, H2, H, P + off_W3, Kp, params + off_b3,
                                                       nullptr, 0, 0, Y32, Kp, nullptr, 0, 0);
  CK_LAUNCH("mlp forward");
}

// weight gradient dW (Kin x Nout) = scale * A^T (rows x Kin) dO (rows x Nout),
// split over rows, partial sums added in a fixed order
void Mlp::weight_grad(const half* Aact, int Kin, const half* dO, int Nout, int rows, float scale, float* out,
                      cudaStream_t s) {
  // enough row chunks to fill the GPU: the output is only Kin x Nout
  const int nz = std::max(1, std::min(64, (int)ceil_div(rows, 256)));
  const int chunk = (int)round_up(ceil_div(rows, nz), TK);
  k_hgemm<true, false><<<ggrid(Kin, Nout, nz), GT, 0, s>>>(Kin, Nout, rows, Aact, Kin, dO, Nout, nullptr, nullptr,
                                                           0, 0, part, Nout, nullptr, 0, chunk);
  k_sum_splits<<<256, 256, 0, s>>>(part, nz, (int64_t)Kin * Nout, scale, out);
}

void Mlp::backward(int rows, float scale, cudaStream_t s) {
  // dY16 (rows x Kp) holds dL/dY from the loss
  weight_grad(H2, H, dY16, Kp, rows, scale, grads + off_W3, s);
  k_col_sum<<<Kp, 256, 0, s>>>(dY16, rows, Kp, scale, grads + off_b3);
  // dH2 = (dY W3^T) * relu'(H2)
  k_hgemm<false, true><<<ggrid(rows, H), GT, 0, s>>>(rows, H, Kp, dY16, Kp, params16 + off_W3, Kp, nullptr, H2, H,
                                                     0, nullptr, 0, dH2, H, 0);
  weight_grad(H1, H, dH2, H, rows, scale, grads + off_W2, s);
  k_col_sum<<<H, 256, 0, s>>>(dH2, rows, H, scale, grads + off_b2);
  // dH1 = (dH2 W2^T) * relu'(H1)
  k_hgemm<false, true><<<ggrid(rows, H), GT, 0, s>>>(rows, H, H, dH2, H, params16 + off_W2, H, nullptr, H1, H, 0,
                                                     nullptr, 0, dH1, H, 0);
  weight_grad(X16, Fp, dH1, H, rows, scale, grads + off_W1, s);
  k_col_sum<<<H, 256, 0, s>>>(dH1, rows, H, scale, grads + off_b1);
  CK_LAUNCH("mlp backward");
}

void Mlp::loss_grad(const float* Z, int ldz, const int64_t* seg, int nseg, double* loss, float* dY32,
                    cudaStream_t s) {
  const size_t smem = sizeof(double) * 7 * K * K;
  if (smem > 48 * 1024)
    CK(cudaFuncSetAttribute(k_subspace_loss, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_subspace_loss<<<nseg, 256, smem, s>>>(Y32, Kp, Z, ldz, seg, K, dY16, Kp, dY32, loss);
  CK_LAUNCH("subspace loss");
}

void Mlp::adam(float lr, cudaStream_t s) {
  ++step;
  k_adam<<<256, 256, 0, s>>>(params, grads, m1, m2, nparams, lr, 0.9f, 0.999f, 1e-8f, step);
  sync_half(s);
}

}  // namespace asmgpu

// ---------------------------------------------------------------------------
// C ABI of the warm-start network
// ---------------------------------------------------------------------------
using namespace asmgpu;

namespace {
template <typename F>
asm_status mlp_guarded(F&& f) {
  try {
    f();
    return ASM_OK;
  } catch (const AsmError& e) {
    return set_last_error(e.status, e.msg);
  } catch (const std::bad_alloc&) {
    return set_last_error(ASM_ERR_OOM, "host allocation failed");
  } catch (...) {
    return set_last_error(ASM_ERR_CUDA, "unexpected internal error");
  }
}

// loss and gradients of one batch; leaves the per-segment losses in dloss
void mlp_loss_and_grad(Mlp& net, const float* X, int rows, const float* T, const int64_t* seg, int nseg,
                       double* dloss, cudaStream_t s) {
  net.forward(X, rows, s);
  net.loss_grad(T, net.K, seg, nseg, dloss, nullptr, s);
  net.backward(rows, 1.0f / (float)nseg, s);
}

double mean_loss(const double* dloss, int nseg, cudaStream_t s) {
  std::vector<double> l(nseg);
  CK(cudaMemcpyAsync(l.data(), dloss, sizeof(double) * nseg, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double t = 0;
  for (double v : l) t += v;
  return t / nseg;
}

struct LossBuf {
  double* p = nullptr;
  cudaStream_t s;
  LossBuf(int n, cudaStream_t st) : s(st) { CK(cudaMallocAsync(&p, sizeof(double) * std::max(n, 1), s)); }
  ~LossBuf() { if (p) cudaFreeAsync(p, s); }
};

asm_status check_batch(const asm_mlp* N, const float* X, int32_t rows, const float* T, const int64_t* seg,
                       int32_t nseg) {
  if (!N || !X || !T || !seg || rows < 1 || nseg < 1)
    return set_last_error(ASM_ERR_INVALID_ARG, "null argument, rows < 1 or nseg < 1");
  return ASM_OK;
}
}  // namespace

extern "C" {

asm_status asm_mlp_create(int32_t hidden, int32_t outputs, uint64_t seed, asm_mlp** out) {
  if (out) *out = nullptr;
  if (!out || hidden < 16 || hidden > 1024 || hidden % 16 != 0 || outputs < 1 || outputs > 32)
    return set_last_error(ASM_ERR_INVALID_ARG, "hidden must be a multiple of 16 in 16..1024, outputs in 1..32");
  asm_mlp* N = nullptr;
  asm_status st = mlp_guarded([&] { N = new asm_mlp(WARM_FEATURES, hidden, outputs, seed); });
  if (st != ASM_OK) { delete N; return st; }
  *out = N;
  return ASM_OK;
}

void asm_mlp_destroy(asm_mlp* N) {
  if (!N) return;
  cudaDeviceSynchronize();
  delete N;
  cudaGetLastError();
}

int64_t asm_mlp_num_params(const asm_mlp* N) { return N ? N->net.nparams : 0; }

asm_status asm_mlp_get_params(const asm_mlp* N, float* params) {
  if (!N || !params) return set_last_error(ASM_ERR_INVALID_ARG, "null argument");
  return mlp_guarded([&] {
    CK(cudaMemcpy(params, N->net.params, sizeof(float) * N->net.nparams, cudaMemcpyDeviceToHost));
  });
}

asm_status asm_mlp_set_params(asm_mlp* N, const float* params) {
  if (!N || !params) return set_last_error(ASM_ERR_INVALID_ARG, "null argument");
  return mlp_guarded([&] {
    CK(cudaMemcpy(N->net.params, params, sizeof(float) * N->net.nparams, cudaMemcpyHostToDevice));
    N->net.sync_half(nullptr);
    CK(cudaDeviceSynchronize());
  });
}

asm_status asm_mlp_forward(asm_mlp* N, const float* X, int32_t rows, float* Y, void* stream) {
  if (!N || !X || !Y || rows < 0) return set_last_error(ASM_ERR_INVALID_ARG, "null argument or rows < 0");
  if (rows == 0) return ASM_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return mlp_guarded([&] {
    Mlp& net = N->net;
    net.forward(X, rows, s);
    CK(cudaMemcpy2DAsync(Y, sizeof(float) * net.K, net.Y32, sizeof(float) * net.Kp, sizeof(float) * net.K, rows,
                         cudaMemcpyDeviceToDevice, s));
  });
}

asm_status asm_mlp_loss_grad(asm_mlp* N, const float* X, int32_t rows, const float* T, const int64_t* seg,
                             int32_t nseg, double* loss, float* grad, void* stream) {
  asm_status c = check_batch(N, X, rows, T, seg, nseg);
  if (c != ASM_OK) return c;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return mlp_guarded([&] {
    Mlp& net = N->net;
    LossBuf lb(nseg, s);
    mlp_loss_and_grad(net, X, rows, T, seg, nseg, lb.p, s);
    const double l = mean_loss(lb.p, nseg, s);
    if (loss) *loss = l;
    if (grad) CK(cudaMemcpy(grad, net.grads, sizeof(float) * net.nparams, cudaMemcpyDeviceToHost));
  });
}

asm_status asm_mlp_train_step(asm_mlp* N, const float* X, int32_t rows, const float* T, const int64_t* seg,
                              int32_t nseg, float lr, double* loss, void* stream) {
  asm_status c = check_batch(N, X, rows, T, seg, nseg);
  if (c != ASM_OK) return c;
  if (!(lr > 0.f)) return set_last_error(ASM_ERR_INVALID_ARG, "lr must be > 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return mlp_guarded([&] {
    Mlp& net = N->net;
    LossBuf lb(nseg, s);
    mlp_loss_and_grad(net, X, rows, T, seg, nseg, lb.p, s);
    net.adam(lr, s);
    if (loss) *loss = mean_loss(lb.p, nseg, s);
  });
}

}  // extern "C"
