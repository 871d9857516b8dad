// Per-node warm-start network (features -> H -> H -> K) with FP16 tensor-core
// GEMMs, FP32 accumulation and FP32 master weights.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace asmgpu {

constexpr int WARM_FEATURES = 16;  // per Gamma_delta node, see k_warm_features

struct Mlp {
  int F, H, K;       // input features, hidden width, outputs
  int Fp, Kp;        // padded to multiples of 16
  int64_t off_W1, off_b1, off_W2, off_b2, off_W3, off_b3, nparams;
  // parameters: W1 (Fp x H), b1 (H), W2 (H x H), b2, W3 (H x Kp), b3 (Kp);
  // rows of W1 beyond F and columns of W3 beyond K are zero and stay zero
  float* params = nullptr;
  float* grads = nullptr;
  float* m1 = nullptr;
  float* m2 = nullptr;
  half* params16 = nullptr;
  int step = 0;
  // activations for `cap` rows
  int cap = 0;
  std::vector<void*> work;
  half *X16 = nullptr, *H1 = nullptr, *H2 = nullptr, *dY16 = nullptr, *dH2 = nullptr, *dH1 = nullptr;
  float* Y32 = nullptr;  // rows x Kp network output
  float* part = nullptr; // split-K partial sums of the weight gradients

  Mlp(int F, int H, int K, uint64_t seed);
  ~Mlp();
  Mlp(const Mlp&) = delete;
  Mlp& operator=(const Mlp&) = delete;
  void ensure(int rows);
  void release_work();
  void sync_half(cudaStream_t s);
  // X: rows x F FP32 (device). Output in Y32 (rows x Kp).
  void forward(const float* X, int rows, cudaStream_t s);
  // subspace loss of Y32 against Z (rows x ldz FP32, first K columns), per
  // segment seg[0..nseg] (device); writes loss[nseg] (device) and the
  // per-segment gradient dL_i/dY to dY16 (and to dY32, rows x K, if set)
  void loss_grad(const float* Z, int ldz, const int64_t* seg, int nseg, double* loss, float* dY32, cudaStream_t s);
  // parameter gradients (scaled by `scale`) from dY16 and the stored activations
  void backward(int rows, float scale, cudaStream_t s);
  void weight_grad(const half* Aact, int Kin, const half* dO, int Nout, int rows, float scale, float* out,
                   cudaStream_t s);
  void adam(float lr, cudaStream_t s);
};

}  // namespace asmgpu

// The C ABI's opaque network handle.
struct asm_mlp {
  asmgpu::Mlp net;
  asm_mlp(int F, int H, int K, uint64_t seed) : net(F, H, K, seed) {}
};
