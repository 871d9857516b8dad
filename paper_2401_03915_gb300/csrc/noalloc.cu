// Allocation-free variant of the fused CSR SpMV + dot product of the Krylov
// loop (y = A x and x^T y in one pass, the dot reduced in a fixed order).
//
// Who needs it: code that must not allocate device memory while it runs,
// e.g. a caller that is recording a CUDA stream capture (cudaMalloc is not
// allowed there), a real-time or latency-critical host thread for which
// cudaMalloc's implicit device synchronisation is unacceptable, or an
// application whose device memory is entirely owned by its own allocator.
// Such callers pass the matrix, x and the outputs; the only scratch this
// entry point uses (one partial sum per thread block) lives in the
// file-scope array below, which every GPU that loads this library holds
// until the process exits.
#include <mutex>

#include "common.cuh"

namespace asmgpu {
namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_VW = 4;                                 // lanes per row
constexpr int NA_ROWS_PER_BLOCK = NA_THREADS / NA_VW;    // 64 rows per block
constexpr int NA_MAX_BLOCKS = 16384;                     // scratch slots
constexpr int64_t NA_MAX_ROWS = (int64_t)NA_MAX_BLOCKS * NA_ROWS_PER_BLOCK;  // 1,048,576

// One partial dot product per thread block; fully rewritten by every call.
static __device__ __align__(256) double g_noalloc_partials[NA_MAX_BLOCKS];

// Block b handles rows [64 b, 64 b + 64): y = A x there, and its share of
// x^T y goes to scratch[b].
__global__ void __launch_bounds__(NA_THREADS) k_na_spmv_dot(int n, const int32_t* __restrict__ rp,
                                                            const int32_t* __restrict__ ci,
                                                            const double* __restrict__ val,
                                                            const double* __restrict__ x, double* __restrict__ y,
                                                            double* __restrict__ scratch) {
  COUNT_LAUNCH();
  __shared__ double red[NA_THREADS / 32];
  const int lane = threadIdx.x % NA_VW;
  const int r = blockIdx.x * NA_ROWS_PER_BLOCK + threadIdx.x / NA_VW;
  double acc = 0;
  if (r < n)
    for (int k = rp[r] + lane; k < rp[r + 1]; k += NA_VW) acc += val[k] * x[ci[k]];
#pragma unroll
  for (int o = NA_VW / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  double d = 0;
  if (r < n && lane == 0) {
    y[r] = acc;
    d = acc * x[r];
  }
  d = block_sum(d, red);
  if (threadIdx.x == 0) scratch[blockIdx.x] = d;
}

// result = sum of the nb partials, in block order.
__global__ void __launch_bounds__(NA_THREADS) k_na_sum(const double* __restrict__ scratch, int nb,
                                                       double* __restrict__ result) {
  COUNT_LAUNCH();
  __shared__ double red[NA_THREADS / 32];
  double s = 0;
  for (int k = threadIdx.x; k < nb; k += NA_THREADS) s += scratch[k];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *result = s;
}

// Device address of the scratch array, looked up once per device.
constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
double* g_na_ptr[NA_MAX_DEVICES] = {};

}  // namespace
}  // namespace asmgpu

extern "C" asm_status asm_spmv_dot_noalloc(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                           const double* val, const double* x, double* y, double* xty,
                                           void* stream) {
  using namespace asmgpu;
  if (n < 0 || !row_ptr || !col_idx || !val || !x || !y || !xty)
    return set_last_error(ASM_ERR_INVALID_ARG, "asm_spmv_dot_noalloc: null pointer or n < 0");
  if ((int64_t)n > NA_MAX_ROWS)
    return set_last_error(ASM_ERR_UNSUPPORTED,
                          "asm_spmv_dot_noalloc: n = " + std::to_string(n) +
                              " exceeds the 1,048,576 rows its static scratch covers; use asm_spmv");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
    cudaGetLastError();
    return set_last_error(ASM_ERR_CUDA, "asm_spmv_dot_noalloc: no usable current device");
  }
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
      // the symbol's host-side name is not a device address: ask the runtime
      // for the address of this device's copy, with this device current
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
      if (e != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return set_last_error(ASM_ERR_CUDA, std::string("asm_spmv_dot_noalloc: cudaGetSymbolAddress failed: ") +
                                                cudaGetErrorString(e));
      }
      g_na_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_na_ptr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nb = n > 0 ? (int)((n + NA_ROWS_PER_BLOCK - 1) / NA_ROWS_PER_BLOCK) : 0;
  if (nb > 0) k_na_spmv_dot<<<nb, NA_THREADS, 0, s>>>(n, row_ptr, col_idx, val, x, y, scratch);
  k_na_sum<<<1, NA_THREADS, 0, s>>>(scratch, nb, xty);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return set_last_error(ASM_ERR_CUDA, std::string("asm_spmv_dot_noalloc: launch failed: ") + cudaGetErrorString(e));
  return ASM_OK;
}
