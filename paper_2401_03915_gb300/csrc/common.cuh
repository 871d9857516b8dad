// Shared device/host helpers of the two-level Schwarz library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "asm.h"

namespace asmgpu {

// ---------------------------------------------------------------------------
// Error handling: internal code throws AsmError; the C ABI layer catches it
// and turns it into a status + thread-local message.
// ---------------------------------------------------------------------------
struct AsmError {
  asm_status status;
  std::string msg;
};

[[noreturn]] void fail(asm_status s, const std::string& msg);
// Record `msg` as the calling thread's asm_last_error() text; returns s.
asm_status set_last_error(asm_status s, const std::string& msg);
void cuda_check(cudaError_t e, const char* what, const char* file, int line);

#define CK(call) ::asmgpu::cuda_check((call), #call, __FILE__, __LINE__)
#define CK_LAUNCH(what) ::asmgpu::cuda_check(cudaGetLastError(), what, __FILE__, __LINE__)

// Device error word bits (set by kernels, read back by the host once per stage).
enum DevErr : int32_t {
  DERR_NOT_SPD = 1,
  DERR_ZERO_PIVOT = 2,
  DERR_NONFINITE = 4,
  DERR_CAPACITY = 8,
  DERR_COARSE = 16,
  DERR_TIMEOUT = 32,  // a bounded device wait gave up
};

// ---------------------------------------------------------------------------
// Device memory owned by a handle (stream-ordered pool allocations).
// ---------------------------------------------------------------------------
struct DevMem {
  std::vector<void*> ptrs;
  cudaStream_t stream = nullptr;
  template <typename T>
  T* alloc(size_t count) {
    if (count == 0) count = 1;
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, count * sizeof(T), stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(e == cudaErrorMemoryAllocation ? ASM_ERR_OOM : ASM_ERR_CUDA,
           std::string("device allocation of ") + std::to_string(count * sizeof(T)) +
               " bytes failed: " + cudaGetErrorString(e));
    }
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  // free one allocation made by alloc (nothing for null)
  void free(void* p) {
    if (p == nullptr) return;
    for (size_t k = 0; k < ptrs.size(); ++k)
      if (ptrs[k] == p) {
        cudaFreeAsync(p, stream);
        ptrs.erase(ptrs.begin() + k);
        return;
      }
  }
  void release() {
    for (void* p : ptrs) cudaFreeAsync(p, stream);
    ptrs.clear();
  }
};

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// Grid-wide deterministic reduction without a second launch: every block
// stores its partial, the last block to arrive (atomic ticket) adds the
// partials in block order and runs fin(total) on thread 0, then re-arms the
// ticket.  No block waits for another.
struct GridSum {
  double* part;       // one slot per block of the launch
  unsigned* ticket;   // zero between launches
};

constexpr int TILE = 64;  // tile edge of the local dense matrices and of the apply

// ---------------------------------------------------------------------------
// Warp / block reductions (deterministic: fixed shuffle tree)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; result valid in all threads.  `sh` needs blockDim/32 slots.
template <typename T>
__device__ T block_sum(T v, T* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T t = 0;
  if (wid == 0) {
    t = lane < nw ? sh[lane] : T(0);
    t = warp_sum(t);
    if (lane == 0) sh[0] = t;
  }
  __syncthreads();
  t = sh[0];
  __syncthreads();
  return t;
}

// The block partial v goes to gs.part[blockIdx.x]; the last block of the
// launch adds all partials in block order and calls fin(total) on thread 0.
// All threads of every block must call it (it contains block barriers).
template <typename F>
__device__ void grid_sum_last(double v, GridSum gs, F&& fin) {
  __shared__ double red_gs[32];
  __shared__ int last_gs;
  v = block_sum(v, red_gs);
  if (threadIdx.x == 0) {
    gs.part[blockIdx.x] = v;
    __threadfence();
    last_gs = atomicAdd(gs.ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last_gs) {
    __threadfence();
    double t = 0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) t += __ldcg(gs.part + k);
    t = block_sum(t, red_gs);
    if (threadIdx.x == 0) {
      fin(t);
      *gs.ticket = 0;
    }
  }
}

// Binary search for `key` in sorted a[lo, hi); returns index or -1.
__device__ __forceinline__ int bsearch_i32(const int32_t* a, int lo, int hi, int32_t key) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    int32_t v = a[mid];
    if (v == key) return mid;
    if (v < key) lo = mid + 1; else hi = mid;
  }
  return -1;
}

// SplitMix64 finaliser (Steele, Lea, Flood 2014) and a counter-based normal
// by Box-Muller: output k of stream s is mix(s + (k+1) * golden gamma).
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double counter_uniform(uint64_t seed, uint64_t k) {
  return (double)(splitmix64(seed + (k + 1) * 0x9E3779B97F4A7C15ull) >> 11) * 0x1.0p-53;
}
__device__ __forceinline__ double counter_normal(uint64_t seed, uint64_t k) {
  double u1 = counter_uniform(seed, 2 * k), u2 = counter_uniform(seed, 2 * k + 1);
  return sqrt(-2.0 * log1p(-u1)) * cospi(2.0 * u2);
}

// ---------------------------------------------------------------------------
// Launch accounting: every kernel of the library bumps a per-translation-unit
// device counter once per launch (block 0, thread 0), so graph replays are
// counted too.  asm_kernel_launches() sums the counters of all units.
// ---------------------------------------------------------------------------
static __device__ unsigned long long g_launch_count = 0;
#define COUNT_LAUNCH()                                                                  \
  do {                                                                                  \
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 &&    \
        threadIdx.y == 0 && threadIdx.z == 0)                                           \
      atomicAdd(&::asmgpu::g_launch_count, 1ull);                                       \
  } while (0)
int register_launch_counter(unsigned long long (*reader)());
static unsigned long long read_tu_launch_count() {
  unsigned long long v = 0;
  if (cudaMemcpyFromSymbol(&v, g_launch_count, sizeof(v)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return v;
}
[[maybe_unused]] static int g_launch_counter_registered = register_launch_counter(&read_tu_launch_count);
unsigned long long total_kernel_launches();

// ---------------------------------------------------------------------------
// Host helpers implemented in util.cu
// ---------------------------------------------------------------------------
// Exclusive scan of n int32 counts into out (n+1 entries, out[n] = total),
// int64 accumulation; device arrays.  Returns the total (synchronises).
int64_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, DevMem& mem,
                           cudaStream_t s);
int64_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, DevMem& mem,
                           cudaStream_t s);

}  // namespace asmgpu
