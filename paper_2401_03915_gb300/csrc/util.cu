// Host error plumbing and device prefix sums.
#include "common.cuh"

namespace asmgpu {

[[noreturn]] void fail(asm_status s, const std::string& msg) { throw AsmError{s, msg}; }

namespace {
std::vector<unsigned long long (*)()>& counters() {
  static std::vector<unsigned long long (*)()> v;
  return v;
}
}  // namespace

int register_launch_counter(unsigned long long (*reader)()) {
  counters().push_back(reader);
  return (int)counters().size();
}

unsigned long long total_kernel_launches() {
  unsigned long long t = 0;
  for (auto f : counters()) t += f();
  return t;
}

void cuda_check(cudaError_t e, const char* what, const char* file, int line) {
  if (e == cudaSuccess) return;
  cudaGetLastError();
  fail(e == cudaErrorMemoryAllocation ? ASM_ERR_OOM : ASM_ERR_CUDA,
       std::string(what) + " failed at " + file + ":" + std::to_string(line) + ": " +
           cudaGetErrorString(e));
}

namespace {
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_PER_THREAD = 8;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_PER_THREAD;  // elements per block

template <typename In>
__global__ void k_chunk_sums(const In* __restrict__ in, int64_t n, int64_t* __restrict__ sums) {
  COUNT_LAUNCH();
  __shared__ int64_t sh[SCAN_THREADS / 32];
  int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK;
  int64_t acc = 0;
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
    if (i < n) acc += (int64_t)in[i];
  }
  acc = block_sum<int64_t>(acc, sh);
  if (threadIdx.x == 0) sums[blockIdx.x] = acc;
}

// Exclusive scan of up to SCAN_THREADS * 32 block sums in one block.
__global__ void k_scan_sums(int64_t* sums, int64_t nb) {
  COUNT_LAUNCH();
  __shared__ int64_t sh[SCAN_THREADS];
  const int per = (int)ceil_div(nb, SCAN_THREADS);
  int64_t local = 0;
  for (int k = 0; k < per; ++k) {
    int64_t i = (int64_t)threadIdx.x * per + k;
    if (i < nb) local += sums[i];
  }
  sh[threadIdx.x] = local;
  __syncthreads();
  for (int o = 1; o < SCAN_THREADS; o <<= 1) {
    int64_t t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  int64_t run = sh[threadIdx.x] - local;
  for (int k = 0; k < per; ++k) {
    int64_t i = (int64_t)threadIdx.x * per + k;
    if (i < nb) {
      int64_t v = sums[i];
      sums[i] = run;
      run += v;
    }
  }
}

template <typename In, typename Out>
__global__ void k_chunk_scan(const In* __restrict__ in, int64_t n, const int64_t* __restrict__ sums,
                             Out* __restrict__ out) {
  COUNT_LAUNCH();
  __shared__ int64_t sh[SCAN_THREADS];
  int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_PER_THREAD;
  int64_t v[SCAN_PER_THREAD];
  int64_t local = 0;
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    int64_t i = base + k;
    v[k] = i < n ? (int64_t)in[i] : 0;
    local += v[k];
  }
  sh[threadIdx.x] = local;
  __syncthreads();
  for (int o = 1; o < SCAN_THREADS; o <<= 1) {
    int64_t t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  int64_t run = sums[blockIdx.x] + sh[threadIdx.x] - local;
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    int64_t i = base + k;
    if (i < n) out[i] = (Out)run;
    run += v[k];
    if (i == n - 1) out[n] = (Out)run;
  }
}

template <typename In, typename Out>
int64_t scan_impl(const In* in, Out* out, int64_t n, DevMem& mem, cudaStream_t s) {
  if (n == 0) {
    CK(cudaMemsetAsync(out, 0, sizeof(Out), s));
    return 0;
  }
  int64_t nb = ceil_div(n, SCAN_CHUNK);
  if (nb > (int64_t)SCAN_THREADS * 64) fail(ASM_ERR_UNSUPPORTED, "prefix sum longer than supported");
  int64_t* sums = mem.alloc<int64_t>(nb);
  k_chunk_sums<In><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, sums);
  k_scan_sums<<<1, SCAN_THREADS, 0, s>>>(sums, nb);
  k_chunk_scan<In, Out><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, sums, out);
  CK_LAUNCH("prefix sum");
  Out total;
  CK(cudaMemcpyAsync(&total, out + n, sizeof(Out), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return (int64_t)total;
}
}  // namespace

int64_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, DevMem& mem, cudaStream_t s) {
  return scan_impl<int32_t, int32_t>(in, out, n, mem, s);
}
int64_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, DevMem& mem, cudaStream_t s) {
  return scan_impl<int64_t, int64_t>(in, out, n, mem, s);
}

}  // namespace asmgpu
