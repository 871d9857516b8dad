// Batched 64 x 64 tile products on the tcgen05 tensor cores (3xTF32).
//
// Each block (4 warps) owns a 64-column FP32 accumulator in tensor memory
// (TMEM) and strides over the jobs.  For every product of a job the block
// stages both 64 x 64 operand tiles from global memory into shared memory in
// the canonical K-major layout without swizzle (8-row x 16-byte core matrices,
// K fastest), split into TF32 high and low parts (x = hi + lo, hi = x rounded
// to TF32, lo = the exact remainder); one thread issues the three products
// lo*hi + hi*lo + hi*hi (8 MMAs of K = 8 each, M = N = 64) and commits them to
// an mbarrier.  The operand loads of the next product are issued into
// registers before the block waits for the MMAs, so they overlap.  The
// dropped lo*lo term and the TF32 rounding of the lo parts leave an error of
// about 2^-21 relative per product term, like an FP32 dot product.
// Epilogue: tcgen05.ld of the accumulator (with M = 64, row r of D sits in
// TMEM lane 32 (r / 16) + r % 16, so warp w reads rows 16 w .. 16 w + 15 in
// its first 16 lanes), through shared memory to coalesced global stores.
#include <algorithm>

#include "tcgemm.cuh"

namespace asmgpu {
namespace {

constexpr int NTH = 128;                 // threads of a block
constexpr int TT = 64;                   // tile edge
constexpr int PER = TT * TT / 4 / NTH;   // float4 pieces of one operand per thread
constexpr int PART = TT * TT;            // floats of one staged operand part
constexpr int STG = TT + 4;              // row stride of the epilogue staging tile
constexpr size_t SMEM = 4 * PART * sizeof(float) + 256;
// instruction descriptor, kind::tf32: D = F32 (bits 4-5), A = B = TF32 (bits
// 7-9, 10-12), both K-major (bits 15, 16 clear), N >> 3 (bits 17-22), M >> 4
// (bits 24-28)
constexpr uint32_t IDESC =
    (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TT >> 3) << 17) | ((uint32_t)(TT >> 4) << 24);
constexpr uint32_t LBO = 128;            // bytes between core matrices along K
constexpr uint32_t SBO = (TT / 4) * 128; // bytes between 8-row groups
constexpr long long WAIT_CYCLES = 2000000000LL;

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((LBO >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((SBO >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// float index of operand element (r, k) in the K-major core-matrix layout
__device__ __forceinline__ int kmaj(int r, int k) { return ((r >> 3) * (TT / 4) + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3); }

__device__ __forceinline__ void split(float x, float& h, float& l) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  h = __uint_as_float(u);
  l = __fsub_rn(x, h);
}

// Thread's piece j of an operand tile: operand row m, columns k0 .. k0 + 3.
// The 8 threads of a quarter warp take 8 consecutive rows at one k0, so the
// 16-byte stores into the core-matrix layout are conflict-free; the global
// loads read 8 rows x 16 bytes (operand as stored) or 4 source rows x 32
// bytes (transposed operand) per warp instruction.
__device__ __forceinline__ void piece(int j, int& m, int& k0) {
  const int f = j * NTH + threadIdx.x;
  const int s = f >> 5, lane = f & 31;
  m = (s & 7) * 8 + (lane & 7);
  k0 = 4 * ((s >> 3) * 4 + (lane >> 3));
}

// operand(m, k) = src[m * ld + k], or src[k * ld + m] when trans.  Plain
// (coherent) loads: an output tile may be an operand of its own job.
__device__ __forceinline__ void load_tile(const float* src, int ld, bool trans, float4 (&v)[PER]) {
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    int m, k0;
    piece(j, m, k0);
    if (!trans) {
      v[j] = *reinterpret_cast<const float4*>(src + (int64_t)m * ld + k0);
    } else {
      const float* p = src + (int64_t)k0 * ld + m;
      v[j] = make_float4(p[0], p[ld], p[2 * (int64_t)ld], p[3 * (int64_t)ld]);
    }
  }
}

__device__ __forceinline__ void store_tile(const float4 (&v)[PER], float* hi, float* lo) {
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    int m, k0;
    piece(j, m, k0);
    float4 h, l;
    split(v[j].x, h.x, l.x);
    split(v[j].y, h.y, l.y);
    split(v[j].z, h.z, l.z);
    split(v[j].w, h.w, l.w);
    const int o = kmaj(m, k0);
    *reinterpret_cast<float4*>(hi + o) = h;
    *reinterpret_cast<float4*>(lo + o) = l;
  }
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
      : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > WAIT_CYCLES) return false;
  }
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// next job of this block at or after index jb that is not skipped; njobs if none
__device__ __forceinline__ int64_t next_job(const TcJob* __restrict__ jobs, int64_t jb, int64_t njobs,
                                            const int8_t* __restrict__ sym, TcJob& J) {
  for (; jb < njobs; jb += gridDim.x) {
    J = jobs[jb];
    if (!(J.flags & TCF_SYMONLY) || sym[J.sub]) return jb;
  }
  return njobs;
}

__global__ void __launch_bounds__(NTH, 3) k_tc_tiles(const TcJob* __restrict__ jobs, int64_t njobs,
                                                     const float* abase, const float* bbase,
                                                     const float* cinbase, float* coutbase,
                                                     const int8_t* __restrict__ sym, int32_t* __restrict__ err) {
  COUNT_LAUNCH();
  extern __shared__ __align__(128) unsigned char smraw[];
  float* base = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smraw) + 127) & ~(uintptr_t)127);
  float* hiA = base;
  float* loA = base + PART;
  float* hiB = base + 2 * PART;
  float* loB = base + 3 * PART;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bar = saddr(&mbar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(saddr(&tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tslot;
  const uint32_t dA = saddr(hiA), dAl = saddr(loA), dB = saddr(hiB), dBl = saddr(loB);
  uint32_t phase = 0;
  float4 va[PER], vb[PER];
  TcJob J, Jn;
  int64_t jb = next_job(jobs, blockIdx.x, njobs, sym, J);
  if (jb < njobs) {
    load_tile(abase + J.a0, J.lda, (J.flags & TCF_AT) != 0, va);
    load_tile(bbase + J.b0, J.ldb, (J.flags & TCF_BT) != 0, vb);
  }
  while (jb < njobs) {
    const int64_t jn = next_job(jobs, jb + gridDim.x, njobs, sym, Jn);
    for (int t = 0; t < J.nprod; ++t) {
      store_tile(va, hiA, loA);
      store_tile(vb, hiB, loB);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        fence_after();
#pragma unroll
        for (int ks = 0; ks < TT / 8; ++ks) {
          const uint32_t o = ks * 2 * 128;  // K = 8 TF32 values: two core matrices
          mma_tf32(tmem, sdesc(dAl + o), sdesc(dB + o), (t > 0 || ks > 0) ? 1u : 0u);
          mma_tf32(tmem, sdesc(dA + o), sdesc(dBl + o), 1u);
          mma_tf32(tmem, sdesc(dA + o), sdesc(dB + o), 1u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                     : "memory");
      }
      // operands of the next product (of this job, else of the next job)
      // load while the MMAs run and, for the last product, the epilogue
      if (t + 1 < J.nprod) {
        load_tile(abase + J.a0 + (int64_t)(t + 1) * J.a_step, J.lda, (J.flags & TCF_AT) != 0, va);
        load_tile(bbase + J.b0 + (int64_t)(t + 1) * J.b_step, J.ldb, (J.flags & TCF_BT) != 0, vb);
      } else if (jn < njobs) {
        load_tile(abase + Jn.a0, Jn.lda, (Jn.flags & TCF_AT) != 0, va);
        load_tile(bbase + Jn.b0, Jn.ldb, (Jn.flags & TCF_BT) != 0, vb);
      }
      if (!mbar_wait(bar, phase)) abort_flag = 1;
      phase ^= 1u;
      __syncthreads();
      if (abort_flag) break;
    }
    if (abort_flag) break;
    fence_after();
    // accumulator rows 16 warp .. +15 (lanes 0-15 of the warp's lane quarter),
    // 16 columns at a time, staged in the (free) A parts
    float* stg = base;
    const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(ta + 16 * q));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (lane < 16) {
        float* row = stg + (16 * warp + lane) * STG + 16 * q;
#pragma unroll
        for (int c = 0; c < 16; c += 4)
          *reinterpret_cast<float4*>(row + c) = make_float4(__uint_as_float(r[c]), __uint_as_float(r[c + 1]),
                                                            __uint_as_float(r[c + 2]), __uint_as_float(r[c + 3]));
      }
    }
    fence_before();
    __syncthreads();
    {
      const bool neg = (J.flags & TCF_NEG) != 0, beta = (J.flags & TCF_BETA) != 0;
#pragma unroll 2
      for (int j = 0; j < PER; ++j) {
        const int idx = j * NTH + tid, r = idx >> 4, c = (idx & 15) * 4;
        float4 v = *reinterpret_cast<const float4*>(stg + r * STG + c);
        if (neg) { v.x = -v.x; v.y = -v.y; v.z = -v.z; v.w = -v.w; }
        if (beta) {
          const float4 ci = *reinterpret_cast<const float4*>(cinbase + J.c_in + (int64_t)r * J.ldc_in + c);
          v.x = __fadd_rn(ci.x, v.x); v.y = __fadd_rn(ci.y, v.y); v.z = __fadd_rn(ci.z, v.z); v.w = __fadd_rn(ci.w, v.w);
        }
        *reinterpret_cast<float4*>(coutbase + J.c_out + (int64_t)r * J.ldc_out + c) = v;
      }
    }
    __syncthreads();  // staging reused by the next job's operands
    J = Jn;
    jb = jn;
  }
  if (abort_flag && tid == 0) atomicOr(err, DERR_TIMEOUT);
  // a gave-up wait: give the MMAs in flight one more bounded wait before the
  // accumulator is released
  if (abort_flag) mbar_wait(bar, phase ^ 1u);
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem));
  }
}

}  // namespace

void tc_tiles(const TcJob* jobs, int64_t njobs, const float* a, const float* b, const float* cin, float* cout,
              const int8_t* sym, int32_t* err, int num_sms, cudaStream_t s) {
  if (njobs <= 0) return;
  static bool attr = false;
  if (!attr) {
    CK(cudaFuncSetAttribute(k_tc_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM));
    attr = true;
  }
  const int64_t grid = std::min<int64_t>(njobs, (int64_t)num_sms * 3);
  k_tc_tiles<<<(unsigned)grid, NTH, SMEM, s>>>(jobs, njobs, a, b, cin, cout, sym, err);
  CK_LAUNCH("tensor-core tile products");
}

}  // namespace asmgpu
