// Batched 64 x 64 tile products on the tcgen05 tensor cores (3xTF32).
//
// One persistent block per SM strides over the jobs with warp-specialised
// roles, connected by mbarriers:
//  * producer warps (0-3): copy both 64 x 64 operand tiles of each product
//    with 16-byte asynchronous copies into a two-stage ring of raw FP32 tiles
//    in shared memory (rows padded to 68 floats), each thread's copies
//    reported to the stage's mbarrier as they land;
//  * split warps (8-11): turn a raw stage into the TF32 high and low parts
//    (x = hi + lo, hi = x rounded to TF32, lo = the exact remainder) of both
//    operands in the canonical K-major layout without swizzle (8-row x 16-byte
//    core matrices, K fastest), double-buffered;
//  * MMA thread (warp 12, lane 0): issues the three products lo*hi + hi*lo +
//    hi*hi (8 MMAs of K = 8 each, M = N = 64) of each product into one of two
//    64-column FP32 accumulators in tensor memory (TMEM), alternating per job,
//    and commits them to mbarriers (operand buffer free; accumulator ready);
//  * epilogue warps (4-7): read a finished accumulator with tcgen05.ld (with
//    M = 64, row r of D sits in TMEM lane 32 (r / 16) + r % 16, so warp w reads
//    rows 16 (w % 4) .. +15 in its first 16 lanes), release it and store the
//    tile (scaled by -1 and added to C_in as the job asks).
// So the copies of product t+2, the split of t+1, the MMAs of t and the
// epilogue of the previous job overlap.  The dropped lo*lo term and the TF32
// rounding of the lo parts leave an error of about 2^-21 relative per product
// term, like an FP32 dot product.  Every mbarrier wait is bounded; one that
// gives up sets DERR_TIMEOUT and the roles wind down.
#include <algorithm>

#include "tcgemm.cuh"

namespace asmgpu {
namespace {

constexpr int NTH = 416;                 // 13 warps: 4 producer, 4 epilogue, 4 split, MMA
constexpr int W_PROD = 0, W_EPI = 4, W_SPLIT = 8, W_MMA = 12;
constexpr int NPROD = 128;               // producer threads
constexpr int NSPLIT = 128;              // split threads
constexpr int TT = 64;                   // tile edge
constexpr int PER = TT * TT / 4 / NSPLIT;  // float4 pieces of one operand per split thread
constexpr int PART = TT * TT;            // floats of one staged operand part
constexpr int RLD = TT + 4;              // row stride of a raw tile (floats)
constexpr int RAW = TT * RLD;            // floats of one raw tile
constexpr size_t SMEM = (size_t)(2 * 2 * RAW + 2 * 4 * PART) * sizeof(float) + 1024;
constexpr int CPT = 2 * TT * TT / 4 / NPROD;  // 16-byte copies per producer thread per product
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

// Split thread u's piece j of an operand tile: operand row m, columns
// k0 .. k0 + 3.  The 8 threads of a quarter warp take 8 consecutive rows at
// one k0: the 16-byte stores into the core-matrix layout are conflict-free,
// and so are the 16-byte reads of a raw tile held as stored (row stride 68).
__device__ __forceinline__ void piece(int j, int u, int& m, int& k0) {
  const int f = j * NSPLIT + u;
  const int s = f >> 5, lane = f & 31;
  m = (s & 7) * 8 + (lane & 7);
  k0 = 4 * ((s >> 3) * 4 + (lane >> 3));
}

// raw tile (source rows, stride RLD) -> hi/lo parts: operand(m, k) =
// raw[m][k], or raw[k][m] when trans
__device__ __forceinline__ void split_tile(const float* raw, bool trans, int u, float* hi, float* lo) {
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    int m, k0;
    piece(j, u, m, k0);
    float4 v;
    if (!trans) {
      v = *reinterpret_cast<const float4*>(raw + m * RLD + k0);
    } else {
      const float* q = raw + k0 * RLD + m;
      v = make_float4(q[0], q[RLD], q[2 * RLD], q[3 * RLD]);
    }
    float4 h, l;
    split(v.x, h.x, l.x);
    split(v.y, h.y, l.y);
    split(v.z, h.z, l.z);
    split(v.w, h.w, l.w);
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

// bounded wait for the phase of the given parity; false if it gave up (or
// another role did: *abort set)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const volatile int* abort) {
  const long long t0 = clock64();
  for (int k = 0;; ++k) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((k & 63) == 63 && *abort) return false;
    if (clock64() - t0 > WAIT_CYCLES) return false;
  }
}
// the same wait taken by a whole warp, its outcome made warp-uniform (so that
// the warp stays converged for __syncwarp and the .sync.aligned instructions)
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, const volatile int* abort) {
  return __all_sync(0xffffffffu, mbar_wait(bar, parity, abort));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// 16-byte asynchronous copy global -> shared (L2 only), and the arrival on
// an mbarrier once all of this thread's earlier copies have landed
__device__ __forceinline__ void cp_async16(uint32_t dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_arrive(uint32_t bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
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

__global__ void __launch_bounds__(NTH, 1) k_tc_tiles(const TcJob* __restrict__ jobs, int64_t njobs,
                                                     const float* abase, const float* bbase,
                                                     const float* cinbase, float* coutbase,
                                                     const int8_t* __restrict__ sym, int32_t* __restrict__ err) {
  COUNT_LAUNCH();
  extern __shared__ __align__(128) unsigned char smraw[];
  float* base = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
  float* raw = base;                 // [stage][A | B] raw tiles, RAW floats each
  float* hl = base + 2 * 2 * RAW;    // [buffer][hiA | loA | hiB | loB], PART floats each
  __shared__ __align__(8) uint64_t bars[13];
  __shared__ uint32_t tslot;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // barriers: raw_full[2], raw_empty[2], hl_full[2], hl_empty[2], acc_full[2], acc_empty[2], fin
  auto bar = [&](int k) { return saddr(&bars[k]); };
  const int RF = 0, RE = 2, HF = 4, HE = 6, AF = 8, AE = 10, FIN = 12;
  if (warp == W_PROD) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(saddr(&tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == W_MMA * 32) {
    for (int k = 0; k < 2; ++k) {
      mbar_init(bar(RF + k), NPROD);  // one arrival per producer thread once its copies land
      mbar_init(bar(RE + k), 4);   // one arrival per split warp
      mbar_init(bar(HF + k), 4);   // one arrival per split warp
      mbar_init(bar(HE + k), 1);   // MMA commit
      mbar_init(bar(AF + k), 1);   // MMA commit
      mbar_init(bar(AE + k), 4);   // one arrival per epilogue warp
    }
    mbar_init(bar(FIN), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tslot;
  auto give_up = [&]() {
    abort_flag = 1;
    atomicOr(err, DERR_TIMEOUT);
  };

  if (warp < W_EPI) {
    // ---------------- producers: raw tiles by 16-byte asynchronous copies
    const int u = tid - W_PROD * 32;
    uint32_t P = 0;
    TcJob J;
    for (int64_t jb = next_job(jobs, blockIdx.x, njobs, sym, J); jb < njobs && !abort_flag;
         jb = next_job(jobs, jb + gridDim.x, njobs, sym, J)) {
      for (int t = 0; t < J.nprod; ++t) {
        const int st = P & 1;
        if (P >= 2 && !warp_wait(bar(RE + st), ((P >> 1) - 1) & 1, &abort_flag)) { give_up(); break; }
        const float* sa = abase + J.a0 + (int64_t)t * J.a_step;
        const float* sb = bbase + J.b0 + (int64_t)t * J.b_step;
        const uint32_t ra = saddr(raw + (2 * st) * RAW), rb = saddr(raw + (2 * st + 1) * RAW);
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          const int id = c * NPROD + u;            // 0 .. 2047: A chunks, then B chunks
          const int tile = id >> 10, row = (id >> 4) & 63, col = (id & 15) * 4;
          if (tile == 0) cp_async16(ra + (row * RLD + col) * 4, sa + (int64_t)row * J.lda + col);
          else cp_async16(rb + (row * RLD + col) * 4, sb + (int64_t)row * J.ldb + col);
        }
        cp_async_arrive(bar(RF + st));
        ++P;
      }
    }
    // this thread's copies in flight land before the block leaves
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (warp >= W_SPLIT && warp < W_SPLIT + 4) {
    // ---------------- split: raw stage -> TF32 hi/lo parts
    const int u = tid - W_SPLIT * 32;
    uint32_t P = 0;
    TcJob J;
    for (int64_t jb = next_job(jobs, blockIdx.x, njobs, sym, J); jb < njobs && !abort_flag;
         jb = next_job(jobs, jb + gridDim.x, njobs, sym, J)) {
      const bool at = (J.flags & TCF_AT) != 0, bt = (J.flags & TCF_BT) != 0;
      for (int t = 0; t < J.nprod; ++t) {
        const int st = P & 1, b = P & 1;
        if (!warp_wait(bar(RF + st), (P >> 1) & 1, &abort_flag)) { give_up(); break; }
        if (P >= 2 && !warp_wait(bar(HE + b), ((P >> 1) - 1) & 1, &abort_flag)) { give_up(); break; }
        float* h4 = hl + b * 4 * PART;
        split_tile(raw + (2 * st) * RAW, at, u, h4, h4 + PART);
        split_tile(raw + (2 * st + 1) * RAW, bt, u, h4 + 2 * PART, h4 + 3 * PART);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(bar(RE + st));
          mbar_arrive(bar(HF + b));
        }
        ++P;
      }
    }
  } else if (warp == W_MMA) {
    // ---------------- MMA issue (one thread)
    if (lane == 0) {
      uint32_t P = 0, q = 0;
      TcJob J;
      for (int64_t jb = next_job(jobs, blockIdx.x, njobs, sym, J); jb < njobs && !abort_flag;
           jb = next_job(jobs, jb + gridDim.x, njobs, sym, J)) {
        const int a = q & 1;
        if (q >= 2 && !mbar_wait(bar(AE + a), ((q >> 1) - 1) & 1, &abort_flag)) { give_up(); break; }
        fence_after();
        const uint32_t acc = tmem + a * TT;
        bool ok = true;
        for (int t = 0; t < J.nprod; ++t) {
          const int b = P & 1;
          if (!mbar_wait(bar(HF + b), (P >> 1) & 1, &abort_flag)) { give_up(); ok = false; break; }
          fence_after();
          const uint32_t d0 = saddr(hl + b * 4 * PART);
          const uint32_t dA = d0, dAl = d0 + PART * 4, dB = d0 + 2 * PART * 4, dBl = d0 + 3 * PART * 4;
#pragma unroll
          for (int ks = 0; ks < TT / 8; ++ks) {
            const uint32_t o = ks * 2 * 128;  // K = 8 TF32 values: two core matrices
            mma_tf32(acc, sdesc(dAl + o), sdesc(dB + o), (t > 0 || ks > 0) ? 1u : 0u);
            mma_tf32(acc, sdesc(dA + o), sdesc(dBl + o), 1u);
            mma_tf32(acc, sdesc(dA + o), sdesc(dB + o), 1u);
          }
          mma_commit(bar(HE + b));
          ++P;
        }
        if (!ok) break;
        mma_commit(bar(AF + a));
        ++q;
      }
      // every MMA of this block has completed before the accumulators are freed
      mma_commit(bar(FIN));
      mbar_wait(bar(FIN), 0, &abort_flag);
    }
  } else if (warp >= W_EPI && warp < W_EPI + 4) {
    // ---------------- epilogue: accumulator -> global tile
    const int quarter = warp & 3;
    uint32_t q = 0;
    TcJob J;
    for (int64_t jb = next_job(jobs, blockIdx.x, njobs, sym, J); jb < njobs && !abort_flag;
         jb = next_job(jobs, jb + gridDim.x, njobs, sym, J)) {
      const int a = q & 1;
      if (!warp_wait(bar(AF + a), (q >> 1) & 1, &abort_flag)) { give_up(); break; }
      fence_after();
      const uint32_t ta = tmem + ((uint32_t)(32 * quarter) << 16) + a * TT;
      uint32_t r[64];
#pragma unroll
      for (int c = 0; c < 4; ++c)
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[16 * c + 0]), "=r"(r[16 * c + 1]), "=r"(r[16 * c + 2]), "=r"(r[16 * c + 3]),
              "=r"(r[16 * c + 4]), "=r"(r[16 * c + 5]), "=r"(r[16 * c + 6]), "=r"(r[16 * c + 7]),
              "=r"(r[16 * c + 8]), "=r"(r[16 * c + 9]), "=r"(r[16 * c + 10]), "=r"(r[16 * c + 11]),
              "=r"(r[16 * c + 12]), "=r"(r[16 * c + 13]), "=r"(r[16 * c + 14]), "=r"(r[16 * c + 15])
            : "r"(ta + 16 * c));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(AE + a));
      if (lane < 16) {
        const int row = 16 * quarter + lane;
        const bool neg = (J.flags & TCF_NEG) != 0, beta = (J.flags & TCF_BETA) != 0;
        float* out = coutbase + J.c_out + (int64_t)row * J.ldc_out;
        const float* cin = cinbase + J.c_in + (int64_t)row * J.ldc_in;
#pragma unroll
        for (int c = 0; c < 64; c += 4) {
          float4 v = make_float4(__uint_as_float(r[c]), __uint_as_float(r[c + 1]), __uint_as_float(r[c + 2]),
                                 __uint_as_float(r[c + 3]));
          if (neg) { v.x = -v.x; v.y = -v.y; v.z = -v.z; v.w = -v.w; }
          if (beta) {
            const float4 ci = *reinterpret_cast<const float4*>(cin + c);
            v.x = __fadd_rn(ci.x, v.x); v.y = __fadd_rn(ci.y, v.y); v.z = __fadd_rn(ci.z, v.z); v.w = __fadd_rn(ci.w, v.w);
          }
          *reinterpret_cast<float4*>(out + c) = v;
        }
      }
      ++q;
    }
  }
  fence_before();
  __syncthreads();
  if (warp == W_PROD) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
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
  const int64_t grid = std::min<int64_t>(njobs, (int64_t)num_sms);
  k_tc_tiles<<<(unsigned)grid, NTH, SMEM, s>>>(jobs, njobs, a, b, cin, cout, sym, err);
  CK_LAUNCH("tensor-core tile products");
}

}  // namespace asmgpu
