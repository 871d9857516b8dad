// Batched 64 x 64 tile products on the 5th-generation tensor cores (tcgen05),
// in single-precision accuracy:
//
//   C = alpha * sum_t op(A_t) op(B_t)^T  (+ C_in),   alpha = +-1,
//
// one job per output tile, the jobs of a launch independent of one another.
// The dense local factorisation (Cholesky by levels of 64-column panels, the
// triangular inverse, S = W^T W) is expressed as launches of such jobs.
#pragma once

#include "common.cuh"

namespace asmgpu {

// One output tile.  Offsets are in elements from the launch's base pointers;
// product t of the sum reads A at a0 + t * a_step and B at b0 + t * b_step.
// Without a transpose flag, A(m, k) = A_src[m * lda + k] and B(n, k) =
// B_src[n * ldb + k]; with TCF_AT, A(m, k) = A_src[k * lda + m] (likewise
// TCF_BT).  C(m, n) is written to cout[c_out + m * ldc_out + n].
struct TcJob {
  int64_t a0, b0, a_step, b_step;
  int64_t c_in, c_out;
  int32_t lda, ldb, ldc_in, ldc_out;
  int32_t nprod;   // products in the sum (>= 1)
  int32_t flags;   // TCF_* below
  int32_t sub;     // subdomain (TCF_SYMONLY)
  int32_t unused;
};
static_assert(sizeof(TcJob) == 80, "TcJob layout");

enum : int32_t {
  TCF_AT = 1,       // A transposed
  TCF_BT = 2,       // B transposed
  TCF_BETA = 4,     // add C_in
  TCF_NEG = 8,      // alpha = -1 (else +1)
  TCF_SYMONLY = 16  // skipped unless sym[sub] != 0
};

// Enqueue the jobs (device array) on s.  Operand, input and output bases are
// FP32 device pointers (cin may equal cout, and an output tile may be the A or
// B operand of its own job: every product is staged before it is written).
// sym may be null when no job carries TCF_SYMONLY.  A bounded wait that gives
// up sets DERR_TIMEOUT in *err.
void tc_tiles(const TcJob* jobs, int64_t njobs, const float* a, const float* b, const float* cin, float* cout,
              const int8_t* sym, int32_t* err, int num_sms, cudaStream_t s);

}  // namespace asmgpu
