/*
 * asm.h -- C ABI of the GB300 (sm_103a) two-level additive Schwarz library.
 *
 * The library implements the fully algebraic two-level additive Schwarz
 * preconditioner of Al Daas, Jolivet, Nataf and Tournier ("A robust
 * two-level Schwarz preconditioner for sparse matrices"):
 *
 *   M^{-1} = sum_{i=1}^N R_i^T A_ii^{-1} R_i  +  Z E^{-1} Z^T,   E = Z^T A Z,
 *
 * (Remark in Section 4.3 with the coarse space of eq. coarse_space_2), and
 * solves A x = b (eq. Ax=b) with it inside FP64 PCG (SPD A) or right-
 * preconditioned FGMRES (general A, Section 5 / Section 6).
 *
 * Conventions shared by every entry point
 *  - All functions return an asm_status; ASM_OK is 0.  On failure a
 *    thread-local message is available from asm_last_error().  No C++
 *    exception crosses this boundary.
 *  - "device" pointers are CUDA global-memory addresses of the current
 *    device; "host" pointers are ordinary process memory.  Each argument says
 *    which it takes.  Pointers are borrowed: the library never frees memory it
 *    did not allocate and keeps no caller pointer after a call returns.
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued on it; calls that return data to host memory
 *    synchronise it.
 *  - Index arrays are int32, values FP64, matrices CSR with sorted column
 *    indices and no duplicates.
 */
#ifndef ASM_H
#define ASM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct asm_handle asm_handle;
typedef struct asm_mlp asm_mlp;   /* warm-start network, see asm_mlp_create */

typedef enum {
  ASM_OK = 0,
  ASM_ERR_INVALID_ARG = 1,      /* malformed CSR, partition, sizes or options   */
  ASM_ERR_NOT_SPD = 2,          /* a local pivot <= 0 on the SPD path            */
  ASM_ERR_ZERO_PIVOT = 3,       /* a zero local pivot on the general path        */
  ASM_ERR_COARSE_SINGULAR = 4,  /* E = Z^T A Z not SPD / singular (Section 4.1)  */
  ASM_ERR_NONFINITE = 5,        /* NaN or Inf in A or produced during setup      */
  ASM_ERR_NO_CONVERGENCE = 6,   /* Krylov iteration cap reached                  */
  ASM_ERR_TIMEOUT = 7,          /* a bounded device wait gave up                 */
  ASM_ERR_CUDA = 8,             /* a CUDA runtime call failed                    */
  ASM_ERR_OOM = 9,              /* device allocation failed                      */
  ASM_ERR_UNSUPPORTED = 10      /* size beyond a kernel's stated capacity        */
} asm_status;

/* ASM_PREC_FP32_H16: single-precision local work, and the explicit local
 * inverses S_i of the SPD method stored in FP16 (products and sums in FP32)
 * wherever 2^-11 ||S_i||_inf ||A^_ii||_inf + |Omega_i| 2^-25 ||A^_ii||_inf <= 1/4,
 * which keeps the eigenvalues of the stored inverse times A^_ii within
 * [3/4, 5/4]; the other subdomains keep FP32 tiles. */
/* ASM_PREC_FP32_B16: single-precision local work, and for SPD A the
 * subspace iteration's operator applications K Y = U (A^_II (U^T Y)) (the
 * block products with U = W[Gamma_delta, I_i]) multiply BF16-rounded operands
 * with FP32 accumulation; its Gram, Rayleigh-Ritz and output products and
 * everything else stay as ASM_PREC_FP32.  The eigen-residual test is that of
 * the BF16 operator (relative accuracy about 2^-8), so the kept vectors
 * approximate those of eq. gevpsvd to that level.  General A: as FP32. */
typedef enum { ASM_PREC_FP64 = 0, ASM_PREC_FP32 = 1, ASM_PREC_FP32_H16 = 2, ASM_PREC_FP32_B16 = 3 } asm_precision;

/* Sparse matrix A (eq. Ax=b).  row_ptr has n+1 entries, col_idx and val nnz.
 * on_device != 0: the three arrays (and the partition passed to asm_setup)
 * are device pointers; otherwise host pointers. */
typedef struct {
  int32_t n;
  int32_t nnz;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const double* val;
  int32_t on_device;
} asm_csr;

typedef struct {
  int32_t spd;              /* 1: SPD method (eq. gevpsvd, Cholesky-type local
                               sweep); 0: general matrices (Section 5: left
                               singular vectors of D_i Pi_i, LU-type sweep)   */
  int32_t local_precision;  /* asm_precision of the local inverses, the eigen
                               iteration and the local part of the apply       */
  int32_t oversample;       /* extra block columns of the subspace iteration   */
  int32_t max_sweeps;       /* cap on subspace-iteration sweeps                 */
  double eig_tol;           /* relative eigen-residual tolerance                */
  double nu;                /* >= 1 (SPD only): also add to each Z_i the
                               eigenvectors u of eq. uppergevp (Section 3.3,
                               D_i A_ii D_i u = lambda A_ii u, Boolean D_i)
                               with lambda > nu, A_ii-normalised, restricted
                               to I_i (eq. Z_i / coarse_space_2), after the
                               eq. gevpsvd columns; 0: off, as in Section 6.
                               Its eigenvalues are >= 1; 0 < nu < 1 is
                               rejected.  With overlap 1 the two problems
                               share one operator (lambda = 1 + the gevpsvd
                               value), so only lifting vectors beyond the
                               kept gevpsvd ones are added                    */
  int32_t nev_lift;         /* at most this many eq. uppergevp vectors per
                               subdomain (0: nev); nev + nev_lift <= 128      */
  int32_t coarse;           /* 1: two-level; 0: one-level (eq. onelevelasm)     */
  uint64_t seed;            /* counter-based random start of the iteration     */
  int32_t warm_start;       /* 1 (SPD only): the first columns of the start
                               block are predicted by warm_net from per-node
                               features; the rest stay random                 */
  int32_t filter_degree;    /* Chebyshev filter degree between Rayleigh-Ritz
                               steps of the subspace iteration (0: 4 in FP64,
                               3 in FP32)                                      */
  int32_t record_warm;      /* 1 (SPD only): keep the network inputs and the
                               converged start blocks for asm_get_warm_data   */
  int32_t one_level;        /* 0: additive ASM (eq. onelevelasm); 1: restricted
                               ASM (eq. onelevelras, Boolean D_i: each node takes
                               the local solution of its owner)              */
  int32_t coarse_mode;      /* 0: additive coarse correction (Remark, Section
                               4.3); 1: deflated, M^{-1} r = Q r + M_1^{-1}
                               (r - A Q r), Q = Z E^{-1} Z^T, the combination of
                               the Section 6 experiments (with one_level = 1)  */
  int32_t reserved[1];
  double tau;               /* > 0: keep only the eigenvalues of eq. gevpsvd
                               above tau^2 (Prop. 5.1), or the singular values
                               of D_i Pi_i above tau (general method), at most
                               nev per subdomain; 0: the top nev             */
  asm_mlp* warm_net;        /* network for warm_start (borrowed: must stay
                               alive and unused elsewhere during asm_setup)    */
} asm_options;

typedef struct {
  int32_t method;           /* 0: PCG for SPD A with the symmetric apply
                               (one_level 0, coarse_mode 0), else FGMRES;
                               1: PCG; 2: FGMRES                               */
  int32_t restart;          /* FGMRES restart length, at most 512 and at most
                               max_it; 0 (default): 512 for the restricted or
                               deflated apply (GMRES without restart, Section
                               6), 30 otherwise, shortened (not below 30) when
                               the 2m + 1 basis vectors would not fit in 3/4
                               of the free device memory                      */
  double rtol;              /* stop at ||b - A x||_2 / ||b||_2 <= rtol         */
  int32_t max_it;           /* iteration cap                                   */
  int32_t use_x0;           /* 1: x holds the initial guess; 0: x0 = 0         */
  int32_t check_every;      /* iterations between host convergence checks      */
  int32_t reserved[5];
} asm_solve_opts;

typedef struct {
  int32_t iterations;       /* SpMVs performed                                 */
  int32_t converged;
  double final_relres;      /* recursive (PCG) / least-squares (FGMRES) estimate */
  double true_relres;       /* ||b - A x|| / ||b|| recomputed at the end       */
  double solve_ms;          /* device time of the Krylov loop                  */
} asm_solve_info;

typedef struct {
  int32_t n, N, overlap, nev;
  int32_t n_C;              /* coarse dimension |Omega_0|                       */
  int64_t nnz_C;            /* stored nonzeros of E                             */
  double gc, oc;            /* GC = 1 + n_C/n, OC = 1 + nnz_C/nnz_A (Section 6) */
  int64_t sum_ni;           /* sum_i |Omega_i|                                  */
  int32_t max_ni;
  int32_t sweeps_max;       /* largest subspace-iteration sweep count           */
  double eig_resid_max;     /* largest relative eigen-residual at exit          */
  double stage_ms[12];      /* device time per setup stage (see asm_stage_name) */
  int32_t coarse_levels;    /* levels of the nested-dissection tree of E        */
  int32_t coarse_fronts;    /* fronts of the multifrontal factorisation of E    */
  int64_t coarse_front_entries; /* FP64 entries stored in the dense fronts      */
  int32_t coarse_max_front; /* order of the largest front                       */
  int32_t tile_ctas;        /* resident tile-pass blocks per SM the apply uses  */
  int32_t local_sym;        /* subdomains whose local solve is the explicit
                               inverse (one pass); the rest use W^T W        */
  int32_t local_fp16;       /* of those, the ones stored in FP16
                               (ASM_PREC_FP32_H16)                           */
} asm_setup_info;

/* Fill *o with defaults: spd 1, FP64, oversample 8, max_sweeps 0 (= 40 in
 * FP64, 12 in FP32), eig_tol 0 (= 1e-8 in FP64, 4e-3 in FP32), nu off, coarse
 * on, seed 0, filter degree 0 (= 4 in FP64, 3 in FP32), no warm start, nothing
 * recorded. */
void asm_default_options(asm_options* o);
void asm_default_solve_opts(asm_solve_opts* o);

/* Build the preconditioner for A with the nonoverlapping partition `part`
 * (n entries, values 0..N-1, Section 2.1), `overlap` = delta >= 1 layers grown
 * through the graph of A + A^T, and `nev` coarse vectors per subdomain.
 * Steps (each a device stage): overlap index sets (Section 2.1), dense A_ii
 * (Section 2.3, symmetrically scaled to unit diagonal), local factor -- SPD:
 * Cholesky A_ii = L L^T and W = L^{-1}, whose block W[Gamma_delta, I_i] gives
 * the reduced form of eq. gevpsvd and W[Omega_i \ I_i, I_i] that of
 * eq. uppergevp; general: a blocked Gauss-Jordan sweep whose midpoint gives
 * X = -B^{-1}C (eq. HOp) -- block subspace iteration for eq. gevpsvd (SPD,
 * plus eq. uppergevp when nu is set) or for the left singular vectors of
 * D_i Pi_i (general), Z and E = Z^T A Z (Section 4.1), FP64 factor of E.
 * A's arrays are copied; the caller may free them after the call.
 * Errors: INVALID_ARG for malformed input (checked on the host), NOT_SPD /
 * ZERO_PIVOT for a bad local pivot, COARSE_SINGULAR, NONFINITE, UNSUPPORTED,
 * CUDA, OOM.  On error *out is NULL. */
asm_status asm_setup(const asm_csr* A, const int32_t* part, int32_t N, int32_t overlap,
                     int32_t nev, const asm_options* opt, void* stream, asm_handle** out);

/* z = M^{-1} r (device r, z of length n, FP64; r and z must not alias).
 * Deterministic: the overlapping sum is a fixed-order pull, no atomics. */
asm_status asm_apply(asm_handle* h, const double* r, double* z, void* stream);

/* Solve A x = b.  b and x are device pointers when the handle was built from
 * device CSR arrays, host pointers otherwise (then the copies in and out are
 * part of the call).  info (host) is always filled.  Returns
 * NO_CONVERGENCE if max_it is reached. */
asm_status asm_solve(asm_handle* h, const double* b, double* x, const asm_solve_opts* o,
                     asm_solve_info* info, void* stream);

/* Independent SPD systems that share one handle: rows [seg_off[k],
 * seg_off[k+1]) form segment k, and A couples no two segments and no
 * subdomain has rows in two of them (so A, every local solve and the coarse
 * correction are block diagonal over the segments; checked on the device,
 * INVALID_ARG otherwise).  PCG runs one recurrence per segment (its own
 * step lengths and stopping test ||b_k - A_k x_k|| / ||b_k|| <= rtol, x0 = 0)
 * while the SpMV and the two-level apply are launched once for all segments:
 * a stream of problems of uneven sizes set up by one asm_setup on their
 * block-diagonal matrix is solved in one call, each to its own tolerance.
 * seg_off: host, nseg + 1 non-decreasing offsets from 0 to n (1 <= nseg <=
 * 65535); b, x as in asm_solve (device, or host for a host-built handle);
 * info: host array of nseg entries (iterations = those of segment k until it
 * converged, solve_ms the whole call).  The additive SPD preconditioner only
 * (UNSUPPORTED otherwise).  Returns NO_CONVERGENCE if a segment reaches
 * max_it; NOT_SPD if a step length's denominator is not positive. */
asm_status asm_solve_segments(asm_handle* h, const double* b, double* x, int32_t nseg, const int32_t* seg_off,
                              const asm_solve_opts* o, asm_solve_info* info, void* stream);

/* y = A x with the handle's copy of A (device x, y). */
asm_status asm_spmv(asm_handle* h, const double* x, double* y, void* stream);

/* y = A x for a CSR matrix given by device arrays (n rows, nnz stored
 * entries; int32 row_ptr (n+1) and col_idx, FP64 val), with the kernel the
 * Krylov loop uses for that shape: rows of at most about 12 entries on
 * average one thread per row, longer rows by lane groups.  No handle and no allocation; x and y (device, n) must not
 * overlap.  Errors: INVALID_ARG (null pointer, negative size, x == y), CUDA. */
asm_status asm_csr_spmv(int32_t n, int32_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                        const double* val, const double* x, double* y, void* stream);

/* Batched 64 x 64 single-precision tile products on the tensor cores, the
 * building block of the local factorisation's single-precision path (the
 * blocked Cholesky, triangular inverse and W^T W of Section 2.3's local
 * solves, by levels): for every job,
 *   C = alpha sum_{t < nprod} op(A_t) op(B_t)^T (+ C_in),  alpha = -1 with
 *   ASM_TILE_NEG, else +1,
 * where A_t is the 64 x 64 tile at a + a0 + t a_step (row stride lda) and
 * op(A_t)(m, k) = A_t[m][k], or A_t[k][m] with ASM_TILE_AT (B likewise with
 * ASM_TILE_BT; the product contracts over k), C_in the tile at cin + c_in
 * (stride ldc_in, ASM_TILE_BETA), C written at cout + c_out (stride ldc_out).
 * Offsets and strides are in elements (FP32); every row start must be 16-byte
 * aligned (offsets and strides multiples of 4).  Products use the 3xTF32
 * split (single-precision accuracy) with FP32 accumulation.  The jobs of one
 * call must be independent (no job reads a tile another job writes); a job's
 * output may be one of its own operands.  jobs: host array (copied); a, b,
 * cin, cout: device.  Errors: INVALID_ARG (null pointer, nprod < 1,
 * misaligned offset or stride), TIMEOUT, CUDA. */
typedef struct asm_tile_job {
  int64_t a0, b0, a_step, b_step;
  int64_t c_in, c_out;
  int32_t lda, ldb, ldc_in, ldc_out;
  int32_t nprod;
  int32_t flags;   /* ASM_TILE_* */
  int32_t sub;     /* unused here (0) */
  int32_t unused;
} asm_tile_job;
enum { ASM_TILE_AT = 1, ASM_TILE_BT = 2, ASM_TILE_BETA = 4, ASM_TILE_NEG = 8 };
asm_status asm_tile_products(const asm_tile_job* jobs, int64_t njobs, const float* a, const float* b,
                             const float* cin, float* cout, void* stream);

asm_status asm_get_info(const asm_handle* h, asm_setup_info* info);

/* Measurement helpers (no counterpart in the paper; used by the benchmark).
 * asm_kernel_launches: kernel launches executed by this library since it was
 * loaded (graph replays included), read from per-unit device counters;
 * synchronises the device.
 * asm_time_apply: runs the apply `iters` times on `stream` with CUDA events
 * around its parts and writes mean milliseconds to ms[6]: [0] the pass over
 * all local tiles (row pass), [1] the whole local part (gather, row pass,
 * the second stage), [2] coarse restriction + coarse
 * solve, [3] pull-sum, [4] the parts run one after the other, [5] the apply
 * as asm_apply runs it (coarse part overlapped on a side stream).
 * r, z: device. */
uint64_t asm_kernel_launches(void);
/* asm_time_spmv: mean milliseconds (ms[0]) of the PCG loop's fused
 * q = A p, p.q launch on the handle's matrix over `iters` launches (after 3
 * untimed ones), CUDA events on `stream`; p, q device vectors of length n. */
asm_status asm_time_spmv(asm_handle* h, const double* p, double* q, int32_t iters, void* stream, double* ms);
asm_status asm_time_apply(asm_handle* h, const double* r, double* z, int32_t iters, void* stream, double* ms);
const char* asm_stage_name(int32_t stage);

/* Overlap index sets, host outputs.  sub_offsets: N+1 entries (start of
 * subdomain i in omega); layer_offsets: N*(overlap+2) entries, for subdomain i
 * the local offsets [0, |I_i|, |I_i|+|Gamma_1|, ..., |Omega_i|]; omega:
 * sum_i |Omega_i| global indices in R_i order.  Any pointer may be NULL. */
asm_status asm_get_overlap(const asm_handle* h, int32_t* sub_offsets, int32_t* layer_offsets,
                           int32_t* omega);

/* Retained local values, host outputs of N*nev entries (row i = subdomain i,
 * descending; unused slots 0): lambda^2 of eq. gevpsvd (SPD) or singular
 * values of D_i Pi_i (general); counts[i] = number kept.  Either may be NULL. */
asm_status asm_get_local_values(const asm_handle* h, double* values, int32_t* counts);

/* Retained eigenvalues of eq. uppergevp (Section 3.3; nu set), host outputs
 * of N*nev_lift entries (row i = subdomain i, descending, lambda > nu; unused
 * slots 0); counts[i] = number kept.  Either may be NULL; nothing is written
 * to values when lifting is off and nev_lift is 0. */
asm_status asm_get_lift_values(const asm_handle* h, double* values, int32_t* counts);

/* Subspace-iteration diagnostics, host outputs: resid (N*nev) the relative
 * eigen-residual of each kept pair at exit (row i = subdomain i, 0 beyond the
 * kept count), sweeps (N) the sweeps each subdomain ran.  Either may be NULL. */
asm_status asm_get_eigen_stats(const asm_handle* h, double* resid, int32_t* sweeps);

/* Coarse basis blocks, host output: for subdomain i a |I_i| x counts[i]
 * row-major FP64 block (rows in I_i order), concatenated over i; col_offsets
 * (N+1) gives the first coarse column of each subdomain.  Either may be NULL. */
asm_status asm_get_coarse_basis(const asm_handle* h, double* Z, int32_t* col_offsets);

/* Dense E = Z^T A Z (n_C x n_C row-major FP64, host) as assembled, before
 * factorisation. */
asm_status asm_get_coarse_matrix(const asm_handle* h, double* E);

void asm_destroy(asm_handle* h);
const char* asm_last_error(void);

/* ------------------------------------------------------------------------
 * Learned warm start of the subspace iteration (the paper has no learned
 * part; its randomized start, Section 5.1, stays the default and the
 * fallback).  A per-node network maps ASM_WARM_FEATURES features of each
 * node of Gamma_delta (the outermost overlap layer, whose nodes index the
 * rows of the iteration's block) to `outputs` values: row v of the start
 * block.  Architecture: 16 -> hidden -> hidden -> outputs, ReLU after the
 * two hidden layers, FP16 operands with FP32 accumulation on the tensor
 * cores, FP32 master weights, Adam.  Training loss per subdomain i with
 * network output Y_i (g_i x k) and converged orthonormal vectors Z_i:
 *   L_i = k - tr((Y_i^T Y_i)^{-1} Y_i^T Z_i Z_i^T Y_i),
 * the sum of squared sines of the principal angles between span(Y_i) and
 * span(Z_i); a batch's loss is the mean of L_i over its subdomains.
 *
 * Features of node v (A^ = D^{-1/2} A D^{-1/2}, la(v) = log10|a_vv|,
 * K = the iteration's operator, 1 = ones/sqrt(g), t_r = r/(g-1) - 1/2 with
 * r the node's row in Gamma_delta, R_i order):
 *   0 (la(v) - mean over Gamma_delta)/6;  1 max over neighbours u inside
 *   Omega_{1:delta-1} of (la(u) - la(v))/6;  2-4 sums of |A^_vu| over
 *   neighbours inside Omega_{1:delta-1}, in Gamma_delta, outside Omega_i;
 *   5-7 the counts of those neighbours / 6;  8 y = K1/max|K1|;
 *   9 log10(1e-4 + |y|)/4 + 1;  10, 11 the same for K(K1);
 *   12 Kt/max|Kt|;  13 t_r;  14 cos(2 pi (t_r + 1/2));  15 sin(2 pi (t_r + 1/2)).
 * ---------------------------------------------------------------------- */
#define ASM_WARM_FEATURES 16

/* New network with He-normal weights drawn from `seed`, zero biases.
 * hidden: multiple of 16 in 16..1024; outputs: 1..32. */
asm_status asm_mlp_create(int32_t hidden, int32_t outputs, uint64_t seed, asm_mlp** out);
void asm_mlp_destroy(asm_mlp* net);

/* Parameter count and FP32 parameter vector (host), in this order:
 * W1 (16 x hidden, row-major), b1 (hidden), W2 (hidden x hidden), b2 (hidden),
 * W3 (hidden x kp, kp = outputs rounded up to 16; columns >= outputs are 0),
 * b3 (kp).  A layer computes h_out = h_in W + b. */
int64_t asm_mlp_num_params(const asm_mlp* net);
asm_status asm_mlp_get_params(const asm_mlp* net, float* params);
asm_status asm_mlp_set_params(asm_mlp* net, const float* params);

/* Y (rows x outputs, device FP32) = network(X (rows x 16, device FP32)). */
asm_status asm_mlp_forward(asm_mlp* net, const float* X, int32_t rows, float* Y, void* stream);

/* Mean subspace loss and its gradient for one batch, without an update.
 * X: rows x 16 features, T: rows x outputs targets (orthonormal columns per
 * subdomain), both device FP32; seg: nseg+1 device int64 row offsets with
 * seg[0] = 0 and seg[nseg] = rows.  loss (host, may be NULL); grad (host,
 * asm_mlp_num_params floats, may be NULL) = d(mean loss)/d(params). */
asm_status asm_mlp_loss_grad(asm_mlp* net, const float* X, int32_t rows, const float* T, const int64_t* seg,
                             int32_t nseg, double* loss, float* grad, void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, step size lr) on the
 * batch's mean loss; arguments as asm_mlp_loss_grad.  loss (host) may be
 * NULL, which keeps the call free of host synchronisation. */
asm_status asm_mlp_train_step(asm_mlp* net, const float* X, int32_t rows, const float* T, const int64_t* seg,
                              int32_t nseg, float lr, double* loss, void* stream);

/* Training data kept by a setup with record_warm = 1 (SPD): row_offsets
 * (host, N+1 int64) gives subdomain i's rows; X (device, rows x 16) the
 * features; T (device, rows x nev) the converged start blocks (zero columns
 * beyond the kept count).  Any pointer may be NULL.  INVALID_ARG if nothing
 * was recorded. */
asm_status asm_get_warm_data(const asm_handle* h, int64_t* row_offsets, float* X, float* T, void* stream);

/* Allocation-free y = A x together with the dot product x^T y (the paper has
 * no counterpart; this is a service for callers that must not allocate).
 * Some callers cannot call cudaMalloc while they run: code recording a CUDA
 * stream capture, where allocation calls are not allowed; latency-critical
 * host threads, for which cudaMalloc's implicit device synchronisation is
 * unacceptable; applications whose device memory is owned by their own
 * allocator.  This entry point allocates nothing and needs no handle.
 *   n, row_ptr (n+1), col_idx, val: A in CSR, device pointers (as asm_csr).
 *   x (n, device): input.  y (n, device): output A x; y must not overlap x
 *   (both are accessed as non-aliased).  xty (device, one
 *   double): output x^T y, summed in a fixed order (deterministic).
 * Scratch: one partial sum per 64 rows in a static device array built into
 * the library (16384 doubles), so n is limited to 1,048,576 rows; larger n is
 * rejected with ASM_ERR_UNSUPPORTED before any device work.  Every GPU that
 * loads the library holds the array until the process exits.  All calls
 * share the array and every call rewrites the slots it reads, so nothing
 * carries over between calls; calls that overlap on the GPU (concurrent
 * streams) race on it and must be serialised by the caller.  The first call
 * on each device looks the array's device address up (cudaGetSymbolAddress,
 * with that device current); make that first call before any stream capture.
 * Errors: INVALID_ARG (null pointer, n < 0), UNSUPPORTED (n too large), CUDA. */
asm_status asm_spmv_dot_noalloc(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                                const double* x, double* y, double* xty, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ASM_H */
