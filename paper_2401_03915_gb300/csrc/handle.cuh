// Internal state of an asm_handle and the stage entry points between files.
#pragma once

#include "common.cuh"
#include "coarse_nd.cuh"
#include "mlp.cuh"

namespace asmgpu {

// Capacities of the overlap builder (one CTA per subdomain, shared memory).
constexpr int OV_HASH = 8192;    // hash slots for the candidates of one layer
constexpr int OV_LAYER = 4096;   // largest single layer
constexpr int MAX_NI = 16384;    // largest |Omega_i| / |I_i| handled

struct Overlap {
  // device
  int32_t* gptr = nullptr;   // graph of A + A^T, no self loops (n+1)
  int32_t* gidx = nullptr;
  int32_t* sub_off = nullptr;  // N+1, start of subdomain i in omega
  int32_t* lay_off = nullptr;  // N*(delta+2) local layer offsets
  int32_t* omega = nullptr;    // sum n_i global indices
  int32_t* pos_sub = nullptr;  // sum n_i: subdomain of each omega position
  int32_t* occ_ptr = nullptr;  // n+1
  int32_t* occ_pos = nullptr;  // sum n_i: omega positions holding node v, ascending
  int32_t* own_pos = nullptr;  // n: omega position of v inside its own I block
  int64_t* ent_off = nullptr;  // sum n_i + 1: entries of the rows of Omega_i
  int32_t* lcol = nullptr;     // local column of each entry, -1 outside Omega_i
  // host
  std::vector<int32_t> h_sub_off, h_lay_off;
  int64_t sum_n = 0, n_ent = 0;
  int32_t max_n = 0;
};

// One work item of the single-precision tile passes, precomputed on the host
// so that a block reads it in one independent load: subdomain, row (or
// column) block, tile count, explicit-inverse flag; the padded-vector offset,
// the first tile (column pass: the subdomain's first tile), the row-block
// bounds and slots of the explicit inverses; |Omega_i|, its first position,
// the tiles per side.
struct __align__(16) TileItem {
  int32_t i, B, cnt, symi;
  int64_t pad, tile0, bias0, slot0;
  int32_t n, sub_off, nt, unused;
};

struct Dense {
  // per subdomain (host and device copies)
  std::vector<int32_t> h_np;          // padded size round_up(n_i, TILE)
  std::vector<int64_t> h_work_off;    // element offset in the working buffer
  std::vector<int64_t> h_xs_off;      // element offset of X_p^T (g x p)
  std::vector<int64_t> h_s_off;       // element offset of S (g x g)
  std::vector<int32_t> h_nt;          // tiles per side
  std::vector<int64_t> h_tile_off;    // first apply tile of subdomain i
  int64_t* work_off = nullptr;
  int64_t* xs_off = nullptr;
  int64_t* s_off = nullptr;
  int32_t* np = nullptr;
  int32_t* nt = nullptr;
  int64_t* tile_off = nullptr;
  int4* tile_desc = nullptr;          // (subdomain, I, J, 0) of every apply tile
  void* work = nullptr;               // A^_ii, then W = L^{-1} (SPD) or A^_ii^{-1} (row-major, ld = np)
  void* XpT = nullptr;                // general A: X_p^T = -(B^{-1} C)[:p]^T (g x p)
  void* S = nullptr;                  // unused
  void* dinv = nullptr;               // SPD: inverses of the diagonal 64x64 blocks of L
  int64_t* dinv_off = nullptr;
  void* tiles = nullptr;              // apply tiles, TILE*TILE each
  int64_t* pad_off = nullptr;         // start of subdomain i in the padded position space (nt_i * TILE each)
  void* xpad = nullptr;               // apply: gathered, scaled r in the padded space (FP64, or float-float
                                      // pairs scaled per subdomain by a power of two in single precision)
  void* tpad = nullptr;               // apply: t = W x (SPD first pass) or the explicit inverses' row part
  double* xunscale = nullptr;         // single precision: per subdomain, the inverse of the scale of xpad
  int64_t* boff = nullptr;            // single precision: first row block of subdomain i in sym_bias
  float* sym_bias = nullptr;          // single precision, explicit inverses: per row block the power of two
                                      // that biases the tile pass's accumulators (bounds all its partial sums)
  int2* row_items = nullptr;          // (subdomain, row block), most tiles first
  int2* col_items = nullptr;          // (subdomain, column block) of two-pass subdomains, most tiles first
  int2* sym_items = nullptr;          // (subdomain, block) of explicit-inverse subdomains
  int n_row_items = 0, n_col_items = 0, n_sym_items = 0;
  int8_t* sym = nullptr;              // per subdomain: 1 = tiles hold S = W^T W (SPD, single precision)
  std::vector<int8_t> h_sym;
  // FP16 storage of the explicit inverses (single precision with half-precision
  // tiles): per subdomain 1 = its S tiles hold FP16 values; the row items split
  // into those subdomains' (h) and the rest (f)
  int8_t* s16 = nullptr;
  std::vector<int8_t> h_s16;
  int2 *row_items_h = nullptr, *row_items_f = nullptr;
  int n_row_items_h = 0, n_row_items_f = 0;
  // single precision: the descriptors of row_items, row_items_h, row_items_f, col_items
  TileItem *row_desc = nullptr, *row_desc_h = nullptr, *row_desc_f = nullptr, *col_desc = nullptr;
  void* slots = nullptr;              // explicit-inverse column contributions, TILE per stored tile
                                      // (FP64, or float-float pairs in single precision)
  double* ypos = nullptr;             // per omega position: local solution before the pull
  int64_t n_tiles = 0, n_work = 0, n_xs = 0, n_s = 0, n_pad = 0;
  int32_t* err = nullptr;             // device error word
};

struct Coarse {
  int32_t s_max = 0;                  // block width of the subspace iteration
  std::vector<int32_t> h_count, h_col_off, h_sweeps;
  std::vector<int64_t> h_z_off;
  int32_t* count = nullptr;           // coarse vectors per subdomain (eq. gevpsvd + lifting)
  int32_t* count_g = nullptr;         // of which from eq. gevpsvd (first columns of Z_i)
  int32_t zld = 0;                    // columns of each Z_i block: nev + nev_lift
  std::vector<int32_t> h_count_g, h_lift_count;
  double* lift_values = nullptr;      // N * nev_lift: lambda of eq. uppergevp kept (descending)
  double* lift_resid = nullptr;       // N * nev_lift eigen-residuals
  int32_t* lift_count = nullptr;      // lifting vectors per subdomain
  int32_t* lift_sweeps = nullptr;
  int32_t* col_off = nullptr;         // N+1 first coarse column
  int64_t* z_off = nullptr;           // offset of Z_i (p_i x zld, row-major FP64)
  double* Z = nullptr;
  float* Zf = nullptr;                // single-precision local work: Z rounded to FP32 for the
                                      // restriction and prolongation (Z itself holds the same values)
  double* values = nullptr;           // N * nev
  double* resid = nullptr;            // N * nev eigen-residuals
  int32_t* sweeps = nullptr;          // N
  void* scratch = nullptr;            // per-subdomain iteration blocks
  int64_t* scr_off = nullptr;
  int32_t n_C = 0;
  int64_t nnz_C = 0;
  double* E = nullptr;                // n_C x n_C, factored in place (lower)
  double* E_copy = nullptr;           // as assembled
  double* Einv_diag = nullptr;        // inverses of the diagonal factor blocks
  double* cvec = nullptr;             // coarse work vectors (2 x n_C)
  float2* ycf = nullptr;              // single precision: the coarse solution as float-float pairs
};

struct Krylov {
  double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *w = nullptr;
  double* part = nullptr;   // block partial sums
  double* scal = nullptr;   // device scalars
  int32_t* flag = nullptr;  // [0] done, [1] iterations
  double* V = nullptr;      // FGMRES basis (restart+1) x n
  double* ZB = nullptr;     // FGMRES preconditioned basis restart x n
  double* H = nullptr;      // Hessenberg and rotations
  double* mpart = nullptr;  // multi-dot partial sums
  double* gpart = nullptr;  // PCG: partials of the fused reductions (3 x RBLK)
  unsigned* ticket = nullptr;  // PCG: tickets of the fused reductions (3)
  int32_t restart = 0;      // FGMRES basis capacity (restart length) allocated
  double* bx = nullptr;     // device copies of b, x for host-pointer solves
  double* hpin = nullptr;   // pinned host staging
};

struct Handle {
  int32_t n = 0, nnz = 0, N = 0, delta = 1, nev = 0;
  asm_options opt{};
  bool host_io = false;
  bool fp32 = false;
  bool s16 = false;                 // explicit local inverses stored in FP16 where the bound allows
  bool b16eig = false;              // SPD subspace iteration: operator applications on BF16 operands
  bool lift = false;                // eq. uppergevp vectors added (opt.nu > 0, SPD)
  int32_t nev_lift = 0;             // at most this many per subdomain
  DevMem mem;
  int32_t *row_ptr = nullptr, *col_idx = nullptr, *part = nullptr;
  double* val = nullptr;
  int32_t *dev_n = nullptr, *dev_m = nullptr, *dev_p = nullptr;  // |Omega_i|, |Omega_{1:d-1}|, |I_i|
  double* dscale = nullptr;         // 1/sqrt(|A_vv|): symmetric diagonal scaling of every A_ii
  double *defl_q = nullptr, *defl_w = nullptr;  // deflated apply: Q r and r - A Q r (n each)
  // learned warm start (SPD path): one row per Gamma_delta node, subdomain i
  // owning rows h_wseg[i] .. h_wseg[i+1]-1
  int64_t warm_rows = 0;
  std::vector<int64_t> h_wseg;
  int64_t* wseg = nullptr;
  float* wfeat = nullptr;           // warm_rows x WARM_FEATURES network inputs
  float* wtgt = nullptr;            // warm_rows x nev converged start blocks (record_warm)
  std::vector<int32_t> h_n, h_p, h_m, h_g;
  Overlap ov;
  Dense dn;
  Coarse co;
  ND nd;
  Krylov kr;
  asm_setup_info info{};
  cudaEvent_t ev[16];
  bool events = false;
  int num_sms = 152;                // multiprocessors of the device
  int tile_ctas = 6;                // resident tile-pass blocks per SM (picked by tune_apply)
  cudaStream_t side = nullptr;      // second stream: the coarse part of the apply runs beside the local part
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

// Stage entry points (each enqueues on `s`; host reads are explicit).
void build_overlap(Handle& h, cudaStream_t s);                 // overlap.cu
void build_local(Handle& h, cudaStream_t s);                   // local.cu: gather + sweep + pack
void build_eigen(Handle& h, cudaStream_t s);                   // eigen.cu
void build_coarse(Handle& h, cudaStream_t s);                  // coarse.cu: E assembly + factor
// Optional dot product r.z fused into the last kernel of the apply (PCG):
// fin receives r.z through scal/flag (see krylov.cu).
struct ApplyDot {
  const double* r = nullptr;
  GridSum gs{};
  double* rz = nullptr;    // in: r.z of the previous iteration; out: the new one
  double* beta = nullptr;  // out: new r.z / previous r.z
};
void apply_preconditioner(Handle& h, const double* r, double* z, cudaStream_t s,
                          const int32_t* done = nullptr, const ApplyDot* dot = nullptr);   // apply.cu
void time_apply(Handle& h, const double* r, double* z, int iters, cudaStream_t s, double* ms);
void tune_apply(Handle& h, cudaStream_t s);                                       // apply.cu
void spmv(Handle& h, const double* x, double* y, cudaStream_t s);                 // krylov.cu
// y = A x for a caller's CSR matrix (device arrays), no handle, no allocation (krylov.cu)
void csr_spmv(int n, int64_t nnz, const int32_t* rp, const int32_t* ci, const double* val, const double* x,
              double* y, cudaStream_t s);
// mean time of the PCG loop's fused q = A p, p.q over iters launches (krylov.cu)
void time_pcg_spmv(Handle& h, const double* p, double* q, int iters, cudaStream_t s, double* ms);
// y = b - A x (krylov.cu); nothing when *done is set
void residual(Handle& h, const double* b, const double* x, double* y, cudaStream_t s, const int32_t* done);
void coarse_solve(Handle& h, const double* c, double* y, cudaStream_t s,
                  const int32_t* done = nullptr);                                 // coarse.cu
void solve_pcg(Handle& h, const double* b, double* x, const asm_solve_opts& o, asm_solve_info& info,
               cudaStream_t s);
// PCG on the independent systems of contiguous row segments h_off[0..nseg]
// (host offsets), one recurrence and one stopping test per segment, info[k]
// per segment (krylov_seg.cu)
void solve_pcg_segments(Handle& h, const double* b, double* x, int nseg, const int32_t* h_off,
                        const asm_solve_opts& o, asm_solve_info* info, cudaStream_t s);
void krylov_buffers(Handle& h, cudaStream_t s);  // the Krylov vectors and pinned flags (krylov.cu)
// auto_restart: the caller left the restart length to the library (it may be
// shortened to fit the basis in device memory)
void solve_fgmres(Handle& h, const double* b, double* x, const asm_solve_opts& o,
                  asm_solve_info& info, cudaStream_t s, bool auto_restart);

// coarse_nd.cu: nested-dissection multifrontal factorisation of E
void nd_setup(Handle& h, const std::vector<std::vector<int>>& adj, cudaStream_t s);
void nd_factor(Handle& h, cudaStream_t s);
void nd_solve(Handle& h, const double* c, double* y, cudaStream_t s, const int32_t* done);
void nd_prepare_smem(Handle& h);

// Read back and clear the device error word; throw the matching status.
void check_device_error(Handle& h, cudaStream_t s, const char* stage);

}  // namespace asmgpu
