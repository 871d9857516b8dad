// Coarse operator E = Z^T A Z (A_00 = R_0 A R_0^T, Section 4.1) and its FP64
// factorisation / solve.
//
// Z is block diagonal in the nonoverlapping partition: the block of
// subdomain j is supported on Omega_{I_j} (the D_j in eq. coarse_space_2
// zeroes every other row).  Hence A Z_j is supported on Omega_j (every
// neighbour of I_j lies in the first layer) and equals A_jj[:, :p_j] Z_j there,
// and E_ij = sum over the nodes of Omega_j owned by subdomain i of
// Z_i[node] (A Z_j)[node].  One block per column block j computes
// E_{.,j}: each entry is written by one thread, summed in a fixed order.
#include <algorithm>
#include <climits>

#include "handle.cuh"

namespace asmgpu {
namespace {

constexpr int NT = 256;
constexpr int EB = 64;  // block size of the dense coarse factorisation

__device__ void bitonic_sort_keys(int32_t* sh, int len) {
  int sz = 1;
  while (sz < len) sz <<= 1;
  for (int k = len + threadIdx.x; k < sz; k += blockDim.x) sh[k] = INT_MAX;
  __syncthreads();
  for (int k = 2; k <= sz; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < sz; t += blockDim.x) {
        int o = t ^ j;
        if (o > t) {
          int32_t x = sh[t], y = sh[o];
          bool up = (t & k) == 0;
          if ((x > y) == up) { sh[t] = y; sh[o] = x; }
        }
      }
      __syncthreads();
    }
}

__global__ void __launch_bounds__(NT) k_assemble_E(
    int ldE, double* __restrict__ E, const double* __restrict__ Z, const int64_t* __restrict__ z_off,
    const int32_t* __restrict__ count, const int32_t* __restrict__ col_off, const int32_t* __restrict__ sub_off,
    const int32_t* __restrict__ omega, const int32_t* __restrict__ part, const int32_t* __restrict__ own_pos,
    const int32_t* __restrict__ rp, const double* __restrict__ val, const int64_t* __restrict__ ent_off,
    const int32_t* __restrict__ lcol, const int32_t* __restrict__ p_arr, const int32_t* __restrict__ n_arr,
    int nev, double* __restrict__ AZ, const int64_t* __restrict__ az_off, unsigned long long* nnz) {
  extern __shared__ int32_t keys[];
  const int j = blockIdx.x;
  const int kj = count[j];
  if (kj == 0) return;
  const int nj = n_arr[j], pj = p_arr[j], b0 = sub_off[j];
  const double* Zj = Z + z_off[j];
  double* V = AZ + az_off[j];
  // (A Z_j) restricted to Omega_j
  for (int idx = threadIdx.x; idx < nj * kj; idx += NT) {
    int a = idx / kj, c = idx % kj;
    int v = omega[b0 + a];
    int64_t e0 = ent_off[b0 + a];
    double acc = 0;
    for (int t = 0; t < rp[v + 1] - rp[v]; ++t) {
      int lc = lcol[e0 + t];
      if (lc >= 0 && lc < pj) acc += val[rp[v] + t] * Zj[(int64_t)lc * nev + c];
    }
    V[(int64_t)a * kj + c] = acc;
  }
  // group the rows of Omega_j by owning subdomain (stable: key = owner * 2^14 + a)
  for (int a = threadIdx.x; a < nj; a += NT) keys[a] = part[omega[b0 + a]] * 16384 + a;
  __syncthreads();
  bitonic_sort_keys(keys, nj);
  int seg_start = 0;
  while (seg_start < nj) {
    const int owner = keys[seg_start] >> 14;
    int seg_end = seg_start;
    while (seg_end < nj && (keys[seg_end] >> 14) == owner) ++seg_end;
    const int ki = count[owner];
    const double* Zi = Z + z_off[owner];
    const int ib0 = sub_off[owner];
    for (int idx = threadIdx.x; idx < ki * kj; idx += NT) {
      int r = idx / kj, c = idx % kj;
      double acc = 0;
      for (int q = seg_start; q < seg_end; ++q) {
        int a = keys[q] & 16383;
        int ipos = own_pos[omega[b0 + a]] - ib0;
        acc += Zi[(int64_t)ipos * nev + r] * V[(int64_t)a * kj + c];
      }
      E[(int64_t)(col_off[owner] + r) * ldE + col_off[j] + c] = acc;
    }
    if (threadIdx.x == 0 && ki > 0) atomicAdd(nnz, (unsigned long long)ki * kj);
    seg_start = seg_end;
    __syncthreads();
  }
}

__global__ void k_pad_identity(double* E, int ldE, int nC) {
  for (int r = nC + blockIdx.x * blockDim.x + threadIdx.x; r < ldE; r += gridDim.x * blockDim.x)
    E[(int64_t)r * ldE + r] = 1.0;
}

// Factor the diagonal block kb of E (all earlier updates applied) and store
// its inverse factor L_kk^{-1} (lower) for the panel solve and for the apply.
__global__ void __launch_bounds__(NT) k_potrf_diag(double* E, int ldE, int kb, double* Linv, int32_t* err) {
  __shared__ double A[EB][EB + 1];
  __shared__ double B[EB][EB + 1];
  __shared__ int bad;
  const int k0 = kb * EB;
  for (int idx = threadIdx.x; idx < EB * EB; idx += NT) {
    int r = idx / EB, c = idx % EB;
    A[r][c] = E[(int64_t)(k0 + r) * ldE + k0 + c];
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < EB; ++j) {
    if (threadIdx.x == 0) {
      double d = A[j][j];
      if (!(d > 0) || !isfinite(d)) { bad = 1; d = 1.0; }
      A[j][j] = sqrt(d);
    }
    __syncthreads();
    double dj = A[j][j];
    for (int r = j + 1 + threadIdx.x; r < EB; r += NT) A[r][j] /= dj;
    __syncthreads();
    for (int idx = threadIdx.x; idx < EB * EB; idx += NT) {
      int r = idx / EB, c = idx % EB;
      if (c > j && r >= c) A[r][c] -= A[r][j] * A[c][j];
    }
    __syncthreads();
  }
  // inverse of the lower factor, one column per thread
  for (int c = threadIdx.x; c < EB; c += NT) {
    for (int r = 0; r < EB; ++r) B[r][c] = 0;
    for (int r = c; r < EB; ++r) {
      double v = r == c ? 1.0 : 0.0;
      for (int t = c; t < r; ++t) v -= A[r][t] * B[t][c];
      B[r][c] = v / A[r][r];
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < EB * EB; idx += NT) {
    int r = idx / EB, c = idx % EB;
    E[(int64_t)(k0 + r) * ldE + k0 + c] = c <= r ? A[r][c] : 0.0;
    Linv[(int64_t)kb * EB * EB + idx] = B[r][c];
  }
  if (threadIdx.x == 0 && bad) atomicOr(err, DERR_COARSE);
}

// L_ik = E_ik L_kk^{-T} for block rows i > kb.
__global__ void __launch_bounds__(NT) k_trsm_panel(double* E, int ldE, int kb, int nb, const double* Linv) {
  __shared__ double Li[EB][EB + 1];
  __shared__ double X[EB][EB + 1];
  const int i = kb + 1 + blockIdx.x;
  if (i >= nb) return;
  const int k0 = kb * EB, i0 = i * EB;
  for (int idx = threadIdx.x; idx < EB * EB; idx += NT) {
    int r = idx / EB, c = idx % EB;
    Li[r][c] = Linv[(int64_t)kb * EB * EB + idx];
    X[r][c] = E[(int64_t)(i0 + r) * ldE + k0 + c];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < EB * EB; idx += NT) {
    int r = idx / EB, c = idx % EB;
    double acc = 0;
    for (int t = 0; t <= c; ++t) acc += X[r][t] * Li[c][t];
    E[(int64_t)(i0 + r) * ldE + k0 + c] = acc;
  }
}

// E_ij -= L_ik L_jk^T for kb < j <= i.
__global__ void __launch_bounds__(NT) k_syrk_update(double* E, int ldE, int kb, int nb) {
  __shared__ double Ai[EB][EB + 1];
  __shared__ double Aj[EB][EB + 1];
  const int m = nb - kb - 1;
  int t = blockIdx.x;
  // map t -> (ii, jj) with 0 <= jj <= ii < m
  int ii = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
  while (ii * (ii + 1) / 2 > t) --ii;
  int jj = t - ii * (ii + 1) / 2;
  if (ii >= m) return;
  const int i0 = (kb + 1 + ii) * EB, j0 = (kb + 1 + jj) * EB, k0 = kb * EB;
  for (int idx = threadIdx.x; idx < EB * EB; idx += NT) {
    int r = idx / EB, c = idx % EB;
    Ai[r][c] = E[(int64_t)(i0 + r) * ldE + k0 + c];
    Aj[r][c] = E[(int64_t)(j0 + r) * ldE + k0 + c];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < EB * EB; idx += NT) {
    int r = idx / EB, c = idx % EB;
    double acc = 0;
    for (int q = 0; q < EB; ++q) acc += Ai[r][q] * Aj[c][q];
    E[(int64_t)(i0 + r) * ldE + j0 + c] -= acc;
  }
}

// y = E^{-1} c with the blocked factor (one block: forward, then backward).
__global__ void __launch_bounds__(NT) k_dense_solve(const double* __restrict__ L, int ldE, int nb,
                                                    const double* __restrict__ Linv, const double* __restrict__ c,
                                                    int nC, double* __restrict__ y, double* __restrict__ tmp,
                                                    const int32_t* __restrict__ done) {
  if (done != nullptr && *done) return;
  __shared__ double rhs[EB];
  __shared__ double red[NT / 32];
  // forward: tmp = L^{-1} c
  for (int k = 0; k < nb; ++k) {
    const int k0 = k * EB;
    for (int r = 0; r < EB; ++r) {
      double part = 0;
      for (int q = threadIdx.x; q < k0; q += NT) part += L[(int64_t)(k0 + r) * ldE + q] * tmp[q];
      part = block_sum(part, red);
      if (threadIdx.x == 0) rhs[r] = (k0 + r < nC ? c[k0 + r] : 0.0) - part;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < EB; r += NT) {
      double acc = 0;
      for (int q = 0; q <= r; ++q) acc += Linv[(int64_t)k * EB * EB + r * EB + q] * rhs[q];
      tmp[k0 + r] = acc;
    }
    __syncthreads();
  }
  // backward: y = L^{-T} tmp
  for (int k = nb - 1; k >= 0; --k) {
    const int k0 = k * EB;
    const int rest = nb * EB - (k0 + EB);
    for (int r = 0; r < EB; ++r) {
      double part = 0;
      for (int q = threadIdx.x; q < rest; q += NT) part += L[(int64_t)(k0 + EB + q) * ldE + k0 + r] * y[k0 + EB + q];
      part = block_sum(part, red);
      if (threadIdx.x == 0) rhs[r] = tmp[k0 + r] - part;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < EB; r += NT) {
      double acc = 0;
      for (int q = r; q < EB; ++q) acc += Linv[(int64_t)k * EB * EB + q * EB + r] * rhs[q];
      y[k0 + r] = acc;
    }
    __syncthreads();
  }
}

}  // namespace

void build_coarse(Handle& h, cudaStream_t s) {
  Coarse& co = h.co;
  const int N = h.N, nev = h.nev;
  DevMem& mem = h.mem;
  co.h_count.assign(N, 0);
  co.h_sweeps.assign(N, 0);
  if (h.nev > 0 && h.opt.coarse) {
    CK(cudaMemcpyAsync(co.h_count.data(), co.count, 4 * N, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(co.h_sweeps.data(), co.sweeps, 4 * N, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  co.h_col_off.assign(N + 1, 0);
  for (int i = 0; i < N; ++i) co.h_col_off[i + 1] = co.h_col_off[i] + co.h_count[i];
  co.n_C = co.h_col_off[N];
  if (co.n_C == 0) return;
  co.col_off = mem.alloc<int32_t>(N + 1);
  CK(cudaMemcpyAsync(co.col_off, co.h_col_off.data(), 4 * (N + 1), cudaMemcpyHostToDevice, s));
  const int ldE = (int)round_up(co.n_C, EB);
  const int nb = ldE / EB;
  co.E = mem.alloc<double>((int64_t)ldE * ldE);
  co.E_copy = mem.alloc<double>((int64_t)ldE * ldE);
  co.Einv_diag = mem.alloc<double>((int64_t)nb * EB * EB);
  co.cvec = mem.alloc<double>(3LL * ldE);
  CK(cudaMemsetAsync(co.E, 0, sizeof(double) * ldE * ldE, s));
  std::vector<int64_t> az(N);
  int64_t t = 0;
  for (int i = 0; i < N; ++i) { az[i] = t; t += (int64_t)h.h_n[i] * std::max(co.h_count[i], 1); }
  double* AZ = mem.alloc<double>(t);
  int64_t* az_off = mem.alloc<int64_t>(N);
  CK(cudaMemcpyAsync(az_off, az.data(), 8 * N, cudaMemcpyHostToDevice, s));
  unsigned long long* nnz = mem.alloc<unsigned long long>(1);
  CK(cudaMemsetAsync(nnz, 0, 8, s));
  const size_t ksm = sizeof(int32_t) * MAX_NI;
  CK(cudaFuncSetAttribute(k_assemble_E, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ksm));
  k_assemble_E<<<N, NT, ksm, s>>>(ldE, co.E, co.Z, co.z_off, co.count, co.col_off, h.ov.sub_off, h.ov.omega,
                                  h.part, h.ov.own_pos, h.row_ptr, h.val, h.ov.ent_off, h.ov.lcol, h.dev_p,
                                  h.dev_n, nev, AZ, az_off, nnz);
  k_pad_identity<<<4, NT, 0, s>>>(co.E, ldE, co.n_C);
  CK_LAUNCH("assemble E");
  CK(cudaMemcpyAsync(co.E_copy, co.E, sizeof(double) * ldE * ldE, cudaMemcpyDeviceToDevice, s));
  unsigned long long hn = 0;
  CK(cudaMemcpyAsync(&hn, nnz, 8, cudaMemcpyDeviceToHost, s));
  if (h.events) CK(cudaEventRecord(h.ev[7], s));
  // dense right-looking blocked Cholesky
  for (int kb = 0; kb < nb; ++kb) {
    k_potrf_diag<<<1, NT, 0, s>>>(co.E, ldE, kb, co.Einv_diag, h.dn.err);
    if (kb + 1 < nb) {
      k_trsm_panel<<<nb - kb - 1, NT, 0, s>>>(co.E, ldE, kb, nb, co.Einv_diag);
      int m = nb - kb - 1;
      k_syrk_update<<<m * (m + 1) / 2, NT, 0, s>>>(co.E, ldE, kb, nb);
    }
  }
  CK_LAUNCH("factor E");
  CK(cudaStreamSynchronize(s));
  co.nnz_C = (int64_t)hn;
  check_device_error(h, s, "coarse factorisation");
}

void coarse_solve(Handle& h, const double* c, double* y, cudaStream_t s, const int32_t* done) {
  Coarse& co = h.co;
  const int ldE = (int)round_up(co.n_C, EB);
  k_dense_solve<<<1, NT, 0, s>>>(co.E, ldE, ldE / EB, co.Einv_diag, c, co.n_C, y, co.cvec + 2 * ldE, done);
}

}  // namespace asmgpu
