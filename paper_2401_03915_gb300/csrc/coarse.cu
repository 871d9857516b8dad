// Coarse operator E = Z^T A Z (A_00 = R_0 A R_0^T, Section 4.1): assembly and
// the subdomain graph of E for the nested-dissection factorisation.
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
constexpr int EB = 64;  // padding of the dense coarse matrix

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
    int nev, double* __restrict__ AZ, const int64_t* __restrict__ az_off, unsigned long long* nnz,
    int2* __restrict__ pairs, unsigned int* __restrict__ npairs) {
  COUNT_LAUNCH();
  extern __shared__ int32_t keys[];
  __shared__ int any_nz;
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
    if (threadIdx.x == 0) any_nz = 0;
    __syncthreads();
    for (int idx = threadIdx.x; idx < ki * kj; idx += NT) {
      int r = idx / kj, c = idx % kj;
      double acc = 0;
      for (int q = seg_start; q < seg_end; ++q) {
        int a = keys[q] & 16383;
        int ipos = own_pos[omega[b0 + a]] - ib0;
        acc += Zi[(int64_t)ipos * nev + r] * V[(int64_t)a * kj + c];
      }
      E[(int64_t)(col_off[owner] + r) * ldE + col_off[j] + c] = acc;
      if (acc != 0.0) any_nz = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0 && ki > 0 && any_nz) {
      atomicAdd(nnz, (unsigned long long)ki * kj);
      pairs[atomicAdd(npairs, 1u)] = make_int2(owner, j);
    }
    seg_start = seg_end;
    __syncthreads();
  }
}


}  // namespace

void build_coarse(Handle& h, cudaStream_t s) {
  Coarse& co = h.co;
  const int N = h.N, nev = co.zld;  // the row stride of the Z_i blocks
  DevMem& mem = h.mem;
  co.h_count.assign(N, 0);
  co.h_count_g.assign(N, 0);
  co.h_lift_count.assign(N, 0);
  co.h_sweeps.assign(N, 0);
  if (co.count) {
    CK(cudaMemcpyAsync(co.h_count.data(), co.count, 4 * N, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(co.h_count_g.data(), co.count_g, 4 * N, cudaMemcpyDeviceToHost, s));
    if (co.lift_count) CK(cudaMemcpyAsync(co.h_lift_count.data(), co.lift_count, 4 * N, cudaMemcpyDeviceToHost, s));
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
  co.E = mem.alloc<double>((int64_t)ldE * ldE);
  co.E_copy = mem.alloc<double>((int64_t)ldE * ldE);
  co.cvec = mem.alloc<double>(3LL * ldE);
  if (co.Zf) co.ycf = mem.alloc<float2>(co.n_C);
  CK(cudaMemsetAsync(co.E, 0, sizeof(double) * ldE * ldE, s));
  std::vector<int64_t> az(N);
  int64_t t = 0;
  for (int i = 0; i < N; ++i) { az[i] = t; t += (int64_t)h.h_n[i] * std::max(co.h_count[i], 1); }
  double* AZ = mem.alloc<double>(t);
  int64_t* az_off = mem.alloc<int64_t>(N);
  CK(cudaMemcpyAsync(az_off, az.data(), 8 * N, cudaMemcpyHostToDevice, s));
  unsigned long long* nnz = mem.alloc<unsigned long long>(1);
  CK(cudaMemsetAsync(nnz, 0, 8, s));
  // nonzero blocks (owner, j): at most one per (j, owner of a node of Omega_j)
  int2* pairs = mem.alloc<int2>(h.ov.sum_n);
  unsigned int* npairs = mem.alloc<unsigned int>(1);
  CK(cudaMemsetAsync(npairs, 0, sizeof(unsigned int), s));
  const size_t ksm = sizeof(int32_t) * MAX_NI;
  CK(cudaFuncSetAttribute(k_assemble_E, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ksm));
  k_assemble_E<<<N, NT, ksm, s>>>(ldE, co.E, co.Z, co.z_off, co.count, co.col_off, h.ov.sub_off, h.ov.omega,
                                  h.part, h.ov.own_pos, h.row_ptr, h.val, h.ov.ent_off, h.ov.lcol, h.dev_p,
                                  h.dev_n, nev, AZ, az_off, nnz, pairs, npairs);
  CK_LAUNCH("assemble E");
  CK(cudaMemcpyAsync(co.E_copy, co.E, sizeof(double) * ldE * ldE, cudaMemcpyDeviceToDevice, s));
  unsigned long long hn = 0;
  unsigned int hp = 0;
  CK(cudaMemcpyAsync(&hn, nnz, 8, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&hp, npairs, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<int2> hpairs(hp);
  if (hp) CK(cudaMemcpy(hpairs.data(), pairs, sizeof(int2) * hp, cudaMemcpyDeviceToHost));
  co.nnz_C = (int64_t)hn;
  if (h.events) CK(cudaEventRecord(h.ev[7], s));
  // subdomain graph of E (symmetrised, subdomains without coarse vectors kept)
  std::vector<std::vector<int>> adj(N);
  for (const int2& pr : hpairs)
    if (pr.x != pr.y) { adj[pr.x].push_back(pr.y); adj[pr.y].push_back(pr.x); }
  for (auto& a : adj) { std::sort(a.begin(), a.end()); a.erase(std::unique(a.begin(), a.end()), a.end()); }
  nd_setup(h, adj, s);
  nd_prepare_smem(h);
  nd_factor(h, s);
  check_device_error(h, s, "coarse factorisation");
}

void coarse_solve(Handle& h, const double* c, double* y, cudaStream_t s, const int32_t* done) {
  nd_solve(h, c, y, s, done);
}

}  // namespace asmgpu
