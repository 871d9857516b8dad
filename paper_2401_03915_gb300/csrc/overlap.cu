// Overlapping subdomains (Section 2.1): the graph of A + A^T, the sets I_i,
// the delta BFS layers, and the maps used by the gathers and the pull-sum.
//
// Ordering of Omega_i: I_i ascending, then layer 1 ascending, ..., layer delta
// ascending (the paper orders layers by distance and leaves the order inside a
// layer open; ascending global index is the reading used throughout).
#include <algorithm>
#include <climits>

#include "handle.cuh"

namespace asmgpu {
namespace {

constexpr int NT = 256;

// ---- CSR checks --------------------------------------------------------------
__global__ void k_validate(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const double* __restrict__ val, const int32_t* __restrict__ part, int n,
                           int nnz, int N, int32_t* err, int32_t* bad_row) {
  COUNT_LAUNCH();
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    int b = rp[r], e = rp[r + 1];
    bool ok = b >= 0 && e >= b && e <= nnz;
    if (ok) {
      for (int k = b; k < e; ++k) {
        int c = ci[k];
        if (c < 0 || c >= n || (k > b && c <= ci[k - 1])) { ok = false; break; }
        if (!isfinite(val[k])) atomicOr(err, DERR_NONFINITE);
      }
    }
    if (part[r] < 0 || part[r] >= N) ok = false;
    if (!ok) { atomicOr(err, DERR_CAPACITY); atomicMin(bad_row, r); }
  }
}

// ---- graph of A + A^T ------------------------------------------------------
__global__ void k_tcount(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int n,
                         int32_t* cnt) {
  COUNT_LAUNCH();
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
    for (int k = rp[r]; k < rp[r + 1]; ++k)
      if (ci[k] != r) atomicAdd(&cnt[ci[k]], 1);
}

__global__ void k_tfill(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int n,
                        const int32_t* __restrict__ tptr, int32_t* cur, int32_t* tidx) {
  COUNT_LAUNCH();
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
    for (int k = rp[r]; k < rp[r + 1]; ++k) {
      int c = ci[k];
      if (c == r) continue;
      int slot = atomicAdd(&cur[c], 1);
      tidx[tptr[c] + slot] = r;
    }
}

// insertion sort of each segment ptr[i]..ptr[i+1] (segments are short)
__global__ void k_sort_rows(const int32_t* __restrict__ ptr, int32_t* idx, int n) {
  COUNT_LAUNCH();
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    int b = ptr[r], e = ptr[r + 1];
    for (int k = b + 1; k < e; ++k) {
      int32_t v = idx[k];
      int t = k - 1;
      while (t >= b && idx[t] > v) { idx[t + 1] = idx[t]; --t; }
      idx[t + 1] = v;
    }
  }
}

// Merge row r of A (without the diagonal) with row r of A^T, dropping duplicates.
// count pass: out_cnt[r] = merged length; fill pass: writes gidx.
template <bool FILL>
__global__ void k_merge(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                        const int32_t* __restrict__ tptr, const int32_t* __restrict__ tidx, int n,
                        const int32_t* __restrict__ gptr, int32_t* out) {
  COUNT_LAUNCH();
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    int a = rp[r], ae = rp[r + 1], b = tptr[r], be = tptr[r + 1];
    int cnt = 0, last = -1;
    int32_t* dst = FILL ? out + gptr[r] : nullptr;
    while (a < ae || b < be) {
      int va = a < ae ? ci[a] : INT_MAX, vb = b < be ? tidx[b] : INT_MAX;
      int v;
      if (va <= vb) { v = va; ++a; if (va == vb) ++b; } else { v = vb; ++b; }
      if (v == r || v == last) continue;
      last = v;
      if (FILL) dst[cnt] = v;
      ++cnt;
    }
    if (!FILL) out[r] = cnt;
  }
}

// ---- I_i lists -----------------------------------------------------------------
__global__ void k_part_count(const int32_t* __restrict__ part, int n, int32_t* cnt) {
  COUNT_LAUNCH();
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    atomicAdd(&cnt[part[v]], 1);
}
__global__ void k_part_fill(const int32_t* __restrict__ part, int n, const int32_t* __restrict__ off,
                            int32_t* cur, int32_t* list) {
  COUNT_LAUNCH();
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    int i = part[v];
    list[off[i] + atomicAdd(&cur[i], 1)] = v;
  }
}

// In-place bitonic sort of sh[0..len) padded to a power of two with INT_MAX.
__device__ void bitonic_sort(int32_t* sh, int len) {
  int sz = 1;
  while (sz < len) sz <<= 1;
  for (int k = len + threadIdx.x; k < sz; k += blockDim.x) sh[k] = INT_MAX;
  __syncthreads();
  for (int k = 2; k <= sz; k <<= 1) {
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
}

// sort each I_i (one block per subdomain, <= MAX_NI entries)
__global__ void k_sort_segments(const int32_t* __restrict__ off, int32_t* list) {
  COUNT_LAUNCH();
  extern __shared__ int32_t sh[];
  int b = off[blockIdx.x], len = off[blockIdx.x + 1] - b;
  for (int k = threadIdx.x; k < len; k += blockDim.x) sh[k] = list[b + k];
  __syncthreads();
  bitonic_sort(sh, len);
  for (int k = threadIdx.x; k < len; k += blockDim.x) list[b + k] = sh[k];
}

// ---- BFS layers --------------------------------------------------------------------
// One block per subdomain.  Layer k = neighbours of layer k-1 that are neither
// in I_i (part check) nor in layers k-1, k-2 (binary search); other layers
// cannot be adjacent to layer k-1.  Candidates are deduplicated in a shared
// hash set and then sorted, so the result does not depend on thread timing.
template <bool WRITE>
__global__ void __launch_bounds__(NT) k_bfs(const int32_t* __restrict__ gptr, const int32_t* __restrict__ gidx,
                      const int32_t* __restrict__ part, const int32_t* __restrict__ ioff,
                      const int32_t* __restrict__ ilist, int delta, int32_t* lay_size,
                      const int32_t* __restrict__ sub_off, const int32_t* __restrict__ lay_off,
                      int32_t* omega, int32_t* err) {
  COUNT_LAUNCH();
  extern __shared__ int32_t sm[];
  int32_t* tab = sm;
  int32_t* buf[3] = {sm + OV_HASH, sm + OV_HASH + OV_LAYER, sm + OV_HASH + 2 * OV_LAYER};
  __shared__ int32_t cnt;
  __shared__ int32_t overflow;
  const int i = blockIdx.x;
  const int32_t* I = ilist + ioff[i];
  const int p = ioff[i + 1] - ioff[i];
  if (WRITE) {
    int32_t* dst = omega + sub_off[i];
    for (int k = threadIdx.x; k < p; k += blockDim.x) dst[k] = I[k];
  }
  const int32_t* prev1 = I;
  int n1 = p;
  bool prev1_I = true;
  const int32_t* prev2 = nullptr;
  int n2 = 0;
  for (int layer = 1; layer <= delta; ++layer) {
    int32_t* cur = buf[(layer - 1) % 3];
    for (int k = threadIdx.x; k < OV_HASH; k += blockDim.x) tab[k] = -1;
    if (threadIdx.x == 0) { cnt = 0; overflow = 0; }
    __syncthreads();
    for (int t = threadIdx.x; t < n1; t += blockDim.x) {
      int v = prev1[t];
      for (int e = gptr[v]; e < gptr[v + 1]; ++e) {
        int w = gidx[e];
        if (part[w] == i) continue;
        if (!prev1_I && bsearch_i32(prev1, 0, n1, w) >= 0) continue;
        if (prev2 && bsearch_i32(prev2, 0, n2, w) >= 0) continue;
        unsigned hsh = ((unsigned)w * 2654435761u) & (OV_HASH - 1);
        bool done = false;
        for (int probe = 0; probe < OV_HASH && !done; ++probe) {
          int old = atomicCAS(&tab[hsh], -1, w);
          if (old == -1 || old == w) done = true;
          else hsh = (hsh + 1) & (OV_HASH - 1);
        }
        if (!done) overflow = 1;
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < OV_HASH; k += blockDim.x) {
      int w = tab[k];
      if (w >= 0) {
        int pos = atomicAdd(&cnt, 1);
        if (pos < OV_LAYER) cur[pos] = w; else overflow = 1;
      }
    }
    __syncthreads();
    int len = min(cnt, OV_LAYER);
    if (threadIdx.x == 0 && (overflow || cnt > OV_LAYER)) atomicOr(err, DERR_CAPACITY);
    bitonic_sort(cur, len);
    if (WRITE) {
      int32_t* dst = omega + sub_off[i] + lay_off[i * (delta + 2) + layer];
      for (int k = threadIdx.x; k < len; k += blockDim.x) dst[k] = cur[k];
    } else if (threadIdx.x == 0) {
      lay_size[i * delta + layer - 1] = len;
    }
    prev2 = prev1_I ? nullptr : prev1;
    n2 = n1;
    prev1 = cur;
    n1 = len;
    prev1_I = false;
    __syncthreads();
  }
}

// s_v = 1 / sqrt(|A_vv|) (1 if the diagonal is absent or zero).
__global__ void k_diag_scale(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const double* __restrict__ val, int n, double* __restrict__ ds) {
  COUNT_LAUNCH();
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    int k = bsearch_i32(ci, rp[r], rp[r + 1], r);
    double d = k >= 0 ? fabs(val[k]) : 0.0;
    ds[r] = d > 0 ? 1.0 / sqrt(d) : 1.0;
  }
}

__global__ void k_pos_sub(const int32_t* __restrict__ sub_off, int32_t* pos_sub) {
  COUNT_LAUNCH();
  int i = blockIdx.x;
  for (int k = sub_off[i] + threadIdx.x; k < sub_off[i + 1]; k += blockDim.x) pos_sub[k] = i;
}

__global__ void k_occ_count(const int32_t* __restrict__ omega, int64_t m, int32_t* cnt) {
  COUNT_LAUNCH();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[omega[k]], 1);
}
__global__ void k_occ_fill(const int32_t* __restrict__ omega, int64_t m, const int32_t* __restrict__ ptr,
                           int32_t* cur, int32_t* pos) {
  COUNT_LAUNCH();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
    int v = omega[k];
    pos[ptr[v] + atomicAdd(&cur[v], 1)] = (int32_t)k;
  }
}

__global__ void k_own_pos(const int32_t* __restrict__ sub_off, const int32_t* __restrict__ lay_off,
                          int delta, const int32_t* __restrict__ omega, int32_t* own) {
  COUNT_LAUNCH();
  int i = blockIdx.x;
  int b = sub_off[i], p = lay_off[i * (delta + 2) + 1];
  for (int a = threadIdx.x; a < p; a += blockDim.x) own[omega[b + a]] = b + a;
}

__global__ void k_rowlen(const int32_t* __restrict__ omega, int64_t m, const int32_t* __restrict__ rp,
                         int64_t* len) {
  COUNT_LAUNCH();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
    int v = omega[k];
    len[k] = rp[v + 1] - rp[v];
  }
}

// local column of every entry of every row of every Omega_i (-1 if outside)
__global__ void k_lcol(const int32_t* __restrict__ omega, int64_t m, const int32_t* __restrict__ pos_sub,
                       const int32_t* __restrict__ sub_off, const int32_t* __restrict__ rp,
                       const int32_t* __restrict__ ci, const int32_t* __restrict__ occ_ptr,
                       const int32_t* __restrict__ occ_pos, const int64_t* __restrict__ ent_off,
                       int32_t* lcol) {
  COUNT_LAUNCH();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
    int v = omega[k], i = pos_sub[k];
    int lo = sub_off[i], hi = sub_off[i + 1];
    int64_t out = ent_off[k];
    for (int e = rp[v]; e < rp[v + 1]; ++e) {
      int c = ci[e], lc = -1;
      for (int t = occ_ptr[c]; t < occ_ptr[c + 1]; ++t) {
        int q = occ_pos[t];
        if (q >= lo && q < hi) { lc = q - lo; break; }
      }
      lcol[out++] = lc;
    }
  }
}

inline unsigned grid_for(int64_t n) { return (unsigned)std::min<int64_t>(std::max<int64_t>(ceil_div(n, NT), 1), 152 * 16); }

}  // namespace

void build_overlap(Handle& h, cudaStream_t s) {
  const int n = h.n, N = h.N, delta = h.delta;
  Overlap& ov = h.ov;
  DevMem& mem = h.mem;
  int32_t* err = h.dn.err;

  // -- validate the CSR and the partition on the device
  {
    int32_t* bad = mem.alloc<int32_t>(1);
    int32_t init = INT_MAX;
    CK(cudaMemcpyAsync(bad, &init, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    k_validate<<<grid_for(n), NT, 0, s>>>(h.row_ptr, h.col_idx, h.val, h.part, n, h.nnz, N, err, bad);
    CK_LAUNCH("validate");
    int32_t e = 0, b = 0;
    CK(cudaMemcpyAsync(&e, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&b, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (e & DERR_CAPACITY)
      fail(ASM_ERR_INVALID_ARG, "malformed CSR or partition at row " + std::to_string(b) +
                                    " (row_ptr, column range/order, or part outside 0..N-1)");
    if (e & DERR_NONFINITE) fail(ASM_ERR_NONFINITE, "A has a NaN or Inf value");
  }

  // -- diagonal scaling used by every local matrix
  h.dscale = mem.alloc<double>(n);
  k_diag_scale<<<grid_for(n), NT, 0, s>>>(h.row_ptr, h.col_idx, h.val, n, h.dscale);

  // -- graph of A + A^T without self loops
  int32_t* tcnt = mem.alloc<int32_t>(n + 1);
  int32_t* tptr = mem.alloc<int32_t>(n + 1);
  CK(cudaMemsetAsync(tcnt, 0, sizeof(int32_t) * (n + 1), s));
  k_tcount<<<grid_for(n), NT, 0, s>>>(h.row_ptr, h.col_idx, n, tcnt);
  int64_t tn = exclusive_scan_i32(tcnt, tptr, n, mem, s);
  int32_t* tidx = mem.alloc<int32_t>(tn);
  CK(cudaMemsetAsync(tcnt, 0, sizeof(int32_t) * (n + 1), s));
  k_tfill<<<grid_for(n), NT, 0, s>>>(h.row_ptr, h.col_idx, n, tptr, tcnt, tidx);
  k_sort_rows<<<grid_for(n), NT, 0, s>>>(tptr, tidx, n);
  k_merge<false><<<grid_for(n), NT, 0, s>>>(h.row_ptr, h.col_idx, tptr, tidx, n, nullptr, tcnt);
  ov.gptr = mem.alloc<int32_t>(n + 1);
  int64_t gn = exclusive_scan_i32(tcnt, ov.gptr, n, mem, s);
  ov.gidx = mem.alloc<int32_t>(gn);
  k_merge<true><<<grid_for(n), NT, 0, s>>>(h.row_ptr, h.col_idx, tptr, tidx, n, ov.gptr, ov.gidx);
  CK_LAUNCH("graph of A + A^T");

  // -- I_i lists
  int32_t* icnt = mem.alloc<int32_t>(N + 1);
  int32_t* ioff = mem.alloc<int32_t>(N + 1);
  int32_t* ilist = mem.alloc<int32_t>(n);
  CK(cudaMemsetAsync(icnt, 0, sizeof(int32_t) * (N + 1), s));
  k_part_count<<<grid_for(n), NT, 0, s>>>(h.part, n, icnt);
  exclusive_scan_i32(icnt, ioff, N, mem, s);
  std::vector<int32_t> h_ioff(N + 1);
  CK(cudaMemcpyAsync(h_ioff.data(), ioff, sizeof(int32_t) * (N + 1), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int i = 0; i < N; ++i) {
    int p = h_ioff[i + 1] - h_ioff[i];
    if (p == 0) fail(ASM_ERR_INVALID_ARG, "subdomain " + std::to_string(i) + " is empty");
    if (p > MAX_NI) fail(ASM_ERR_UNSUPPORTED, "subdomain " + std::to_string(i) + " has more than 16384 nodes");
  }
  CK(cudaMemsetAsync(icnt, 0, sizeof(int32_t) * (N + 1), s));
  k_part_fill<<<grid_for(n), NT, 0, s>>>(h.part, n, ioff, icnt, ilist);
  CK(cudaFuncSetAttribute(k_sort_segments, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_NI * 4));
  k_sort_segments<<<N, 1024, MAX_NI * 4, s>>>(ioff, ilist);
  CK_LAUNCH("I lists");

  // -- BFS layers: sizes, then the sets
  const size_t bfs_smem = sizeof(int32_t) * (OV_HASH + 3 * OV_LAYER);
  CK(cudaFuncSetAttribute(k_bfs<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bfs_smem));
  CK(cudaFuncSetAttribute(k_bfs<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bfs_smem));
  int32_t* lsize = mem.alloc<int32_t>((int64_t)N * delta);
  k_bfs<false><<<N, NT, bfs_smem, s>>>(ov.gptr, ov.gidx, h.part, ioff, ilist, delta, lsize, nullptr,
                                       nullptr, nullptr, err);
  CK_LAUNCH("overlap layers (sizes)");
  std::vector<int32_t> h_lsize((size_t)N * delta);
  int32_t e = 0;
  CK(cudaMemcpyAsync(h_lsize.data(), lsize, sizeof(int32_t) * h_lsize.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&e, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (e & DERR_CAPACITY)
    fail(ASM_ERR_UNSUPPORTED, "an overlap layer has more than 4096 nodes (overlap builder capacity)");

  ov.h_sub_off.assign(N + 1, 0);
  ov.h_lay_off.assign((size_t)N * (delta + 2), 0);
  h.h_n.resize(N); h.h_p.resize(N); h.h_m.resize(N); h.h_g.resize(N);
  int64_t total = 0;
  ov.max_n = 0;
  for (int i = 0; i < N; ++i) {
    int32_t* lo = &ov.h_lay_off[(size_t)i * (delta + 2)];
    lo[0] = 0;
    lo[1] = h_ioff[i + 1] - h_ioff[i];
    for (int k = 1; k <= delta; ++k) lo[k + 1] = lo[k] + h_lsize[(size_t)i * delta + k - 1];
    int ni = lo[delta + 1];
    if (ni > MAX_NI) fail(ASM_ERR_UNSUPPORTED, "overlapping subdomain " + std::to_string(i) + " exceeds 16384 nodes");
    h.h_n[i] = ni; h.h_p[i] = lo[1]; h.h_m[i] = lo[delta]; h.h_g[i] = ni - lo[delta];
    ov.h_sub_off[i] = (int32_t)total;
    total += ni;
    ov.max_n = std::max(ov.max_n, ni);
    if (total > INT32_MAX) fail(ASM_ERR_UNSUPPORTED, "sum of subdomain sizes exceeds 2^31");
  }
  ov.h_sub_off[N] = (int32_t)total;
  ov.sum_n = total;
  ov.sub_off = mem.alloc<int32_t>(N + 1);
  ov.lay_off = mem.alloc<int32_t>((int64_t)N * (delta + 2));
  ov.omega = mem.alloc<int32_t>(total);
  CK(cudaMemcpyAsync(ov.sub_off, ov.h_sub_off.data(), sizeof(int32_t) * (N + 1), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ov.lay_off, ov.h_lay_off.data(), sizeof(int32_t) * ov.h_lay_off.size(),
                     cudaMemcpyHostToDevice, s));
  k_bfs<true><<<N, NT, bfs_smem, s>>>(ov.gptr, ov.gidx, h.part, ioff, ilist, delta, nullptr, ov.sub_off,
                                      ov.lay_off, ov.omega, err);
  CK_LAUNCH("overlap layers (sets)");

  // -- maps
  ov.pos_sub = mem.alloc<int32_t>(total);
  k_pos_sub<<<N, NT, 0, s>>>(ov.sub_off, ov.pos_sub);
  int32_t* ocnt = mem.alloc<int32_t>(n + 1);
  ov.occ_ptr = mem.alloc<int32_t>(n + 1);
  ov.occ_pos = mem.alloc<int32_t>(total);
  CK(cudaMemsetAsync(ocnt, 0, sizeof(int32_t) * (n + 1), s));
  k_occ_count<<<grid_for(total), NT, 0, s>>>(ov.omega, total, ocnt);
  exclusive_scan_i32(ocnt, ov.occ_ptr, n, mem, s);
  CK(cudaMemsetAsync(ocnt, 0, sizeof(int32_t) * (n + 1), s));
  k_occ_fill<<<grid_for(total), NT, 0, s>>>(ov.omega, total, ov.occ_ptr, ocnt, ov.occ_pos);
  k_sort_rows<<<grid_for(n), NT, 0, s>>>(ov.occ_ptr, ov.occ_pos, n);
  ov.own_pos = mem.alloc<int32_t>(n);
  k_own_pos<<<N, NT, 0, s>>>(ov.sub_off, ov.lay_off, delta, ov.omega, ov.own_pos);
  int64_t* rlen = mem.alloc<int64_t>(total + 1);
  ov.ent_off = mem.alloc<int64_t>(total + 1);
  k_rowlen<<<grid_for(total), NT, 0, s>>>(ov.omega, total, h.row_ptr, rlen);
  ov.n_ent = exclusive_scan_i64(rlen, ov.ent_off, total, mem, s);
  ov.lcol = mem.alloc<int32_t>(ov.n_ent);
  k_lcol<<<grid_for(total), NT, 0, s>>>(ov.omega, total, ov.pos_sub, ov.sub_off, h.row_ptr, h.col_idx,
                                        ov.occ_ptr, ov.occ_pos, ov.ent_off, ov.lcol);
  CK_LAUNCH("overlap maps");
}

}  // namespace asmgpu
