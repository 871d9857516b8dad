// FP64 factorisation and solve of the coarse matrix E = Z^T A Z.
//
// E inherits the sparsity of the subdomain graph (block (i, j) is zero
// unless A couples I_i and I_j), so it is factored by nested dissection on
// that graph with a multifrontal scheme:
//   host:   BFS level-set bisection of the subdomain graph -> separator tree,
//           symbolic factorisation (front variables V_t, boundary B_t),
//           index maps for the extend-add, per-level task lists;
//   device: fronts of one tree level are assembled from E and the children's
//           update matrices, then eliminated on V_t by a blocked Gauss-Jordan
//           sweep.  On a front [F_VV F_VB; F_BV F_BB] the sweep leaves
//               [ F_VV^{-1}           F_VV^{-1} F_VB ]
//               [ -F_BV F_VV^{-1}     U = F_BB - F_BV F_VV^{-1} F_VB ]
//           and U is the update matrix passed to the parent.
// Solve E y = c, level by level:
//   forward (leaves up):  f = [c_V; 0] + children's u;  u_t = f_B + M_BV f_V
//   backward (root down): y_V = M_VV f_V - M_VB y_B
// Every kernel of the apply is a set of dense matrix-vector products over
// the fronts of one level; the sums run in a fixed order (deterministic).
#include <algorithm>
#include <cmath>
#include <functional>
#include <unordered_map>

#include "handle.cuh"
#include "coarse_nd.cuh"

namespace asmgpu {
namespace {

constexpr int NT = 256;
// Block size of the fronts.  Each elimination step inverts one FB x FB pivot
// block in a single CTA, FB^3 FP64 FMAs at GB300's 2 per cycle per SM, on
// the critical path of its level: 32 costs an eighth of 64 per step.
constexpr int FB = 32;
constexpr int RB = FB / 16;  // rows (and columns) per thread in a 16 x 16 thread grid
// Blocks per FB-row task of the forward/backward solve: one row per warp.
// The solve is bound by GB300's FP64 FMA rate (2 per cycle per SM), so every
// level is spread over as many SMs as it has rows to give.
constexpr int SPLIT = FB / (NT / 32);

// ---------------------------------------------------------------------------
// device kernels
// ---------------------------------------------------------------------------
// F = E restricted to (V u B) x (V u B) with at least one index in V, identity
// on padded pivots, plus the children's update matrices.  One task = one
// FB-row slab of one front.
__global__ void __launch_bounds__(NT) k_front_assemble(const FrontDev* __restrict__ fr, const int2* __restrict__ tasks,
                                                       const double* __restrict__ E, int ldE,
                                                       const int32_t* __restrict__ dofs,
                                                       const int32_t* __restrict__ children,
                                                       const int32_t* __restrict__ invmap, double* __restrict__ M) {
  COUNT_LAUNCH();
  const int2 tk = tasks[blockIdx.x];
  const FrontDev f = fr[tk.x];
  const int r0 = tk.y * FB;
  double* F = M + f.mat_off;
  const int32_t* dof = dofs + f.dof_off;
  for (int idx = threadIdx.x; idx < FB * f.m; idx += NT) {
    const int a = r0 + idx / f.m, b = idx % f.m;
    double v = 0;
    if (a < f.nvp || b < f.nvp) {
      const int da = dof[a], db = dof[b];
      if (da >= 0 && db >= 0) v = E[(int64_t)da * ldE + db];
      else if (a == b && a < f.nvp) v = 1.0;  // padded pivot
    }
    for (int c = 0; c < f.nchild; ++c) {
      const FrontDev ch = fr[children[f.child_off + c]];
      const int32_t* im = invmap + f.inv_off + (int64_t)c * f.m;
      const int ia = im[a], ib = im[b];
      if (ia >= 0 && ib >= 0) v += M[ch.mat_off + (int64_t)(ch.nvp + ia) * ch.m + ch.nvp + ib];
    }
    F[(int64_t)a * f.m + b] = v;
  }
}

// Invert pivot block k of each listed front (Gauss-Jordan in shared memory).
__global__ void __launch_bounds__(NT) k_front_pivot(const FrontDev* __restrict__ fr, const int32_t* __restrict__ list,
                                                    int k, double* __restrict__ M, double* __restrict__ piv,
                                                    int spd, int32_t* err) {
  COUNT_LAUNCH();
  // Gauss-Jordan inversion of the FB x FB pivot block, ping-ponging between
  // two copies so that each elimination step needs one block barrier: step q
  // reads row q, column q and the pivot of the current copy and writes every
  // entry of the other (the same operations, in the same order per entry, as
  // in place).
  __shared__ double P[2][FB][FB + 1];
  __shared__ int bad;
  const int t = list[blockIdx.x];
  const FrontDev f = fr[t];
  const double* F = M + f.mat_off;
  const int k0 = k * FB;
  for (int idx = threadIdx.x; idx < FB * FB; idx += NT) {
    int r = idx / FB, c = idx % FB;
    P[0][r][c] = F[(int64_t)(k0 + r) * f.m + k0 + c];
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  int cur = 0;
  for (int q = 0; q < FB; ++q) {
    const double (*Pc)[FB + 1] = P[cur];
    double (*Pn)[FB + 1] = P[cur ^ 1];
    const double pv = Pc[q][q];
    if (threadIdx.x == 0 && (!isfinite(pv) || (spd ? !(pv > 0) : pv == 0.0))) bad = 1;
    const double inv = 1.0 / pv;
    for (int idx = threadIdx.x; idx < FB * FB; idx += NT) {
      const int r = idx / FB, c = idx % FB;
      double v;
      if (r == q) v = c == q ? inv : Pc[q][c] * inv;
      else if (c == q) v = Pc[r][q] * -inv;
      else v = Pc[r][c] - Pc[r][q] * Pc[q][c] * inv;
      Pn[r][c] = v;
    }
    cur ^= 1;
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) atomicOr(err, DERR_COARSE);
    for (int idx = threadIdx.x; idx < FB * FB; idx += NT) {
      int r = idx / FB, c = idx % FB;
      P[cur][r][c] = r == c ? 1.0 : 0.0;
    }
    __syncthreads();
  }
  double* out = piv + (int64_t)t * FB * FB;
  for (int idx = threadIdx.x; idx < FB * FB; idx += NT) out[idx] = P[cur][idx / FB][idx % FB];
}

// Row panel: M[K][C] <- P M[K][C] for column tiles C != K.
__global__ void __launch_bounds__(NT) k_front_rowpanel(const FrontDev* __restrict__ fr, const int2* __restrict__ tasks,
                                                       int k, double* __restrict__ M, const double* __restrict__ piv) {
  COUNT_LAUNCH();
  __shared__ double P[FB][FB + 1];
  __shared__ double X[FB][FB + 1];
  const int2 tk = tasks[blockIdx.x];
  const FrontDev f = fr[tk.x];
  double* F = M + f.mat_off;
  const int k0 = k * FB, c0 = tk.y * FB;
  const double* pv = piv + (int64_t)tk.x * FB * FB;
  for (int idx = threadIdx.x; idx < FB * FB; idx += NT) {
    int r = idx / FB, c = idx % FB;
    P[r][c] = pv[idx];
    X[r][c] = F[(int64_t)(k0 + r) * f.m + c0 + c];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < FB * FB; idx += NT) {
    int r = idx / FB, c = idx % FB;
    double acc = 0;
    for (int q = 0; q < FB; ++q) acc += P[r][q] * X[q][c];
    F[(int64_t)(k0 + r) * f.m + c0 + c] = acc;
  }
}

// Rank-FB update: M[R][C] -= M[R][K] M[K][C] for R, C != K (row panel already new).
__global__ void __launch_bounds__(NT) k_front_update(const FrontDev* __restrict__ fr, const int4* __restrict__ tasks,
                                                     int k, double* __restrict__ M) {
  COUNT_LAUNCH();
  __shared__ double A[FB][FB + 1];
  __shared__ double B[FB][FB + 1];
  const int4 tk = tasks[blockIdx.x];
  const FrontDev f = fr[tk.x];
  double* F = M + f.mat_off;
  const int k0 = k * FB, r0 = tk.y * FB, c0 = tk.z * FB;
  for (int idx = threadIdx.x; idx < FB * FB; idx += NT) {
    int r = idx / FB, c = idx % FB;
    A[r][c] = F[(int64_t)(r0 + r) * f.m + k0 + c];
    B[r][c] = F[(int64_t)(k0 + r) * f.m + c0 + c];
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[RB][RB] = {};
  for (int q = 0; q < FB; ++q) {
    double av[RB], bv[RB];
#pragma unroll
    for (int a = 0; a < RB; ++a) av[a] = A[ty + 16 * a][q];
#pragma unroll
    for (int b = 0; b < RB; ++b) bv[b] = B[q][tx + 16 * b];
#pragma unroll
    for (int a = 0; a < RB; ++a)
#pragma unroll
      for (int b = 0; b < RB; ++b) acc[a][b] += av[a] * bv[b];
  }
#pragma unroll
  for (int a = 0; a < RB; ++a)
#pragma unroll
    for (int b = 0; b < RB; ++b) F[(int64_t)(r0 + ty + 16 * a) * f.m + c0 + tx + 16 * b] -= acc[a][b];
}

// Column panel: M[R][K] <- -M[R][K] P for R != K; the task with R == K
// writes P into the pivot block.
__global__ void __launch_bounds__(NT) k_front_colpanel(const FrontDev* __restrict__ fr, const int2* __restrict__ tasks,
                                                       int k, double* __restrict__ M, const double* __restrict__ piv) {
  COUNT_LAUNCH();
  __shared__ double P[FB][FB + 1];
  __shared__ double X[FB][FB + 1];
  const int2 tk = tasks[blockIdx.x];
  const FrontDev f = fr[tk.x];
  double* F = M + f.mat_off;
  const int k0 = k * FB, r0 = tk.y * FB;
  const double* pv = piv + (int64_t)tk.x * FB * FB;
  if (tk.y == k) {
    for (int idx = threadIdx.x; idx < FB * FB; idx += NT)
      F[(int64_t)(k0 + idx / FB) * f.m + k0 + idx % FB] = pv[idx];
    return;
  }
  for (int idx = threadIdx.x; idx < FB * FB; idx += NT) {
    int r = idx / FB, c = idx % FB;
    P[r][c] = pv[idx];
    X[r][c] = F[(int64_t)(r0 + r) * f.m + k0 + c];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < FB * FB; idx += NT) {
    int r = idx / FB, c = idx % FB;
    double acc = 0;
    for (int q = 0; q < FB; ++q) acc += X[r][q] * P[q][c];
    F[(int64_t)(r0 + r) * f.m + k0 + c] = -acc;
  }
}

// Entries of the front right-hand side f (first nvp entries: V, then B) into
// shared memory: [0, nvp) and, if nb > 0, [nvp + b0, nvp + b0 + nb).
__device__ void assemble_rhs(const FrontDev& f, const FrontDev* __restrict__ fr, const int32_t* __restrict__ dof,
                             const int32_t* __restrict__ children, const int32_t* __restrict__ invmap,
                             const double* __restrict__ vecs, const double* __restrict__ c, double* sf, int b0,
                             int nb) {
  for (int t = threadIdx.x; t < f.nvp + nb; t += NT) {
    const int a = t < f.nvp ? t : f.nvp + b0 + (t - f.nvp);
    double v = 0;
    if (a < f.nvp) {
      int d = dof[a];
      v = d >= 0 ? c[d] : 0.0;
    }
    for (int q = 0; q < f.nchild; ++q) {
      const FrontDev ch = fr[children[f.child_off + q]];
      int ia = invmap[f.inv_off + (int64_t)q * f.m + a];
      if (ia >= 0) v += vecs[ch.vec_off + ch.nvp + ia];
    }
    sf[a] = v;
  }
  __syncthreads();
}

// Forward: task (front, B row tile) computes u rows; tile -1 stores f_V.
// SPLIT blocks per task, one row per warp; a warp reads its row contiguously.
__global__ void __launch_bounds__(NT) k_front_forward(const FrontDev* __restrict__ fr, const int2* __restrict__ tasks,
                                                      const int32_t* __restrict__ dofs,
                                                      const int32_t* __restrict__ children,
                                                      const int32_t* __restrict__ invmap, const double* __restrict__ M,
                                                      double* __restrict__ vecs, const double* __restrict__ c,
                                                      const int32_t* __restrict__ done) {
  COUNT_LAUNCH();
  if (done != nullptr && *done) return;
  extern __shared__ double sf[];
  const int2 tk = tasks[blockIdx.x / SPLIT];
  const int quarter = blockIdx.x % SPLIT;
  const FrontDev f = fr[tk.x];
  if (tk.y < 0 && quarter != 0) return;
  // f_V and this block's own B rows only
  const int b0 = tk.y * FB + quarter * (FB / SPLIT);
  assemble_rhs(f, fr, dofs + f.dof_off, children, invmap, vecs, c, sf, b0, tk.y < 0 ? 0 : FB / SPLIT);
  double* vec = vecs + f.vec_off;
  if (tk.y < 0) {
    for (int a = threadIdx.x; a < f.nvp; a += NT) vec[a] = sf[a];
    return;
  }
  const double* F = M + f.mat_off;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int rr = wid; rr < FB / SPLIT; rr += NT / 32) {
    const int r = tk.y * FB + quarter * (FB / SPLIT) + rr;
    const double* row = F + (int64_t)(f.nvp + r) * f.m;
    double acc = 0;
    for (int q = lane; q < f.nvp; q += 32) acc += row[q] * sf[q];
    acc = warp_sum(acc);
    if (lane == 0) vec[f.nvp + r] = sf[f.nvp + r] + acc;
  }
}

// Backward: task (front, V row tile): y_V = M_VV f_V - M_VB y_B; SPLIT blocks per task.
__global__ void __launch_bounds__(NT) k_front_backward(const FrontDev* __restrict__ fr, const int2* __restrict__ tasks,
                                                       const int32_t* __restrict__ dofs, const double* __restrict__ M,
                                                       const double* __restrict__ vecs, double* __restrict__ y,
                                                       const int32_t* __restrict__ done) {
  COUNT_LAUNCH();
  if (done != nullptr && *done) return;
  extern __shared__ double sx[];  // [f_V ; -y_B]
  const int2 tk = tasks[blockIdx.x / SPLIT];
  const int quarter = blockIdx.x % SPLIT;
  const FrontDev f = fr[tk.x];
  const int32_t* dof = dofs + f.dof_off;
  const double* vec = vecs + f.vec_off;
  for (int a = threadIdx.x; a < f.m; a += NT) {
    if (a < f.nvp) sx[a] = vec[a];
    else { int d = dof[a]; sx[a] = d >= 0 ? -y[d] : 0.0; }
  }
  __syncthreads();
  const double* F = M + f.mat_off;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int rr = wid; rr < FB / SPLIT; rr += NT / 32) {
    const int r = tk.y * FB + quarter * (FB / SPLIT) + rr;
    const double* row = F + (int64_t)r * f.m;
    double acc = 0;
    for (int q = lane; q < f.m; q += 32) acc += row[q] * sx[q];
    acc = warp_sum(acc);
    const int d = dof[r];
    if (lane == 0 && d >= 0) y[d] = acc;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host: nested dissection, symbolic factorisation, task lists
// ---------------------------------------------------------------------------
namespace {

struct HostFront {
  std::vector<int> vsubs, bsubs, children;
  int parent = -1, level = 0;
  int nv = 0, nb = 0, nvp = 0, nbp = 0, m = 0;
  int first_pos = 0, last_pos = -1;  // subtree range in the elimination order
};

struct NDTree {
  std::vector<HostFront> fronts;  // in postorder
  std::vector<int> pos;           // elimination position of each subdomain
  int cursor = 0;
};

// Connected components of the vertex set V (mask marks membership).
std::vector<std::vector<int>> components(const std::vector<int>& V, const std::vector<std::vector<int>>& adj,
                                         std::vector<int>& mark, int tag) {
  for (int v : V) mark[v] = tag;
  std::vector<std::vector<int>> comps;
  std::vector<int> q;
  for (int v : V) {
    if (mark[v] != tag) continue;
    comps.emplace_back();
    q.assign(1, v);
    mark[v] = tag + 1;
    for (size_t h = 0; h < q.size(); ++h) {
      int u = q[h];
      comps.back().push_back(u);
      for (int w : adj[u])
        if (mark[w] == tag) { mark[w] = tag + 1; q.push_back(w); }
    }
  }
  return comps;
}

// BFS levels inside a connected set (mark == tag), from `start`.
std::vector<std::vector<int>> bfs_levels(int start, const std::vector<std::vector<int>>& adj, std::vector<int>& mark,
                                         int tag, int visited_tag) {
  std::vector<std::vector<int>> lv;
  std::vector<int> cur(1, start);
  mark[start] = visited_tag;
  while (!cur.empty()) {
    std::sort(cur.begin(), cur.end());
    lv.push_back(cur);
    std::vector<int> nxt;
    for (int u : cur)
      for (int w : adj[u])
        if (mark[w] == tag) { mark[w] = visited_tag; nxt.push_back(w); }
    cur.swap(nxt);
  }
  return lv;
}

struct NDBuilder {
  const std::vector<std::vector<int>>& adj;
  std::vector<int> mark;
  int tagc = 1;
  int leaf;
  NDTree& T;
  NDBuilder(const std::vector<std::vector<int>>& a, int lf, NDTree& t) : adj(a), mark(a.size(), 0), leaf(lf), T(t) {}

  int new_tag() { tagc += 4; return tagc; }

  // returns the front ids of the roots of the subtrees covering V
  std::vector<int> build(const std::vector<int>& V) {
    std::vector<int> roots;
    if (V.empty()) return roots;
    int tag = new_tag();
    auto comps = components(V, adj, mark, tag);
    for (auto& comp : comps) roots.push_back(build_connected(comp));
    return roots;
  }

  int make_front(std::vector<int> vs, std::vector<int> children) {
    std::sort(vs.begin(), vs.end());
    HostFront f;
    f.vsubs = vs;
    f.children = children;
    f.first_pos = T.cursor;
    for (int c : children) f.first_pos = std::min(f.first_pos, T.fronts[c].first_pos);
    for (int v : vs) T.pos[v] = T.cursor++;
    f.last_pos = T.cursor - 1;
    int lvl = 0;
    for (int c : children) lvl = std::max(lvl, T.fronts[c].level + 1);
    f.level = lvl;
    T.fronts.push_back(f);
    int id = (int)T.fronts.size() - 1;
    for (int c : children) T.fronts[c].parent = id;
    return id;
  }

  int build_connected(const std::vector<int>& V) {
    if ((int)V.size() <= leaf) return make_front(V, {});
    int tag = new_tag();
    for (int v : V) mark[v] = tag;
    // pseudo-peripheral start: two sweeps
    int start = V[0];
    for (int v : V)
      if (adj[v].size() < adj[start].size()) start = v;
    auto lv = bfs_levels(start, adj, mark, tag, tag + 1);
    int far = lv.back().front();
    for (int v : V) mark[v] = tag;
    lv = bfs_levels(far, adj, mark, tag, tag + 1);
    const int D = (int)lv.size();
    if (D < 3) return make_front(V, {});
    int half = (int)V.size() / 2, acc = 0, mid = 1;
    for (int l = 0; l < D; ++l) {
      acc += (int)lv[l].size();
      if (acc >= half) { mid = l; break; }
    }
    mid = std::max(1, std::min(mid, D - 2));
    std::vector<int> V1, V2;
    for (int l = 0; l < mid; ++l) V1.insert(V1.end(), lv[l].begin(), lv[l].end());
    for (int l = mid + 1; l < D; ++l) V2.insert(V2.end(), lv[l].begin(), lv[l].end());
    std::vector<int> sep = lv[mid];
    std::vector<int> ch = build(V1);
    std::vector<int> ch2 = build(V2);
    ch.insert(ch.end(), ch2.begin(), ch2.end());
    return make_front(sep, ch);
  }
};

}  // namespace

void nd_setup(Handle& h, const std::vector<std::vector<int>>& adj, cudaStream_t s) {
  ND& nd = h.nd;
  const int N = h.N;
  const std::vector<int32_t>& col = h.co.h_col_off;
  NDTree T;
  T.pos.assign(N, -1);
  const int nevmax = std::max(1, h.nev);
  const int leaf = std::max(2, 128 / nevmax);
  NDBuilder B(adj, leaf, T);
  std::vector<int> all(N);
  for (int i = 0; i < N; ++i) all[i] = i;
  B.build(all);
  const int nf = (int)T.fronts.size();
  // symbolic: boundary sets in postorder
  std::vector<int> stamp(N, -1);
  for (int t = 0; t < nf; ++t) {
    HostFront& f = T.fronts[t];
    std::vector<int> cand;
    for (int v : f.vsubs)
      for (int w : adj[v])
        if (T.pos[w] > f.last_pos && stamp[w] != t) { stamp[w] = t; cand.push_back(w); }
    for (int c : f.children)
      for (int w : T.fronts[c].bsubs)
        if (T.pos[w] > f.last_pos && stamp[w] != t) { stamp[w] = t; cand.push_back(w); }
    std::sort(cand.begin(), cand.end(), [&](int a, int b) { return T.pos[a] < T.pos[b]; });
    f.bsubs = cand;
    for (int v : f.vsubs) f.nv += col[v + 1] - col[v];
    for (int v : f.bsubs) f.nb += col[v + 1] - col[v];
    f.nvp = (int)round_up(f.nv, FB);
    f.nbp = (int)round_up(f.nb, FB);
    f.m = f.nvp + f.nbp;
  }
  // device descriptors, dofs, children, inverse maps
  std::vector<FrontDev> fd(nf);
  std::vector<int32_t> dofs, children, invmap;
  int64_t mat = 0, vec = 0;
  int maxlvl = 0, maxm = 0;
  for (int t = 0; t < nf; ++t) {
    HostFront& f = T.fronts[t];
    FrontDev& d = fd[t];
    d.m = f.m; d.nvp = f.nvp; d.nbp = f.nbp;
    d.mat_off = mat; mat += (int64_t)f.m * f.m;
    d.vec_off = vec; vec += f.m;
    d.dof_off = (int32_t)dofs.size();
    std::vector<int32_t> local;
    for (int v : f.vsubs) for (int c = col[v]; c < col[v + 1]; ++c) local.push_back(c);
    local.resize(f.nvp, -1);
    for (int v : f.bsubs) for (int c = col[v]; c < col[v + 1]; ++c) local.push_back(c);
    local.resize(f.m, -1);
    dofs.insert(dofs.end(), local.begin(), local.end());
    d.nchild = (int)f.children.size();
    d.child_off = (int32_t)children.size();
    d.inv_off = (int64_t)invmap.size();
    std::unordered_map<int, int> where;
    for (int a = 0; a < f.m; ++a)
      if (local[a] >= 0) where[local[a]] = a;
    for (int c : f.children) {
      children.push_back(c);
      const HostFront& cf = T.fronts[c];
      std::vector<int32_t> im(f.m, -1);
      int bi = 0;
      for (int v : cf.bsubs)
        for (int q = col[v]; q < col[v + 1]; ++q, ++bi) {
          auto it = where.find(q);
          if (it == where.end()) fail(ASM_ERR_CUDA, "coarse symbolic factorisation: boundary dof missing in parent");
          im[it->second] = bi;
        }
      invmap.insert(invmap.end(), im.begin(), im.end());
    }
    maxlvl = std::max(maxlvl, f.level);
    maxm = std::max(maxm, f.m);
  }
  nd.nfronts = nf;
  nd.nlevels = maxlvl + 1;
  nd.max_m = maxm;
  nd.n_mat = mat;
  // task lists per level
  nd.lv_assemble.assign(nd.nlevels + 1, 0);
  nd.lv_fwd.assign(nd.nlevels + 1, 0);
  nd.lv_bwd.assign(nd.nlevels + 1, 0);
  std::vector<int2> t_asm, t_fwd, t_bwd;
  std::vector<std::vector<int>> bylevel(nd.nlevels);
  for (int t = 0; t < nf; ++t) bylevel[T.fronts[t].level].push_back(t);
  nd.steps.clear();
  std::vector<int32_t> t_piv;
  std::vector<int2> t_row, t_col;
  std::vector<int4> t_upd;
  for (int L = 0; L < nd.nlevels; ++L) {
    nd.lv_assemble[L] = (int)t_asm.size();
    nd.lv_fwd[L] = (int)t_fwd.size();
    nd.lv_bwd[L] = (int)t_bwd.size();
    int maxk = 0;
    for (int t : bylevel[L]) {
      const HostFront& f = T.fronts[t];
      for (int r = 0; r < f.m / FB; ++r) t_asm.push_back(make_int2(t, r));
      t_fwd.push_back(make_int2(t, -1));
      for (int r = 0; r < f.nbp / FB; ++r) t_fwd.push_back(make_int2(t, r));
      for (int r = 0; r < f.nvp / FB; ++r) t_bwd.push_back(make_int2(t, r));
      maxk = std::max(maxk, f.nvp / FB);
    }
    for (int k = 0; k < maxk; ++k) {
      NDStep st;
      st.level = L; st.k = k;
      st.piv0 = (int)t_piv.size(); st.row0 = (int)t_row.size();
      st.upd0 = (int)t_upd.size(); st.col0 = (int)t_col.size();
      for (int t : bylevel[L]) {
        const HostFront& f = T.fronts[t];
        if (k >= f.nvp / FB) continue;
        const int nt = f.m / FB;
        t_piv.push_back(t);
        for (int c = 0; c < nt; ++c) if (c != k) t_row.push_back(make_int2(t, c));
        for (int r = 0; r < nt; ++r)
          for (int c = 0; c < nt; ++c)
            if (r != k && c != k) t_upd.push_back(make_int4(t, r, c, 0));
        for (int r = 0; r < nt; ++r) t_col.push_back(make_int2(t, r));
      }
      st.npiv = (int)t_piv.size() - st.piv0; st.nrow = (int)t_row.size() - st.row0;
      st.nupd = (int)t_upd.size() - st.upd0; st.ncol = (int)t_col.size() - st.col0;
      nd.steps.push_back(st);
    }
  }
  nd.lv_assemble[nd.nlevels] = (int)t_asm.size();
  nd.lv_fwd[nd.nlevels] = (int)t_fwd.size();
  nd.lv_bwd[nd.nlevels] = (int)t_bwd.size();
  // upload
  DevMem& mem = h.mem;
  auto up = [&](auto& vecv, auto*& dst) {
    using V = typename std::remove_reference<decltype(vecv)>::type::value_type;
    dst = mem.alloc<V>(std::max<size_t>(vecv.size(), 1));
    if (!vecv.empty()) CK(cudaMemcpyAsync(dst, vecv.data(), sizeof(V) * vecv.size(), cudaMemcpyHostToDevice, s));
  };
  up(fd, nd.fr);
  up(dofs, nd.dofs);
  up(children, nd.children);
  up(invmap, nd.invmap);
  up(t_asm, nd.t_asm);
  up(t_fwd, nd.t_fwd);
  up(t_bwd, nd.t_bwd);
  up(t_piv, nd.t_piv);
  up(t_row, nd.t_row);
  up(t_upd, nd.t_upd);
  up(t_col, nd.t_col);
  nd.M = mem.alloc<double>(std::max<int64_t>(mat, 1));
  nd.vecs = mem.alloc<double>(std::max<int64_t>(vec, 1));
  nd.piv = mem.alloc<double>((int64_t)std::max(nf, 1) * FB * FB);
  // statistics: stored entries of the factor
  int64_t stored = 0;
  for (const HostFront& f : T.fronts) stored += (int64_t)f.nv * f.nv + 2LL * f.nv * f.nb;
  nd.factor_entries = stored;
}

void nd_factor(Handle& h, cudaStream_t s) {
  ND& nd = h.nd;
  const int ldE = (int)round_up(h.co.n_C, 64);
  size_t si = 0;
  for (int L = 0; L < nd.nlevels; ++L) {
    int na = nd.lv_assemble[L + 1] - nd.lv_assemble[L];
    if (na) k_front_assemble<<<na, NT, 0, s>>>(nd.fr, nd.t_asm + nd.lv_assemble[L], h.co.E, ldE, nd.dofs,
                                               nd.children, nd.invmap, nd.M);
    for (; si < nd.steps.size() && nd.steps[si].level == L; ++si) {
      const NDStep& st = nd.steps[si];
      k_front_pivot<<<st.npiv, NT, 0, s>>>(nd.fr, nd.t_piv + st.piv0, st.k, nd.M, nd.piv, h.opt.spd, h.dn.err);
      if (st.nrow) k_front_rowpanel<<<st.nrow, NT, 0, s>>>(nd.fr, nd.t_row + st.row0, st.k, nd.M, nd.piv);
      if (st.nupd) k_front_update<<<st.nupd, NT, 0, s>>>(nd.fr, nd.t_upd + st.upd0, st.k, nd.M);
      k_front_colpanel<<<st.ncol, NT, 0, s>>>(nd.fr, nd.t_col + st.col0, st.k, nd.M, nd.piv);
    }
  }
  CK_LAUNCH("coarse multifrontal factorisation");
}

void nd_solve(Handle& h, const double* c, double* y, cudaStream_t s, const int32_t* done) {
  ND& nd = h.nd;
  const size_t smem = sizeof(double) * std::max(nd.max_m, 1);
  for (int L = 0; L < nd.nlevels; ++L) {
    int nf = nd.lv_fwd[L + 1] - nd.lv_fwd[L];
    if (nf) k_front_forward<<<SPLIT * nf, NT, smem, s>>>(nd.fr, nd.t_fwd + nd.lv_fwd[L], nd.dofs, nd.children, nd.invmap,
                                                 nd.M, nd.vecs, c, done);
  }
  for (int L = nd.nlevels - 1; L >= 0; --L) {
    int nb = nd.lv_bwd[L + 1] - nd.lv_bwd[L];
    if (nb) k_front_backward<<<SPLIT * nb, NT, smem, s>>>(nd.fr, nd.t_bwd + nd.lv_bwd[L], nd.dofs, nd.M, nd.vecs, y, done);
  }
}

void nd_prepare_smem(Handle& h) {
  const int smem = (int)(sizeof(double) * std::max(h.nd.max_m, 1));
  if (smem > 48 * 1024) {
    CK(cudaFuncSetAttribute(k_front_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    CK(cudaFuncSetAttribute(k_front_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  }
}

}  // namespace asmgpu
