// Nested-dissection multifrontal factorisation of the coarse matrix (types).
#pragma once

#include <vector>

#include "common.cuh"

namespace asmgpu {

struct FrontDev {
  int64_t mat_off;   // m x m front matrix (row-major)
  int64_t vec_off;   // m entries: f_V then u
  int64_t inv_off;   // nchild x m inverse extend-add maps
  int32_t m, nvp, nbp;
  int32_t dof_off;   // m coarse indices (-1: padding)
  int32_t nchild, child_off;
};

struct NDStep {
  int level, k;
  int piv0, npiv, row0, nrow, upd0, nupd, col0, ncol;
};

struct ND {
  int nfronts = 0, nlevels = 0, max_m = 0;
  int64_t n_mat = 0, factor_entries = 0;
  std::vector<int> lv_assemble, lv_fwd, lv_bwd;
  std::vector<NDStep> steps;
  FrontDev* fr = nullptr;
  int32_t *dofs = nullptr, *children = nullptr, *invmap = nullptr, *t_piv = nullptr;
  int2 *t_asm = nullptr, *t_fwd = nullptr, *t_bwd = nullptr, *t_row = nullptr, *t_col = nullptr;
  int4* t_upd = nullptr;
  double *M = nullptr, *vecs = nullptr, *piv = nullptr;
};

}  // namespace asmgpu
