// Solver driver interface between the C API and the engines.
#pragma once

#include <vector>

#include "kr_engine.h"

namespace kr {

// method numbering of the C interface (kr_method)
enum : int {
  KRM_BL_BICG = 0, KRM_BL_BICG_RQ = 1, KRM_GL_BICG = 2, KRM_EGL_BICG = 3, KRM_BL_BICGSTAB = 4,
  KRM_BL_BICGSTAB_RQ = 5, KRM_GL_BICGSTAB = 6, KRM_BL_QMR = 7, KRM_GL_QMR = 8, KRM_EGL_QMR = 9,
  KRM_LI_BICG = 10, KRM_LI_BICGSTAB = 11, KRM_LI_QMR = 12, KRM_COUNT = 13
};

struct SolveIn {
  double tol = 1e-8;
  int maxit = 500;
  int check_every = 8;
  int shadow_mode = 0;
  const void* shadow = nullptr;
  double time_limit_s = 0.0;
  int stall = 0;  // > 0: stop when above the starting residual with no new minimum for max(stall, best_iter) iterations
  int graphs = 0;  // replay the iterations as a CUDA graph
  int precond = 0;  // solve A M^{-1} Y = B with the operator's ILU(0) (FP64, kr_solve only)
};

struct SolveOut {
  int iters = 0;
  int status = 4;
  int matvecs = 0;
  double res0 = 0.0;
  double relres_recursive = 0.0;
  std::vector<double> hist;
};

template <typename T>
SolveOut run_solve(Operator& op, int method, int s, const void* B, void* X, const SolveIn& in, cudaStream_t st,
                   bool adjoint);

double true_residual(Operator& op, int s, const void* B, const void* X, void* Rbuf, cudaStream_t st, bool adjoint);

// workspace key (element size field) of the orthonormalised right-hand sides: a workspace of its
// own, so that the solve that follows cannot overwrite Q, Y or S
constexpr size_t kOrthoKey = 32;
double orthonormal_rhs(Operator& op, int s, const void* B, const void* X, void** Q, void** Y, cudaStream_t st,
                       bool adjoint);
void add_back_rhs_factor(Operator& op, int s, void* X, cudaStream_t st);
void ensure_orig_pattern(Operator& op);
void rebuild_operator_values(Operator& op);
void standalone_qr(Operator& op, Workspace& ws, int64_t n, int s, void* Q, cudaStream_t st);

}  // namespace kr
