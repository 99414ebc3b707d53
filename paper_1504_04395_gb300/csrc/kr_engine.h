// Solver engine: device state, coefficient arena layout, operator storage.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <vector>

#include "kr_internal.h"

namespace kr {

// ----- device-resident solver state (one per solve) -------------------------------------
struct DevState {
  int status;  // kr_status numbering: 0 converged, 1 breakdown, 2 diverged, 3 nan, 4 maxit
  int done;    // set once the iteration must stop; every later kernel returns immediately
  int iter;    // completed iterations
  int maxit;
  int k;       // Lanczos step counter (QMR)
  int econ;    // economic shadow (norm of W = sqrt(s) * norm of w)
  int s;
  int pad;
  double tol;
  double res0;  // ||R_0||_F
  double rel;   // last relative residual
  double rho_k, xi_k;      // QMR: norms that scaled the current Lanczos blocks
  double rho_n, xi_n;      // QMR: norms of the new unnormalised blocks
  double2 sc_rho;          // BiCG / BiCGStab: carried inner product
  double2 delta, delta_prev;
  double2 t;               // QMR: current entry of the rotated right-hand side
  double2 rot1_c, rot1_s, rot2_c, rot2_s;  // QMR: Givens rotations of the last two steps (c real)
  int have_rot1, have_rot2;
  int pad2[2];
  // stagnation stop (complex64 inner solves of the defect correction; stall == 0: off): stop
  // once the residual is above its starting norm and has not reached a new minimum for
  // max(stall, best_iter) iterations
  double best;
  int best_iter;
  int stall;
};

// ----- coefficient arena slots (each slot holds up to (2*kMaxS)^2 complex entries) -----
enum Slot : int {
  SL_ALPHA = 0, SL_ALPHAH, SL_BETA, SL_BETAH, SL_G, SL_GNEW, SL_M, SL_AC,
  SL_C, SL_CH, SL_S, SL_SH, SL_OMEGA, SL_NOMEGA, SL_GAMMA, SL_RTT,
  SL_B2, SL_B3, SL_OC, SL_ONES,
  SL_QR_R1, SL_QR_R1INV, SL_QR_R2INV, SL_QR_S,
  SL_DELTA, SL_DELTAP, SL_RHOK, SL_XIK, SL_RHON, SL_XIN, SL_T,
  SL_OM1, SL_OM2, SL_OMK, SL_UKK, SL_UKINV, SL_CV, SL_CD1, SL_CD2, SL_TAU,
  SL_INVRHO, SL_INVXI, SL_NTAU,
  SL_TMP0, SL_TMP1, SL_TMP2, SL_TMP3, SL_TMP4, SL_TMP5,
  SL_COUNT
};
constexpr int kSlotElems = 4 * kMaxS * kMaxS;

// ----- coefficient phases -----------------------------------------------------------------
enum Phase : int {
  PH_INIT = 0, PH_MONITOR,
  PH_SC_RHO0, PH_SC_ALPHA, PH_SC_BETA,                 // Gl/eGl-BiCG (scalar)
  PH_LI_RHO0, PH_LI_ALPHA, PH_LI_BETA,                 // Li-BiCG (diagonal)
  PH_LS_ALPHA, PH_LS_OMEGA, PH_LS_BETA,                // Li-BiCGStab (diagonal)
  PH_LQ_INIT, PH_LQ_DELTA, PH_LQ_COEF1, PH_LQ_COEF2, PH_LQ_MON,  // Li-QMR (per column)
  PH_BL_G0, PH_BL_ALPHA, PH_BL_BETA,                   // Bl-BiCG
  PH_QR1, PH_QR2,                                      // CholQR passes
  PH_RQ_INIT, PH_RQ_ALPHA, PH_RQ_C, PH_RQ_BETA,        // Bl-BiCG-rQ
  PH_GS_ALPHA, PH_GS_OMEGA, PH_GS_BETA,                // Gl-BiCGStab
  PH_BS_G0, PH_BS_ALPHA, PH_BS_OMEGA, PH_BS_BETA,      // Bl-BiCGStab
  PH_BSR_INIT, PH_BSR_ALPHA, PH_BSR_OMEGA, PH_BSR_C,   // Bl-BiCGStab-rQ
  PH_QMR_INIT, PH_QMR_DELTA, PH_QMR_COEF1, PH_QMR_COEF2, PH_QMR_MON,   // Gl/eGl-QMR
  PH_BQ_INIT, PH_BQ_COEF1, PH_BQ_COEF2, PH_BQ_MON,     // Bl-QMR
  PH_FILL_ONES,
  PH_SC_ALPHA_CONJ,                                    // Gl-BiCG with alpha from the adjoint product
};

struct CoefArgs {
  int phase;
  int s;
  DevState* st;
  double* hist;
  const double2* red;  // reduced slots
  double2* ar;         // arena: slot i at ar + i * kSlotElems
  int i0, i1, i2, i3;
  double x0;
};

void launch_coef(const CoefArgs& a, cudaStream_t st);

// ----- operator ---------------------------------------------------------------------------
constexpr size_t kCsrPad = 64;

template <typename T>
struct CsrDev {
  int64_t n = 0, nnz = 0;
  int64_t maxrow = 0;     // most stored entries in one row
  int split = 0;
  // the arrays are allocated kCsrPad bytes longer than their contents, so that 16-byte
  // rounded bulk copies of a row range never read past an allocation
  int64_t* rowptr = nullptr;
  int32_t* colidx = nullptr;
  C2<T>* vals = nullptr;  // split == 0
  T* offr = nullptr;      // split == 1
  C2<T>* diag = nullptr;  // split == 1
  void free_all();
};

struct Workspace;

struct StencilSpec {
  int d = 0;                 // 0: not a stencil operator
  int real = 0;              // neighbour coefficients all real
  int64_t dims[3] = {1, 1, 1};
  int64_t str[3] = {0, 0, 0};
  double2 c{}, m[3]{}, p[3]{};
};

// matrix-free 4D lattice operator (kr_op_create_lattice4d)
struct LatticeSpec {
  int on = 0;
  int64_t dims[4] = {1, 1, 1, 1};
  int64_t str[4] = {0, 0, 0, 0};
  double2 diag{}, diagH{};     // A and A^H
  LatHop hops[8], hopsH[8];    // projector tables of A and A^H (gamma -> -gamma)
  double2* links = nullptr;    // device [4][sites][9], scaled by the hop coefficient
  float2* links32 = nullptr;   // complex64 copy (mixed precision), built on first use
  std::vector<double> h_links; // host copy (interleaved re, im), scaled
};

// one triangular factor of the ILU(0) preconditioner on the device (kr_precond.cu)
struct TriDev {
  int64_t n = 0, h_nnz = 0;
  int nlev = 0;
  std::vector<int64_t> h_lev_ptr;  // host: first row of each level in lev_rows
  int64_t* rowptr = nullptr;       // off-diagonal entries (CSR)
  int32_t* colidx = nullptr;
  double2* vals = nullptr;
  double2* invdiag = nullptr;      // inverse diagonal; null: unit diagonal
  int32_t* lev_rows = nullptr;     // rows ordered by level
  void free_all();
};

struct IluDev {
  bool on = false;
  TriDev L, U, UH, LH;  // M = L U; M^{-H} = L^{-H} U^{-H}
  void free_all();
};

struct Operator {
  int device = 0;
  LatticeSpec lat;
  IluDev ilu;  // ILU(0) right preconditioner (kr_op_set_preconditioner)
  int64_t n = 0, nnz = 0;
  int real_offdiag = 0;
  StencilSpec stA, stAH;     // matrix-free operator (and its adjoint) when stA.d > 0
  CsrDev<double> A, AH;
  CsrDev<float> A32, AH32;
  bool have32 = false;
  // host copies kept for value updates / mixed precision set-up
  std::vector<int64_t> h_rowptr;
  std::vector<int32_t> h_colidx;
  std::vector<double> h_vals;  // interleaved re, im
  std::map<long long, std::unique_ptr<Workspace>> ws;
  void* pinned = nullptr;  // small pinned host buffer for state read-back
  int64_t* orig_rowptr = nullptr;  // CSR pattern as given (gradient output order)
  int32_t* orig_colidx = nullptr;
  ~Operator();
};

template <typename T>
const CsrDev<T>& op_mat(const Operator& op, bool adjoint);

// product arguments for op(A) (CSR or stencil), without V / Y / Z / scaling
template <typename T>
SpmmArgs<T> op_spmm_args(const Operator& op, bool adjoint, int s);

void build_operator_device(Operator& op, bool want32);

// ----- workspace --------------------------------------------------------------------------
struct Workspace {
  int64_t n = 0;
  int s = 0;
  size_t elem = 0;  // bytes per complex element
  std::vector<void*> blocks;  // n x s blocks
  std::vector<void*> vecs;    // n-vectors
  void* partials = nullptr;
  size_t partial_bytes = 0;
  double2* red = nullptr;
  double2* arena = nullptr;
  DevState* st = nullptr;
  double* hist = nullptr;
  int hist_cap = 0;
  void* colbuf = nullptr;  // one column of a block (Gram fallback for s > 16)
  void* ptmp[2] = {nullptr, nullptr};  // preconditioner scratch blocks
  cudaStream_t gstream = nullptr;  // private stream for CUDA-graph capture and replay
  cudaEvent_t gevent = nullptr;    // orders the caller's stream and the private stream
  ~Workspace();
};

Workspace& get_workspace(Operator& op, int s, size_t elem, int nblocks, int nvecs, int maxit);

}  // namespace kr
