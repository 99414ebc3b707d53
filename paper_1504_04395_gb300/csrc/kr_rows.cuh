// Row kernels over n x s blocks: block sparse product (SpMM), row-local linear
// combinations, and the fused reductions (Gram, trace, sum, norm) they feed.
//
// Thread mapping: G threads per row (G a power of two >= s), thread c of a row
// group owning column c; 32/G rows per warp; 256 threads per CTA; a grid-stride
// loop over rows with a grid size fixed by n, so every CTA's partial sums, and
// hence every reduction, are formed in a fixed order (bitwise reproducible).
#pragma once

#include "kr_common.cuh"

namespace kr {

constexpr int kMaxRed = 4;     // fused reductions per launch
constexpr int kMaxOut = 6;     // outputs of one linear-combination launch
constexpr int kMaxTerm = 4;    // terms per output
constexpr int kMaxMat = 6;     // s x s / diagonal coefficient matrices per launch

struct RedSpec {
  int kind;        // RedKind
  int ysrc;        // which computed value is Y (linear combination: output index; SpMM: 0)
  int ureg;        // >= 0: U is computed output ureg of this launch; -1: U is read from memory
  int gacc;        // accumulator index for RED_GRAM
  const void* U;   // memory operand: n x s block (GRAM, TRACE) or n-vector (SUMV, GRAMV)
  int slot;        // first slot of this reduction in a CTA's partial record
  int pad;
};

struct RedSet {
  int nred;
  int nslots;      // slots per CTA record
  void* partials;  // [gridDim.x][nslots] complex (C2<T>)
  RedSpec r[kMaxRed];
};

// One hop of the 4D lattice operator (direction mu, forward or backward) for one thread's
// column: the neighbour's spinor psi (4 spins x 3 colours) is projected onto the two spin
// components h_t = psi[rep_t] + pc_t psi[sig_t] (t = 0, 1), each is multiplied by the
// link (U for a forward hop, U^H for a backward one: g_t = U h_t), and spin a of the output
// receives rc_a * g_{rsrc_a}.  For a projector I + e gamma with gamma a phase permutation
// (gamma[a][sigma a] = phi_a, sigma without fixed points, phi_a phi_{sigma a} = 1) the
// rank-2 structure gives rep_t / sig_t = an orbit {r, sigma r}, pc_t = e phi_r,
// rc_r = 1 and rc_{sigma r} = e phi_{sigma r}.
struct LatHop {
  int rep[2];
  int sig[2];
  int rsrc[4];
  double2 pc[2];
  double2 rc[4];
};

// Division of a 32-bit unsigned index by an invariant divisor d >= 1 with one high multiply
// (Granlund and Montgomery, "Division by invariant integers using multiplication", PLDI 1994,
// Sec. 4): with l = ceil(log2 d) and mag = floor(2^32 (2^l - d) / d) + 1,
// floor(x / d) = (t + ((x - t) >> min(l, 1))) >> max(l - 1, 0), t = floor(x mag / 2^32),
// exact for every 0 <= x < 2^32.  Grid coordinates of the matrix-free operators use it in place
// of a 64-bit division, which costs tens of instructions per row.
struct FastDivU32 {
  uint32_t d, mag;
  int sh1, sh2;
};
inline FastDivU32 make_fastdiv(uint32_t d) {
  int l = 0;
  while (l < 32 && (uint64_t(1) << l) < d) ++l;
  FastDivU32 f;
  f.d = d;
  // (2^l - d) < d <= 2^32, so the 64-bit product cannot overflow
  f.mag = (uint32_t)((((uint64_t(1) << l) - d) << 32) / d + 1);
  f.sh1 = l < 1 ? l : 1;
  f.sh2 = l > 1 ? l - 1 : 0;
  return f;
}
#ifdef __CUDACC__
__device__ __forceinline__ uint32_t fastdiv(uint32_t x, const FastDivU32& f) {
  const uint32_t t = __umulhi(x, f.mag);
  return (t + ((x - t) >> f.sh1)) >> f.sh2;
}
#endif

// ---------------------------------------------------------------------------------------
// SpMM: Y = ay * (A V) + bz * Z  (ay, bz real; optionally ay scaled by a device scalar)
// ---------------------------------------------------------------------------------------
template <typename T>
struct SpmmArgs {
  int64_t n;
  int s;
  int split;                 // 1: real off-diagonal entries + complex diagonal
  const int64_t* rowptr;
  const int32_t* colidx;
  const C2<T>* vals;         // complex entries (split == 0)
  const T* offr;             // real off-diagonal entries (split == 1)
  const C2<T>* diag;         // complex diagonal (split == 1)
  const C2<T>* V;            // input block, row stride s
  C2<T>* Y;                  // output block (may be null: reductions only)
  const C2<T>* Z;            // optional addend block
  double ay, bz;             // real scales
  const double2* ys;         // optional device scalar multiplying ay (complex)
  int ys_conj, ys_neg;
  int64_t nnz;               // stored entries (host-side bookkeeping for the launch profile)
  int64_t maxrow;            // most stored entries in one row (CSR; host-side kernel choice)
  // matrix-free (2d+1)-point stencil with Dirichlet boundaries (nst = d > 0 replaces the CSR):
  // y_j = c V_j + sum_a m_a V_{j - st_a} [x_a > 0] + p_a V_{j + st_a} [x_a < N_a - 1]
  int nst;
  int sreal;                 // all neighbour coefficients real
  int sdiv32;                // n < 2^32: coordinates through sdiv (else 64-bit division)
  int64_t sdims[3];
  int64_t sstr[3];
  FastDivU32 sdiv[3];        // divisors sdims[q]
  double2 sc;                // centre
  double2 sm[3], sp[3];      // minus / plus neighbour along each axis
  // matrix-free 4D lattice operator (lat = 1 replaces the CSR; rows (site * 4 + spin) * 3 + colour):
  // y_x = ldiag psi_x + sum_mu [ (I - e gamma_mu) U_mu(x) psi_{x+mu} + (I + e gamma_mu) U_mu(x-mu)^H psi_{x-mu} ]
  // with the hop coefficient folded into the links and the projector tables in lh
  int lat;
  int64_t ldims[4];          // sites per axis (axis 0 fastest), periodic
  int64_t lstr[4];           // site strides
  int ldiv32;                // sites < 2^32: coordinates through ldiv
  FastDivU32 ldiv[4];        // divisors ldims[q]
  const C2<T>* links;        // [4][sites][3][3] (row-major 3 x 3), scaled by the hop coefficient
  double2 ldiag;
  LatHop lh[8];              // hop 2 mu: forward (+mu), hop 2 mu + 1: backward (-mu)
};

#ifdef __CUDACC__
// Coordinates (axis 0 fastest) of index j < prod(dims[0..nd)) of a grid with nd <= ND axes; the
// last axis takes the quotient left over and needs no division.  use32: j and every extent fit in
// 32 bits, so the divisions go through the precomputed FastDivU32.
template <int ND>
__device__ __forceinline__ void grid_coords(int64_t j, int nd, int use32, const int64_t* dims,
                                            const FastDivU32* div, int64_t (&xc)[ND]) {
  if (use32) {
    uint32_t rem = (uint32_t)j;
#pragma unroll
    for (int q = 0; q < ND; ++q) {
      xc[q] = 0;
      if (q + 1 < nd) {
        const uint32_t qt = fastdiv(rem, div[q]);
        xc[q] = (int64_t)(rem - qt * div[q].d);
        rem = qt;
      } else if (q + 1 == nd) {
        xc[q] = (int64_t)rem;
      }
    }
  } else {
    int64_t rem = j;
#pragma unroll
    for (int q = 0; q < ND; ++q) {
      xc[q] = 0;
      if (q + 1 < nd) {
        xc[q] = rem % dims[q];
        rem /= dims[q];
      } else if (q + 1 == nd) {
        xc[q] = rem;
      }
    }
  }
}
#endif

// ---------------------------------------------------------------------------------------
// Linear combinations: out_o = sum_t  src_t * coef_t
// ---------------------------------------------------------------------------------------
// SRC_SPMM: the value (A V)[j][c] of the launch's sparse product, computed in the same pass
// (the product operand is a separate kernel argument); it needs no memory block of its own.
enum SrcKind : int { SRC_BLOCK = 0, SRC_VEC = 1, SRC_REG = 2, SRC_SPMM = 3 };
enum CoefKind : int { COEF_ONE = 0, COEF_SCALAR = 1, COEF_MAT = 2, COEF_DIAG = 3, COEF_REAL = 4 };

struct Term {
  int src_kind;        // SrcKind
  int src_reg;         // SRC_REG: index of an earlier output
  const void* src;     // SRC_BLOCK / SRC_VEC pointer
  int coef_kind;       // CoefKind
  int coef_idx;        // COEF_MAT / COEF_DIAG: index into the launch's matrix table
  const double2* coef; // COEF_SCALAR: device complex scalar
  double creal;        // COEF_REAL: host real scalar
  int neg, conj;       // flags on the coefficient (negate; conjugate scalar / diagonal)
  int xconj;           // conjugate the source value
};

struct Out {
  int nterm;
  int is_vec;          // output is an n-vector (stored by column-0 threads)
  void* dst;           // null: temporary (kept only for reductions / later terms)
  Term t[kMaxTerm];
};

struct LinArgs {
  int64_t n;
  int s;
  int nout;
  int nmat;
  const double2* mat[kMaxMat];   // device s x s (row-major) or s-vector (diagonal) coefficients
  int mat_is_diag[kMaxMat];
  int mat_neg[kMaxMat];          // stored negated in shared memory
  Out o[kMaxOut];
};

// A reduction whose memory operand U is also written by the same launch is redirected to
// that output's register: it reduces the updated value (outputs are stored at the end of
// each row).  Always returns true.
inline bool resolve_sources(LinArgs& a, RedSet& rs) {
  for (int i = 0; i < rs.nred; ++i) {
    RedSpec& r = rs.r[i];
    if (r.ureg >= 0 || r.U == nullptr) continue;
    const int vec = (r.kind == RED_SUMV || r.kind == RED_GRAMV) ? 1 : 0;
    // a U that this launch writes is reduced with its new value (the output's register)
    int written = -1;
    for (int o = 0; o < a.nout; ++o)
      if (a.o[o].dst == r.U && a.o[o].is_vec == vec) written = o;
    if (written >= 0) r.ureg = written;
  }
  return true;
}

}  // namespace kr
