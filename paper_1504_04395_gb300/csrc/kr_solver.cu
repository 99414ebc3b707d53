// Host-side solver engines: launch sequences of each simultaneous method.
//
// Each method is the same sequence of steps as its definition in the paper
// (Algorithms 1-5, Secs. 2 and 4) with these GB300 mappings:
//  * every block product A V / A^H W is one SpMM launch reading A once for all
//    s columns, with the Gram / trace / sum reduction of its output fused in;
//  * the row-local block updates of one step are one launch, with the Grams of
//    the updated blocks (e.g. Rh_{k+1}^H R_{k+1} and ||R_{k+1}||_F) fused in;
//  * the small FP64 coefficient algebra runs in one-CTA kernels, so all
//    coefficients stay on the device; the host only reads the convergence state
//    back every `check_every` iterations.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <limits>

#include "kr_engine.h"
#include "kr_precond.h"
#include "kr_profile.h"
#include "kr_solver.h"

namespace kr {

// =========================================================================================
// operator storage
// =========================================================================================
template <typename T>
void CsrDev<T>::free_all() {
  cudaFree(rowptr); cudaFree(colidx); cudaFree(vals); cudaFree(offr); cudaFree(diag);
  rowptr = nullptr; colidx = nullptr; vals = nullptr; offr = nullptr; diag = nullptr;
}
template struct CsrDev<double>;
template struct CsrDev<float>;

Operator::~Operator() {
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  ws.clear();
  A.free_all(); AH.free_all(); A32.free_all(); AH32.free_all();
  cudaFree(orig_rowptr); cudaFree(orig_colidx);
  cudaFree(lat.links); cudaFree(lat.links32);
  ilu.free_all();
  if (pinned) cudaFreeHost(pinned);
  cudaSetDevice(prev);
}

Workspace::~Workspace() {
  for (void* p : blocks) cudaFree(p);
  for (void* p : vecs) cudaFree(p);
  cudaFree(partials); cudaFree(red); cudaFree(arena); cudaFree(st); cudaFree(hist); cudaFree(colbuf);
  cudaFree(ptmp[0]); cudaFree(ptmp[1]);
  if (gevent) cudaEventDestroy(gevent);
  if (gstream) cudaStreamDestroy(gstream);
}

template <>
const CsrDev<double>& op_mat<double>(const Operator& op, bool adjoint) { return adjoint ? op.AH : op.A; }
template <>
const CsrDev<float>& op_mat<float>(const Operator& op, bool adjoint) { return adjoint ? op.AH32 : op.A32; }

template <typename T>
SpmmArgs<T> op_spmm_args(const Operator& op, bool adjoint, int s) {
  SpmmArgs<T> a{};
  a.n = op.n;
  a.s = s;
  a.ay = 1.0;
  if (op.lat.on) {
    const LatticeSpec& L = op.lat;
    a.lat = 1;
    int64_t sites = 1;
    for (int q = 0; q < 4; ++q) {
      a.ldims[q] = L.dims[q];
      a.lstr[q] = L.str[q];
      sites *= L.dims[q];
    }
    a.ldiv32 = sites <= (int64_t)UINT32_MAX;
    for (int q = 0; q < 4; ++q) a.ldiv[q] = make_fastdiv(a.ldiv32 ? (uint32_t)L.dims[q] : 1u);
    if constexpr (sizeof(T) == 8) a.links = reinterpret_cast<const C2<T>*>(L.links);
    else a.links = reinterpret_cast<const C2<T>*>(L.links32);
    a.ldiag = adjoint ? L.diagH : L.diag;
    for (int h = 0; h < 8; ++h) a.lh[h] = adjoint ? L.hopsH[h] : L.hops[h];
    a.nnz = op.nnz;
    return a;
  }
  if (op.stA.d > 0) {
    const StencilSpec& st = adjoint ? op.stAH : op.stA;
    a.nst = st.d;
    a.sreal = st.real;
    for (int q = 0; q < 3; ++q) {
      a.sdims[q] = st.dims[q];
      a.sstr[q] = st.str[q];
      a.sm[q] = st.m[q];
      a.sp[q] = st.p[q];
    }
    a.sdiv32 = op.n <= (int64_t)UINT32_MAX;
    for (int q = 0; q < 3; ++q) a.sdiv[q] = make_fastdiv(a.sdiv32 ? (uint32_t)st.dims[q] : 1u);
    a.sc = st.c;
    a.split = 1;  // profile accounting: real neighbours
    a.nnz = op.nnz - op.n;
    return a;
  }
  const CsrDev<T>& M = op_mat<T>(op, adjoint);
  a.split = M.split;
  a.rowptr = M.rowptr;
  a.colidx = M.colidx;
  a.vals = M.vals;
  a.offr = M.offr;
  a.diag = M.diag;
  a.nnz = M.nnz;
  a.maxrow = M.maxrow;
  return a;
}
template SpmmArgs<double> op_spmm_args<double>(const Operator&, bool, int);
template SpmmArgs<float> op_spmm_args<float>(const Operator&, bool, int);

namespace {

struct HostCsr {
  std::vector<int64_t> rowptr;
  std::vector<int32_t> colidx;
  std::vector<double> vals;  // interleaved
};

HostCsr transpose_conj(int64_t n, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                       const std::vector<double>& v) {
  const int64_t nnz = rp[n];
  HostCsr t;
  t.rowptr.assign(n + 1, 0);
  for (int64_t k = 0; k < nnz; ++k) t.rowptr[ci[k] + 1]++;
  for (int64_t i = 0; i < n; ++i) t.rowptr[i + 1] += t.rowptr[i];
  t.colidx.resize(nnz);
  t.vals.resize(2 * nnz);
  std::vector<int64_t> fill(t.rowptr.begin(), t.rowptr.end() - 1);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {  // rows visited in order: columns of A^H ascending
      const int64_t d = fill[ci[k]]++;
      t.colidx[d] = (int32_t)i;
      t.vals[2 * d] = v[2 * k];
      t.vals[2 * d + 1] = -v[2 * k + 1];
    }
  return t;
}

bool offdiag_real(int64_t n, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                  const std::vector<double>& v) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] != i && v[2 * k + 1] != 0.0) return false;
  return true;
}

// A stored value in the element type.  For complex64 copies the conversion follows IEEE round to
// nearest, with the overflow case written out: magnitudes from 2^128 - 2^103 (half an ulp above
// the largest float) up become infinities, those between the largest float and that bound round
// to it, NaN stays NaN.  An operator beyond the complex64 range then gives non-finite inner
// solves, which the defect correction detects (it finishes in FP64).
template <typename T>
static inline T narrow(double x) {
  if constexpr (sizeof(T) == 8) {
    return x;
  } else {
    constexpr float inf = std::numeric_limits<float>::infinity();
    constexpr float fmax = std::numeric_limits<float>::max();
    const double ax = std::fabs(x);
    if (std::isnan(x)) return std::numeric_limits<float>::quiet_NaN();
    if (ax >= 0x1.ffffffp+127) return x < 0 ? -inf : inf;
    if (ax > (double)fmax) return x < 0 ? -fmax : fmax;
    return (float)x;
  }
}

template <typename T>
void upload(CsrDev<T>& d, int64_t n, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
            const std::vector<double>& v, bool split) {
  d.free_all();
  d.n = n;
  d.nnz = rp[n];
  d.split = split ? 1 : 0;
  if (!split) {
    std::vector<C2<T>> hv(d.nnz);
    for (int64_t k = 0; k < d.nnz; ++k) hv[k] = mk<T>(narrow<T>(v[2 * k]), narrow<T>(v[2 * k + 1]));
    KR_CUDA(cudaMalloc(&d.rowptr, sizeof(int64_t) * (n + 1) + kCsrPad));
    KR_CUDA(cudaMalloc(&d.colidx, sizeof(int32_t) * std::max<int64_t>(d.nnz, 1) + kCsrPad));
    KR_CUDA(cudaMalloc(&d.vals, sizeof(C2<T>) * std::max<int64_t>(d.nnz, 1) + kCsrPad));
    for (int64_t i = 0; i < n; ++i) d.maxrow = std::max<int64_t>(d.maxrow, rp[i + 1] - rp[i]);
    KR_CUDA(cudaMemcpy(d.rowptr, rp.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice));
    KR_CUDA(cudaMemcpy(d.colidx, ci.data(), sizeof(int32_t) * d.nnz, cudaMemcpyHostToDevice));
    KR_CUDA(cudaMemcpy(d.vals, hv.data(), sizeof(C2<T>) * d.nnz, cudaMemcpyHostToDevice));
    return;
  }
  // real off-diagonal part (CSR without the diagonal) + complex diagonal
  std::vector<int64_t> orp(n + 1, 0);
  std::vector<int32_t> oci;
  std::vector<T> ov;
  std::vector<C2<T>> dg(n, mk<T>(T(0), T(0)));
  oci.reserve(d.nnz);
  ov.reserve(d.nnz);
  for (int64_t i = 0; i < n; ++i) {
    double dr = 0.0, di = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      if (ci[k] == i) { dr += v[2 * k]; di += v[2 * k + 1]; }
      else { oci.push_back(ci[k]); ov.push_back(narrow<T>(v[2 * k])); }
    }
    dg[i] = mk<T>(narrow<T>(dr), narrow<T>(di));
    orp[i + 1] = (int64_t)oci.size();
  }
  d.nnz = orp[n];
  for (int64_t i = 0; i < n; ++i) d.maxrow = std::max<int64_t>(d.maxrow, orp[i + 1] - orp[i]);
  KR_CUDA(cudaMalloc(&d.rowptr, sizeof(int64_t) * (n + 1) + kCsrPad));
  KR_CUDA(cudaMalloc(&d.colidx, sizeof(int32_t) * std::max<int64_t>(d.nnz, 1) + kCsrPad));
  KR_CUDA(cudaMalloc(&d.offr, sizeof(T) * std::max<int64_t>(d.nnz, 1) + kCsrPad));
  KR_CUDA(cudaMalloc(&d.diag, sizeof(C2<T>) * n + kCsrPad));
  KR_CUDA(cudaMemcpy(d.rowptr, orp.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice));
  if (d.nnz) {
    KR_CUDA(cudaMemcpy(d.colidx, oci.data(), sizeof(int32_t) * d.nnz, cudaMemcpyHostToDevice));
    KR_CUDA(cudaMemcpy(d.offr, ov.data(), sizeof(T) * d.nnz, cudaMemcpyHostToDevice));
  }
  KR_CUDA(cudaMemcpy(d.diag, dg.data(), sizeof(C2<T>) * n, cudaMemcpyHostToDevice));
}

}  // namespace

void rebuild_operator_values(Operator& op) {
  op.ilu.free_all();  // factors of the old values
  const bool had32 = op.have32;
  op.A.free_all();
  op.AH.free_all();
  op.A32.free_all();
  op.AH32.free_all();
  op.have32 = false;
  build_operator_device(op, had32);
}

void build_operator_device(Operator& op, bool want32) {
  if (op.lat.on) {  // matrix-free lattice: the links (and their complex64 copy)
    LatticeSpec& L = op.lat;
    const size_t cnt = L.h_links.size() / 2;
    if (!L.links) {
      KR_CUDA(cudaMalloc(&L.links, sizeof(double2) * cnt));
      KR_CUDA(cudaMemcpy(L.links, L.h_links.data(), sizeof(double2) * cnt, cudaMemcpyHostToDevice));
    }
    if (want32 && !L.links32) {
      std::vector<float2> h32(cnt);
      for (size_t i = 0; i < cnt; ++i) h32[i] = make_float2(narrow<float>(L.h_links[2 * i]), narrow<float>(L.h_links[2 * i + 1]));
      KR_CUDA(cudaMalloc(&L.links32, sizeof(float2) * cnt));
      KR_CUDA(cudaMemcpy(L.links32, h32.data(), sizeof(float2) * cnt, cudaMemcpyHostToDevice));
    }
    return;
  }
  if (op.stA.d > 0) return;  // matrix-free: nothing to upload
  if (op.A.rowptr && (!want32 || op.have32)) return;  // already resident
  const bool split = offdiag_real(op.n, op.h_rowptr, op.h_colidx, op.h_vals);
  op.real_offdiag = split ? 1 : 0;
  HostCsr t = transpose_conj(op.n, op.h_rowptr, op.h_colidx, op.h_vals);
  if (!op.A.rowptr) {
    upload<double>(op.A, op.n, op.h_rowptr, op.h_colidx, op.h_vals, split);
    upload<double>(op.AH, op.n, t.rowptr, t.colidx, t.vals, split);
  }
  if (want32 && !op.have32) {
    upload<float>(op.A32, op.n, op.h_rowptr, op.h_colidx, op.h_vals, split);
    upload<float>(op.AH32, op.n, t.rowptr, t.colidx, t.vals, split);
    op.have32 = true;
  }
}

void ensure_orig_pattern(Operator& op) {
  if (op.orig_rowptr) return;
  KR_CUDA(cudaMalloc(&op.orig_rowptr, sizeof(int64_t) * (op.n + 1)));
  KR_CUDA(cudaMalloc(&op.orig_colidx, sizeof(int32_t) * std::max<int64_t>(op.nnz, 1)));
  KR_CUDA(cudaMemcpy(op.orig_rowptr, op.h_rowptr.data(), sizeof(int64_t) * (op.n + 1), cudaMemcpyHostToDevice));
  if (op.nnz)
    KR_CUDA(cudaMemcpy(op.orig_colidx, op.h_colidx.data(), sizeof(int32_t) * op.nnz, cudaMemcpyHostToDevice));
}

// =========================================================================================
// workspace
// =========================================================================================
constexpr int kMaxSlots = 2 * kMaxS * kMaxS + 4 * kMaxS + 8;
constexpr int kRedCap = 1 << 16;

Workspace& get_workspace(Operator& op, int s, size_t elem, int nblocks, int nvecs, int maxit) {
  // elem is the key of the workspace: 8 (complex64) and 16 (complex128) are the solvers' own;
  // larger values name further complex128 workspaces (defect correction, preconditioning,
  // orthonormalised right-hand sides), whose blocks hold complex128 entries
  const long long key = (long long)s * 64 + (long long)elem;
  if (elem > sizeof(double2)) elem = sizeof(double2);
  auto it = op.ws.find(key);
  if (it == op.ws.end()) {
    auto w = std::make_unique<Workspace>();
    w->n = op.n;
    w->s = s;
    w->elem = elem;
    w->partial_bytes = (size_t)max_row_grid() * kMaxSlots * 16;
    KR_CUDA(cudaMalloc(&w->partials, w->partial_bytes));
    KR_CUDA(cudaMalloc(&w->red, sizeof(double2) * kRedCap));
    KR_CUDA(cudaMalloc(&w->arena, sizeof(double2) * (size_t)kSlotElems * SL_COUNT));
    KR_CUDA(cudaMemset(w->arena, 0, sizeof(double2) * (size_t)kSlotElems * SL_COUNT));
    KR_CUDA(cudaMalloc(&w->st, sizeof(DevState)));
    it = op.ws.emplace(key, std::move(w)).first;
  }
  Workspace& w = *it->second;
  while ((int)w.blocks.size() < nblocks) {
    void* p = nullptr;
    KR_CUDA(cudaMalloc(&p, std::max<size_t>((size_t)op.n * s * elem, 16)));
    w.blocks.push_back(p);
  }
  while ((int)w.vecs.size() < nvecs) {
    void* p = nullptr;
    KR_CUDA(cudaMalloc(&p, std::max<size_t>((size_t)op.n * elem, 16)));
    w.vecs.push_back(p);
  }
  if (w.hist_cap < maxit + 1) {
    cudaFree(w.hist);
    w.hist = nullptr;
    KR_CUDA(cudaMalloc(&w.hist, sizeof(double) * (maxit + 1)));
    w.hist_cap = maxit + 1;
  }
  return w;
}

// =========================================================================================
// launch helpers
// =========================================================================================
namespace {

struct Cf {
  int kind = COEF_ONE;
  const double2* p = nullptr;
  double r = 0.0;
  int neg = 0, conj = 0, xconj = 0;
};
inline Cf one() { return Cf{}; }
inline Cf minus() { Cf c; c.neg = 1; return c; }
inline Cf conjx() { Cf c; c.xconj = 1; return c; }
inline Cf sc(const double2* p, bool conj = false, bool neg = false) {
  Cf c; c.kind = COEF_SCALAR; c.p = p; c.conj = conj; c.neg = neg; return c;
}
inline Cf mat(const double2* p, bool neg = false) { Cf c; c.kind = COEF_MAT; c.p = p; c.neg = neg; return c; }
inline Cf dg(const double2* p, bool conj = false, bool neg = false) {
  Cf c; c.kind = COEF_DIAG; c.p = p; c.conj = conj; c.neg = neg; return c;
}
inline Cf real(double r) { Cf c; c.kind = COEF_REAL; c.r = r; return c; }

struct Reds {
  RedSet rs{};
  int ngram = 0;
  int add(int kind, int ysrc, int ureg, const void* U, int s) {
    RedSpec& r = rs.r[rs.nred++];
    r.kind = kind;
    r.ysrc = ysrc;
    r.ureg = ureg;
    r.U = U;
    r.slot = rs.nslots;
    r.gacc = 0;
    if (kind == RED_GRAM) { r.gacc = ngram++; rs.nslots += s * s; }
    else if (kind == RED_GRAMV || kind == RED_CDOT) rs.nslots += s;
    else rs.nslots += 1;
    return r.slot;
  }
};

struct Lin {
  LinArgs a{};
  Lin(int64_t n, int s) { a.n = n; a.s = s; }
  int out(void* dst, bool vec = false) {
    const int o = a.nout++;
    a.o[o].dst = dst;
    a.o[o].is_vec = vec ? 1 : 0;
    a.o[o].nterm = 0;
    return o;
  }
  int matidx(const double2* p, bool is_diag, bool neg) {
    for (int i = 0; i < a.nmat; ++i)
      if (a.mat[i] == p && a.mat_neg[i] == (neg ? 1 : 0)) return i;
    a.mat[a.nmat] = p;
    a.mat_is_diag[a.nmat] = is_diag ? 1 : 0;
    a.mat_neg[a.nmat] = neg ? 1 : 0;
    return a.nmat++;
  }
  void term(int o, int src_kind, const void* src, int reg, const Cf& c) {
    Term& t = a.o[o].t[a.o[o].nterm++];
    t.src_kind = src_kind;
    t.src = src;
    t.src_reg = reg;
    t.coef_kind = c.kind;
    t.coef = c.p;
    t.creal = c.r;
    t.neg = c.neg;
    t.conj = c.conj;
    t.xconj = c.xconj;
    // matrix negation is folded into the shared-memory copy; diagonal negation stays a flag
    const bool mneg = c.kind == COEF_MAT && c.neg;
    if (mneg) t.neg = 0;
    t.coef_idx = (c.kind == COEF_MAT || c.kind == COEF_DIAG) ? matidx(c.p, c.kind == COEF_DIAG, mneg) : 0;
  }
  void blk(int o, const void* src, const Cf& c = Cf{}) { term(o, SRC_BLOCK, src, 0, c); }
  void product(int o, const Cf& c = Cf{}) { term(o, SRC_SPMM, nullptr, 0, c); }  // (op(A) V)[j], see lin_product
  void vec(int o, const void* src, const Cf& c = Cf{}) { term(o, SRC_VEC, src, 0, c); }
  void reg(int o, int r, const Cf& c = Cf{}) { term(o, SRC_REG, nullptr, r, c); }
};

}  // namespace

template <typename T>
struct Engine {
  Operator& op;
  bool swap;  // adjoint solve: A and A^H exchange roles
  int s;
  int64_t n;
  cudaStream_t st;
  Workspace& ws;
  int red_top = 0;  // next free offset in ws.red for this iteration's reductions

  bool prec = false;  // right preconditioning: the products are A M^{-1} and M^{-H} A^H

  Engine(Operator& o, bool sw, int s_, cudaStream_t stream, Workspace& w)
      : op(o), swap(sw), s(s_), n(o.n), st(stream), ws(w) {}

  double2* ptmp(int i) {  // n x s scratch blocks of the preconditioner
    if (!ws.ptmp[i]) KR_CUDA(cudaMalloc(&ws.ptmp[i], std::max<size_t>((size_t)n * s * sizeof(double2), 16)));
    return reinterpret_cast<double2*>(ws.ptmp[i]);
  }

  // Y = ay op(A) V + bz Z with fused reductions (op(A) preconditioned when prec); returns red offset
  int spmm(bool adjA, int sdim, const void* V, void* Y, Reds r = Reds{}, const void* Z = nullptr, double ay = 1.0,
           double bz = 0.0, const double2* ys = nullptr, bool ysconj = false, bool ysneg = false) {
    if constexpr (sizeof(T) == 8) {
      if (prec) {
        if (!adjA) {  // A (M^{-1} V): the input preconditioned, the product as usual
          apply_ilu0(op, false, sdim, reinterpret_cast<const double2*>(V), ptmp(0), ptmp(1), st);
          return spmm_op(false, sdim, ptmp(0), Y, r, Z, ay, bz, ys, ysconj, ysneg);
        }
        // M^{-H} (A^H V): the product, the adjoint solve, then scaling, addend and reductions
        spmm_op(true, sdim, V, ptmp(0));
        if (r.rs.nred == 0 && Z == nullptr && ys == nullptr && ay == 1.0) {
          apply_ilu0(op, true, sdim, ptmp(0), reinterpret_cast<double2*>(Y), ptmp(1), st);
          return -1;
        }
        apply_ilu0(op, true, sdim, ptmp(0), ptmp(0), ptmp(1), st);
        if (ys != nullptr && ay != 1.0) throw CudaError{cudaErrorInvalidValue, "preconditioned product: ay with ys"};
        Lin L(n, sdim);
        const int o = L.out(Y);
        L.blk(o, ptmp(0), ys != nullptr ? sc(ys, ysconj, ysneg) : (ay == 1.0 ? one() : real(ay)));
        if (Z != nullptr) L.blk(o, Z, real(bz));
        return lin(L, r);
      }
    }
    return spmm_op(adjA, sdim, V, Y, r, Z, ay, bz, ys, ysconj, ysneg);
  }

  const int* done() const { return &ws.st->done; }
  C2<T>* blk(int i) const { return reinterpret_cast<C2<T>*>(ws.blocks[i]); }
  C2<T>* vecp(int i) const { return reinterpret_cast<C2<T>*>(ws.vecs[i]); }
  double2* slot(int i) const { return ws.arena + (size_t)i * kSlotElems; }

  // Y = ay op(A) V + bz Z, op(A) = A or A^H, with fused reductions; returns red offset
  int spmm_op(bool adjA, int sdim, const void* V, void* Y, Reds r = Reds{}, const void* Z = nullptr, double ay = 1.0,
              double bz = 0.0, const double2* ys = nullptr, bool ysconj = false, bool ysneg = false) {
    SpmmArgs<T> a = op_spmm_args<T>(op, adjA != swap, sdim);
    a.n = n;
    a.V = reinterpret_cast<const C2<T>*>(V);
    a.Y = reinterpret_cast<C2<T>*>(Y);
    a.Z = reinterpret_cast<const C2<T>*>(Z);
    a.ay = ay;
    a.bz = bz;
    a.ys = ys;
    a.ys_conj = ysconj;
    a.ys_neg = ysneg;
    r.rs.partials = ws.partials;
    const int grid0 = row_grid(n, sdim);
    if (count_grams(r.rs) <= ng_capacity(threads_per_row(sdim))) {
      const int grid = launch_spmm<T>(a, r.rs, grid0, done(), st);
      return reduce(r, grid);
    }
    // register budget exceeded: product stored with the other reductions fused, Grams from memory
    if (!Y) throw CudaError{cudaErrorInvalidValue, "Gram of an unstored block product"};
    if (red_top + 2 * r.rs.nslots > kRedCap) red_top = 0;
    const int off = red_top;
    red_top += r.rs.nslots;
    Reds nong;
    int map[kMaxRed];
    for (int i = 0; i < r.rs.nred; ++i) {
      const RedSpec& q = r.rs.r[i];
      map[i] = q.kind == RED_GRAM ? -1 : nong.add(q.kind, q.ysrc, q.ureg, q.U, sdim);
    }
    nong.rs.partials = ws.partials;
    const int grid = launch_spmm<T>(a, nong.rs, grid0, done(), st);
    const int tmp = nong.rs.nred ? reduce(nong, grid) : -1;
    for (int i = 0; i < r.rs.nred; ++i) {
      const RedSpec& q = r.rs.r[i];
      if (q.kind != RED_GRAM) {
        const int cnt = (q.kind == RED_GRAMV || q.kind == RED_CDOT) ? sdim : 1;
        KR_CUDA(cudaMemcpyAsync(ws.red + off + q.slot, ws.red + tmp + map[i], sizeof(double2) * cnt,
                                cudaMemcpyDeviceToDevice, st));
      } else {
        gram_from_memory(q.U, Y, sdim, ws.red + off + q.slot);
      }
    }
    return off;
  }

  // memory holding output o of L (its destination, or the block it merely copies)
  static const void* mem_of(const LinArgs& a, int o) {
    const Out& q = a.o[o];
    if (q.dst) return q.dst;
    if (q.nterm == 1 && q.t[0].src_kind == SRC_BLOCK && q.t[0].coef_kind == COEF_ONE && !q.t[0].neg &&
        !q.t[0].xconj)
      return q.t[0].src;
    return nullptr;
  }

  // row-local linear combination with fused reductions; returns red offset
  int lin(Lin& L, Reds r = Reds{}) {
    r.rs.partials = ws.partials;
    const int grid0 = row_grid(n, L.a.s);
    const int G = threads_per_row(L.a.s);
    if (count_grams(r.rs) <= ng_capacity(G)) {
      const int grid = launch_lincomb<T>(L.a, r.rs, grid0, done(), st);
      return reduce(r, grid);
    }
    // register budget exceeded: non-Gram reductions fused, each Gram from memory afterwards
    if (red_top + 2 * r.rs.nslots > kRedCap) red_top = 0;
    const int off = red_top;
    red_top += r.rs.nslots;
    Reds nong;
    int map[kMaxRed];
    for (int i = 0; i < r.rs.nred; ++i) {
      const RedSpec& q = r.rs.r[i];
      map[i] = q.kind == RED_GRAM ? -1 : nong.add(q.kind, q.ysrc, q.ureg, q.U, L.a.s);
    }
    nong.rs.partials = ws.partials;
    const int grid = launch_lincomb<T>(L.a, nong.rs, grid0, done(), st);
    const int tmp = nong.rs.nred ? reduce(nong, grid) : -1;
    for (int i = 0; i < r.rs.nred; ++i) {
      const RedSpec& q = r.rs.r[i];
      if (q.kind != RED_GRAM) {
        const int cnt = (q.kind == RED_GRAMV || q.kind == RED_CDOT) ? L.a.s : 1;
        KR_CUDA(cudaMemcpyAsync(ws.red + off + q.slot, ws.red + tmp + map[i], sizeof(double2) * cnt,
                                cudaMemcpyDeviceToDevice, st));
        continue;
      }
      const void* Ymem = mem_of(L.a, q.ysrc);
      const void* Umem = q.ureg >= 0 ? mem_of(L.a, q.ureg) : q.U;
      if (!Ymem || !Umem) throw CudaError{cudaErrorInvalidValue, "Gram of an unstored combination"};
      // two-pass Gram: G = U^H Y accumulated by a dedicated launch with one Gram
      gram_from_memory(Umem, Ymem, L.a.s, ws.red + off + q.slot);
    }
    return off;
  }

  // Row-local combination L whose SRC_SPMM terms are the product op(A) V (op(A) = A or A^H).  The
  // product is formed in the same pass (never stored) when the operator allows it -- CSR or
  // stencil storage, no preconditioner, at most one fused Gram -- and fused products are on;
  // otherwise it is stored in `scratch` first and the terms read it.  Both give the same values:
  // every product kernel forms each entry with the same operations in the same order.
  int lin_product(Lin& L, bool adjA, const void* V, void* scratch, Reds r = Reds{}) {
    const bool fuse = fused_products_enabled() && !prec && !op.lat.on && count_grams(r.rs) <= 1 &&
                      ng_capacity(threads_per_row(s)) >= count_grams(r.rs);
    if (fuse) {
      SpmmArgs<T> sp = op_spmm_args<T>(op, adjA != swap, s);
      sp.n = n;
      sp.V = reinterpret_cast<const C2<T>*>(V);
      r.rs.partials = ws.partials;
      const int grid = launch_lincomb_spmm<T>(L.a, r.rs, sp, row_grid(n, s), done(), st);
      return reduce(r, grid);
    }
    spmm(adjA, s, V, scratch);
    for (int o = 0; o < L.a.nout; ++o)
      for (int t = 0; t < L.a.o[o].nterm; ++t)
        if (L.a.o[o].t[t].src_kind == SRC_SPMM) {
          L.a.o[o].t[t].src_kind = SRC_BLOCK;
          L.a.o[o].t[t].src = scratch;
        }
    return lin(L, r);
  }

  // U^H Y (n x sdim blocks in memory) -> dst (sdim^2 entries), any sdim <= 32
  void gram_from_memory(const void* U, const void* Y, int sdim, double2* dst) {
    const int grid0 = row_grid(n, sdim);
    if (ng_capacity(threads_per_row(sdim)) >= 1) {
      Lin g(n, sdim);
      const int go = g.out(nullptr);
      g.blk(go, Y);
      Reds gr;
      gr.add(RED_GRAM, go, -1, U, sdim);
      gr.rs.partials = ws.partials;
      const int grid = launch_lincomb<T>(g.a, gr.rs, grid0, done(), st);
      launch_reduce<T>(ws.partials, grid, gr.rs.nslots, dst, done(), st);
      return;
    }
    // s > 16: column-dot reductions of Y against each column of U broadcast as a vector
    for (int a = 0; a < sdim; ++a) {
      Lin g(n, sdim);
      const int go = g.out(nullptr);
      g.blk(go, Y);
      Reds gr;
      gr.add(RED_GRAMV, go, -1, nullptr, sdim);
      gr.rs.r[0].U = nullptr;
      gr.rs.partials = ws.partials;
      // U column a as a strided vector is not addressable directly: copy it out first
      extract_column(U, sdim, a);
      gr.rs.r[0].U = colbuf();
      const int grid = launch_lincomb<T>(g.a, gr.rs, grid0, done(), st);
      launch_reduce<T>(ws.partials, grid, gr.rs.nslots, dst + (size_t)a * sdim, done(), st);
    }
  }

  void* colbuf() {
    if (!ws.colbuf) KR_CUDA(cudaMalloc(&ws.colbuf, std::max<size_t>((size_t)n * sizeof(C2<T>), 16)));
    return ws.colbuf;
  }
  void extract_column(const void* U, int sdim, int a) {
    KR_CUDA(cudaMemcpy2DAsync(colbuf(), sizeof(C2<T>), reinterpret_cast<const char*>(U) + a * sizeof(C2<T>),
                              sdim * sizeof(C2<T>), sizeof(C2<T>), n, cudaMemcpyDeviceToDevice, st));
  }

  int reduce(const Reds& r, int grid) {
    if (r.rs.nred == 0) return -1;
    if (red_top + r.rs.nslots > kRedCap) red_top = 0;
    const int off = red_top;
    launch_reduce<T>(ws.partials, grid, r.rs.nslots, ws.red + off, done(), st);
    red_top += r.rs.nslots;
    return off;
  }

  void coef(int phase, int i0 = 0, int i1 = 0, int i2 = 0, int i3 = 0, double x0 = 0.0) {
    CoefArgs a{};
    a.phase = phase;
    a.s = s;
    a.st = ws.st;
    a.hist = ws.hist;
    a.red = ws.red;
    a.ar = ws.arena;
    a.i0 = i0; a.i1 = i1; a.i2 = i2; a.i3 = i3;
    a.x0 = x0;
    launch_coef(a, st);
  }

  // CholQR2 of Z (n x s, in place -> Q); S = R2 R1 written to arena slot sslot.
  // Optional fused Gram of the final Q: ufin^H Q (ufin memory block) -> returns its red offset.
  int thin_qr(void* Z, int sslot, const void* ufin = nullptr, bool q_is_y = true) {
    Lin g(n, s);
    const int o = g.out(nullptr);
    g.blk(o, Z);
    Reds r1;
    r1.add(RED_GRAM, o, o, nullptr, s);
    const int g1 = lin(g, r1);
    coef(PH_QR1, g1, SL_QR_R1, SL_QR_R1INV, 0, (double)n);
    Lin q1(n, s);
    const int o1 = q1.out(Z);
    q1.blk(o1, Z, mat(slot(SL_QR_R1INV)));
    Reds r2;
    r2.add(RED_GRAM, o1, o1, nullptr, s);
    const int g2 = lin(q1, r2);
    coef(PH_QR2, g2, SL_QR_R1, SL_QR_R2INV, sslot);
    Lin q2(n, s);
    const int o2 = q2.out(Z);
    q2.blk(o2, Z, mat(slot(SL_QR_R2INV)));
    Reds r3;
    if (ufin) {
      if (q_is_y) r3.add(RED_GRAM, o2, -1, ufin, s);  // ufin^H Q
    }
    return lin(q2, r3);
  }
};

// =========================================================================================
// methods
// =========================================================================================
namespace {

template <typename T>
struct Ctx {
  Engine<T>& E;
  const void* B;
  void* X;
  const void* shadow;
  int shadow_mode;
  int matvecs_per_iter;
};

// R = B - op(A) X with ||R||^2 -> PH_INIT
template <typename T>
void init_residual(Engine<T>& E, const void* B, void* X, void* R) {
  Reds r;
  const int sl = r.add(RED_NORM2, 0, -1, nullptr, E.s);
  const int off = E.spmm(false, E.s, X, R, r, B, -1.0, 1.0);
  E.coef(PH_INIT, off + sl);
}

// shadow block Rh from R (default / conj / user)
template <typename T>
void make_shadow(Engine<T>& E, const void* R, void* Rh, int mode, const void* user) {
  Lin L(E.n, E.s);
  const int o = L.out(Rh);
  if (mode == 2) L.blk(o, user);
  else if (mode == 1) L.blk(o, R, conjx());
  else L.blk(o, R);
  E.lin(L);
}

// Gl-BiCG (Algorithm 2) with alpha from the adjoint product and the update fused with the
// product: tr(Ph^H A P) = tr(Qh^H P) with Qh = A^H Ph, so alpha's denominator is a reduction of the
// direction update of P, and X += alpha P, R -= alpha A P (formed in the pass, not stored),
// Rh -= conj(alpha) Qh run in one pass.  Per iteration 2M + 17 Bv instead of 2M + 19 Bv; the
// iterates equal Algorithm 2's in exact arithmetic.
template <typename T>
void run_gl_bicg_fused(Ctx<T>& c, int maxit, const std::function<bool(int)>& poll) {
  Engine<T>& E = c.E;
  void *R = E.blk(0), *Rh = E.blk(1), *P = E.blk(2), *Ph = E.blk(3), *Q = E.blk(4), *Qh = E.blk(5);
  init_residual(E, c.B, c.X, R);
  make_shadow(E, R, Rh, c.shadow_mode, c.shadow);
  {
    Lin L(E.n, E.s);
    const int op_ = L.out(P), oph = L.out(Ph);
    L.blk(op_, R);
    L.blk(oph, Rh);
    Reds r;
    const int sl = r.add(RED_TRACE, op_, oph, nullptr, E.s);  // tr(Rh^H R)
    const int off = E.lin(L, r);
    E.coef(PH_SC_RHO0, off + sl);
  }
  {
    Reds r;
    const int sl = r.add(RED_TRACE, 0, -1, P, E.s);  // tr(P^H Qh) = conj(tr(Qh^H P))
    const int off = E.spmm(true, E.s, Ph, Qh, r);
    E.coef(PH_SC_ALPHA_CONJ, off + sl);
  }
  for (int it = 0; it < maxit; ++it) {
    E.red_top = 0;
    Lin L(E.n, E.s);
    const int ox = L.out(c.X), orr = L.out(R), orh = L.out(Rh);
    L.blk(ox, c.X);
    L.blk(ox, P, sc(E.slot(SL_ALPHA)));
    L.blk(orr, R);
    L.product(orr, sc(E.slot(SL_ALPHA), false, true));
    L.blk(orh, Rh);
    L.blk(orh, Qh, sc(E.slot(SL_ALPHA), true, true));
    Reds r2;
    const int s2 = r2.add(RED_TRACE, orr, orh, nullptr, E.s);  // tr(Rh^H R)
    const int s3 = r2.add(RED_NORM2, orr, -1, nullptr, E.s);
    const int o2 = E.lin_product(L, false, P, Q, r2);
    E.coef(PH_SC_BETA, o2 + s2, o2 + s3);
    if (poll(it + 1)) break;
    Lin Uh(E.n, E.s);
    const int oph = Uh.out(Ph);
    Uh.blk(oph, Rh);
    Uh.blk(oph, Ph, sc(E.slot(SL_BETA), true));
    E.lin(Uh);
    E.spmm(true, E.s, Ph, Qh);
    Lin U(E.n, E.s);
    const int op_ = U.out(P);
    U.blk(op_, R);
    U.blk(op_, P, sc(E.slot(SL_BETA)));
    Reds r1;
    const int s1 = r1.add(RED_TRACE, op_, -1, Qh, E.s);  // tr(Qh^H P)
    const int o1 = E.lin(U, r1);
    E.coef(PH_SC_ALPHA, o1 + s1);
  }
}

template <typename T>
void run_gl_bicg(Ctx<T>& c, int maxit, const std::function<bool(int)>& poll) {
  Engine<T>& E = c.E;
  void *R = E.blk(0), *Rh = E.blk(1), *P = E.blk(2), *Ph = E.blk(3), *Q = E.blk(4);
  init_residual(E, c.B, c.X, R);
  make_shadow(E, R, Rh, c.shadow_mode, c.shadow);
  {
    Lin L(E.n, E.s);
    const int op_ = L.out(P), oph = L.out(Ph);
    L.blk(op_, R);
    L.blk(oph, Rh);
    Reds r;
    const int sl = r.add(RED_TRACE, op_, oph, nullptr, E.s);  // tr(Rh^H R)
    const int off = E.lin(L, r);
    E.coef(PH_SC_RHO0, off + sl);
  }
  for (int it = 0; it < maxit; ++it) {
    E.red_top = 0;
    Reds r1;
    const int s1 = r1.add(RED_TRACE, 0, -1, Ph, E.s);  // tr(Ph^H Q)
    const int o1 = E.spmm(false, E.s, P, Q, r1);
    E.coef(PH_SC_ALPHA, o1 + s1);
    // Rh <- Rh - conj(alpha) A^H Ph
    E.spmm(true, E.s, Ph, Rh, Reds{}, Rh, 1.0, 1.0, E.slot(SL_ALPHA), true, true);
    Lin L(E.n, E.s);
    const int ox = L.out(c.X), orr = L.out(R);
    L.blk(ox, c.X);
    L.blk(ox, P, sc(E.slot(SL_ALPHA)));
    L.blk(orr, R);
    L.blk(orr, Q, sc(E.slot(SL_ALPHA), false, true));
    Reds r2;
    const int s2 = r2.add(RED_TRACE, orr, -1, Rh, E.s);  // tr(Rh^H R)
    const int s3 = r2.add(RED_NORM2, orr, -1, nullptr, E.s);
    const int o2 = E.lin(L, r2);
    E.coef(PH_SC_BETA, o2 + s2, o2 + s3);
    Lin U(E.n, E.s);
    const int op_ = U.out(P), oph = U.out(Ph);
    U.blk(op_, R);
    U.blk(op_, P, sc(E.slot(SL_BETA)));
    U.blk(oph, Rh);
    U.blk(oph, Ph, sc(E.slot(SL_BETA), true));
    E.lin(U);
    if (poll(it + 1)) break;
  }
}

// eGl-BiCG (Algorithm 4) with the coefficient alpha taken from the adjoint product and the update
// fused with the product.  sum(ph^H A P) = sum((A^H ph)^H P) = sum(qh^H P) with qh = A^H ph, so
// after the n-vector product qh the denominator of alpha is a reduction of the direction update
// P = R + beta P itself, and X += alpha P, R -= alpha A P, rh -= conj(alpha) qh run in one pass
// that forms A P row by row without storing it.  Per iteration 2M + 8 Bv instead of 2M + 11 Bv
// (M: one read of A; Bv: one n x s block); the iterates equal Algorithm 4's in exact arithmetic.
template <typename T>
void run_egl_bicg_fused(Ctx<T>& c, int maxit, const std::function<bool(int)>& poll) {
  Engine<T>& E = c.E;
  void *R = E.blk(0), *P = E.blk(1), *Q = E.blk(2);
  void *rh = E.vecp(0), *ph = E.vecp(1), *qh = E.vecp(2);
  init_residual(E, c.B, c.X, R);
  E.coef(PH_FILL_ONES);
  {
    Lin L(E.n, E.s);
    const int orh = L.out(rh, true);
    if (c.shadow_mode == 2) L.vec(orh, c.shadow);
    else L.blk(orh, R, mat(E.slot(SL_ONES)));  // mean of the columns of R_0 (Sec. 5)
    E.lin(L);
    if (c.shadow_mode == 1) {  // conj(mean)
      Lin L2(E.n, 1);
      const int o2 = L2.out(rh, true);
      L2.vec(o2, rh, conjx());
      E.lin(L2);
    }
  }
  {
    Lin L(E.n, E.s);
    const int op_ = L.out(P);
    L.blk(op_, R);
    Reds r;
    const int sl = r.add(RED_SUMV, op_, -1, rh, E.s);  // rho_0 = sum(rh^H R)
    const int off = E.lin(L, r);
    E.coef(PH_SC_RHO0, off + sl);
    Lin V(E.n, 1);
    const int ov = V.out(ph, true);
    V.vec(ov, rh);
    E.lin(V);
  }
  // alpha_0 = rho_0 / sum(qh^H P) with qh = A^H ph
  E.spmm(true, 1, ph, qh);
  {
    Lin L(E.n, E.s);
    const int o = L.out(nullptr);
    L.blk(o, P);
    Reds r;
    const int sl = r.add(RED_SUMV, o, -1, qh, E.s);
    const int off = E.lin(L, r);
    E.coef(PH_SC_ALPHA, off + sl);
  }
  for (int it = 0; it < maxit; ++it) {
    E.red_top = 0;
    // rh -= conj(alpha) qh (an n-vector, its own launch: the block pass then has block outputs
    // only and runs on column pairs in complex64)
    Lin Lv(E.n, 1);
    const int orh = Lv.out(rh, true);
    Lv.vec(orh, rh);
    Lv.vec(orh, qh, sc(E.slot(SL_ALPHA), true, true));
    E.lin(Lv);
    // X += alpha P; R -= alpha A P (formed in this pass); rho = sum(rh^H R), ||R||^2
    Lin L(E.n, E.s);
    const int ox = L.out(c.X), orr = L.out(R);
    L.blk(ox, c.X);
    L.blk(ox, P, sc(E.slot(SL_ALPHA)));
    L.blk(orr, R);
    L.product(orr, sc(E.slot(SL_ALPHA), false, true));
    Reds r2;
    const int s2 = r2.add(RED_SUMV, orr, -1, rh, E.s);
    const int s3 = r2.add(RED_NORM2, orr, -1, nullptr, E.s);
    const int o2 = E.lin_product(L, false, P, Q, r2);
    E.coef(PH_SC_BETA, o2 + s2, o2 + s3);
    if (poll(it + 1)) break;
    // ph = rh + conj(beta) ph; qh = A^H ph; P = R + beta P with alpha's denominator sum(qh^H P)
    Lin Uv(E.n, 1);
    const int ov = Uv.out(ph, true);
    Uv.vec(ov, rh);
    Uv.vec(ov, ph, sc(E.slot(SL_BETA), true));
    E.lin(Uv);
    E.spmm(true, 1, ph, qh);
    Lin U(E.n, E.s);
    const int op_ = U.out(P);
    U.blk(op_, R);
    U.blk(op_, P, sc(E.slot(SL_BETA)));
    Reds r1;
    const int s1 = r1.add(RED_SUMV, op_, -1, qh, E.s);
    const int o1 = E.lin(U, r1);
    E.coef(PH_SC_ALPHA, o1 + s1);
  }
}

template <typename T>
void run_egl_bicg(Ctx<T>& c, int maxit, const std::function<bool(int)>& poll) {
  Engine<T>& E = c.E;
  void *R = E.blk(0), *P = E.blk(1), *Q = E.blk(2);
  void *rh = E.vecp(0), *ph = E.vecp(1);
  init_residual(E, c.B, c.X, R);
  E.coef(PH_FILL_ONES);
  {
    Lin L(E.n, E.s);
    const int orh = L.out(rh, true);
    if (c.shadow_mode == 2) L.vec(orh, c.shadow);
    else L.blk(orh, R, mat(E.slot(SL_ONES)));  // mean of the columns of R_0 (Sec. 5)
    E.lin(L);
    if (c.shadow_mode == 1) {  // conj(mean)
      Lin L2(E.n, 1);
      const int o2 = L2.out(rh, true);
      L2.vec(o2, rh, conjx());
      E.lin(L2);
    }
  }
  {
    Lin L(E.n, E.s);
    const int op_ = L.out(P);
    L.blk(op_, R);
    Reds r;
    const int sl = r.add(RED_SUMV, op_, -1, rh, E.s);  // sum(rh^H R)
    const int off = E.lin(L, r);
    E.coef(PH_SC_RHO0, off + sl);
    Lin V(E.n, 1);
    const int ov = V.out(ph, true);
    V.vec(ov, rh);
    E.lin(V);
  }
  for (int it = 0; it < maxit; ++it) {
    E.red_top = 0;
    Reds r1;
    const int s1 = r1.add(RED_SUMV, 0, -1, ph, E.s);  // sum(ph^H Q)
    const int o1 = E.spmm(false, E.s, P, Q, r1);
    E.coef(PH_SC_ALPHA, o1 + s1);
    // rh <- rh - conj(alpha) A^H ph   (one n-vector)
    E.spmm(true, 1, ph, rh, Reds{}, rh, 1.0, 1.0, E.slot(SL_ALPHA), true, true);
    Lin L(E.n, E.s);
    const int ox = L.out(c.X), orr = L.out(R);
    L.blk(ox, c.X);
    L.blk(ox, P, sc(E.slot(SL_ALPHA)));
    L.blk(orr, R);
    L.blk(orr, Q, sc(E.slot(SL_ALPHA), false, true));
    Reds r2;
    const int s2 = r2.add(RED_SUMV, orr, -1, rh, E.s);
    const int s3 = r2.add(RED_NORM2, orr, -1, nullptr, E.s);
    const int o2 = E.lin(L, r2);
    E.coef(PH_SC_BETA, o2 + s2, o2 + s3);
    Lin U(E.n, E.s);
    const int op_ = U.out(P);
    U.blk(op_, R);
    U.blk(op_, P, sc(E.slot(SL_BETA)));
    E.lin(U);
    Lin Uv(E.n, 1);
    const int ov = Uv.out(ph, true);
    Uv.vec(ov, rh);
    Uv.vec(ov, ph, sc(E.slot(SL_BETA), true));
    E.lin(Uv);
    if (poll(it + 1)) break;
  }
}

template <typename T>
void run_li_bicg(Ctx<T>& c, int maxit, const std::function<bool(int)>& poll) {
  Engine<T>& E = c.E;
  void *R = E.blk(0), *Rh = E.blk(1), *P = E.blk(2), *Ph = E.blk(3), *Q = E.blk(4), *Qh = E.blk(5);
  init_residual(E, c.B, c.X, R);
  make_shadow(E, R, Rh, c.shadow_mode, c.shadow);
  {
    Lin L(E.n, E.s);
    const int op_ = L.out(P), oph = L.out(Ph);
    L.blk(op_, R);
    L.blk(oph, Rh);
    Reds r;
    const int sl = r.add(RED_CDOT, op_, oph, nullptr, E.s);  // rh_i^H r_i
    const int off = E.lin(L, r);
    E.coef(PH_LI_RHO0, off + sl);
  }
  for (int it = 0; it < maxit; ++it) {
    E.red_top = 0;
    Reds r1;
    const int s1 = r1.add(RED_CDOT, 0, -1, Ph, E.s);  // ph_i^H q_i
    const int o1 = E.spmm(false, E.s, P, Q, r1);
    E.coef(PH_LI_ALPHA, o1 + s1);
    E.spmm(true, E.s, Ph, Qh, Reds{});
    Lin L(E.n, E.s);
    const int ox = L.out(c.X), orr = L.out(R), orh = L.out(Rh);
    L.blk(ox, c.X);
    L.blk(ox, P, dg(E.slot(SL_ALPHA)));
    L.blk(orr, R);
    L.blk(orr, Q, dg(E.slot(SL_ALPHA), false, true));
    L.blk(orh, Rh);
    L.blk(orh, Qh, dg(E.slot(SL_ALPHA), true, true));  // Rh - (A^H Ph) conj(diag(alpha))
    Reds r2;
    const int s2 = r2.add(RED_CDOT, orr, -1, Rh, E.s);
    const int s3 = r2.add(RED_NORM2, orr, -1, nullptr, E.s);
    const int o2 = E.lin(L, r2);
    E.coef(PH_LI_BETA, o2 + s2, o2 + s3);
    Lin U(E.n, E.s);
    const int op_ = U.out(P), oph = U.out(Ph);
    U.blk(op_, R);
    U.blk(op_, P, dg(E.slot(SL_BETA)));
    U.blk(oph, Rh);
    U.blk(oph, Ph, dg(E.slot(SL_BETA), true));
    E.lin(U);
    if (poll(it + 1)) break;
  }
}

template <typename T>
void run_li_bicgstab(Ctx<T>& c, int maxit, const std::function<bool(int)>& poll) {
  Engine<T>& E = c.E;
  void *R = E.blk(0), *Rt = E.blk(1), *P = E.blk(2), *V = E.blk(3), *S = E.blk(4), *T_ = E.blk(5);
  init_residual(E, c.B, c.X, R);
  make_shadow(E, R, Rt, c.shadow_mode, c.shadow);
  {
    Lin L(E.n, E.s);
    const int op_ = L.out(P);
    L.blk(op_, R);
    Reds r;
    const int sl = r.add(RED_CDOT, op_, -1, Rt, E.s);  // rt_c^H r_c
    const int off = E.lin(L, r);
    E.coef(PH_LI_RHO0, off + sl);
  }
  for (int it = 0; it < maxit; ++it) {
    E.red_top = 0;
    Reds r1;
    const int s1 = r1.add(RED_CDOT, 0, -1, Rt, E.s);  // rt_c^H v_c
    const int o1 = E.spmm(false, E.s, P, V, r1);
    E.coef(PH_LS_ALPHA, o1 + s1);
    Lin L(E.n, E.s);
    const int os = L.out(S);
    L.blk(os, R);
    L.blk(os, V, dg(E.slot(SL_ALPHA), false, true));
    E.lin(L);
    Reds r2;
    const int s2 = r2.add(RED_CDOT, 0, -1, S, E.s);        // s_c^H t_c
    const int s3 = r2.add(RED_CDOT, 0, -1, nullptr, E.s);  // t_c^H t_c
    const int o2 = E.spmm(false, E.s, S, T_, r2);
    E.coef(PH_LS_OMEGA, o2 + s2, o2 + s3);
    Lin U(E.n, E.s);
    const int ox = U.out(c.X), orr = U.out(R);
    U.blk(ox, c.X);
    U.blk(ox, P, dg(E.slot(SL_ALPHA)));
    U.blk(ox, S, dg(E.slot(SL_OMEGA)));
    U.blk(orr, S);
    U.blk(orr, T_, dg(E.slot(SL_NOMEGA)));
    Reds r3;
    const int s4 = r3.add(RED_CDOT, orr, -1, Rt, E.s);
    const int s5 = r3.add(RED_NORM2, orr, -1, nullptr, E.s);
    const int o3 = E.lin(U, r3);
    E.coef(PH_LS_BETA, o3 + s4, o3 + s5);
    Lin W(E.n, E.s);
    const int op_ = W.out(P);
    W.blk(op_, R);
    W.blk(op_, P, dg(E.slot(SL_BETA)));
    W.blk(op_, V, dg(E.slot(SL_GAMMA)));  // -beta omega
    E.lin(W);
    if (poll(it + 1)) break;
  }
}

template <typename T>
void run_bl_bicg(Ctx<T>& c, int maxit, const std::function<bool(int)>& poll) {
  Engine<T>& E = c.E;
  void *R = E.blk(0), *Rh = E.blk(1), *P = E.blk(2), *Ph = E.blk(3), *Q = E.blk(4), *Qh = E.blk(5);
  init_residual(E, c.B, c.X, R);
  make_shadow(E, R, Rh, c.shadow_mode, c.shadow);
  {
    Lin L(E.n, E.s);
    const int op_ = L.out(P), oph = L.out(Ph);
    L.blk(op_, R);
    L.blk(oph, Rh);
    Reds r;
    const int sl = r.add(RED_GRAM, op_, oph, nullptr, E.s);  // Rh^H R
    const int off = E.lin(L, r);
    E.coef(PH_BL_G0, off + sl);
  }
  for (int it = 0; it < maxit; ++it) {
    E.red_top = 0;
    Reds r1;
    const int s1 = r1.add(RED_GRAM, 0, -1, Ph, E.s);  // Ph^H Q
    const int o1 = E.spmm(false, E.s, P, Q, r1);
    E.spmm(true, E.s, Ph, Qh);
    E.coef(PH_BL_ALPHA, o1 + s1);
    Lin L(E.n, E.s);
    const int ox = L.out(c.X), orr = L.out(R), orh = L.out(Rh);
    L.blk(ox, c.X);
    L.blk(ox, P, mat(E.slot(SL_ALPHA)));
    L.blk(orr, R);
    L.blk(orr, Q, mat(E.slot(SL_ALPHA), true));
    L.blk(orh, Rh);
    L.blk(orh, Qh, mat(E.slot(SL_ALPHAH), true));
    Reds r2;
    const int s2 = r2.add(RED_GRAM, orr, orh, nullptr, E.s);  // Rh_new^H R_new
    const int s3 = r2.add(RED_NORM2, orr, -1, nullptr, E.s);
    const int o2 = E.lin(L, r2);
    E.coef(PH_BL_BETA, o2 + s2, o2 + s3);
    Lin U(E.n, E.s);
    const int op_ = U.out(P), oph = U.out(Ph);
    U.blk(op_, R);
    U.blk(op_, P, mat(E.slot(SL_BETA)));
    U.blk(oph, Rh);
    U.blk(oph, Ph, mat(E.slot(SL_BETAH)));
    E.lin(U);
    if (poll(it + 1)) break;
  }
}

template <typename T>
void run_bl_bicg_rq(Ctx<T>& c, int maxit, const std::function<bool(int)>& poll) {
  Engine<T>& E = c.E;
  void *Zq = E.blk(0), *Q = E.blk(1), *Qh = E.blk(2), *V = E.blk(3), *Vh = E.blk(4), *W = E.blk(5),
       *Wh = E.blk(6), *Zh = E.blk(7);
  init_residual(E, c.B, c.X, Q);
  make_shadow(E, Q, Qh, c.shadow_mode, c.shadow);
  E.thin_qr(Qh, SL_CH);
  E.thin_qr(Q, SL_C);
  {
    Lin L(E.n, E.s);
    const int ov = L.out(V), ovh = L.out(Vh);
    L.blk(ov, Q);
    L.blk(ovh, Qh);
    Reds r;
    const int sl = r.add(RED_GRAM, ov, ovh, nullptr, E.s);  // Qh^H Q
    const int off = E.lin(L, r);
    E.coef(PH_RQ_INIT, off + sl);
  }
  for (int it = 0; it < maxit; ++it) {
    E.red_top = 0;
    Reds r1;
    const int s1 = r1.add(RED_GRAM, 0, -1, Vh, E.s);  // Vh^H W
    const int o1 = E.spmm(false, E.s, V, W, r1);
    E.spmm(true, E.s, Vh, Wh);
    E.coef(PH_RQ_ALPHA, o1 + s1);
    Lin L(E.n, E.s);
    const int ox = L.out(c.X), oz = L.out(Zq), ozh = L.out(Zh);
    L.blk(ox, c.X);
    L.blk(ox, V, mat(E.slot(SL_AC)));
    L.blk(oz, Q);
    L.blk(oz, W, mat(E.slot(SL_ALPHA), true));
    L.blk(ozh, Qh);
    L.blk(ozh, Wh, mat(E.slot(SL_ALPHAH), true));
    E.lin(L);
    E.thin_qr(Zq, SL_S);
    E.thin_qr(Zh, SL_SH);
    E.coef(PH_RQ_C);
    Lin g(E.n, E.s);
    const int oq = g.out(nullptr), oqh = g.out(nullptr);
    g.blk(oq, Zq);
    g.blk(oqh, Zh);
    Reds r2;
    const int s2 = r2.add(RED_GRAM, oq, oqh, nullptr, E.s);  // Qh_new^H Q_new
    const int o2 = E.lin(g, r2);
    E.coef(PH_RQ_BETA, o2 + s2);
    Lin U(E.n, E.s);
    const int ov = U.out(V), ovh = U.out(Vh);
    U.blk(ov, Zq);
    U.blk(ov, V, mat(E.slot(SL_BETA)));
    U.blk(ovh, Zh);
    U.blk(ovh, Vh, mat(E.slot(SL_BETAH)));
    E.lin(U);
    std::swap(Q, Zq);
    std::swap(Qh, Zh);
    if (poll(it + 1)) break;
  }
}

template <typename T>
void run_gl_bicgstab(Ctx<T>& c, int maxit, const std::function<bool(int)>& poll) {
  Engine<T>& E = c.E;
  void *R = E.blk(0), *Rt = E.blk(1), *P = E.blk(2), *V = E.blk(3), *S = E.blk(4), *T_ = E.blk(5);
  init_residual(E, c.B, c.X, R);
  make_shadow(E, R, Rt, c.shadow_mode, c.shadow);
  {
    Lin L(E.n, E.s);
    const int op_ = L.out(P);
    L.blk(op_, R);
    Reds r;
    const int sl = r.add(RED_TRACE, op_, -1, Rt, E.s);
    const int off = E.lin(L, r);
    E.coef(PH_SC_RHO0, off + sl);
  }
  for (int it = 0; it < maxit; ++it) {
    E.red_top = 0;
    Reds r1;
    const int s1 = r1.add(RED_TRACE, 0, -1, Rt, E.s);  // tr(Rt^H V)
    const int o1 = E.spmm(false, E.s, P, V, r1);
    E.coef(PH_GS_ALPHA, o1 + s1);
    Lin L(E.n, E.s);
    const int os = L.out(S);
    L.blk(os, R);
    L.blk(os, V, sc(E.slot(SL_ALPHA), false, true));
    E.lin(L);
    Reds r2;
    const int s2 = r2.add(RED_TRACE, 0, -1, S, E.s);  // tr(S^H T)
    const int s3 = r2.add(RED_NORM2, 0, -1, nullptr, E.s);
    const int o2 = E.spmm(false, E.s, S, T_, r2);
    E.coef(PH_GS_OMEGA, o2 + s2, o2 + s3);
    Lin U(E.n, E.s);
    const int ox = U.out(c.X), orr = U.out(R);
    U.blk(ox, c.X);
    U.blk(ox, P, sc(E.slot(SL_ALPHA)));
    U.blk(ox, S, sc(E.slot(SL_OMEGA)));
    U.blk(orr, S);
    U.blk(orr, T_, sc(E.slot(SL_NOMEGA)));
    Reds r3;
    const int s4 = r3.add(RED_TRACE, orr, -1, Rt, E.s);
    const int s5 = r3.add(RED_NORM2, orr, -1, nullptr, E.s);
    const int o3 = E.lin(U, r3);
    E.coef(PH_GS_BETA, o3 + s4, o3 + s5);
    Lin W(E.n, E.s);
    const int op_ = W.out(P);
    W.blk(op_, R);
    W.blk(op_, P, sc(E.slot(SL_BETA)));
    W.blk(op_, V, sc(E.slot(SL_GAMMA)));  // -beta omega
    E.lin(W);
    if (poll(it + 1)) break;
  }
}

template <typename T>
void run_bl_bicgstab(Ctx<T>& c, int maxit, const std::function<bool(int)>& poll) {
  Engine<T>& E = c.E;
  void *R = E.blk(0), *Rt = E.blk(1), *P = E.blk(2), *V = E.blk(3), *S = E.blk(4), *T_ = E.blk(5);
  init_residual(E, c.B, c.X, R);
  make_shadow(E, R, Rt, c.shadow_mode, c.shadow);
  {
    Lin L(E.n, E.s);
    const int op_ = L.out(P);
    L.blk(op_, R);
    Reds r;
    const int sl = r.add(RED_GRAM, op_, -1, Rt, E.s);  // Rt^H R
    const int off = E.lin(L, r);
    E.coef(PH_BS_G0, off + sl);
  }
  for (int it = 0; it < maxit; ++it) {
    E.red_top = 0;
    Reds r1;
    const int s1 = r1.add(RED_GRAM, 0, -1, Rt, E.s);  // Rt^H V
    const int o1 = E.spmm(false, E.s, P, V, r1);
    E.coef(PH_BS_ALPHA, o1 + s1);
    Lin L(E.n, E.s);
    const int os = L.out(S);
    L.blk(os, R);
    L.blk(os, V, mat(E.slot(SL_ALPHA), true));
    E.lin(L);
    Reds r2;
    const int s2 = r2.add(RED_TRACE, 0, -1, S, E.s);
    const int s3 = r2.add(RED_NORM2, 0, -1, nullptr, E.s);
    const int s4 = r2.add(RED_GRAM, 0, -1, Rt, E.s);  // Rt^H T
    const int o2 = E.spmm(false, E.s, S, T_, r2);
    E.coef(PH_BS_OMEGA, o2 + s2, o2 + s3, o2 + s4);
    Lin U(E.n, E.s);
    const int ox = U.out(c.X), orr = U.out(R);
    U.blk(ox, c.X);
    U.blk(ox, P, mat(E.slot(SL_ALPHA)));
    U.blk(ox, S, sc(E.slot(SL_OMEGA)));
    U.blk(orr, S);
    U.blk(orr, T_, sc(E.slot(SL_NOMEGA)));
    Reds r3;
    const int s5 = r3.add(RED_GRAM, orr, -1, Rt, E.s);
    const int s6 = r3.add(RED_NORM2, orr, -1, nullptr, E.s);
    const int o3 = E.lin(U, r3);
    E.coef(PH_BS_BETA, o3 + s5, o3 + s6);
    Lin W(E.n, E.s);
    const int op_ = W.out(P);
    W.blk(op_, R);
    W.blk(op_, P, mat(E.slot(SL_BETA)));
    W.blk(op_, V, mat(E.slot(SL_B2)));  // -omega beta
    E.lin(W);
    if (poll(it + 1)) break;
  }
}

template <typename T>
void run_bl_bicgstab_rq(Ctx<T>& c, int maxit, const std::function<bool(int)>& poll) {
  Engine<T>& E = c.E;
  void *Z = E.blk(0), *Rt = E.blk(1), *Q = E.blk(2), *V = E.blk(3), *W = E.blk(4), *Sp = E.blk(5),
       *Tp = E.blk(6);
  init_residual(E, c.B, c.X, Q);
  make_shadow(E, Q, Rt, c.shadow_mode, c.shadow);
  {
    const int off = E.thin_qr(Q, SL_C, Rt);  // R_0 = Q C; fused Rt^H Q
    E.coef(PH_BSR_INIT, off);
    Lin L(E.n, E.s);
    const int ov = L.out(V);
    L.blk(ov, Q);
    E.lin(L);
  }
  for (int it = 0; it < maxit; ++it) {
    E.red_top = 0;
    Reds r1;
    const int s1 = r1.add(RED_GRAM, 0, -1, Rt, E.s);  // Rt^H W
    const int o1 = E.spmm(false, E.s, V, W, r1);
    E.coef(PH_BSR_ALPHA, o1 + s1);
    Lin L(E.n, E.s);
    const int os = L.out(Sp);
    L.blk(os, Q);
    L.blk(os, W, mat(E.slot(SL_ALPHA), true));
    E.lin(L);
    Reds r2;
    const int s2 = r2.add(RED_GRAM, 0, -1, Sp, E.s);  // Sp^H Tp
    const int s3 = r2.add(RED_GRAM, 0, -1, Rt, E.s);  // Rt^H Tp
    const int o2 = E.spmm(false, E.s, Sp, Tp, r2);
    // Tp^H Tp
    Lin g(E.n, E.s);
    const int og = g.out(nullptr);
    g.blk(og, Tp);
    Reds r3;
    const int s4 = r3.add(RED_GRAM, og, og, nullptr, E.s);
    const int o3 = E.lin(g, r3);
    E.coef(PH_BSR_OMEGA, o2 + s2, o3 + s4, o2 + s3);
    Lin U(E.n, E.s);
    const int ox = U.out(c.X), oz = U.out(Z);
    U.blk(ox, c.X);
    U.blk(ox, V, mat(E.slot(SL_AC)));
    U.blk(ox, Sp, mat(E.slot(SL_OC)));
    U.blk(oz, Sp);
    U.blk(oz, Tp, sc(E.slot(SL_NOMEGA)));
    E.lin(U);
    const int o4 = E.thin_qr(Z, SL_S, Rt);  // Z = Q_new Sigma; fused Rt^H Q_new
    E.coef(PH_BSR_C, o4);
    Lin Wv(E.n, E.s);
    const int ov = Wv.out(V);
    Wv.blk(ov, Z);
    Wv.blk(ov, V, mat(E.slot(SL_B2)));
    Wv.blk(ov, W, mat(E.slot(SL_B3)));
    E.lin(Wv);
    std::swap(Q, Z);
    if (poll(it + 1)) break;
  }
}

template <typename T>
void run_gl_qmr(Ctx<T>& c, int maxit, const std::function<bool(int)>& poll, bool econ) {
  Engine<T>& E = c.E;
  void *R = E.blk(0), *V = E.blk(1), *Vp = E.blk(2), *Y = E.blk(3), *D1 = E.blk(4), *D2 = E.blk(5),
       *AD1 = E.blk(6), *AD2 = E.blk(7);
  void *W, *Wp, *Yh, *Wstart;
  if (econ) { W = E.vecp(0); Wp = E.vecp(1); Yh = E.vecp(2); Wstart = E.vecp(3); }
  else { W = E.blk(8); Wp = E.blk(9); Yh = E.blk(10); Wstart = E.blk(11); }
  const int ws = econ ? 1 : E.s;
  init_residual(E, c.B, c.X, R);
  // shadow start block / vector
  if (econ) {
    E.coef(PH_FILL_ONES);
    Lin L(E.n, E.s);
    const int o = L.out(Wstart, true);
    if (c.shadow_mode == 2) L.vec(o, c.shadow);
    else L.blk(o, R, mat(E.slot(SL_ONES)));
    E.lin(L);
    if (c.shadow_mode == 1) {
      Lin L2(E.n, 1);
      const int o2 = L2.out(Wstart, true);
      L2.vec(o2, Wstart, conjx());
      E.lin(L2);
    }
  } else {
    make_shadow(E, R, Wstart, c.shadow_mode, c.shadow);
  }
  int offR, slR, offW, slW;
  {
    Lin L(E.n, E.s);
    const int o = L.out(nullptr);
    L.blk(o, R);
    Reds r;
    slR = r.add(RED_NORM2, o, -1, nullptr, E.s);
    offR = E.lin(L, r);
    Lin Lw(E.n, ws);
    const int ow = Lw.out(nullptr, econ);
    if (econ) Lw.vec(ow, Wstart); else Lw.blk(ow, Wstart);
    Reds rw;
    slW = rw.add(RED_NORM2, ow, -1, nullptr, ws);
    offW = E.lin(Lw, rw);
  }
  E.coef(PH_QMR_INIT, offR + slR, offW + slW);
  // zero the direction blocks and previous Lanczos blocks
  KR_CUDA(cudaMemsetAsync(D1, 0, (size_t)E.n * E.s * sizeof(C2<T>), E.st));
  KR_CUDA(cudaMemsetAsync(D2, 0, (size_t)E.n * E.s * sizeof(C2<T>), E.st));
  KR_CUDA(cudaMemsetAsync(AD1, 0, (size_t)E.n * E.s * sizeof(C2<T>), E.st));
  KR_CUDA(cudaMemsetAsync(AD2, 0, (size_t)E.n * E.s * sizeof(C2<T>), E.st));
  KR_CUDA(cudaMemsetAsync(Vp, 0, (size_t)E.n * E.s * sizeof(C2<T>), E.st));
  KR_CUDA(cudaMemsetAsync(Wp, 0, (size_t)E.n * ws * sizeof(C2<T>), E.st));
  {
    Lin Lw(E.n, ws);
    const int ow = Lw.out(W, econ);
    if (econ) Lw.vec(ow, Wstart, sc(E.slot(SL_INVXI))); else Lw.blk(ow, Wstart, sc(E.slot(SL_INVXI)));
    E.lin(Lw);
    Lin L(E.n, E.s);
    const int ov = L.out(V);
    L.blk(ov, R, sc(E.slot(SL_INVRHO)));
    Reds r;
    const int sl = r.add(econ ? RED_SUMV : RED_TRACE, ov, -1, W, E.s);  // tr(W^H V)
    const int off = E.lin(L, r);
    E.coef(PH_QMR_DELTA, off + sl);
  }
  for (int it = 0; it < maxit; ++it) {
    E.red_top = 0;
    Reds r1;
    const int s1 = r1.add(econ ? RED_SUMV : RED_TRACE, 0, -1, W, E.s);  // tr(W^H Y)
    const int o1 = E.spmm(false, E.s, V, Y, r1);
    E.spmm(true, ws, W, Yh);
    E.coef(PH_QMR_COEF1, o1 + s1);
    // Wt = Yh - conj(alpha) W - gamma Wp  (into Wp)
    Lin Lw(E.n, ws);
    const int ow = Lw.out(Wp, econ);
    if (econ) {
      Lw.vec(ow, Yh);
      Lw.vec(ow, W, sc(E.slot(SL_ALPHA), true, true));
      Lw.vec(ow, Wp, sc(E.slot(SL_GAMMA), false, true));
    } else {
      Lw.blk(ow, Yh);
      Lw.blk(ow, W, sc(E.slot(SL_ALPHA), true, true));
      Lw.blk(ow, Wp, sc(E.slot(SL_GAMMA), false, true));
    }
    Reds rw;
    const int sw = rw.add(RED_NORM2, ow, -1, nullptr, ws);
    const int offw = E.lin(Lw, rw);
    // Vt = Y - alpha V - beta Vp  (into Vp)
    Lin Lv(E.n, E.s);
    const int ov = Lv.out(Vp);
    Lv.blk(ov, Y);
    Lv.blk(ov, V, sc(E.slot(SL_ALPHA), false, true));
    Lv.blk(ov, Vp, sc(E.slot(SL_BETA), false, true));
    Reds rv;
    const int sv = rv.add(RED_NORM2, ov, -1, nullptr, E.s);
    const int st_ = rv.add(econ ? RED_SUMV : RED_TRACE, ov, -1, Wp, E.s);  // tr(Wt^H Vt)
    const int offv = E.lin(Lv, rv);
    E.coef(PH_QMR_COEF2, offv + sv, offw + sw, offv + st_);
    // directions, iterate, residual, normalised next Lanczos block
    Lin U(E.n, E.s);
    const int od = U.out(D2), oad = U.out(AD2), ox = U.out(c.X), orr = U.out(R), ovn = U.out(Vp);
    U.blk(od, V, sc(E.slot(SL_CV)));
    U.blk(od, D2, sc(E.slot(SL_CD2)));
    U.blk(od, D1, sc(E.slot(SL_CD1)));
    U.blk(oad, Y, sc(E.slot(SL_CV)));
    U.blk(oad, AD2, sc(E.slot(SL_CD2)));
    U.blk(oad, AD1, sc(E.slot(SL_CD1)));
    U.blk(ox, c.X);
    U.reg(ox, od, sc(E.slot(SL_TAU)));
    U.blk(orr, R);
    U.reg(orr, oad, sc(E.slot(SL_NTAU)));
    U.blk(ovn, Vp, sc(E.slot(SL_INVRHO)));
    Reds r2;
    const int s2 = r2.add(RED_NORM2, orr, -1, nullptr, E.s);
    const int o2 = E.lin(U, r2);
    Lin Wn(E.n, ws);
    const int own = Wn.out(Wp, econ);
    if (econ) Wn.vec(own, Wp, sc(E.slot(SL_INVXI))); else Wn.blk(own, Wp, sc(E.slot(SL_INVXI)));
    E.lin(Wn);
    E.coef(PH_QMR_MON, o2 + s2);
    std::swap(V, Vp);
    std::swap(W, Wp);
    std::swap(D1, D2);
    std::swap(AD1, AD2);
    if (poll(it + 1)) break;
  }
}

// Li-QMR: s scalar QMR iterations (no look-ahead) in lockstep, the loop interchange of
// Sec. 2 applied to QMR; every coefficient is a per-column (diagonal) one and every inner
// product a column-wise one (RED_CDOT).  Stops on ||R||_F.
template <typename T>
void run_li_qmr(Ctx<T>& c, int maxit, const std::function<bool(int)>& poll) {
  Engine<T>& E = c.E;
  void *R = E.blk(0), *V = E.blk(1), *Vp = E.blk(2), *Y = E.blk(3), *D1 = E.blk(4), *D2 = E.blk(5),
       *AD1 = E.blk(6), *AD2 = E.blk(7), *W = E.blk(8), *Wp = E.blk(9), *Yh = E.blk(10), *Wstart = E.blk(11);
  init_residual(E, c.B, c.X, R);
  make_shadow(E, R, Wstart, c.shadow_mode, c.shadow);
  int offR, slR, offW, slW;
  {
    Lin L(E.n, E.s);
    const int o = L.out(nullptr);
    L.blk(o, R);
    Reds r;
    slR = r.add(RED_CDOT, o, o, nullptr, E.s);  // ||r_c||^2
    offR = E.lin(L, r);
    Lin Lw(E.n, E.s);
    const int ow = Lw.out(nullptr);
    Lw.blk(ow, Wstart);
    Reds rw;
    slW = rw.add(RED_CDOT, ow, ow, nullptr, E.s);  // ||w_c||^2
    offW = E.lin(Lw, rw);
  }
  E.coef(PH_LQ_INIT, offR + slR, offW + slW);
  const size_t bytes = (size_t)E.n * E.s * sizeof(C2<T>);
  KR_CUDA(cudaMemsetAsync(D1, 0, bytes, E.st));
  KR_CUDA(cudaMemsetAsync(D2, 0, bytes, E.st));
  KR_CUDA(cudaMemsetAsync(AD1, 0, bytes, E.st));
  KR_CUDA(cudaMemsetAsync(AD2, 0, bytes, E.st));
  KR_CUDA(cudaMemsetAsync(Vp, 0, bytes, E.st));
  KR_CUDA(cudaMemsetAsync(Wp, 0, bytes, E.st));
  {
    Lin Lw(E.n, E.s);
    const int ow = Lw.out(W);
    Lw.blk(ow, Wstart, dg(E.slot(SL_INVXI)));
    E.lin(Lw);
    Lin L(E.n, E.s);
    const int ov = L.out(V);
    L.blk(ov, R, dg(E.slot(SL_INVRHO)));
    Reds r;
    const int sl = r.add(RED_CDOT, ov, -1, W, E.s);  // w_c^H v_c
    const int off = E.lin(L, r);
    E.coef(PH_LQ_DELTA, off + sl);
  }
  for (int it = 0; it < maxit; ++it) {
    E.red_top = 0;
    Reds r1;
    const int s1 = r1.add(RED_CDOT, 0, -1, W, E.s);  // w_c^H (A v_c)
    const int o1 = E.spmm(false, E.s, V, Y, r1);
    E.spmm(true, E.s, W, Yh);
    E.coef(PH_LQ_COEF1, o1 + s1);
    // wt = A^H w - conj(alpha) w - gamma w_prev  (into Wp), column-wise norms
    Lin Lw(E.n, E.s);
    const int ow = Lw.out(Wp);
    Lw.blk(ow, Yh);
    Lw.blk(ow, W, dg(E.slot(SL_ALPHA), true, true));
    Lw.blk(ow, Wp, dg(E.slot(SL_GAMMA), false, true));
    Reds rw;
    const int sw = rw.add(RED_CDOT, ow, ow, nullptr, E.s);
    const int offw = E.lin(Lw, rw);
    // vt = A v - alpha v - beta v_prev  (into Vp), column-wise norms and wt_c^H vt_c
    Lin Lv(E.n, E.s);
    const int ov = Lv.out(Vp);
    Lv.blk(ov, Y);
    Lv.blk(ov, V, dg(E.slot(SL_ALPHA), false, true));
    Lv.blk(ov, Vp, dg(E.slot(SL_BETA), false, true));
    Reds rv;
    const int sv = rv.add(RED_CDOT, ov, ov, nullptr, E.s);
    const int st_ = rv.add(RED_CDOT, ov, -1, Wp, E.s);
    const int offv = E.lin(Lv, rv);
    E.coef(PH_LQ_COEF2, offv + sv, offw + sw, offv + st_);
    // directions, iterate, residual, normalised next Lanczos block
    Lin U(E.n, E.s);
    const int od = U.out(D2), oad = U.out(AD2), ox = U.out(c.X), orr = U.out(R), ovn = U.out(Vp);
    U.blk(od, V, dg(E.slot(SL_CV)));
    U.blk(od, D2, dg(E.slot(SL_CD2)));
    U.blk(od, D1, dg(E.slot(SL_CD1)));
    U.blk(oad, Y, dg(E.slot(SL_CV)));
    U.blk(oad, AD2, dg(E.slot(SL_CD2)));
    U.blk(oad, AD1, dg(E.slot(SL_CD1)));
    U.blk(ox, c.X);
    U.reg(ox, od, dg(E.slot(SL_TAU)));
    U.blk(orr, R);
    U.reg(orr, oad, dg(E.slot(SL_NTAU)));
    U.blk(ovn, Vp, dg(E.slot(SL_INVRHO)));
    Reds r2;
    const int s2 = r2.add(RED_NORM2, orr, -1, nullptr, E.s);
    const int o2 = E.lin(U, r2);
    Lin Wn(E.n, E.s);
    const int own = Wn.out(Wp);
    Wn.blk(own, Wp, dg(E.slot(SL_INVXI)));
    E.lin(Wn);
    E.coef(PH_LQ_MON, o2 + s2);
    std::swap(V, Vp);
    std::swap(W, Wp);
    std::swap(D1, D2);
    std::swap(AD1, AD2);
    if (poll(it + 1)) break;
  }
}

template <typename T>
void run_bl_qmr(Ctx<T>& c, int maxit, const std::function<bool(int)>& poll) {
  Engine<T>& E = c.E;
  void *R = E.blk(0), *V = E.blk(1), *Vp = E.blk(2), *W = E.blk(3), *Wp = E.blk(4), *Y = E.blk(5),
       *Yh = E.blk(6), *D1 = E.blk(7), *D2 = E.blk(8), *AD1 = E.blk(9), *AD2 = E.blk(10);
  init_residual(E, c.B, c.X, R);
  make_shadow(E, R, W, c.shadow_mode, c.shadow);
  {
    Lin L(E.n, E.s);
    const int ov = L.out(V);
    L.blk(ov, R);
    E.lin(L);
  }
  E.thin_qr(W, SL_XIK);             // Rh_0 = W_1 xi_1
  const int off = E.thin_qr(V, SL_RHOK, W);  // R_0 = V_1 rho_0; fused W^H V
  E.coef(PH_BQ_INIT, off);
  const size_t bytes = (size_t)E.n * E.s * sizeof(C2<T>);
  KR_CUDA(cudaMemsetAsync(D1, 0, bytes, E.st));
  KR_CUDA(cudaMemsetAsync(D2, 0, bytes, E.st));
  KR_CUDA(cudaMemsetAsync(AD1, 0, bytes, E.st));
  KR_CUDA(cudaMemsetAsync(AD2, 0, bytes, E.st));
  KR_CUDA(cudaMemsetAsync(Vp, 0, bytes, E.st));
  KR_CUDA(cudaMemsetAsync(Wp, 0, bytes, E.st));
  for (int it = 0; it < maxit; ++it) {
    E.red_top = 0;
    Reds r1;
    const int s1 = r1.add(RED_GRAM, 0, -1, W, E.s);  // W^H Y
    const int o1 = E.spmm(false, E.s, V, Y, r1);
    E.spmm(true, E.s, W, Yh);
    E.coef(PH_BQ_COEF1, o1 + s1);
    Lin L(E.n, E.s);
    const int ov = L.out(Vp), ow = L.out(Wp);
    L.blk(ov, Y);
    L.blk(ov, V, mat(E.slot(SL_ALPHA), true));
    L.blk(ov, Vp, mat(E.slot(SL_BETA), true));
    L.blk(ow, Yh);
    L.blk(ow, W, mat(E.slot(SL_ALPHAH), true));
    L.blk(ow, Wp, mat(E.slot(SL_BETAH), true));
    E.lin(L);
    E.thin_qr(Wp, SL_XIN);
    const int o2 = E.thin_qr(Vp, SL_RHON, Wp);  // fused W_new^H V_new
    E.coef(PH_BQ_COEF2, o2);
    Lin U(E.n, E.s);
    const int od = U.out(D2), oad = U.out(AD2), ox = U.out(c.X), orr = U.out(R);
    U.blk(od, V, mat(E.slot(SL_CV)));
    U.blk(od, D2, mat(E.slot(SL_CD2)));
    U.blk(od, D1, mat(E.slot(SL_CD1)));
    U.blk(oad, Y, mat(E.slot(SL_CV)));
    U.blk(oad, AD2, mat(E.slot(SL_CD2)));
    U.blk(oad, AD1, mat(E.slot(SL_CD1)));
    U.blk(ox, c.X);
    U.reg(ox, od, mat(E.slot(SL_TAU)));
    U.blk(orr, R);
    U.reg(orr, oad, mat(E.slot(SL_NTAU)));
    Reds r2;
    const int s2 = r2.add(RED_NORM2, orr, -1, nullptr, E.s);
    const int o3 = E.lin(U, r2);
    E.coef(PH_BQ_MON, o3 + s2);
    std::swap(V, Vp);
    std::swap(W, Wp);
    std::swap(D1, D2);
    std::swap(AD1, AD2);
    if (poll(it + 1)) break;
  }
}

int blocks_needed(int method) {
  switch (method) {
    case KRM_GL_QMR: return 12;
    case KRM_LI_QMR: return 12;
    case KRM_BL_QMR: return 11;
    case KRM_EGL_QMR: return 8;
    case KRM_BL_BICG_RQ: return 8;
    case KRM_BL_BICGSTAB_RQ: return 7;
    default: return 6;
  }
}
int vecs_needed(int method) {
  if (method == KRM_EGL_BICG) return 3;
  if (method == KRM_EGL_QMR) return 4;
  return 0;
}
int matvecs_per_iter(int method, int s) {
  if (method == KRM_EGL_BICG || method == KRM_EGL_QMR) return s + 1;
  return 2 * s;
}

}  // namespace

// =========================================================================================
// driver for one precision
// =========================================================================================
template <typename T>
SolveOut run_solve(Operator& op, int method, int s, const void* B, void* X, const SolveIn& in, cudaStream_t user_st,
                   bool adjoint) {
  Workspace& ws = get_workspace(op, s, sizeof(C2<T>), blocks_needed(method), vecs_needed(method), in.maxit);
  // CUDA-graph replay: iteration 0 runs eagerly (it also makes every lazy allocation), the
  // launches of iterations 1 and 2 are captured on a private stream (the caller's may be the
  // legacy default stream, which cannot be captured), and the graph is replayed until the
  // device state says done.  The launch profile counts launches on the host, so it disables it.
  const bool graphs = in.graphs && in.maxit >= 3 && !prof_active();
  cudaStream_t st = user_st;
  if (graphs) {
    if (!ws.gstream) KR_CUDA(cudaStreamCreateWithFlags(&ws.gstream, cudaStreamNonBlocking));
    if (!ws.gevent) KR_CUDA(cudaEventCreateWithFlags(&ws.gevent, cudaEventDisableTiming));
    KR_CUDA(cudaEventRecord(ws.gevent, user_st));
    KR_CUDA(cudaStreamWaitEvent(ws.gstream, ws.gevent, 0));
    st = ws.gstream;
  }
  struct CaptureGuard {  // ends a capture left open by an exception
    cudaStream_t s = nullptr;
    ~CaptureGuard() {
      if (s) {
        cudaGraph_t g = nullptr;
        if (cudaStreamEndCapture(s, &g) == cudaSuccess && g) cudaGraphDestroy(g);
      }
    }
  } guard;
  Engine<T> E(op, adjoint, s, st, ws);
  E.prec = in.precond && op.ilu.on && !adjoint;
  DevState h{};
  h.maxit = in.maxit;
  h.tol = in.tol;
  h.s = s;
  h.econ = (method == KRM_EGL_QMR) ? 1 : 0;
  h.status = 4;
  h.best = HUGE_VAL;
  h.stall = in.stall;
  KR_CUDA(cudaMemcpyAsync(ws.st, &h, sizeof(DevState), cudaMemcpyHostToDevice, st));
  KR_CUDA(cudaMemsetAsync(ws.hist, 0, sizeof(double) * (in.maxit + 1), st));
  DevState* pin = reinterpret_cast<DevState*>(op.pinned);
  const auto t0 = std::chrono::steady_clock::now();
  bool timed_out = false;
  const int every = in.check_every > 0 ? in.check_every : 8;
  // read the device state back; true when the iteration must stop
  auto check = [&]() -> bool {
    KR_CUDA(cudaMemcpyAsync(pin, ws.st, sizeof(DevState), cudaMemcpyDeviceToHost, st));
    KR_CUDA(cudaStreamSynchronize(st));
    if (pin->done) return true;
    if (in.time_limit_s > 0) {
      const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (el > in.time_limit_s) { timed_out = true; return true; }
    }
    return false;
  };
  std::function<bool(int)> poll = [&](int it) -> bool {
    if (graphs) {
      if (it == 1) {
        KR_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        guard.s = st;
        return false;
      }
      if (it == 2) return false;
      // it == 3: iterations 1 and 2 are recorded, not run; replay them in pairs
      cudaGraph_t g = nullptr;
      guard.s = nullptr;
      KR_CUDA(cudaStreamEndCapture(st, &g));
      cudaGraphExec_t ge = nullptr;
      const cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      KR_CUDA(e);
      const int per_check = every >= 4 ? every / 2 : 1;
      int launched = 1, replays = 0;  // iterations launched so far
      bool stop = false;
      while (!stop) {
        const cudaError_t le = cudaGraphLaunch(ge, st);
        if (le != cudaSuccess) { cudaGraphExecDestroy(ge); KR_CUDA(le); }
        launched += 2;
        ++replays;
        if (launched >= in.maxit || replays % per_check == 0) stop = check() || launched >= in.maxit;
      }
      cudaGraphExecDestroy(ge);
      return true;
    }
    if (it % every != 0 && it < in.maxit) return false;
    return check();
  };
  Ctx<T> c{E, B, X, in.shadow, in.shadow_mode, 0};
  // the fused-product schedules except on the matrix-free stencil: there the fused pass forms the
  // product with one neighbour load at a time (its registers leave no room for more), and the
  // algorithms' own order, whose products run on the product kernels, is faster (128^3, s = 8,
  // 50 FP64 eGl-BiCG iterations: 106 ms against 131 ms)
  const bool fused_schedule = fused_products_enabled() && op.stA.d == 0;
  switch (method) {
    case KRM_GL_BICG:
      if (fused_schedule) run_gl_bicg_fused<T>(c, in.maxit, poll);
      else run_gl_bicg<T>(c, in.maxit, poll);
      break;
    case KRM_EGL_BICG:
      if (fused_schedule) run_egl_bicg_fused<T>(c, in.maxit, poll);
      else run_egl_bicg<T>(c, in.maxit, poll);
      break;
    case KRM_LI_BICG: run_li_bicg<T>(c, in.maxit, poll); break;
    case KRM_LI_BICGSTAB: run_li_bicgstab<T>(c, in.maxit, poll); break;
    case KRM_LI_QMR: run_li_qmr<T>(c, in.maxit, poll); break;
    case KRM_BL_BICG: run_bl_bicg<T>(c, in.maxit, poll); break;
    case KRM_BL_BICG_RQ: run_bl_bicg_rq<T>(c, in.maxit, poll); break;
    case KRM_GL_BICGSTAB: run_gl_bicgstab<T>(c, in.maxit, poll); break;
    case KRM_BL_BICGSTAB: run_bl_bicgstab<T>(c, in.maxit, poll); break;
    case KRM_BL_BICGSTAB_RQ: run_bl_bicgstab_rq<T>(c, in.maxit, poll); break;
    case KRM_GL_QMR: run_gl_qmr<T>(c, in.maxit, poll, false); break;
    case KRM_EGL_QMR: run_gl_qmr<T>(c, in.maxit, poll, true); break;
    case KRM_BL_QMR: run_bl_qmr<T>(c, in.maxit, poll); break;
    default: throw CudaError{cudaErrorInvalidValue, "unknown method"};
  }
  KR_CUDA(cudaMemcpyAsync(pin, ws.st, sizeof(DevState), cudaMemcpyDeviceToHost, st));
  KR_CUDA(cudaStreamSynchronize(st));
  SolveOut o;
  o.iters = pin->iter;
  o.status = timed_out && !pin->done ? 5 : pin->status;
  o.res0 = pin->res0;
  o.relres_recursive = pin->iter > 0 ? pin->rel : (pin->res0 == 0.0 ? 0.0 : 1.0);
  o.matvecs = pin->iter * matvecs_per_iter(method, s);
  o.hist.resize(pin->iter + 1);
  KR_CUDA(cudaMemcpy(o.hist.data(), ws.hist, sizeof(double) * (pin->iter + 1), cudaMemcpyDeviceToHost));
  if (graphs) {  // later work on the caller's stream follows the solve
    KR_CUDA(cudaEventRecord(ws.gevent, st));
    KR_CUDA(cudaStreamWaitEvent(user_st, ws.gevent, 0));
  }
  return o;
}

template SolveOut run_solve<double>(Operator&, int, int, const void*, void*, const SolveIn&, cudaStream_t, bool);
template SolveOut run_solve<float>(Operator&, int, int, const void*, void*, const SolveIn&, cudaStream_t, bool);

// thin QR of an n x s device block in place (Q) with S written to arena slot SL_QR_S
void standalone_qr(Operator& op, Workspace& ws, int64_t n, int s, void* Q, cudaStream_t st) {
  Engine<double> E(op, false, s, st, ws);
  E.n = n;
  E.thin_qr(Q, SL_QR_S);
}

// Orthonormalised right-hand sides (the set-up of Sec. 5: B replaced by the factor Q of a thin
// QR).  R_0 = B - op(A) X_0 is formed in block 0 of a workspace of its own and factorised in
// place, R_0 = Q S, with S kept in that workspace's arena; block 1 is zeroed for the solution Y
// of op(A) Y = Q.  Returns ||R_0||_F, or a negative value when R_0 is numerically rank deficient.
double orthonormal_rhs(Operator& op, int s, const void* B, const void* X, void** Q, void** Y, cudaStream_t st,
                       bool adjoint) {
  Workspace& ws = get_workspace(op, s, kOrthoKey, 2, 0, 1);
  *Q = ws.blocks[0];
  *Y = ws.blocks[1];
  const double res0 = true_residual(op, s, B, X, *Q, st, adjoint);
  KR_CUDA(cudaMemsetAsync(*Y, 0, sizeof(double2) * (size_t)op.n * s, st));
  if (!(res0 > 0.0)) return res0;  // zero (X_0 solves the system) or non-finite: nothing to factorise
  DevState h{};
  h.maxit = 1;
  KR_CUDA(cudaMemcpyAsync(ws.st, &h, sizeof(DevState), cudaMemcpyHostToDevice, st));
  standalone_qr(op, ws, op.n, s, *Q, st);
  DevState back{};
  std::vector<double2> S((size_t)s * s);
  KR_CUDA(cudaMemcpyAsync(&back, ws.st, sizeof(DevState), cudaMemcpyDeviceToHost, st));
  KR_CUDA(cudaMemcpyAsync(S.data(), ws.arena + (size_t)SL_QR_S * kSlotElems, sizeof(double2) * s * s,
                          cudaMemcpyDeviceToHost, st));
  KR_CUDA(cudaStreamSynchronize(st));
  if (back.done && back.status == 1) return -1.0;
  // numerically rank deficient when a diagonal entry of S is at most 64 eps ||S||_F (the
  // breakdown rule of the s x s solves): CholQR2's shifted first pass still returns a factor
  double fro = 0.0, dmin = HUGE_VAL;
  for (int i = 0; i < s; ++i)
    for (int k = 0; k < s; ++k) fro += S[(size_t)i * s + k].x * S[(size_t)i * s + k].x + S[(size_t)i * s + k].y * S[(size_t)i * s + k].y;
  for (int i = 0; i < s; ++i) dmin = std::min(dmin, std::hypot(S[(size_t)i * s + i].x, S[(size_t)i * s + i].y));
  if (!(dmin > 64.0 * 2.220446049250313e-16 * std::sqrt(fro))) return -1.0;
  return res0;
}

// X += Y S with Y and S from the last orthonormal_rhs on this operator and s
void add_back_rhs_factor(Operator& op, int s, void* X, cudaStream_t st) {
  Workspace& ws = get_workspace(op, s, kOrthoKey, 2, 0, 1);
  Engine<double> E(op, false, s, st, ws);
  DevState h{};
  KR_CUDA(cudaMemcpyAsync(ws.st, &h, sizeof(DevState), cudaMemcpyHostToDevice, st));
  Lin L(op.n, s);
  const int o = L.out(X);
  L.blk(o, X);
  L.blk(o, ws.blocks[1], mat(E.slot(SL_QR_S)));
  E.lin(L);
}

// ||B - op(A) X||_F in FP64 (R written to Rbuf when given)
double true_residual(Operator& op, int s, const void* B, const void* X, void* Rbuf, cudaStream_t st, bool adjoint) {
  Workspace& ws = get_workspace(op, s, sizeof(double2), 1, 0, 1);
  Engine<double> E(op, adjoint, s, st, ws);
  DevState h{};
  KR_CUDA(cudaMemcpyAsync(ws.st, &h, sizeof(DevState), cudaMemcpyHostToDevice, st));
  Reds r;
  const int sl = r.add(RED_NORM2, 0, -1, nullptr, s);
  const int off = E.spmm(false, s, X, Rbuf ? Rbuf : ws.blocks[0], r, B, -1.0, 1.0);
  double2 v;
  KR_CUDA(cudaMemcpyAsync(&v, ws.red + off + sl, sizeof(double2), cudaMemcpyDeviceToHost, st));
  KR_CUDA(cudaStreamSynchronize(st));
  return std::sqrt(v.x);
}

}  // namespace kr
