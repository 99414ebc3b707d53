// ILU(0) right preconditioning (Sec. 5, second set of experiments): A M^{-1} Y = B, X = M^{-1} Y,
// M = L U with L unit lower and U upper triangular on the sparsity pattern of A.
//
// The factorisation runs once on the host in FP64 (row-by-row elimination restricted to the
// pattern of A).  The four triangular factors used by the solvers -- L and U for M^{-1},
// U^H and L^H for M^{-H} = L^{-H} U^{-H} -- are stored as CSR of their off-diagonal entries
// plus the inverse of their diagonal (none for the unit factors), each with a level
// schedule: a row's level is one more than the deepest level among the rows it depends on,
// so all rows of one level can be solved at once.  A triangular solve of an n x s block is
// one launch per level, G threads per row (one per column), rows of the level spread over
// the grid; the launches of a level read only rows finished by earlier launches.  The level
// launches are programmatic dependent launches: each is scheduled while the previous one is
// still running and waits (griddepcontrol.wait) until that one has completed and its writes are
// visible, so the launch latency between levels is hidden.
#include <algorithm>
#include <cmath>

#include "../../include/kr.h"
#include "kr_engine.h"
#include "kr_precond.h"
#include "kr_profile.h"

namespace kr {

namespace {

struct HostTri {
  std::vector<int64_t> rowptr;  // off-diagonal entries
  std::vector<int32_t> colidx;
  std::vector<double2> vals;
  std::vector<double2> invdiag;  // empty: unit diagonal
  bool lower = true;
};

// level schedule: rows grouped by dependency depth (forward for lower, backward for upper)
void schedule(const HostTri& t, int64_t n, std::vector<int64_t>& lev_ptr, std::vector<int32_t>& lev_rows) {
  std::vector<int32_t> level(n, 0);
  int32_t nlev = 0;
  auto visit = [&](int64_t i) {
    int32_t lv = 0;
    for (int64_t k = t.rowptr[i]; k < t.rowptr[i + 1]; ++k) lv = std::max(lv, level[t.colidx[k]] + 1);
    level[i] = lv;
    nlev = std::max(nlev, lv + 1);
  };
  if (t.lower)
    for (int64_t i = 0; i < n; ++i) visit(i);
  else
    for (int64_t i = n - 1; i >= 0; --i) visit(i);
  lev_ptr.assign(nlev + 1, 0);
  for (int64_t i = 0; i < n; ++i) lev_ptr[level[i] + 1]++;
  for (int32_t l = 0; l < nlev; ++l) lev_ptr[l + 1] += lev_ptr[l];
  lev_rows.assign(n, 0);
  std::vector<int64_t> fill(lev_ptr.begin(), lev_ptr.end() - 1);
  for (int64_t i = 0; i < n; ++i) lev_rows[fill[level[i]]++] = (int32_t)i;
}

// conjugate transpose of the off-diagonal part (lower <-> upper)
HostTri adjoint_of(const HostTri& t, int64_t n) {
  HostTri a;
  a.lower = !t.lower;
  a.rowptr.assign(n + 1, 0);
  for (int64_t k = 0; k < (int64_t)t.colidx.size(); ++k) a.rowptr[t.colidx[k] + 1]++;
  for (int64_t i = 0; i < n; ++i) a.rowptr[i + 1] += a.rowptr[i];
  a.colidx.resize(t.colidx.size());
  a.vals.resize(t.vals.size());
  std::vector<int64_t> fill(a.rowptr.begin(), a.rowptr.end() - 1);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = t.rowptr[i]; k < t.rowptr[i + 1]; ++k) {
      const int64_t p = fill[t.colidx[k]]++;
      a.colidx[p] = (int32_t)i;
      a.vals[p] = make_double2(t.vals[k].x, -t.vals[k].y);
    }
  if (!t.invdiag.empty()) {
    a.invdiag.resize(n);
    for (int64_t i = 0; i < n; ++i) a.invdiag[i] = make_double2(t.invdiag[i].x, -t.invdiag[i].y);
  }
  return a;
}

template <typename V>
V* upload(const std::vector<V>& h) {
  V* d = nullptr;
  KR_CUDA(cudaMalloc(&d, sizeof(V) * std::max<size_t>(h.size(), 1)));
  if (!h.empty()) KR_CUDA(cudaMemcpy(d, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice));
  return d;
}

TriDev to_device(const HostTri& t, int64_t n) {
  TriDev d;
  d.n = n;
  std::vector<int64_t> lev_ptr;
  std::vector<int32_t> lev_rows;
  schedule(t, n, lev_ptr, lev_rows);
  d.h_lev_ptr = lev_ptr;
  d.nlev = (int)lev_ptr.size() - 1;
  d.rowptr = upload(t.rowptr);
  d.colidx = upload(t.colidx);
  d.vals = upload(t.vals);
  d.invdiag = t.invdiag.empty() ? nullptr : upload(t.invdiag);
  d.lev_rows = upload(lev_rows);
  return d;
}

// y_i = (v_i - sum_j t_ij y_j) * invdiag_i for the rows of one level; thread c of a row group
// owns column c
template <int G>
__global__ void __launch_bounds__(kThreads) trsv_level_kernel(const int32_t* __restrict__ rows, int64_t count,
                                                              const int64_t* __restrict__ rowptr,
                                                              const int32_t* __restrict__ colidx,
                                                              const double2* __restrict__ vals,
                                                              const double2* __restrict__ invdiag, int s,
                                                              const double2* V, double2* Y) {
  constexpr int RPW = 32 / G;
  // the previous level's launch has completed and its rows are visible; then this level's own
  // dependent (the next level) may be scheduled
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = lane & (G - 1);
  const int64_t r = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * RPW + lane / G;
  if (r >= count || c >= s) return;
  const int64_t i = rows[r];
  double2 acc = V[i * s + c];
  for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
    const double2 t = vals[k];
    const double2 y = Y[(int64_t)colidx[k] * s + c];
    acc.x = fma(-t.x, y.x, acc.x);
    acc.x = fma(t.y, y.y, acc.x);
    acc.y = fma(-t.x, y.y, acc.y);
    acc.y = fma(-t.y, y.x, acc.y);
  }
  if (invdiag != nullptr) acc = cmul<double>(invdiag[i], acc);
  Y[i * s + c] = acc;
}

template <int G>
void trsv_go(const TriDev& t, int s, const double2* V, double2* Y, cudaStream_t st) {
  const int64_t rows_per_cta = (kThreads / 32) * (32 / G);
  for (int l = 0; l < t.nlev; ++l) {
    const int64_t b = t.h_lev_ptr[l], cnt = t.h_lev_ptr[l + 1] - b;
    if (cnt == 0) continue;
    const int64_t grid = (cnt + rows_per_cta - 1) / rows_per_cta;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    KR_CUDA(cudaLaunchKernelEx(&cfg, trsv_level_kernel<G>, (const int32_t*)(t.lev_rows + b), cnt,
                               (const int64_t*)t.rowptr, (const int32_t*)t.colidx, (const double2*)t.vals,
                               (const double2*)t.invdiag, s, V, Y));
  }
  KR_CUDA(cudaGetLastError());
}

// Y = T^{-1} V for one triangular factor (Y may equal V)
void trsv(const TriDev& t, int s, const double2* V, double2* Y, cudaStream_t st) {
  ProfToken tk = prof_begin(KC_OTHER, st);
  switch (threads_per_row(s)) {
    case 1: trsv_go<1>(t, s, V, Y, st); break;
    case 2: trsv_go<2>(t, s, V, Y, st); break;
    case 4: trsv_go<4>(t, s, V, Y, st); break;
    case 8: trsv_go<8>(t, s, V, Y, st); break;
    case 16: trsv_go<16>(t, s, V, Y, st); break;
    default: trsv_go<32>(t, s, V, Y, st); break;
  }
  const double nnz = (double)t.h_nnz, n = (double)t.n;
  // per entry a 4-byte index and a 16-byte value; row pointers, level rows, inverse diagonal;
  // the right-hand side read and the solution written once
  prof_end(tk, st, (double)s * (8.0 * nnz + (t.invdiag ? 6.0 * n : 0.0)),
           20.0 * nnz + 8.0 * (n + 1) + 4.0 * n + (t.invdiag ? 16.0 * n : 0.0) + 32.0 * n * s);
}

}  // namespace

void TriDev::free_all() {
  cudaFree(rowptr); cudaFree(colidx); cudaFree(vals); cudaFree(invdiag); cudaFree(lev_rows);
  rowptr = nullptr; colidx = nullptr; vals = nullptr; invdiag = nullptr; lev_rows = nullptr;
}

void IluDev::free_all() {
  L.free_all(); U.free_all(); UH.free_all(); LH.free_all();
  on = false;
}

int build_ilu0(Operator& op) {
  const int64_t n = op.n;
  const std::vector<int64_t>& rp = op.h_rowptr;
  // rows with sorted columns (values kept with their column)
  std::vector<int32_t> ci(op.h_colidx);
  std::vector<double2> v(op.h_colidx.size());
  for (int64_t k = 0; k < (int64_t)v.size(); ++k) v[k] = make_double2(op.h_vals[2 * k], op.h_vals[2 * k + 1]);
  std::vector<int32_t> diagpos(n, -1);
  {
    std::vector<std::pair<int32_t, double2>> tmp;
    for (int64_t i = 0; i < n; ++i) {
      tmp.clear();
      for (int64_t k = rp[i]; k < rp[i + 1]; ++k) tmp.push_back({ci[k], v[k]});
      std::stable_sort(tmp.begin(), tmp.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
      for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
        ci[k] = tmp[k - rp[i]].first;
        v[k] = tmp[k - rp[i]].second;
        if (k > rp[i] && ci[k] == ci[k - 1]) return KR_BAD_ARG;  // duplicate entry
        if (ci[k] == i) diagpos[i] = (int32_t)(k - rp[i]);
      }
      if (diagpos[i] < 0) return KR_BAD_ARG;  // ILU(0) needs the diagonal stored
    }
  }
  // row-by-row elimination on the pattern; pos[j] = position of column j in the current row
  std::vector<int64_t> pos(n, -1);
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) pos[ci[k]] = k;
    for (int64_t p = rp[i]; p < rp[i + 1] && ci[p] < i; ++p) {
      const int32_t k = ci[p];
      const double2 ukk = v[rp[k] + diagpos[k]];
      if (ukk.x == 0.0 && ukk.y == 0.0) {
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) pos[ci[q]] = -1;
        return KR_BREAKDOWN;
      }
      const double den = ukk.x * ukk.x + ukk.y * ukk.y;
      const double2 lik = make_double2((v[p].x * ukk.x + v[p].y * ukk.y) / den, (v[p].y * ukk.x - v[p].x * ukk.y) / den);
      v[p] = lik;
      for (int64_t q = rp[k] + diagpos[k] + 1; q < rp[k + 1]; ++q) {
        const int64_t at = pos[ci[q]];
        if (at >= 0) {
          v[at].x -= lik.x * v[q].x - lik.y * v[q].y;
          v[at].y -= lik.x * v[q].y + lik.y * v[q].x;
        }
      }
    }
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) pos[ci[k]] = -1;
  }
  for (int64_t i = 0; i < n; ++i) {
    const double2 d = v[rp[i] + diagpos[i]];
    if (!(std::isfinite(d.x) && std::isfinite(d.y)) || (d.x == 0.0 && d.y == 0.0)) return KR_BREAKDOWN;
  }
  // split into strict L, strict U + inverse diagonal
  HostTri L, U;
  L.lower = true;
  U.lower = false;
  L.rowptr.assign(n + 1, 0);
  U.rowptr.assign(n + 1, 0);
  U.invdiag.resize(n);
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      if (ci[k] < i) { L.colidx.push_back(ci[k]); L.vals.push_back(v[k]); }
      else if (ci[k] > i) { U.colidx.push_back(ci[k]); U.vals.push_back(v[k]); }
      else {
        const double den = v[k].x * v[k].x + v[k].y * v[k].y;
        U.invdiag[i] = make_double2(v[k].x / den, -v[k].y / den);
      }
    }
    L.rowptr[i + 1] = (int64_t)L.colidx.size();
    U.rowptr[i + 1] = (int64_t)U.colidx.size();
  }
  IluDev& d = op.ilu;
  d.free_all();
  d.L = to_device(L, n);
  d.L.h_nnz = (int64_t)L.colidx.size();
  d.U = to_device(U, n);
  d.U.h_nnz = (int64_t)U.colidx.size();
  HostTri UH = adjoint_of(U, n), LH = adjoint_of(L, n);
  d.UH = to_device(UH, n);
  d.UH.h_nnz = (int64_t)UH.colidx.size();
  d.LH = to_device(LH, n);
  d.LH.h_nnz = (int64_t)LH.colidx.size();
  d.on = true;
  return KR_OK;
}

void apply_ilu0(const Operator& op, bool adjoint, int s, const double2* V, double2* Y, double2* tmp,
                cudaStream_t st) {
  const IluDev& d = op.ilu;
  if (!adjoint) {  // M^{-1} V = U^{-1} (L^{-1} V)
    trsv(d.L, s, V, tmp, st);
    trsv(d.U, s, tmp, Y, st);
  } else {  // M^{-H} V = L^{-H} (U^{-H} V)
    trsv(d.UH, s, V, tmp, st);
    trsv(d.LH, s, tmp, Y, st);
  }
}

}  // namespace kr
