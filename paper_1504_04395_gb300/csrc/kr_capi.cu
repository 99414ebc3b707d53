// extern "C" boundary of the library (declared in include/kr.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>

#include "../../include/kr.h"
#include "kr_engine.h"
#include "kr_precond.h"
#include "kr_profile.h"
#include "kr_solver.h"

struct kr_op_s {
  kr::Operator op;
};

namespace kr {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
const char* get_error() { return g_err.c_str(); }

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  static std::map<int, int> cache;
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
  cache[dev] = n;
  return n;
}

namespace {

// elementwise helpers of the defect-correction loop and the gradient
__global__ void to_c64_kernel(const double2* __restrict__ a, float2* __restrict__ b, int64_t cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = make_float2((float)a[i].x, (float)a[i].y);
}
__global__ void add_c128_kernel(double2* __restrict__ x, const double2* __restrict__ d, int64_t cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
    x[i].x += d[i].x;
    x[i].y += d[i].y;
  }
}
__global__ void add_c64_kernel(double2* __restrict__ x, const float2* __restrict__ d, int64_t cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = d[i];
    x[i].x += (double)v.x;
    x[i].y += (double)v.y;
  }
}

// dvals[k] = - sum_c Lambda[i][c] conj(X[j][c]) for stored entry k = (i, j); G threads per row
template <int G>
__global__ void __launch_bounds__(256) grad_kernel(int64_t n, int s, const int64_t* __restrict__ rowptr,
                                                   const int32_t* __restrict__ colidx,
                                                   const double2* __restrict__ Lam, const double2* __restrict__ X,
                                                   double2* __restrict__ dv) {
  constexpr int RPW = 32 / G;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = lane & (G - 1);
  const int64_t rows_per_cta = (int64_t)(blockDim.x >> 5) * RPW;
  for (int64_t base = blockIdx.x * rows_per_cta; base < n; base += (int64_t)gridDim.x * rows_per_cta) {
    const int64_t i = base + warp * RPW + lane / G;
    const bool rowok = i < n;
    const bool act = rowok && c < s;
    const double2 l = act ? Lam[i * s + c] : make_double2(0.0, 0.0);
    int64_t k0 = 0, k1 = 0;
    if (rowok) { k0 = rowptr[i]; k1 = rowptr[i + 1]; }
    // iterate to the longest row in the warp so that every lane joins the shuffles
    int64_t len = k1 - k0, mx = len;
    for (int off = 16; off >= 1; off >>= 1) {
      const int64_t o = __shfl_xor_sync(0xffffffffu, mx, off);
      mx = o > mx ? o : mx;
    }
    for (int64_t q = 0; q < mx; ++q) {
      double2 p = make_double2(0.0, 0.0);
      const bool has = q < len;
      if (act && has) {
        const int64_t j = colidx[k0 + q];
        const double2 x = X[j * s + c];
        p.x = l.x * x.x + l.y * x.y;   // l * conj(x)
        p.y = l.y * x.x - l.x * x.y;
      }
      for (int off = G / 2; off >= 1; off >>= 1) {
        p.x += __shfl_down_sync(0xffffffffu, p.x, off, G);
        p.y += __shfl_down_sync(0xffffffffu, p.y, off, G);
      }
      if (c == 0 && rowok && has) dv[k0 + q] = make_double2(-p.x, -p.y);
    }
  }
}

int grid1d(int64_t cnt) {
  int64_t g = (cnt + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * 8;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

kr_status map_exc(const std::exception* e) {
  if (e) set_error(e->what());
  return KR_CUDA_ERROR;
}

#define KR_API_BEGIN try {
#define KR_API_END                                                                         \
  }                                                                                        \
  catch (const ::kr::CudaError& e) {                                                       \
    ::kr::set_error(std::string(cudaGetErrorString(e.code)) + " (" + e.where + ")");       \
    return (e.code == cudaErrorMemoryAllocation) ? KR_OOM : KR_CUDA_ERROR;                  \
  }                                                                                        \
  catch (const std::bad_alloc&) {                                                          \
    ::kr::set_error("host allocation failed");                                             \
    return KR_OOM;                                                                         \
  }                                                                                        \
  catch (const std::exception& e) {                                                        \
    return map_exc(&e);                                                                    \
  }

// scratch context for the kernel-level entry points (one per device, grown on demand)
struct Scratch {
  Operator op;  // empty operator: only n / device are used
};
std::map<int, std::unique_ptr<Scratch>> g_scratch;
std::mutex g_scratch_mu;

Workspace& scratch_ws(int64_t n, int s) {
  int dev = 0;
  KR_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  auto& sc = g_scratch[dev];
  if (!sc) sc = std::make_unique<Scratch>();
  sc->op.device = dev;
  if (sc->op.n < n) {  // workspace blocks are sized by n: rebuild when n grows
    sc->op.ws.clear();
    sc->op.n = n;
  }
  return get_workspace(sc->op, s, sizeof(double2), 0, 0, 1);
}

bool bad_s(int s) { return s < 1 || s > kMaxS; }

}  // namespace
}  // namespace kr

using namespace kr;

extern "C" {

void kr_options_default(kr_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->tol = 1e-8;
  opt->maxit = 500;
  opt->precision = KR_FP64;
  opt->inner_tol = 1e-4;
  opt->max_outer = 30;
  opt->shadow_mode = KR_SHADOW_DEFAULT;
  opt->check_every = 8;
  opt->deterministic = 1;
}

const char* kr_last_error(void) { return get_error(); }

kr_status kr_set_lattice_rows_per_thread(int32_t rows) {
  if (rows != 0 && rows != 4 && rows != 12) { set_error("rows must be 0, 4 or 12"); return KR_BAD_ARG; }
  kr::set_lattice_rows_per_thread(rows);
  return KR_OK;
}

kr_status kr_set_column_pairs(int32_t enable) {
  kr::set_pair_kernels(enable != 0);
  return KR_OK;
}

kr_status kr_set_tile_kernels(int32_t enable) {
  kr::set_tile_kernels(enable != 0);
  return KR_OK;
}

kr_status kr_set_fused_products(int32_t enable) {
  kr::set_fused_products(enable != 0);
  return KR_OK;
}

kr_status kr_op_create_csr(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                           const double* vals, int32_t device, kr_op* out) {
  if (!out) { set_error("out is NULL"); return KR_BAD_ARG; }
  *out = nullptr;
  if (n <= 0 || nnz < 0 || !rowptr || (nnz > 0 && (!colidx || !vals))) {
    set_error("invalid CSR sizes or NULL arrays");
    return KR_BAD_ARG;
  }
  if (n > 0x7fffffffLL) { set_error("n exceeds int32 column index range"); return KR_BAD_ARG; }
  if (rowptr[0] != 0 || rowptr[n] != nnz) { set_error("rowptr[0] must be 0 and rowptr[n] == nnz"); return KR_BAD_ARG; }
  for (int64_t i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) { set_error("rowptr not monotone"); return KR_BAD_ARG; }
  for (int64_t k = 0; k < nnz; ++k)
    if (colidx[k] < 0 || colidx[k] >= n) { set_error("column index out of range"); return KR_BAD_ARG; }
  KR_API_BEGIN
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) { set_error("no CUDA device"); return KR_CUDA_ERROR; }
  if (device < 0 || device >= ndev) { set_error("device ordinal out of range"); return KR_BAD_ARG; }
  KR_CUDA(cudaSetDevice(device));
  auto h = std::make_unique<kr_op_s>();
  Operator& op = h->op;
  op.device = device;
  op.n = n;
  op.nnz = nnz;
  op.h_rowptr.assign(rowptr, rowptr + n + 1);
  op.h_colidx.assign(colidx, colidx + nnz);
  op.h_vals.assign(vals, vals + 2 * nnz);
  build_operator_device(op, false);
  KR_CUDA(cudaMallocHost(&op.pinned, 4096));
  *out = h.release();
  return KR_OK;
  KR_API_END
}

kr_status kr_op_create_csr_async(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                                 const double* vals, int32_t on_device, void* stream, kr_op* out) {
  if (!out) { set_error("out is NULL"); return KR_BAD_ARG; }
  *out = nullptr;
  if (n <= 0 || nnz < 0 || !rowptr || (nnz > 0 && (!colidx || !vals))) {
    set_error("invalid CSR sizes or NULL arrays");
    return KR_BAD_ARG;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  if (st != nullptr) {
    if (cudaStreamGetDevice(st, &dev) != cudaSuccess) {
      cudaGetLastError();
      set_error("cannot determine the device of the stream");
      return KR_BAD_ARG;
    }
  } else if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    set_error("no CUDA device");
    return KR_CUDA_ERROR;
  }
  if (!on_device) return kr_op_create_csr(n, nnz, rowptr, colidx, vals, dev, out);
  KR_API_BEGIN
  KR_CUDA(cudaSetDevice(dev));
  // staged through pinned host memory on the caller's stream; the host builds A^H and checks
  // the arrays exactly as for host input
  int64_t* hr = nullptr;
  int32_t* hc = nullptr;
  double* hv = nullptr;
  struct PinGuard {
    void* p[3] = {nullptr, nullptr, nullptr};
    ~PinGuard() { for (void* q : p) if (q) cudaFreeHost(q); }
  } pg;
  KR_CUDA(cudaMallocHost(&hr, sizeof(int64_t) * (n + 1)));
  pg.p[0] = hr;
  KR_CUDA(cudaMallocHost(&hc, sizeof(int32_t) * std::max<int64_t>(nnz, 1)));
  pg.p[1] = hc;
  KR_CUDA(cudaMallocHost(&hv, sizeof(double2) * std::max<int64_t>(nnz, 1)));
  pg.p[2] = hv;
  KR_CUDA(cudaMemcpyAsync(hr, rowptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, st));
  if (nnz > 0) {
    KR_CUDA(cudaMemcpyAsync(hc, colidx, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, st));
    KR_CUDA(cudaMemcpyAsync(hv, vals, sizeof(double2) * nnz, cudaMemcpyDeviceToHost, st));
  }
  KR_CUDA(cudaStreamSynchronize(st));
  return kr_op_create_csr(n, nnz, hr, hc, hv, dev, out);
  KR_API_END
}

kr_status kr_op_create_stencil(int32_t dim, const int64_t* dims, const double* coeffs, int32_t device, kr_op* out) {
  if (!out) { set_error("out is NULL"); return KR_BAD_ARG; }
  *out = nullptr;
  if (dim < 1 || dim > 3 || !dims || !coeffs) { set_error("dim must be 1, 2 or 3 with dims and coeffs"); return KR_BAD_ARG; }
  int64_t n = 1;
  for (int q = 0; q < dim; ++q) {
    if (dims[q] < 1) { set_error("grid extents must be >= 1"); return KR_BAD_ARG; }
    n *= dims[q];
    if (n > 0x7fffffffLL) { set_error("grid too large"); return KR_BAD_ARG; }
  }
  for (int q = 0; q < 2 + 4 * dim; ++q)
    if (!std::isfinite(coeffs[q])) { set_error("non-finite stencil coefficient"); return KR_BAD_ARG; }
  KR_API_BEGIN
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) { set_error("no CUDA device"); return KR_CUDA_ERROR; }
  if (device < 0 || device >= ndev) { set_error("device ordinal out of range"); return KR_BAD_ARG; }
  KR_CUDA(cudaSetDevice(device));
  auto h = std::make_unique<kr_op_s>();
  Operator& op = h->op;
  op.device = device;
  op.n = n;
  StencilSpec& A = op.stA;
  StencilSpec& AH = op.stAH;
  A.d = AH.d = dim;
  int64_t stride = 1, nnz = n;
  bool real = true;
  A.c = make_double2(coeffs[0], coeffs[1]);
  AH.c = make_double2(coeffs[0], -coeffs[1]);
  for (int q = 0; q < dim; ++q) {
    A.dims[q] = AH.dims[q] = dims[q];
    A.str[q] = AH.str[q] = stride;
    nnz += 2 * (n - n / dims[q]);
    stride *= dims[q];
    A.m[q] = make_double2(coeffs[2 + 4 * q], coeffs[3 + 4 * q]);
    A.p[q] = make_double2(coeffs[4 + 4 * q], coeffs[5 + 4 * q]);
    real = real && coeffs[3 + 4 * q] == 0.0 && coeffs[5 + 4 * q] == 0.0;
    // adjoint: (A^H)_{i, i+st} = conj(A_{i+st, i}) = conj(m), (A^H)_{i, i-st} = conj(p)
    AH.p[q] = make_double2(A.m[q].x, -A.m[q].y);
    AH.m[q] = make_double2(A.p[q].x, -A.p[q].y);
  }
  A.real = AH.real = real ? 1 : 0;
  op.nnz = nnz;
  op.real_offdiag = real ? 1 : 0;
  KR_CUDA(cudaMallocHost(&op.pinned, 4096));
  *out = h.release();
  return KR_OK;
  KR_API_END
}

kr_status kr_op_create_lattice4d(const int64_t* dims, const double* diag, double hop, const double* gamma,
                                 const double* links, int32_t device, kr_op* out) {
  if (!out) { set_error("out is NULL"); return KR_BAD_ARG; }
  *out = nullptr;
  if (!dims || !diag || !gamma || !links) { set_error("dims, diag, gamma and links must be non-NULL"); return KR_BAD_ARG; }
  int64_t sites = 1;
  for (int q = 0; q < 4; ++q) {
    if (dims[q] < 3) { set_error("every lattice extent must be >= 3"); return KR_BAD_ARG; }
    sites *= dims[q];
    if (sites * 12 > 0x7fffffffLL) { set_error("lattice too large"); return KR_BAD_ARG; }
  }
  if (!std::isfinite(hop) || !std::isfinite(diag[0]) || !std::isfinite(diag[1])) {
    set_error("non-finite diagonal or hop coefficient");
    return KR_BAD_ARG;
  }
  // each gamma_mu: one unit-modulus entry per row, off the diagonal, Hermitian
  int sig[4][4];
  double2 phi[4][4];
  for (int mu = 0; mu < 4; ++mu) {
    for (int r = 0; r < 4; ++r) {
      int found = -1;
      for (int col = 0; col < 4; ++col) {
        const double re = gamma[((mu * 4 + r) * 4 + col) * 2], im = gamma[((mu * 4 + r) * 4 + col) * 2 + 1];
        if (!std::isfinite(re) || !std::isfinite(im)) { set_error("non-finite gamma entry"); return KR_BAD_ARG; }
        const double m2 = re * re + im * im;
        if (m2 == 0.0) continue;
        if (found >= 0 || std::fabs(m2 - 1.0) > 1e-12) {
          set_error("gamma matrices must have one entry of modulus 1 per row");
          return KR_BAD_ARG;
        }
        found = col;
        phi[mu][r] = make_double2(re, im);
      }
      if (found < 0 || found == r) { set_error("gamma matrices need one off-diagonal entry per row"); return KR_BAD_ARG; }
      sig[mu][r] = found;
    }
    for (int r = 0; r < 4; ++r) {
      const int q = sig[mu][r];
      if (sig[mu][q] != r || std::fabs(phi[mu][q].x - phi[mu][r].x) > 1e-12 ||
          std::fabs(phi[mu][q].y + phi[mu][r].y) > 1e-12) {
        set_error("gamma matrices must be Hermitian");
        return KR_BAD_ARG;
      }
    }
  }
  const size_t nlink = (size_t)4 * sites * 9;
  for (size_t i = 0; i < 2 * nlink; ++i)
    if (!std::isfinite(links[i])) { set_error("non-finite link entry"); return KR_BAD_ARG; }
  KR_API_BEGIN
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) { set_error("no CUDA device"); return KR_CUDA_ERROR; }
  if (device < 0 || device >= ndev) { set_error("device ordinal out of range"); return KR_BAD_ARG; }
  KR_CUDA(cudaSetDevice(device));
  auto h = std::make_unique<kr_op_s>();
  Operator& op = h->op;
  op.device = device;
  op.n = 12 * sites;
  op.nnz = 49 * op.n;  // entries of the equivalent sparse matrix
  op.real_offdiag = 0;
  LatticeSpec& L = op.lat;
  L.on = 1;
  int64_t stride = 1;
  for (int q = 0; q < 4; ++q) {
    L.dims[q] = dims[q];
    L.str[q] = stride;
    stride *= dims[q];
  }
  L.diag = make_double2(diag[0], diag[1]);
  L.diagH = make_double2(diag[0], -diag[1]);
  // projector I + e gamma_mu: e = -1 forward, +1 backward for A; the opposite for A^H
  auto table = [&](int mu, double e) {
    LatHop t{};
    const int r0 = 0, s0 = sig[mu][0];
    int r1 = 1;
    while (r1 == r0 || r1 == s0) ++r1;
    const int reps[2] = {r0, r1};
    for (int k = 0; k < 2; ++k) {
      const int r = reps[k], q = sig[mu][r];
      t.rep[k] = r;
      t.sig[k] = q;
      t.pc[k] = make_double2(e * phi[mu][r].x, e * phi[mu][r].y);
      t.rsrc[r] = k;
      t.rc[r] = make_double2(1.0, 0.0);
      t.rsrc[q] = k;
      t.rc[q] = make_double2(e * phi[mu][q].x, e * phi[mu][q].y);
    }
    return t;
  };
  for (int mu = 0; mu < 4; ++mu) {
    L.hops[2 * mu] = table(mu, -1.0);
    L.hops[2 * mu + 1] = table(mu, +1.0);
    L.hopsH[2 * mu] = table(mu, +1.0);
    L.hopsH[2 * mu + 1] = table(mu, -1.0);
  }
  L.h_links.assign(links, links + 2 * nlink);
  for (double& v : L.h_links) v *= hop;
  build_operator_device(op, false);
  KR_CUDA(cudaMallocHost(&op.pinned, 4096));
  *out = h.release();
  return KR_OK;
  KR_API_END
}

kr_status kr_op_set_preconditioner(kr_op op, int32_t kind) {
  if (!op) { set_error("op is NULL"); return KR_BAD_ARG; }
  if (kind != KR_PREC_NONE && kind != KR_PREC_ILU0) { set_error("unknown preconditioner"); return KR_BAD_ARG; }
  if (kind == KR_PREC_ILU0 && (op->op.stA.d > 0 || op->op.lat.on)) {
    set_error("ILU(0) needs a CSR operator");
    return KR_UNSUPPORTED;
  }
  KR_API_BEGIN
  Operator& o = op->op;
  KR_CUDA(cudaSetDevice(o.device));
  KR_CUDA(cudaDeviceSynchronize());
  o.ilu.free_all();
  if (kind == KR_PREC_NONE) return KR_OK;
  const int r = build_ilu0(o);
  if (r != KR_OK) {
    o.ilu.free_all();
    set_error(r == KR_BREAKDOWN ? "ILU(0): zero pivot" : "ILU(0): a diagonal entry is missing or an entry repeated");
    return static_cast<kr_status>(r);
  }
  return KR_OK;
  KR_API_END
}

kr_status kr_op_apply_precond(kr_op op, int32_t adjoint, int32_t s, const double* V, double* Y, void* stream) {
  if (!op || !V || !Y || bad_s(s)) { set_error("invalid op, V, Y or s"); return KR_BAD_ARG; }
  if (!op->op.ilu.on) { set_error("no preconditioner set"); return KR_BAD_ARG; }
  KR_API_BEGIN
  Operator& o = op->op;
  KR_CUDA(cudaSetDevice(o.device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Workspace& ws = get_workspace(o, s, 24, 4, 0, 1);
  apply_ilu0(o, adjoint != 0, s, reinterpret_cast<const double2*>(V), reinterpret_cast<double2*>(Y),
             reinterpret_cast<double2*>(ws.blocks[3]), st);
  return KR_OK;
  KR_API_END
}

kr_status kr_op_update_values(kr_op op, const double* vals, int32_t on_device) {
  if (!op || (!vals && op->op.nnz > 0)) { set_error("op and vals must be non-NULL"); return KR_BAD_ARG; }
  if (op->op.stA.d > 0 || op->op.lat.on) { set_error("matrix-free operators have no CSR values"); return KR_UNSUPPORTED; }
  KR_API_BEGIN
  Operator& o = op->op;
  KR_CUDA(cudaSetDevice(o.device));
  if (on_device) {
    KR_CUDA(cudaDeviceSynchronize());
    KR_CUDA(cudaMemcpy(o.h_vals.data(), vals, sizeof(double) * 2 * o.nnz, cudaMemcpyDeviceToHost));
  } else {
    o.h_vals.assign(vals, vals + 2 * o.nnz);
  }
  rebuild_operator_values(o);
  return KR_OK;
  KR_API_END
}

kr_status kr_op_destroy(kr_op op) {
  if (!op) return KR_OK;
  KR_API_BEGIN
  delete op;
  return KR_OK;
  KR_API_END
}

kr_status kr_op_info(kr_op op, int64_t* n, int64_t* nnz, int32_t* real_offdiag) {
  if (!op) { set_error("op is NULL"); return KR_BAD_ARG; }
  if (n) *n = op->op.n;
  if (nnz) *nnz = op->op.nnz;
  if (real_offdiag) *real_offdiag = op->op.real_offdiag;
  return KR_OK;
}

extern "C++" {
template <typename T>
static kr_status apply_impl(kr_op op, int32_t adjoint, int32_t s, const T* V, T* Y, const T* U, int32_t kind,
                            double* out, void* stream) {
  if (!op || !V || bad_s(s)) { set_error("invalid op, V or s"); return KR_BAD_ARG; }
  if (kind && (!out || (kind != KR_RED_NORM2 && !U))) { set_error("reduction needs U and out"); return KR_BAD_ARG; }
  if (kind < 0 || kind > KR_RED_NORM2) { set_error("unknown reduction kind"); return KR_BAD_ARG; }
  if (!kind && !Y) { set_error("Y is NULL"); return KR_BAD_ARG; }
  KR_API_BEGIN
  Operator& o = op->op;
  KR_CUDA(cudaSetDevice(o.device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (sizeof(T) == 4) build_operator_device(o, true);
  Workspace& ws = get_workspace(o, s, sizeof(C2<T>), 0, 0, 1);
  DevState h{};
  KR_CUDA(cudaMemcpyAsync(ws.st, &h, sizeof(DevState), cudaMemcpyHostToDevice, st));
  SpmmArgs<T> a = op_spmm_args<T>(o, adjoint != 0, s);
  a.V = reinterpret_cast<const C2<T>*>(V);
  a.Y = reinterpret_cast<C2<T>*>(Y);
  a.ay = 1.0;
  RedSet rs{};
  rs.partials = ws.partials;
  if (kind) {
    rs.nred = 1;
    rs.r[0].kind = kind;
    rs.r[0].ureg = -1;
    rs.r[0].U = U;
    rs.nslots = kind == KR_RED_GRAM ? s * s : 1;
  }
  const int grid = launch_spmm<T>(a, rs, row_grid(o.n, s), nullptr, st);
  if (kind) launch_reduce<T>(ws.partials, grid, rs.nslots, reinterpret_cast<double2*>(out), nullptr, st);
  return KR_OK;
  KR_API_END
}
}  // extern "C++"

kr_status kr_op_apply(kr_op op, int32_t adjoint, int32_t s, const double* V, double* Y, void* stream) {
  if (!Y) { set_error("Y is NULL"); return KR_BAD_ARG; }
  return apply_impl<double>(op, adjoint, s, V, Y, nullptr, 0, nullptr, stream);
}

kr_status kr_op_apply_reduce(kr_op op, int32_t adjoint, int32_t s, const double* V, double* Y, const double* U,
                             int32_t kind, double* out, void* stream) {
  if (kind < KR_RED_GRAM || kind > KR_RED_NORM2) { set_error("unknown reduction kind"); return KR_BAD_ARG; }
  return apply_impl<double>(op, adjoint, s, V, Y, U, kind, out, stream);
}

kr_status kr_op_apply_reduce_c64(kr_op op, int32_t adjoint, int32_t s, const float* V, float* Y, const float* U,
                                 int32_t kind, double* out, void* stream) {
  return apply_impl<float>(op, adjoint, s, V, Y, U, kind, out, stream);
}

extern "C++" {
template <typename T>
static kr_status block_reduce_impl(int64_t n, int32_t s, const T* U, const T* Y, int32_t kind, double* out,
                                   void* stream) {
  if (n <= 0 || bad_s(s) || !Y || !out || (kind != KR_RED_NORM2 && !U) || kind < KR_RED_GRAM || kind > KR_RED_NORM2) {
    set_error("invalid arguments");
    return KR_BAD_ARG;
  }
  KR_API_BEGIN
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Workspace& ws = scratch_ws(n, s);
  LinArgs a{};
  a.n = n;
  a.s = s;
  a.nout = 1;
  a.o[0].nterm = 1;
  a.o[0].t[0].src_kind = SRC_BLOCK;
  a.o[0].t[0].src = Y;
  a.o[0].t[0].coef_kind = COEF_ONE;
  RedSet rs{};
  rs.partials = ws.partials;
  rs.nred = 1;
  rs.r[0].kind = kind;
  rs.r[0].ysrc = 0;
  rs.r[0].ureg = -1;
  rs.r[0].U = U;
  rs.nslots = kind == KR_RED_GRAM ? s * s : 1;
  const int G = threads_per_row(s);
  if (kind == KR_RED_GRAM && ng_capacity(G) < 1) { set_error("Gram with s > 16 not fused here"); return KR_UNSUPPORTED; }
  const int grid = launch_lincomb<T>(a, rs, row_grid(n, s), nullptr, st);
  launch_reduce<T>(ws.partials, grid, rs.nslots, reinterpret_cast<double2*>(out), nullptr, st);
  return KR_OK;
  KR_API_END
}
}  // extern "C++"

kr_status kr_block_reduce(int64_t n, int32_t s, const double* U, const double* Y, int32_t kind, double* out,
                          void* stream) {
  return block_reduce_impl<double>(n, s, U, Y, kind, out, stream);
}

kr_status kr_block_reduce_c64(int64_t n, int32_t s, const float* U, const float* Y, int32_t kind, double* out,
                              void* stream) {
  return block_reduce_impl<float>(n, s, U, Y, kind, out, stream);
}

kr_status kr_thin_qr(int64_t n, int32_t s, const double* Z, double* Q, double* S, void* stream) {
  if (n <= 0 || bad_s(s) || !Z || !Q || !S) { set_error("invalid arguments"); return KR_BAD_ARG; }
  if (s > 16) { set_error("kr_thin_qr supports s <= 16"); return KR_UNSUPPORTED; }
  KR_API_BEGIN
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Workspace& ws = scratch_ws(n, s);
  if (Q != Z) KR_CUDA(cudaMemcpyAsync(Q, Z, sizeof(double2) * n * s, cudaMemcpyDeviceToDevice, st));
  DevState h{};
  h.maxit = 1;
  KR_CUDA(cudaMemcpyAsync(ws.st, &h, sizeof(DevState), cudaMemcpyHostToDevice, st));
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  int dev = 0;
  KR_CUDA(cudaGetDevice(&dev));
  Operator& o = g_scratch[dev]->op;
  standalone_qr(o, ws, n, s, Q, st);
  KR_CUDA(cudaMemcpyAsync(S, ws.arena + (size_t)SL_QR_S * kSlotElems, sizeof(double2) * s * s,
                          cudaMemcpyDeviceToDevice, st));
  DevState back{};
  KR_CUDA(cudaMemcpyAsync(&back, ws.st, sizeof(DevState), cudaMemcpyDeviceToHost, st));
  KR_CUDA(cudaStreamSynchronize(st));
  if (back.done && back.status == 1) { set_error("rank-deficient block"); return KR_BREAKDOWN; }
  return KR_OK;
  KR_API_END
}

static kr_status solve_impl(kr_op op, int32_t method, int32_t s, const double* B, double* X, const kr_options* optp,
                            void* stream, kr_info* info, bool adjoint) {
  if (!op || !B || !X) { set_error("op, B and X must be non-NULL"); return KR_BAD_ARG; }
  if (method < 0 || method >= KRM_COUNT) { set_error("unknown method"); return KR_BAD_ARG; }
  if (bad_s(s)) { set_error("s must be in [1, 32]"); return KR_UNSUPPORTED; }
  kr_options opt;
  if (optp) opt = *optp; else kr_options_default(&opt);
  if (!(opt.tol >= 0.0) || opt.maxit < 0) { set_error("tol must be >= 0 and maxit >= 0"); return KR_BAD_ARG; }
  if (opt.shadow_mode == KR_SHADOW_USER && !opt.shadow) { set_error("user shadow is NULL"); return KR_BAD_ARG; }
  if (opt.precision != KR_FP64 && opt.precision != KR_FP32_REFINE) { set_error("unknown precision"); return KR_BAD_ARG; }
  if (opt.graphs < 0 || opt.graphs > 2) { set_error("graphs must be 0 (automatic), 1 (on) or 2 (off)"); return KR_BAD_ARG; }
  if (op->op.ilu.on && (adjoint || opt.precision != KR_FP64)) {
    set_error("the ILU(0) preconditioner is supported for kr_solve in FP64");
    return KR_UNSUPPORTED;
  }
  if (opt.orthonormalize_B != 0 && opt.orthonormalize_B != 1) { set_error("orthonormalize_B must be 0 or 1"); return KR_BAD_ARG; }
  if (opt.deterministic != 0 && opt.deterministic != 1) { set_error("deterministic must be 0 or 1"); return KR_BAD_ARG; }
  if (opt.orthonormalize_B && op->op.ilu.on) {
    set_error("orthonormalize_B is not supported together with a preconditioner");
    return KR_UNSUPPORTED;
  }
  KR_API_BEGIN
  Operator& o = op->op;
  KR_CUDA(cudaSetDevice(o.device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t bytes = sizeof(double2) * (size_t)o.n * s;
  const double* dB = B;
  double* dX = X;
  void *tB = nullptr, *tX = nullptr;
  struct Guard {
    void** a; void** b;
    ~Guard() { if (*a) cudaFree(*a); if (*b) cudaFree(*b); }
  } guard{&tB, &tX};
  if (opt.host_buffers) {
    KR_CUDA(cudaMalloc(&tB, bytes));
    KR_CUDA(cudaMalloc(&tX, bytes));
    KR_CUDA(cudaMemcpyAsync(tB, B, bytes, cudaMemcpyHostToDevice, st));
    KR_CUDA(cudaMemcpyAsync(tX, X, bytes, cudaMemcpyHostToDevice, st));
    dB = reinterpret_cast<const double*>(tB);
    dX = reinterpret_cast<double*>(tX);
  }
  SolveIn in;
  in.tol = opt.tol;
  in.maxit = opt.maxit;
  in.check_every = opt.check_every > 0 ? opt.check_every : 8;
  in.shadow_mode = opt.shadow_mode;
  in.shadow = opt.shadow;
  in.time_limit_s = opt.time_limit_s;
  // automatic graphs: small problems, and every preconditioned solve (one launch per level of the
  // triangular solves makes those iterations launch-bound)
  in.graphs = (opt.graphs == 1 || (opt.graphs == 0 && ((int64_t)o.n * s <= ((int64_t)1 << 22) || o.ilu.on))) ? 1 : 0;
  kr_info inf{};
  // orthonormalised right-hand sides (Sec. 5): R_0 = B - A X_0 = Q S, solve A Y = Q from Y = 0,
  // then X = X_0 + Y S; the iteration and its history are those of the system with Q
  const double* uB = dB;
  double* uX = dX;
  double ortho_res0 = 0.0;
  bool ortho_skip = false;
  if (opt.orthonormalize_B) {
    void *Qp = nullptr, *Yp = nullptr;
    ortho_res0 = orthonormal_rhs(o, s, dB, dX, &Qp, &Yp, st, adjoint);
    if (ortho_res0 < 0.0) {
      inf.status = KR_BREAKDOWN;
      inf.relres_recursive = inf.relres_true = 1.0;
      if (opt.history) opt.history[0] = 1.0;
      set_error("orthonormalize_B: the initial residual block is numerically rank deficient");
      ortho_skip = true;
    } else if (!(ortho_res0 > 0.0)) {  // X_0 solves the system (0) or the residual is not finite
      inf.status = ortho_res0 == 0.0 ? KR_OK : KR_NAN;
      inf.relres_true = inf.relres_recursive = ortho_res0 == 0.0 ? 0.0 : ortho_res0;
      if (opt.history) opt.history[0] = 1.0;
      ortho_skip = true;
    }
    dB = reinterpret_cast<const double*>(Qp);
    dX = reinterpret_cast<double*>(Yp);
  }
  if (ortho_skip) {
    // nothing to iterate
  } else if (opt.precision == KR_FP64 && o.ilu.on) {
    // right preconditioning: A M^{-1} Y = B - A X0 from Y = 0, then X = X0 + M^{-1} Y
    Workspace& rw = get_workspace(o, s, 24, 4, 0, 1);
    void *R0 = rw.blocks[0], *Yb = rw.blocks[1], *Tb = rw.blocks[2];
    const int64_t cnt = o.n * (int64_t)s;
    const double res0 = true_residual(o, s, dB, dX, R0, st, false);
    KR_CUDA(cudaMemsetAsync(Yb, 0, sizeof(double2) * cnt, st));
    SolveIn pin = in;
    pin.precond = 1;
    SolveOut so = run_solve<double>(o, method, s, R0, Yb, pin, st, false);
    apply_ilu0(o, false, s, reinterpret_cast<const double2*>(Yb), reinterpret_cast<double2*>(Yb),
               reinterpret_cast<double2*>(Tb), st);
    {
      ProfToken tk = prof_begin(KC_OTHER, st);
      add_c128_kernel<<<grid1d(cnt), 256, 0, st>>>(reinterpret_cast<double2*>(dX),
                                                    reinterpret_cast<const double2*>(Yb), cnt);
      KR_CUDA(cudaGetLastError());
      prof_end(tk, st, 2.0 * cnt, 48.0 * cnt);
    }
    inf.iters = so.iters;
    inf.matvecs = so.matvecs;
    inf.status = so.status;
    inf.relres_recursive = so.relres_recursive;
    const double tr = true_residual(o, s, dB, dX, nullptr, st, false);
    inf.relres_true = res0 > 0 ? tr / res0 : tr;
    if (opt.history)
      for (size_t k = 0; k < so.hist.size() && (int)k <= opt.maxit; ++k) opt.history[k] = so.hist[k];
  } else if (opt.precision == KR_FP64) {
    SolveOut so = run_solve<double>(o, method, s, dB, dX, in, st, adjoint);
    inf.iters = so.iters;
    inf.matvecs = so.matvecs;
    inf.status = so.status;
    inf.relres_recursive = so.relres_recursive;
    const double tr = true_residual(o, s, dB, dX, nullptr, st, adjoint);
    inf.relres_true = so.res0 > 0 ? tr / so.res0 : tr;
    if (opt.history)
      for (size_t k = 0; k < so.hist.size() && (int)k <= opt.maxit; ++k) opt.history[k] = so.hist[k];
  } else {
    // defect correction: R = B - A X in FP64; inner complex64 solve of A D = R; X += D
    build_operator_device(o, true);
    Workspace& rw = get_workspace(o, s, 24, 4, 0, 1);  // R64, R32, D32, X backup (sized for complex128)
    void *R64 = rw.blocks[0], *R32 = rw.blocks[1], *D32 = rw.blocks[2], *Xkeep = rw.blocks[3];
    const int64_t cnt = o.n * (int64_t)s;
    double res0 = true_residual(o, s, dB, dX, R64, st, adjoint);
    double res = res0;
    SolveIn inner = in;
    inner.tol = opt.inner_tol > 0 ? opt.inner_tol : 1e-4;
    inner.shadow_mode = opt.shadow_mode == KR_SHADOW_USER ? KR_SHADOW_DEFAULT : opt.shadow_mode;
    const int max_outer = opt.max_outer > 0 ? opt.max_outer : 30;
    int status = KR_MAXIT, outer = 0;
    bool fallback = false;
    inner.stall = 100;
    if (opt.history) opt.history[0] = 1.0;
    if (res0 == 0.0) status = KR_OK;
    else if (!std::isfinite(res0)) status = KR_NAN;
    while (status == KR_MAXIT && outer < max_outer && inf.iters < opt.maxit) {
      inner.maxit = opt.maxit - inf.iters;
      {
        ProfToken tk = prof_begin(KC_OTHER, st);
        to_c64_kernel<<<grid1d(cnt), 256, 0, st>>>(reinterpret_cast<const double2*>(R64),
                                                    reinterpret_cast<float2*>(R32), cnt);
        KR_CUDA(cudaGetLastError());
        prof_end(tk, st, 0.0, 24.0 * cnt);
      }
      KR_CUDA(cudaMemsetAsync(D32, 0, sizeof(float2) * cnt, st));
      SolveOut so = run_solve<float>(o, method, s, R32, D32, inner, st, adjoint);
      inf.iters += so.iters;
      inf.matvecs += so.matvecs;
      KR_CUDA(cudaMemcpyAsync(Xkeep, dX, bytes, cudaMemcpyDeviceToDevice, st));
      {
        ProfToken tk = prof_begin(KC_OTHER, st);
        add_c64_kernel<<<grid1d(cnt), 256, 0, st>>>(reinterpret_cast<double2*>(dX),
                                                     reinterpret_cast<const float2*>(D32), cnt);
        KR_CUDA(cudaGetLastError());
        prof_end(tk, st, 2.0 * cnt, 40.0 * cnt);
      }
      const double prev = res;
      res = true_residual(o, s, dB, dX, R64, st, adjoint);
      ++outer;
      if (opt.history && outer <= opt.maxit) opt.history[outer] = res / res0;
      if (!std::isfinite(res) || res >= prev) {
        // the complex64 inner solve did not reduce the FP64 residual (for the block methods the
        // FP32-accumulated s x s Gram products can make it diverge): restore X, finish in FP64
        KR_CUDA(cudaMemcpyAsync(dX, Xkeep, bytes, cudaMemcpyDeviceToDevice, st));
        res = prev;
        fallback = true;
        break;
      }
      if (res <= opt.tol * res0) status = KR_OK;
      else if (res > 1e8 * res0) status = KR_DIVERGED;
    }
    if (fallback && inf.iters < opt.maxit) {
      // finish in FP64 from the current X, to the caller's tolerance relative to the first residual
      SolveIn in64 = in;
      in64.maxit = opt.maxit - inf.iters;
      in64.tol = res > 0 ? opt.tol * res0 / res : opt.tol;
      SolveOut so = run_solve<double>(o, method, s, dB, dX, in64, st, adjoint);
      inf.iters += so.iters;
      inf.matvecs += so.matvecs;
      inf.fp64_iters = so.iters;
      res = true_residual(o, s, dB, dX, R64, st, adjoint);
      status = res <= opt.tol * res0 ? KR_OK : (so.status == KR_OK ? KR_MAXIT : so.status);
      if (opt.history && outer + 1 <= opt.maxit) opt.history[outer + 1] = res / res0;
      ++outer;
    } else if (fallback) {
      status = KR_MAXIT;
    }
    inf.outer_iters = outer;
    inf.status = status;
    inf.relres_recursive = res0 > 0 ? res / res0 : res;
    inf.relres_true = inf.relres_recursive;
  }
  if (opt.orthonormalize_B && !ortho_skip) {
    add_back_rhs_factor(o, s, uX, st);
    const double tr = true_residual(o, s, uB, uX, nullptr, st, adjoint);
    inf.relres_true = tr / ortho_res0;
  }
  if (inf.status == KR_MAXIT && inf.relres_true > 1.0) inf.status = KR_DIVERGED;
  if (!std::isfinite(inf.relres_true) && inf.status != KR_BREAKDOWN) inf.status = KR_NAN;
  inf.breakdown_iter = inf.status == KR_BREAKDOWN ? inf.iters + 1 : 0;
  if (opt.host_buffers) {
    KR_CUDA(cudaMemcpyAsync(X, tX, bytes, cudaMemcpyDeviceToHost, st));
    KR_CUDA(cudaStreamSynchronize(st));
  }
  if (info) *info = inf;
  return static_cast<kr_status>(inf.status);
  KR_API_END
}

kr_status kr_solve(kr_op op, int32_t method, int32_t s, const double* B, double* X, const kr_options* opt,
                   void* stream, kr_info* info) {
  return solve_impl(op, method, s, B, X, opt, stream, info, false);
}

kr_status kr_adjoint_solve(kr_op op, int32_t method, int32_t s, const double* G, double* Lambda,
                           const kr_options* opt, void* stream, kr_info* info) {
  return solve_impl(op, method, s, G, Lambda, opt, stream, info, true);
}

kr_status kr_grad_values(kr_op op, int32_t s, const double* Lambda, const double* X, double* dvals, void* stream) {
  if (!op || !Lambda || !X || !dvals || bad_s(s)) { set_error("invalid arguments"); return KR_BAD_ARG; }
  if (op->op.stA.d > 0 || op->op.lat.on) { set_error("gradient on the CSR pattern needs a CSR operator"); return KR_UNSUPPORTED; }
  KR_API_BEGIN
  Operator& o = op->op;
  KR_CUDA(cudaSetDevice(o.device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  ensure_orig_pattern(o);
  const int G = threads_per_row(s);
  const int grid = row_grid(o.n, s);
  const auto* L = reinterpret_cast<const double2*>(Lambda);
  const auto* Xp = reinterpret_cast<const double2*>(X);
  auto* dv = reinterpret_cast<double2*>(dvals);
  ProfToken tk = prof_begin(KC_OTHER, st);
  switch (G) {
    case 1: grad_kernel<1><<<grid, 256, 0, st>>>(o.n, s, o.orig_rowptr, o.orig_colidx, L, Xp, dv); break;
    case 2: grad_kernel<2><<<grid, 256, 0, st>>>(o.n, s, o.orig_rowptr, o.orig_colidx, L, Xp, dv); break;
    case 4: grad_kernel<4><<<grid, 256, 0, st>>>(o.n, s, o.orig_rowptr, o.orig_colidx, L, Xp, dv); break;
    case 8: grad_kernel<8><<<grid, 256, 0, st>>>(o.n, s, o.orig_rowptr, o.orig_colidx, L, Xp, dv); break;
    case 16: grad_kernel<16><<<grid, 256, 0, st>>>(o.n, s, o.orig_rowptr, o.orig_colidx, L, Xp, dv); break;
    default: grad_kernel<32><<<grid, 256, 0, st>>>(o.n, s, o.orig_rowptr, o.orig_colidx, L, Xp, dv); break;
  }
  KR_CUDA(cudaGetLastError());
  prof_end(tk, st, 8.0 * s * o.nnz, 12.0 * o.nnz + 8.0 * (o.n + 1) + 32.0 * o.n * s);
  return KR_OK;
  KR_API_END
}

}  // extern "C"
