// Host launcher of the row-local combinations with a fused sparse product (SRC_SPMM terms),
// instantiated per element type in kr_rowsp_f64.cu / kr_rowsp_f32.cu (separate units keep the
// build parallel).
#pragma once

#include "kr_rows_launch.cuh"

namespace kr {

template <typename T, int G, int NG>
static void linsp_go(const LinArgs& a, const RedSet& rs, const SpmmArgs<T>& sp, int& grid, const int* done,
                     cudaStream_t st) {
  static std::atomic<uint64_t> attr{0};
  allow_smem(lincomb_spmm_kernel<T, G, NG>, attr);
  size_t smem = (size_t)a.nmat * a.s * a.s * sizeof(C2<T>);
  if (rs.nred > 0) smem += (size_t)(kThreads / 32) * rs.nslots * sizeof(C2<T>);
  if (smem > (size_t)kMaxDynSmem) throw CudaError{cudaErrorInvalidValue, "lincomb: shared memory budget exceeded"};
  thread_local std::unordered_map<size_t, int> occ;
  grid = resident_grid(lincomb_spmm_kernel<T, G, NG>, smem, grid, occ);
  lincomb_spmm_kernel<T, G, NG><<<grid, kThreads, smem, st>>>(a, rs, sp, done);
  KR_CUDA(cudaGetLastError());
}

template <typename T, int G>
static void linsp_ng(int ng, const LinArgs& a, const RedSet& rs, const SpmmArgs<T>& sp, int& grid, const int* done,
                     cudaStream_t st) {
  if (ng == 0) return linsp_go<T, G, 0>(a, rs, sp, grid, done, st);
  if constexpr (NGCap<1, G>::ok) {
    if (ng == 1) return linsp_go<T, G, 1>(a, rs, sp, grid, done, st);
  }
  throw CudaError{cudaErrorInvalidValue, "lincomb with product: fused Gram count exceeds the register budget"};
}

template <int GP>
static void lin2sp_go(const LinArgs& a, const RedSet& rs, const SpmmArgs<float>& sp, int& grid, const int* done,
                      cudaStream_t st, size_t smem) {
  thread_local std::unordered_map<size_t, int> occ;
  grid = resident_grid(lincomb2_spmm_kernel<GP>, smem, grid, occ);
  lincomb2_spmm_kernel<GP><<<grid, kThreads, smem, st>>>(a, rs, sp, done);
  KR_CUDA(cudaGetLastError());
}

// Row-local combination whose terms include the sparse product of `sp` (SRC_SPMM terms), formed
// in the same pass.  No output may be the product's operand sp.V (its rows are gathered by other
// threads while outputs are stored).  At most one fused Gram.
template <typename T>
int launch_lincomb_spmm(const LinArgs& a_in, const RedSet& rs_in, const SpmmArgs<T>& sp, int grid, const int* done,
                        cudaStream_t st) {
  LinArgs a = a_in;
  RedSet rs = rs_in;
  resolve_sources(a, rs);
  for (int o = 0; o < a.nout; ++o)
    if (a.o[o].dst != nullptr && a.o[o].dst == static_cast<const void*>(sp.V))
      throw CudaError{cudaErrorInvalidValue, "lincomb with product: an output overwrites the product's operand"};
  if (sp.lat || sp.s != a.s) throw CudaError{cudaErrorInvalidValue, "lincomb with product: unsupported operand"};
  ProfToken tk = prof_begin(sizeof(T) == 4 ? KC_LINCOMB32 : KC_LINCOMB, st);
  const int ng = count_grams(rs);
  bool pairs = false;
  if constexpr (sizeof(T) == 4) {
    pairs = pair_kernels_enabled() && pair_ok_lin(a, rs) && aligned16(sp.V);
    if (pairs) {
      size_t smem = (size_t)a.nmat * a.s * sizeof(float2);
      if (rs.nred > 0) smem += (size_t)(kThreads / 32) * rs.nslots * sizeof(float2);
      if (smem > 48 * 1024) throw CudaError{cudaErrorInvalidValue, "lincomb: shared memory budget exceeded"};
      switch (threads_per_row(a.s / 2)) {
        case 1: lin2sp_go<1>(a, rs, sp, grid, done, st, smem); break;
        case 2: lin2sp_go<2>(a, rs, sp, grid, done, st, smem); break;
        case 4: lin2sp_go<4>(a, rs, sp, grid, done, st, smem); break;
        case 8: lin2sp_go<8>(a, rs, sp, grid, done, st, smem); break;
        default: lin2sp_go<16>(a, rs, sp, grid, done, st, smem); break;
      }
    }
  }
  if (!pairs) switch (threads_per_row(a.s)) {
    case 1: linsp_ng<T, 1>(ng, a, rs, sp, grid, done, st); break;
    case 2: linsp_ng<T, 2>(ng, a, rs, sp, grid, done, st); break;
    case 4: linsp_ng<T, 4>(ng, a, rs, sp, grid, done, st); break;
    case 8: linsp_ng<T, 8>(ng, a, rs, sp, grid, done, st); break;
    case 16: linsp_ng<T, 16>(ng, a, rs, sp, grid, done, st); break;
    case 32: linsp_ng<T, 32>(ng, a, rs, sp, grid, done, st); break;
    default: throw CudaError{cudaErrorInvalidValue, "lincomb with product: s out of range"};
  }
  double f = 0.0, b = 0.0;
  const double E = sizeof(C2<T>);
  lin_account(a, rs, E, f, b);
  // the product: matrix (or nothing for a stencil) and its operand, read once; its flops
  const double n = (double)sp.n, s = (double)sp.s, nnz = (double)sp.nnz;
  f += sp.split ? s * (4.0 * nnz + 6.0 * n) : s * 8.0 * nnz;
  if (sp.nst > 0 && !sp.sreal) f = s * 8.0 * (nnz + n);
  if (sp.nst == 0) b += 8.0 * (n + 1) + 4.0 * nnz + (sp.split ? sizeof(T) * nnz + E * n : E * nnz);
  bool operand_counted = false;  // the product's operand is often also a term (X += alpha P)
  for (int o = 0; o < a.nout; ++o)
    for (int t = 0; t < a.o[o].nterm; ++t)
      operand_counted = operand_counted ||
                        (a.o[o].t[t].src_kind == SRC_BLOCK && a.o[o].t[t].src == static_cast<const void*>(sp.V));
  if (!operand_counted) b += E * n * s;
  prof_end(tk, st, f, b);
  return grid;
}


#define KR_INSTANTIATE_ROWSP(T)                                                                               \
  template int launch_lincomb_spmm<T>(const LinArgs&, const RedSet&, const SpmmArgs<T>&, int, const int*,   \
                                      cudaStream_t);

}  // namespace kr
