// Host launchers for the row kernels, instantiated once per element type.
#pragma once

#include "kr_internal.h"
#include "kr_rows_impl.cuh"

namespace kr {

constexpr int kMaxDynSmem = 200 * 1024;

template <typename K>
static void allow_smem(K kernel, bool& flag) {
  if (!flag) {
    KR_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem));
    flag = true;
  }
}

template <typename T, int G, int NG>
static void spmm_go(const SpmmArgs<T>& a, const RedSet& rs, int grid, const int* done, cudaStream_t st) {
  static bool attr = false;
  allow_smem(spmm_kernel<T, G, NG>, attr);
  const size_t smem = rs.nred > 0 ? (size_t)(kThreads / 32) * rs.nslots * sizeof(C2<T>) : 0;
  if (smem > (size_t)kMaxDynSmem) throw CudaError{cudaErrorInvalidValue, "spmm: too many reduction slots"};
  spmm_kernel<T, G, NG><<<grid, kThreads, smem, st>>>(a, rs, done);
  KR_CUDA(cudaGetLastError());
}

template <typename T, int G>
static void spmm_ng(int ng, const SpmmArgs<T>& a, const RedSet& rs, int grid, const int* done, cudaStream_t st) {
  if (ng == 0) return spmm_go<T, G, 0>(a, rs, grid, done, st);
  if constexpr (NGCap<1, G>::ok) {
    if (ng == 1) return spmm_go<T, G, 1>(a, rs, grid, done, st);
  }
  if constexpr (NGCap<2, G>::ok) {
    if (ng == 2) return spmm_go<T, G, 2>(a, rs, grid, done, st);
  }
  throw CudaError{cudaErrorInvalidValue, "spmm: fused Gram count exceeds the register budget"};
}

template <typename T>
void launch_spmm(const SpmmArgs<T>& a, const RedSet& rs, int grid, const int* done, cudaStream_t st) {
  const int G = threads_per_row(a.s);
  const int ng = count_grams(rs);
  switch (G) {
    case 1: return spmm_ng<T, 1>(ng, a, rs, grid, done, st);
    case 2: return spmm_ng<T, 2>(ng, a, rs, grid, done, st);
    case 4: return spmm_ng<T, 4>(ng, a, rs, grid, done, st);
    case 8: return spmm_ng<T, 8>(ng, a, rs, grid, done, st);
    case 16: return spmm_ng<T, 16>(ng, a, rs, grid, done, st);
    case 32: return spmm_ng<T, 32>(ng, a, rs, grid, done, st);
  }
  throw CudaError{cudaErrorInvalidValue, "spmm: s out of range"};
}

template <typename T, int G, int NG>
static void lin_go(const LinArgs& a, const RedSet& rs, int grid, const int* done, cudaStream_t st) {
  static bool attr = false;
  allow_smem(lincomb_kernel<T, G, NG>, attr);
  size_t smem = (size_t)a.nmat * a.s * a.s * sizeof(C2<T>);
  if (rs.nred > 0) smem += (size_t)(kThreads / 32) * rs.nslots * sizeof(C2<T>);
  if (smem > (size_t)kMaxDynSmem) throw CudaError{cudaErrorInvalidValue, "lincomb: shared memory budget exceeded"};
  lincomb_kernel<T, G, NG><<<grid, kThreads, smem, st>>>(a, rs, done);
  KR_CUDA(cudaGetLastError());
}

template <typename T, int G>
static void lin_ng(int ng, const LinArgs& a, const RedSet& rs, int grid, const int* done, cudaStream_t st) {
  if (ng == 0) return lin_go<T, G, 0>(a, rs, grid, done, st);
  if constexpr (NGCap<1, G>::ok) {
    if (ng == 1) return lin_go<T, G, 1>(a, rs, grid, done, st);
  }
  if constexpr (NGCap<2, G>::ok) {
    if (ng == 2) return lin_go<T, G, 2>(a, rs, grid, done, st);
  }
  throw CudaError{cudaErrorInvalidValue, "lincomb: fused Gram count exceeds the register budget"};
}

template <typename T>
void launch_lincomb(const LinArgs& a, const RedSet& rs, int grid, const int* done, cudaStream_t st) {
  const int G = threads_per_row(a.s);
  const int ng = count_grams(rs);
  switch (G) {
    case 1: return lin_ng<T, 1>(ng, a, rs, grid, done, st);
    case 2: return lin_ng<T, 2>(ng, a, rs, grid, done, st);
    case 4: return lin_ng<T, 4>(ng, a, rs, grid, done, st);
    case 8: return lin_ng<T, 8>(ng, a, rs, grid, done, st);
    case 16: return lin_ng<T, 16>(ng, a, rs, grid, done, st);
    case 32: return lin_ng<T, 32>(ng, a, rs, grid, done, st);
  }
  throw CudaError{cudaErrorInvalidValue, "lincomb: s out of range"};
}

template <typename T>
void launch_reduce(const void* partials, int nparts, int nslots, double2* out, const int* done, cudaStream_t st) {
  if (nslots <= 0) return;
  reduce_slots_kernel<T><<<nslots, kThreads, 0, st>>>(reinterpret_cast<const C2<T>*>(partials), nparts, nslots,
                                                       out, done);
  KR_CUDA(cudaGetLastError());
}

#define KR_INSTANTIATE_ROWS(T)                                                                               \
  template void launch_spmm<T>(const SpmmArgs<T>&, const RedSet&, int, const int*, cudaStream_t);           \
  template void launch_lincomb<T>(const LinArgs&, const RedSet&, int, const int*, cudaStream_t);            \
  template void launch_reduce<T>(const void*, int, int, double2*, const int*, cudaStream_t);

}  // namespace kr
