// Host-side declarations shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "kr_rows.cuh"

namespace kr {

// ----- errors -------------------------------------------------------------------------
void set_error(const std::string& msg);
const char* get_error();

struct CudaError {
  cudaError_t code;
  std::string where;
};

#define KR_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e__ = (call);                                                           \
    if (e__ != cudaSuccess) throw ::kr::CudaError{e__, std::string(#call) + " @ " +     \
                                                        std::string(__FILE__) + ":" +   \
                                                        std::to_string(__LINE__)};      \
  } while (0)

// ----- launch geometry ----------------------------------------------------------------
int sm_count();                       // SMs of the current device
inline int threads_per_row(int s) {   // G: smallest power of two >= s
  int g = 1;
  while (g < s) g <<= 1;
  return g;
}
inline int ng_capacity(int G) { return G <= 8 ? 2 : (G == 16 ? 1 : 0); }
constexpr int kCtasPerSm = kCtasPerSmRows;
inline int max_row_grid() { return sm_count() * kCtasPerSm; }
inline int row_grid(int64_t n, int s) {
  const int G = threads_per_row(s);
  const int64_t rows_per_cta = (int64_t)(kThreads / 32) * (32 / G);
  int64_t g = (n + rows_per_cta - 1) / rows_per_cta;
  if (g < 1) g = 1;
  const int64_t cap = max_row_grid();
  return (int)(g < cap ? g : cap);
}

// complex64 row kernels on column pairs (kr_set_column_pairs; on by default)
bool pair_kernels_enabled();
void set_pair_kernels(bool on);
// Gl-/eGl-BiCG with alpha from the adjoint product and the update fused with the product
// (kr_set_fused_products; on by default)
bool fused_products_enabled();
void set_fused_products(bool on);
// complex64 CSR products on TMA-staged row tiles (kr_set_tile_kernels; on by default)
bool tile_kernels_enabled();
void set_tile_kernels(bool on);
// rows per thread of the matrix-free lattice product (4: (site, colour) units, 12: whole sites)
int lattice_rows_per_thread(size_t real_bytes);
void set_lattice_rows_per_thread(int rows);

// ----- row kernels (kr_rows_f64.cu / kr_rows_f32.cu) -------------------------------------
// Both return the grid actually launched (the requested grid clamped to the resident CTAs);
// reductions of the launch's partial records must use that count.
template <typename T>
int launch_spmm(const SpmmArgs<T>& a, const RedSet& rs, int grid, const int* done, cudaStream_t st);
template <typename T>
int launch_lincomb(const LinArgs& a, const RedSet& rs, int grid, const int* done, cudaStream_t st);
template <typename T>
void launch_reduce(const void* partials, int nparts, int nslots, double2* out, const int* done, cudaStream_t st);
// row-local combination with SRC_SPMM terms: the product of sp formed in the same pass
template <typename T>
int launch_lincomb_spmm(const LinArgs& a, const RedSet& rs, const SpmmArgs<T>& sp, int grid, const int* done,
                        cudaStream_t st);

// number of GRAM reductions in a set
inline int count_grams(const RedSet& rs) {
  int k = 0;
  for (int i = 0; i < rs.nred; ++i)
    if (rs.r[i].kind == RED_GRAM) ++k;
  return k;
}

}  // namespace kr
