// complex64 instantiation of the row kernels
#include <string>

#include "../../include/kr.h"
#include "kr_rows_launch.cuh"
namespace kr {
KR_INSTANTIATE_ROWS(float)
}

#include <atomic>

namespace kr {
namespace {
std::atomic<int> g_column_pairs{1};
std::atomic<int> g_tile_kernels{1};
std::atomic<int> g_fused_products{1};
std::atomic<int> g_lattice_rows{0};  // 0: the default per precision
}
bool pair_kernels_enabled() { return g_column_pairs.load(std::memory_order_relaxed) != 0; }
void set_pair_kernels(bool on) { g_column_pairs.store(on ? 1 : 0, std::memory_order_relaxed); }
bool tile_kernels_enabled() { return g_tile_kernels.load(std::memory_order_relaxed) != 0; }
void set_tile_kernels(bool on) { g_tile_kernels.store(on ? 1 : 0, std::memory_order_relaxed); }
bool fused_products_enabled() { return g_fused_products.load(std::memory_order_relaxed) != 0; }
void set_fused_products(bool on) { g_fused_products.store(on ? 1 : 0, std::memory_order_relaxed); }
int lattice_rows_per_thread(size_t real_bytes) {
  const int r = g_lattice_rows.load(std::memory_order_relaxed);
  if (r == 4 || r == 12) return r;
  (void)real_bytes;
  return 12;  // whole sites measured faster in both precisions (1.4x complex128, 2x complex64)
}
void set_lattice_rows_per_thread(int rows) { g_lattice_rows.store(rows, std::memory_order_relaxed); }
}  // namespace kr
