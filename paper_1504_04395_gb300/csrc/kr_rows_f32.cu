// complex64 instantiation of the row kernels
#include "kr_rows_launch.cuh"
namespace kr {
KR_INSTANTIATE_ROWS(float)
}

#include <atomic>

namespace kr {
namespace {
std::atomic<int> g_column_pairs{1};
}
bool pair_kernels_enabled() { return g_column_pairs.load(std::memory_order_relaxed) != 0; }
void set_pair_kernels(bool on) { g_column_pairs.store(on ? 1 : 0, std::memory_order_relaxed); }
}  // namespace kr
