// complex64 row-tile product: kernel instantiations and launcher (kr_tile_c64.cuh)
#include <algorithm>
#include <atomic>
#include <string>
#include <unordered_map>

#include "../../include/kr.h"
#include "kr_tile_c64.cuh"

namespace kr {

constexpr int kTileMaxDynSmem = 200 * 1024;

template <int GP, int MODE, int NG>
static int tile_go(const SpmmArgs<float>& a, const RedSet& rs, const TileLayout& L, const int* done,
                   cudaStream_t st) {
  static std::atomic<uint64_t> attr{0};
  int dev = 0;
  KR_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = (dev >= 0 && dev < 64) ? (uint64_t{1} << dev) : 0;
  if (bit == 0 || !(attr.load(std::memory_order_acquire) & bit)) {
    KR_CUDA(cudaFuncSetAttribute(spmm_tile_kernel<GP, MODE, NG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kTileMaxDynSmem));
    if (bit != 0) attr.fetch_or(bit, std::memory_order_acq_rel);
  }
  const int T = GP * L.R;
  // resident CTAs per SM for this shared-memory size (cached per device and size): the grid
  // depends only on the launch's shape, so its partial sums always have the same order
  thread_local std::unordered_map<size_t, int> occ_cache;
  const size_t key = (size_t)L.total * 256 + (size_t)dev;
  int occ;
  auto it = occ_cache.find(key);
  if (it != occ_cache.end()) {
    occ = it->second;
  } else {
    KR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, spmm_tile_kernel<GP, MODE, NG>, T, L.total));
    occ = std::max(1, std::min(occ, kCtasPerSm));
    occ_cache.emplace(key, occ);
  }
  const int64_t ntiles = (a.n + L.R - 1) / L.R;
  const int grid = (int)std::min<int64_t>(ntiles, (int64_t)sm_count() * occ);
  spmm_tile_kernel<GP, MODE, NG><<<grid, T, L.total, st>>>(a, rs, L, done);
  KR_CUDA(cudaGetLastError());
  return grid;
}

template <int GP, int MODE>
static int tile_ng(const SpmmArgs<float>& a, const RedSet& rs, const TileLayout& L, const int* done,
                   cudaStream_t st) {
  if (L.ngram == 0) return tile_go<GP, MODE, 0>(a, rs, L, done, st);
  if (L.ngram == 1) return tile_go<GP, MODE, 1>(a, rs, L, done, st);
  return tile_go<GP, MODE, 2>(a, rs, L, done, st);
}

template <int GP>
static int tile_mode(const SpmmArgs<float>& a, const RedSet& rs, const TileLayout& L, const int* done,
                     cudaStream_t st) {
  if (L.mode == TILE_STENCIL) return tile_ng<GP, TILE_STENCIL>(a, rs, L, done, st);
  if (L.mode == TILE_SPLIT) return tile_ng<GP, TILE_SPLIT>(a, rs, L, done, st);
  return tile_ng<GP, TILE_CSR>(a, rs, L, done, st);
}

int launch_spmm_tile(const SpmmArgs<float>& a, const RedSet& rs, const TileLayout& L, int grid, const int* done,
                     cudaStream_t st) {
  (void)grid;
  switch (a.s) {
    case 4: return tile_mode<2>(a, rs, L, done, st);
    case 8: return tile_mode<4>(a, rs, L, done, st);
    case 16: return tile_mode<8>(a, rs, L, done, st);
    case 32: return tile_mode<16>(a, rs, L, done, st);
  }
  throw CudaError{cudaErrorInvalidValue, "tile product: s out of range"};
}

}  // namespace kr

// waits of the tile kernels that ran out since the last call (g_kr_wait_timeouts of this unit)
extern "C" kr_status kr_take_device_timeouts(int32_t reset, int64_t* count) {
  if (!count) {
    kr::set_error("kr_take_device_timeouts: count is NULL");
    return KR_BAD_ARG;
  }
  unsigned int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, kr::g_kr_wait_timeouts, sizeof(v));
  if (e == cudaSuccess && reset) {
    const unsigned int zero = 0;
    e = cudaMemcpyToSymbol(kr::g_kr_wait_timeouts, &zero, sizeof(zero));
  }
  if (e != cudaSuccess) {
    kr::set_error(std::string("kr_take_device_timeouts: ") + cudaGetErrorString(e));
    return KR_CUDA_ERROR;
  }
  *count = v;
  return KR_OK;
}
