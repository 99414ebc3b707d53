// complex64 staged products: row tiles (kr_tile_c64.cuh) and stencil planes (kr_plane_c64.cuh),
// kernel instantiations and launchers (one unit: both kernels count their device waits that ran
// out in the same g_kr_wait_timeouts)
#include <algorithm>
#include <atomic>
#include <string>
#include <unordered_map>

#include "../../include/kr.h"
#include <cudaTypedefs.h>

#include "kr_plane_c64.cuh"
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

// ---- stencil planes
// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (null if the driver
// does not provide it)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder_or_null() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) (void)cudaGetLastError();  // leave no sticky error behind for the next check
    return (e == cudaSuccess && q == cudaDriverEntryPointSuccess) ? reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p)
                                                                  : nullptr;
  }();
  return fn;
}
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder_or_null();
  if (!fn) throw CudaError{cudaErrorNotSupported, "plane product: cuTensorMapEncodeTiled unavailable"};
  return fn;
}

bool plane_kernels_available() { return tensor_map_encoder_or_null() != nullptr; }

// 4D map of an n x s complex64 block on an nx x ny x nz grid as floats {2s, nx, ny, nz}, box
// {2s, bx, by, 1}; points outside the grid read as zeros
static CUtensorMap block_map(const void* base, const PlaneGeom& P, int s, int bx, int by) {
  CUtensorMap m;
  const cuuint64_t dims[4] = {(cuuint64_t)(2 * s), (cuuint64_t)P.nx, (cuuint64_t)P.ny, (cuuint64_t)P.nz};
  const cuuint64_t strides[3] = {(cuuint64_t)s * 8, (cuuint64_t)P.nx * s * 8, (cuuint64_t)P.nx * P.ny * s * 8};
  const cuuint32_t box[4] = {(cuuint32_t)(2 * s), (cuuint32_t)bx, (cuuint32_t)by, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = tensor_map_encoder()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(base), dims, strides,
                                          box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw CudaError{cudaErrorInvalidValue, "plane product: tensor map encoding failed"};
  return m;
}

template <int GP, int NG, int IPT>
static int plane_go(const SpmmArgs<float>& a, const RedSet& rs, const TileLayout& L, const PlaneGeom& P,
                    const int* done, cudaStream_t st) {
  static std::atomic<uint64_t> attr{0};
  int dev = 0;
  KR_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = (dev >= 0 && dev < 64) ? (uint64_t{1} << dev) : 0;
  if (bit == 0 || !(attr.load(std::memory_order_acquire) & bit)) {
    KR_CUDA(cudaFuncSetAttribute(spmm_plane_kernel<GP, NG, IPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kTileMaxDynSmem));
    if (bit != 0) attr.fetch_or(bit, std::memory_order_acq_rel);
  }
  thread_local std::unordered_map<size_t, int> occ_cache;
  const size_t key = (size_t)P.total * 256 + (size_t)dev;
  int occ;
  auto it = occ_cache.find(key);
  if (it != occ_cache.end()) {
    occ = it->second;
  } else {
    KR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, spmm_plane_kernel<GP, NG, IPT>, kPlaneThreads, P.total + 128));
    occ = std::max(1, std::min(occ, kCtasPerSm));
    occ_cache.emplace(key, occ);
  }
  const int s = 2 * GP;
  const CUtensorMap mv = block_map(a.V, P, s, P.tx + 2, P.ty + 2);
  const CUtensorMap mu = block_map(L.nu > 0 ? L.U[0] : a.V, P, s, P.tx, P.ty);
  const int64_t units = (int64_t)P.ntx * P.nty * P.nz;
  const int grid = (int)std::min<int64_t>(units, (int64_t)sm_count() * occ);
  spmm_plane_kernel<GP, NG, IPT><<<grid, kPlaneThreads, P.total + 128, st>>>(a, rs, L, P, mv, mu, done);
  KR_CUDA(cudaGetLastError());
  return grid;
}

template <int GP, int NG>
static int plane_ipt(const SpmmArgs<float>& a, const RedSet& rs, const TileLayout& L, const PlaneGeom& P,
                     const int* done, cudaStream_t st) {
  if (P.ipt == 1) return plane_go<GP, NG, 1>(a, rs, L, P, done, st);
  return plane_go<GP, NG, 2>(a, rs, L, P, done, st);
}

template <int GP>
static int plane_ng(const SpmmArgs<float>& a, const RedSet& rs, const TileLayout& L, const PlaneGeom& P,
                    const int* done, cudaStream_t st) {
  if (L.ngram == 0) return plane_ipt<GP, 0>(a, rs, L, P, done, st);
  if (L.ngram == 1) return plane_ipt<GP, 1>(a, rs, L, P, done, st);
  return plane_ipt<GP, 2>(a, rs, L, P, done, st);
}

int launch_spmm_plane(const SpmmArgs<float>& a, const RedSet& rs, const TileLayout& L, const PlaneGeom& P,
                      const int* done, cudaStream_t st) {
  switch (a.s) {
    case 2: return plane_ng<1>(a, rs, L, P, done, st);
    case 4: return plane_ng<2>(a, rs, L, P, done, st);
    case 8: return plane_ng<4>(a, rs, L, P, done, st);
    case 16: return plane_ng<8>(a, rs, L, P, done, st);
    case 32: return plane_ng<16>(a, rs, L, P, done, st);
  }
  throw CudaError{cudaErrorInvalidValue, "plane product: s out of range"};
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
