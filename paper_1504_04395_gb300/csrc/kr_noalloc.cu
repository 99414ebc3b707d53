// kr_block_reduce_noalloc: the block reduction of kr_block_reduce without any
// device allocation by the library.
//
// Some callers cannot let a library allocate device memory: applications that
// hand all device memory to their own pool allocator up front and forbid any
// other allocation, and latency-critical loops where cudaMalloc / cudaFree,
// which can synchronise the device, are not acceptable.  For them this entry
// point keeps its only scratch buffer (the per-CTA partial sums of the
// reduction) in a fixed, statically sized device array that is part of the
// loaded library.
//
// Limits and behaviour:
//  * scratch: kNoAllocMaxCtas x kNoAllocMaxSlots complex128 = 256 x 256 x 16 B = 1 MiB,
//    held by every GPU on which the library is loaded until the process exits;
//  * s <= 16 (a Gram needs s*s <= 256 slots per CTA); larger s is rejected with
//    KR_UNSUPPORTED, before any GPU work;
//  * the call runs on the device that holds Y (made current for the call and the
//    previous device restored); U, out and a non-null stream must belong to the same
//    device, otherwise KR_BAD_ARG before any GPU work;
//  * the device address of the array is looked up (cudaGetSymbolAddress, with that
//    device current) on every call that is not being captured into a CUDA graph, so a
//    device reset or a new primary context does not leave a stale address behind;
//    while a stream capture is in progress the address of the last uncaptured call on
//    that device is used, so make one call on each device before capturing;
//  * the grid is capped at 256 CTAs (kr_block_reduce uses up to 4 CTAs per SM), so for
//    large n the partial sums are grouped differently: results agree with
//    kr_block_reduce to rounding, not bitwise;
//  * all calls share the one array: every CTA overwrites all of its slots, so
//    nothing needs clearing between calls, but calls whose GPU work overlaps
//    (different streams, or different host threads) race on the array.
#include <mutex>

#include "../../include/kr.h"
#include "kr_internal.h"
#include "kr_rows_impl.cuh"

namespace kr {
namespace {

constexpr int kNoAllocMaxCtas = 256;
constexpr int kNoAllocMaxSlots = 256;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double2 g_noalloc_partials[kNoAllocMaxCtas * kNoAllocMaxSlots];

std::mutex g_noalloc_mu;
double2* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

// Device address of g_noalloc_partials on the current device.  Looked up again on every
// call outside a stream capture (cheap; survives a device reset); during a capture the
// address recorded by the last uncaptured call on this device is used.
cudaError_t noalloc_scratch(bool capturing, double2** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!capturing) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = reinterpret_cast<double2*>(p);
  } else if (g_noalloc_ptr[dev] == nullptr) {
    return cudaErrorStreamCaptureUnsupported;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

// Device that holds a pointer (-1: not device-accessible memory the runtime knows of).
int pointer_device(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // clear the (non-sticky) error left by the failed query
    return -1;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return -1;
  return at.device;
}

// Makes `dev` current for the lifetime of the guard and restores the previous device.
struct DeviceGuard {
  int prev = -1;
  bool switched = false;
  cudaError_t enter(int dev) {
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return e;
    if (prev == dev) return cudaSuccess;
    e = cudaSetDevice(dev);
    switched = e == cudaSuccess;
    return e;
  }
  ~DeviceGuard() {
    if (switched) cudaSetDevice(prev);
  }
};

template <int G, int NG>
void launch_noalloc(const LinArgs& a, const RedSet& rs, int grid, cudaStream_t st) {
  const size_t smem = (size_t)(kThreads / 32) * rs.nslots * sizeof(double2);  // <= 32 KiB
  lincomb_kernel<double, G, NG><<<grid, kThreads, smem, st>>>(a, rs, nullptr);
}

template <int G>
void launch_noalloc_g(bool gram, const LinArgs& a, const RedSet& rs, int grid, cudaStream_t st) {
  if (gram) launch_noalloc<G, 1>(a, rs, grid, st);
  else launch_noalloc<G, 0>(a, rs, grid, st);
}

}  // namespace
}  // namespace kr

using namespace kr;

extern "C" kr_status kr_block_reduce_noalloc(int64_t n, int32_t s, const double* U, const double* Y, int32_t kind,
                                             double* out, void* stream) {
  if (n <= 0 || !Y || !out || kind < KR_RED_GRAM || kind > KR_RED_NORM2 || (kind != KR_RED_NORM2 && !U)) {
    set_error("kr_block_reduce_noalloc: invalid arguments");
    return KR_BAD_ARG;
  }
  if (s < 1 || s > 16) {
    set_error("kr_block_reduce_noalloc: s must be in [1, 16] (static scratch holds 256 slots per CTA)");
    return KR_UNSUPPORTED;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // every operand on one device, the one the call runs on
  const int dev = pointer_device(Y);
  if (dev < 0 || pointer_device(out) != dev || (kind != KR_RED_NORM2 && pointer_device(U) != dev)) {
    set_error("kr_block_reduce_noalloc: U, Y and out must be device memory of one GPU");
    return KR_BAD_ARG;
  }
  if (st != nullptr) {
    int sdev = -1;
    if (cudaStreamGetDevice(st, &sdev) != cudaSuccess || sdev != dev) {
      cudaGetLastError();
      set_error("kr_block_reduce_noalloc: the stream does not belong to the device that holds Y");
      return KR_BAD_ARG;
    }
  }
  DeviceGuard guard;
  cudaError_t e = guard.enter(dev);
  if (e != cudaSuccess) {
    set_error(std::string("kr_block_reduce_noalloc: cannot select the device of Y: ") + cudaGetErrorString(e));
    return KR_CUDA_ERROR;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) {
    set_error(std::string("kr_block_reduce_noalloc: stream query failed: ") + cudaGetErrorString(e));
    return KR_CUDA_ERROR;
  }
  double2* scratch = nullptr;
  e = noalloc_scratch(cap != cudaStreamCaptureStatusNone, &scratch);
  if (e != cudaSuccess) {
    set_error(std::string("kr_block_reduce_noalloc: scratch lookup failed (during a stream capture the first "
                          "call on a device must have been made before the capture): ") + cudaGetErrorString(e));
    return KR_CUDA_ERROR;
  }
  LinArgs a{};
  a.n = n;
  a.s = s;
  a.nout = 1;
  a.o[0].nterm = 1;
  a.o[0].t[0].src_kind = SRC_BLOCK;
  a.o[0].t[0].src = Y;
  a.o[0].t[0].coef_kind = COEF_ONE;
  RedSet rs{};
  rs.nred = 1;
  rs.r[0].kind = kind;
  rs.r[0].ysrc = 0;
  rs.r[0].ureg = -1;
  rs.r[0].U = U;
  rs.nslots = kind == KR_RED_GRAM ? s * s : 1;
  rs.partials = scratch;
  resolve_sources(a, rs);  // two operands at most: always fits
  int grid = row_grid(n, s);
  if (grid > kNoAllocMaxCtas) grid = kNoAllocMaxCtas;
  const bool gram = kind == KR_RED_GRAM;
  switch (threads_per_row(s)) {
    case 1: launch_noalloc_g<1>(gram, a, rs, grid, st); break;
    case 2: launch_noalloc_g<2>(gram, a, rs, grid, st); break;
    case 4: launch_noalloc_g<4>(gram, a, rs, grid, st); break;
    case 8: launch_noalloc_g<8>(gram, a, rs, grid, st); break;
    default: launch_noalloc_g<16>(gram, a, rs, grid, st); break;
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    reduce_slots_kernel<double><<<rs.nslots, kThreads, 0, st>>>(scratch, grid, rs.nslots,
                                                                reinterpret_cast<double2*>(out), nullptr);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    set_error(std::string("kr_block_reduce_noalloc: launch failed: ") + cudaGetErrorString(e));
    return KR_CUDA_ERROR;
  }
  return KR_OK;
}
