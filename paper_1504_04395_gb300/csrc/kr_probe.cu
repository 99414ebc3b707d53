// kr_probe_fma: arithmetic-throughput probe used as the roofline denominator of the FP64 path.
//
// GB300 issues few FP64 FMAs per clock, so every complex128 kernel of the solvers is bound by
// the FP64 pipe rather than by HBM.  The achieved fraction of that pipe needs a measured peak:
// this kernel runs kChains independent FMA chains per thread on a resident grid (4 CTAs of 256
// threads per SM), which keeps every FMA pipe busy; the chain loop is unrolled by four so that
// the loop's own instructions stay negligible.  The caller times it with CUDA events; the
// probe itself only launches and reports the algorithmic flop count.
#include <cmath>

#include "../../include/kr.h"
#include "kr_internal.h"

namespace kr {
namespace {

constexpr int kChains = 16;

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(int64_t iters, T b, T c, T sentinel, T* out) {
  T a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (T)(threadIdx.x + i);
#pragma unroll 4
  for (int64_t k = 0; k < iters; ++k) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  T sum = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) sum += a[i];
  // with b = 1 and c = 0 the values stay bounded.  Every thread may store (sentinel is a NaN
  // passed at run time, which no sum equals, but the compiler cannot know that), so no thread's
  // chains can be removed as dead code; only thread 0 of CTA 0 actually writes out[0]
  if (sum == sentinel || (threadIdx.x == 0 && blockIdx.x == 0)) out[0] = sum;
}

}  // namespace
}  // namespace kr

using namespace kr;

extern "C" kr_status kr_probe_fma(int32_t precision, int64_t iters, double* out, double* flops, void* stream) {
  if (iters <= 0 || !out || !flops || (precision != KR_FP64 && precision != 2)) {
    set_error("kr_probe_fma: precision must be KR_FP64 (0) or 2 (FP32), iters > 0, out and flops non-NULL");
    return KR_BAD_ARG;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int grid = sm_count() * 4;
  if (precision == KR_FP64)
    fma_probe_kernel<double><<<grid, 256, 0, st>>>(iters, 1.0, 0.0, std::nan(""), out);
  else
    fma_probe_kernel<float><<<grid, 256, 0, st>>>(iters, 1.0f, 0.0f, std::nanf(""), reinterpret_cast<float*>(out));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("kr_probe_fma: launch failed: ") + cudaGetErrorString(e));
    return KR_CUDA_ERROR;
  }
  *flops = 2.0 * kChains * (double)iters * 256.0 * grid;
  return KR_OK;
}
