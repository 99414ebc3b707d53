// Shared device helpers: complex arithmetic on (re, im) pairs, warp reductions, launch constants.
//
// Block vectors are row-interleaved: an n x s complex block is n*s consecutive
// (re, im) pairs, row i holding the s entries of unknown i (the layout of a
// C-contiguous (n, s) complex array).  The same kernels serve complex128
// (T = double, pairs are double2) and complex64 (T = float, pairs are float2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kr {

template <typename T> struct cplx;
template <> struct cplx<double> { typedef double2 type; };
template <> struct cplx<float> { typedef float2 type; };

template <typename T> using C2 = typename cplx<T>::type;

template <typename T> __host__ __device__ __forceinline__ C2<T> mk(T re, T im) {
  C2<T> r; r.x = re; r.y = im; return r;
}
template <typename T> __host__ __device__ __forceinline__ C2<T> czero() { return mk<T>(T(0), T(0)); }

// c + a*b (4 FMAs)
template <typename T> __device__ __forceinline__ C2<T> cfma(C2<T> a, C2<T> b, C2<T> c) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
  return c;
}
// c + conj(a)*b (4 FMAs)
template <typename T> __device__ __forceinline__ C2<T> cfmaconj(C2<T> a, C2<T> b, C2<T> c) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(-a.y, b.x, c.y);
  return c;
}
// c + r*b for real r (2 FMAs)
template <typename T> __device__ __forceinline__ C2<T> cfmareal(T r, C2<T> b, C2<T> c) {
  c.x = fma(r, b.x, c.x);
  c.y = fma(r, b.y, c.y);
  return c;
}
template <typename T> __host__ __device__ __forceinline__ C2<T> cadd(C2<T> a, C2<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __host__ __device__ __forceinline__ C2<T> csub(C2<T> a, C2<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
// a*b with explicit FMAs, so that every kernel rounds a complex product the same way
template <typename T> __host__ __device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
  return mk<T>(fma(a.x, b.x, -(a.y * b.y)), fma(a.x, b.y, a.y * b.x));
}
// v or -v by a runtime flag.  For doubles the sign bit is flipped on the integer pipe: a
// negation that cannot be folded into an FMA operand costs an FP64 add, and the FP64 pipe
// is the scarce unit (bitwise the same result as the floating-point negation).
__device__ __forceinline__ double neg_if(double v, bool f) {
  return __hiloint2double(__double2hiint(v) ^ (f ? (int)0x80000000 : 0), __double2loint(v));
}
__device__ __forceinline__ float neg_if(float v, bool f) { return f ? -v : v; }
template <typename T> __host__ __device__ __forceinline__ C2<T> cconj(C2<T> a) {
#ifdef __CUDA_ARCH__
  return mk<T>(a.x, neg_if(a.y, true));
#else
  return mk<T>(a.x, -a.y);
#endif
}
template <typename T> __host__ __device__ __forceinline__ T cabs2(C2<T> a) { return a.x * a.x + a.y * a.y; }

__device__ __forceinline__ double2 to_d2(double2 a) { return a; }
__device__ __forceinline__ double2 to_d2(float2 a) { return make_double2((double)a.x, (double)a.y); }
template <typename T> __device__ __forceinline__ C2<T> from_d2(double2 a);
template <> __device__ __forceinline__ double2 from_d2<double>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from_d2<float>(double2 a) { return make_float2((float)a.x, (float)a.y); }

template <typename T> __device__ __forceinline__ C2<T> shfl(C2<T> v, int src, int width = 32) {
  v.x = __shfl_sync(0xffffffffu, v.x, src, width);
  v.y = __shfl_sync(0xffffffffu, v.y, src, width);
  return v;
}
template <typename T> __device__ __forceinline__ C2<T> shfl_down(C2<T> v, int d) {
  v.x = __shfl_down_sync(0xffffffffu, v.x, d);
  v.y = __shfl_down_sync(0xffffffffu, v.y, d);
  return v;
}

// Number of CTAs used by the grid-stride kernels: a fixed multiple of the SM count so
// that per-CTA partial sums (and hence every reduction) have a fixed order.
constexpr int kThreads = 256;
constexpr int kCtasPerSmRows = 4;  // resident CTAs per SM the row kernels are sized for
constexpr int kMaxS = 32;

// Reduction kinds of the fused epilogues.
enum RedKind : int {
  RED_NONE = 0,
  RED_GRAM = 1,   // s x s  U^H Y      (U an n x s block)
  RED_TRACE = 2,  // 1      tr(U^H Y)  (U an n x s block)
  RED_SUMV = 3,   // 1      sum(u^H Y) (u an n-vector)
  RED_NORM2 = 4,  // 1      ||Y||_F^2  (real part only)
  RED_GRAMV = 5,  // 1 x s  u^H Y      (u an n-vector)
  RED_CDOT = 6,   // 1 x s  diag(U^H Y) (column-wise inner products)
};

}  // namespace kr
