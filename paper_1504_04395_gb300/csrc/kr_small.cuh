// Single-CTA FP64 dense algebra on s x s complex matrices held in shared memory.
//
// Every routine is called by all threads of the CTA (they synchronise
// internally).  Matrices are row-major double2 arrays M[i*ld + j].  Used for the
// coefficient matrices of the block methods (alpha, beta, ... of Algorithms 3
// and 5), the Cholesky factors of CholQR, and the block rotations of Bl-QMR.
#pragma once

#include "kr_common.cuh"

namespace kr {
namespace small {

constexpr double kEps = 2.220446049250313e-16;

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double cabsd(double2 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ bool finite2(double2 a) { return isfinite(a.x) && isfinite(a.y); }

__device__ __forceinline__ void copy(double2* dst, const double2* src, int cnt) {
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}
__device__ __forceinline__ void fill(double2* dst, int cnt, double2 v) {
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) dst[i] = v;
  __syncthreads();
}
__device__ __forceinline__ void identity(double2* dst, int s) {
  for (int i = threadIdx.x; i < s * s; i += blockDim.x)
    dst[i] = make_double2((i / s) == (i % s) ? 1.0 : 0.0, 0.0);
  __syncthreads();
}
// dst = A^H (s x s); dst must not alias A
__device__ __forceinline__ void adjoint(double2* dst, const double2* A, int s) {
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
    const int r = i / s, c = i % s;
    const double2 v = A[c * s + r];
    dst[i] = make_double2(v.x, -v.y);
  }
  __syncthreads();
}
// C (m x p) = op(A) (m x k) * op(B) (k x p); ha/hb: use the adjoint of A / B.
// A is m x k (or k x m when ha), B is k x p (or p x k when hb). C must not alias A or B.
__device__ void matmul(double2* C, const double2* A, const double2* B, int m, int k, int p, bool ha = false,
                       bool hb = false, double scale = 1.0) {
  for (int i = threadIdx.x; i < m * p; i += blockDim.x) {
    const int r = i / p, c = i % p;
    double2 acc = make_double2(0.0, 0.0);
    for (int q = 0; q < k; ++q) {
      double2 a = ha ? A[q * m + r] : A[r * k + q];
      if (ha) a.y = -a.y;
      double2 b = hb ? B[c * k + q] : B[q * p + c];
      if (hb) b.y = -b.y;
      acc.x = fma(a.x, b.x, acc.x);
      acc.x = fma(-a.y, b.y, acc.x);
      acc.y = fma(a.x, b.y, acc.y);
      acc.y = fma(a.y, b.x, acc.y);
    }
    C[i] = make_double2(scale * acc.x, scale * acc.y);
  }
  __syncthreads();
}
__device__ __forceinline__ void axpy(double2* Y, const double2* X, double2 a, int cnt) {  // Y += a X
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    const double2 x = X[i];
    Y[i].x += a.x * x.x - a.y * x.y;
    Y[i].y += a.x * x.y + a.y * x.x;
  }
  __syncthreads();
}

// Frobenius norm (all threads get the result); scratch >= 32 doubles
__device__ double fro(const double2* A, int cnt, double* scratch) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) acc += A[i].x * A[i].x + A[i].y * A[i].y;
  for (int off = 16; off >= 1; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[warp] = acc;
  __syncthreads();
  double tot = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += scratch[w];
  __syncthreads();
  return sqrt(tot);
}

// X <- M^{-1} X by LU with partial pivoting (M s x s overwritten, X s x nrhs).
// Returns false (breakdown) when a pivot |u_ii| <= 64 eps ||M||_F or a value is not finite.
__device__ bool lu_solve(double2* M, double2* X, int s, int nrhs, double* scratch, int* iscratch) {
  const double nrm = fro(M, s * s, scratch);
  const double tolp = 64.0 * kEps * nrm;
  bool ok = isfinite(nrm);
  for (int k = 0; k < s && ok; ++k) {
    if (threadIdx.x == 0) {
      // pivot: largest |re| + |im| in the column (the LAPACK convention for complex LU)
      int p = k;
      double best = fabs(M[k * s + k].x) + fabs(M[k * s + k].y);
      for (int i = k + 1; i < s; ++i) {
        const double v = fabs(M[i * s + k].x) + fabs(M[i * s + k].y);
        if (v > best) { best = v; p = i; }
      }
      iscratch[0] = p;
      const double piv = cabsd(M[p * s + k]);
      iscratch[1] = (piv <= tolp || !isfinite(piv)) ? 1 : 0;
    }
    __syncthreads();
    const int p = iscratch[0];
    if (iscratch[1]) ok = false;
    __syncthreads();
    if (!ok) break;
    if (p != k) {
      for (int j = threadIdx.x; j < s; j += blockDim.x) {
        const double2 t = M[k * s + j]; M[k * s + j] = M[p * s + j]; M[p * s + j] = t;
      }
      for (int j = threadIdx.x; j < nrhs; j += blockDim.x) {
        const double2 t = X[k * nrhs + j]; X[k * nrhs + j] = X[p * nrhs + j]; X[p * nrhs + j] = t;
      }
      __syncthreads();
    }
    const double2 piv = M[k * s + k];
    // multipliers
    for (int i = k + 1 + threadIdx.x; i < s; i += blockDim.x) M[i * s + k] = cdiv(M[i * s + k], piv);
    __syncthreads();
    const int rows = s - k - 1;
    const int cols = (s - k - 1) + nrhs;
    for (int idx = threadIdx.x; idx < rows * cols; idx += blockDim.x) {
      const int i = k + 1 + idx / cols;
      const int jj = idx % cols;
      const double2 l = M[i * s + k];
      if (jj < s - k - 1) {
        const int j = k + 1 + jj;
        const double2 u = M[k * s + j];
        M[i * s + j].x -= l.x * u.x - l.y * u.y;
        M[i * s + j].y -= l.x * u.y + l.y * u.x;
      } else {
        const int r = jj - (s - k - 1);
        const double2 u = X[k * nrhs + r];
        X[i * nrhs + r].x -= l.x * u.x - l.y * u.y;
        X[i * nrhs + r].y -= l.x * u.y + l.y * u.x;
      }
    }
    __syncthreads();
  }
  if (!ok) return false;
  // back substitution, one right-hand side column per thread
  for (int k = s - 1; k >= 0; --k) {
    for (int r = threadIdx.x; r < nrhs; r += blockDim.x) {
      double2 acc = X[k * nrhs + r];
      for (int j = k + 1; j < s; ++j) {
        const double2 u = M[k * s + j], x = X[j * nrhs + r];
        acc.x -= u.x * x.x - u.y * x.y;
        acc.y -= u.x * x.y + u.y * x.x;
      }
      X[k * nrhs + r] = cdiv(acc, M[k * s + k]);
    }
    __syncthreads();
  }
  bool fin = true;
  for (int i = 0; i < s * nrhs; ++i) fin = fin && finite2(X[i]);
  return fin;
}

// Upper Cholesky factor R (R^H R = A) in place in A; lower triangle zeroed.
// Returns false when a diagonal entry is not positive or not finite.
__device__ bool chol_upper(double2* A, int s, int* iscratch) {
  for (int k = 0; k < s; ++k) {
    if (threadIdx.x == 0) {
      double d = A[k * s + k].x;
      for (int i = 0; i < k; ++i) d -= A[i * s + k].x * A[i * s + k].x + A[i * s + k].y * A[i * s + k].y;
      iscratch[0] = (d > 0.0 && isfinite(d)) ? 1 : 0;
      A[k * s + k] = make_double2(d > 0.0 ? sqrt(d) : 0.0, 0.0);
    }
    __syncthreads();
    if (!iscratch[0]) return false;
    const double rkk = A[k * s + k].x;
    for (int j = k + 1 + threadIdx.x; j < s; j += blockDim.x) {
      double2 v = A[k * s + j];
      for (int i = 0; i < k; ++i) {  // v -= conj(R[i][k]) R[i][j]
        const double2 a = A[i * s + k], b = A[i * s + j];
        v.x -= a.x * b.x + a.y * b.y;
        v.y -= a.x * b.y - a.y * b.x;
      }
      A[k * s + j] = make_double2(v.x / rkk, v.y / rkk);
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < s * s; i += blockDim.x)
    if (i / s > i % s) A[i] = make_double2(0.0, 0.0);
  __syncthreads();
  return true;
}

// Rinv = R^{-1} for upper triangular R (column-parallel back substitution on the identity)
__device__ void tri_inv_upper(double2* Rinv, const double2* R, int s) {
  for (int c = threadIdx.x; c < s; c += blockDim.x) {
    for (int k = s - 1; k >= 0; --k) {
      double2 acc = make_double2(k == c ? 1.0 : 0.0, 0.0);
      for (int j = k + 1; j < s; ++j) {
        const double2 u = R[k * s + j], x = Rinv[j * s + c];
        acc.x -= u.x * x.x - u.y * x.y;
        acc.y -= u.x * x.y + u.y * x.x;
      }
      Rinv[k * s + c] = (k > c) ? make_double2(0.0, 0.0) : cdiv(acc, R[k * s + k]);
    }
  }
  __syncthreads();
}

// Complete QR of the 2s x s matrix Mx by Householder reflections:
// Om (2s x 2s unitary) with Om * Mx = [U; 0], U (s x s) upper triangular, written to U.
// Mx is destroyed.  scratch2s >= 2s double2.
__device__ void householder_2s(double2* Om, double2* U, double2* Mx, int s, double2* v, double* scratch) {
  const int m = 2 * s;
  identity(Om, m);
  for (int k = 0; k < s; ++k) {
    // v = x - alpha e_k on rows k..m-1 of column k; alpha = -e^{i arg x_k} ||x||
    if (threadIdx.x == 0) {
      double nx = 0.0;
      for (int i = k; i < m; ++i) nx += Mx[i * s + k].x * Mx[i * s + k].x + Mx[i * s + k].y * Mx[i * s + k].y;
      nx = sqrt(nx);
      const double2 xk = Mx[k * s + k];
      const double axk = cabsd(xk);
      const double2 ph = axk > 0.0 ? make_double2(xk.x / axk, xk.y / axk) : make_double2(1.0, 0.0);
      const double2 alpha = make_double2(-ph.x * nx, -ph.y * nx);
      double vn = 0.0;
      for (int i = 0; i < m; ++i) {
        double2 vi = (i < k) ? make_double2(0.0, 0.0) : Mx[i * s + k];
        if (i == k) { vi.x -= alpha.x; vi.y -= alpha.y; }
        v[i] = vi;
        vn += vi.x * vi.x + vi.y * vi.y;
      }
      scratch[0] = vn;
    }
    __syncthreads();
    const double vn = scratch[0];
    __syncthreads();
    if (vn > 0.0) {
      // H = I - 2 v v^H / (v^H v): apply to Mx (columns k..s-1) and to Om (all columns)
      for (int c = threadIdx.x; c < (s - k) + m; c += blockDim.x) {
        double2* base;
        int ld, col;
        if (c < s - k) { base = Mx; ld = s; col = k + c; } else { base = Om; ld = m; col = c - (s - k); }
        double2 d = make_double2(0.0, 0.0);  // v^H x
        for (int i = k; i < m; ++i) {
          const double2 vi = v[i], xi = base[i * ld + col];
          d.x += vi.x * xi.x + vi.y * xi.y;
          d.y += vi.x * xi.y - vi.y * xi.x;
        }
        const double f = 2.0 / vn;
        for (int i = k; i < m; ++i) {
          const double2 vi = v[i];
          base[i * ld + col].x -= f * (vi.x * d.x - vi.y * d.y);
          base[i * ld + col].y -= f * (vi.x * d.y + vi.y * d.x);
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
    const int r = i / s, c = i % s;
    U[i] = (r <= c) ? Mx[r * s + c] : make_double2(0.0, 0.0);
  }
  __syncthreads();
}

}  // namespace small
}  // namespace kr
