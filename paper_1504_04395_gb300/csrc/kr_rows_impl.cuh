// Kernel bodies for the row kernels (included by the per-precision translation units).
#pragma once

#include "kr_rows.cuh"

namespace kr {

// Gram accumulators per thread: NG s x s Grams (column c = this thread's column, G rows of it).
template <typename T, int G, int NG>
struct Acc {
  C2<T> g0[NG >= 1 ? G : 1];     // first fused Gram
  C2<T> g1[NG >= 2 ? G : 1];     // second fused Gram
  C2<T> v[kMaxRed];
};

template <int NG, int G>
struct NGCap {  // register budget: at most 16 Gram accumulators per thread
  static constexpr bool ok = (NG * G <= 16) || NG == 0;
};

template <typename T, int G, int NG>
__device__ __forceinline__ void acc_zero(Acc<T, G, NG>& a) {
#pragma unroll
  for (int i = 0; i < (NG >= 1 ? G : 1); ++i) a.g0[i] = czero<T>();
#pragma unroll
  for (int i = 0; i < (NG >= 2 ? G : 1); ++i) a.g1[i] = czero<T>();
#pragma unroll
  for (int i = 0; i < kMaxRed; ++i) a.v[i] = czero<T>();
}

template <typename T, int G>
__device__ __forceinline__ void gram_add(C2<T> (&g)[G], C2<T> u, C2<T> y, int s, int grpbase) {
  // (U^H Y)[a][c] += conj(U[j][a]) * Y[j][c]; U[j][a] lives in lane grpbase + a
#pragma unroll
  for (int a = 0; a < G; ++a) {
    C2<T> ua = shfl<T>(u, grpbase + a);
    if (a < s) g[a] = cfmaconj<T>(ua, y, g[a]);
  }
}

template <typename T, int G, int NG>
__device__ __forceinline__ void red_add(const RedSpec& r, int ri, Acc<T, G, NG>& acc, C2<T> y, C2<T> u,
                                        int s, int grpbase) {
  if (r.kind == RED_GRAM) {
    if constexpr (NG >= 1) {
      if (r.gacc == 0) gram_add<T, G>(acc.g0, u, y, s, grpbase);
    }
    if constexpr (NG >= 2) {
      if (r.gacc == 1) gram_add<T, G>(acc.g1, u, y, s, grpbase);
    }
  } else if (r.kind != RED_NONE) {
    // select accumulator ri with constant indices only (keeps Acc in registers)
    C2<T> cur = acc.v[0];
#pragma unroll
    for (int q = 1; q < kMaxRed; ++q)
      if (q == ri) cur = acc.v[q];
    if (r.kind == RED_NORM2) {
      cur.x = fma(y.x, y.x, fma(y.y, y.y, cur.x));
    } else {  // TRACE, SUMV, GRAMV: conj(u) * y
      cur = cfmaconj<T>(u, y, cur);
    }
#pragma unroll
    for (int q = 0; q < kMaxRed; ++q)
      if (q == ri) acc.v[q] = cur;
  }
}

template <typename T, int G, int NG>
__device__ __forceinline__ C2<T> acc_v(const Acc<T, G, NG>& acc, int ri) {
  C2<T> cur = acc.v[0];
#pragma unroll
  for (int q = 1; q < kMaxRed; ++q)
    if (q == ri) cur = acc.v[q];
  return cur;
}

template <typename T, int G>
__device__ __forceinline__ void gram_stage(const C2<T> (&g)[G], C2<T>* dst, int s, int lane) {
#pragma unroll
  for (int a = 0; a < G; ++a) {
    C2<T> v = g[a];
#pragma unroll
    for (int off = 16; off >= G; off >>= 1) v = cadd<T>(v, shfl_down<T>(v, off));
    if (lane < s && a < s) dst[a * s + lane] = v;
  }
}

// Fixed-order CTA reduction of the accumulators into this CTA's partial record.
template <typename T, int G, int NG>
__device__ __forceinline__ void cta_reduce(const RedSet& rs, Acc<T, G, NG>& acc, int s, C2<T>* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int ns = rs.nslots;
#pragma unroll
  for (int ri = 0; ri < kMaxRed; ++ri) {
    if (ri < rs.nred) {
      const RedSpec& r = rs.r[ri];
      if (r.kind == RED_GRAM) {
        if constexpr (NG >= 1) {
          if (r.gacc == 0) gram_stage<T, G>(acc.g0, sm + warp * ns + r.slot, s, lane);
        }
        if constexpr (NG >= 2) {
          if (r.gacc == 1) gram_stage<T, G>(acc.g1, sm + warp * ns + r.slot, s, lane);
        }
      } else if (r.kind == RED_GRAMV || r.kind == RED_CDOT) {
        C2<T> v = acc_v<T, G, NG>(acc, ri);
#pragma unroll
        for (int off = 16; off >= G; off >>= 1) v = cadd<T>(v, shfl_down<T>(v, off));
        if (lane < s) sm[warp * ns + r.slot + lane] = v;
      } else {
        C2<T> v = acc_v<T, G, NG>(acc, ri);
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) v = cadd<T>(v, shfl_down<T>(v, off));
        if (lane == 0) sm[warp * ns + r.slot] = v;
      }
    }
  }
  __syncthreads();
  C2<T>* out = reinterpret_cast<C2<T>*>(rs.partials) + (size_t)blockIdx.x * ns;
  for (int t = threadIdx.x; t < ns; t += blockDim.x) {
    C2<T> sum = czero<T>();
    for (int w = 0; w < nw; ++w) sum = cadd<T>(sum, sm[w * ns + t]);
    out[t] = sum;
  }
}

template <typename T>
__device__ __forceinline__ C2<T> pick(const C2<T> (&o)[kMaxOut], int r) {
  C2<T> x = o[0];
#pragma unroll
  for (int i = 1; i < kMaxOut; ++i)
    if (r == i) x = o[i];
  return x;
}

template <typename T>
__device__ __forceinline__ C2<T> scalar_coef(const double2* p, int conj, int neg) {
  double2 d = *p;
  if (conj) d.y = -d.y;
  if (neg) { d.x = -d.x; d.y = -d.y; }
  return from_d2<T>(d);
}

// ---------------------------------------------------------------------------------------
// SpMM with fused reductions
// ---------------------------------------------------------------------------------------

// Stencil coefficients in the element type, converted once per CTA (a double -> float
// conversion runs on the FP64 pipe): centre, minus neighbours, plus neighbours per axis.
template <typename T>
struct StencilCoef {
  C2<T> c, m[3], p[3];
};
template <typename T>
__device__ __forceinline__ StencilCoef<T> stencil_coef(const SpmmArgs<T>& a) {
  StencilCoef<T> k;
  k.c = mk<T>((T)a.sc.x, (T)a.sc.y);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    k.m[q] = mk<T>((T)a.sm[q].x, (T)a.sm[q].y);
    k.p[q] = mk<T>((T)a.sp[q].x, (T)a.sp[q].y);
  }
  return k;
}

// (A V)[j][c] for one thread of row j's group (G threads per row): the matrix-free stencil or
// the CSR product, before any scaling.  act = row j exists and c < s; rowok = row j exists.
// SM: 0 = the operator decides at run time (the fused linear-combination kernels: one stencil
// load at a time); 1 = CSR only; 2 = stencil only, its loads issued in two groups ahead of their
// FMAs (the product kernel has one instantiation for each storage, so the CSR one keeps its
// registers).
template <typename T, int G, int SM>
__device__ __forceinline__ C2<T> spmm_row(const SpmmArgs<T>& a, const StencilCoef<T>& sk, int64_t j, int c,
                                          bool rowok, bool act) {
  constexpr bool GROUPED = SM == 2;
  const int s = a.s;
  C2<T> y = czero<T>();
  const bool sten = SM == 2 || (SM == 0 && a.nst > 0);
  if (rowok && sten) {
    // matrix-free stencil, same summation order as the real-off-diagonal CSR storage:
    // centre, then -axis d-1 .. -axis 0, then +axis 0 .. +axis d-1
    const C2<T> stc = sk.c;
    int64_t xc[3];
    grid_coords<3>(j, a.nst, a.sdiv32, a.sdims, a.sdiv, xc);
    if (act) {
      if constexpr (GROUPED) {
        // the loads of a group (centre and minus neighbours, then plus neighbours) are issued before
        // its FMAs (an absent neighbour loads the centre again and is not used), so they are in
        // flight together; two groups keep the registers of the complex128 kernels in bounds
        bool has[6];
        int64_t nb[6];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int qa = 2 - q;
          has[q] = qa < a.nst && xc[qa] > 0;
          nb[q] = has[q] ? j - a.sstr[qa] : j;
          has[3 + q] = q < a.nst && xc[q] < a.sdims[q] - 1;
          nb[3 + q] = has[3 + q] ? j + a.sstr[q] : j;
        }
        const C2<T> xv = a.V[j * s + c];
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          C2<T> x[3];
#pragma unroll
          for (int m = 0; m < 3; ++m) x[m] = a.V[nb[3 * g + m] * s + c];
          if (g == 0) y = cmul<T>(stc, xv);
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            if (has[3 * g + m]) {
              const C2<T> k = g == 0 ? sk.m[2 - m] : sk.p[m];
              if (a.sreal) y = cfmareal<T>(k.x, x[m], y);
              else y = cfma<T>(k, x[m], y);
            }
          }
        }
      } else {
        y = cmul<T>(stc, a.V[j * s + c]);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int qa = 2 - q;
          if (qa < a.nst && xc[qa] > 0) {
            const C2<T> xv = a.V[(j - a.sstr[qa]) * s + c];
            const C2<T> m = sk.m[qa];
            if (a.sreal) y = cfmareal<T>(m.x, xv, y);
            else y = cfma<T>(m, xv, y);
          }
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          if (q < a.nst && xc[q] < a.sdims[q] - 1) {
            const C2<T> xv = a.V[(j + a.sstr[q]) * s + c];
            const C2<T> pp = sk.p[q];
            if (a.sreal) y = cfmareal<T>(pp.x, xv, y);
            else y = cfma<T>(pp, xv, y);
          }
        }
      }
    }
  } else if (rowok && SM != 2) {
    const int64_t k0 = a.rowptr[j], k1 = a.rowptr[j + 1];
    // batches of kBatch entries: all index, value and gathered-row loads of a batch are
    // issued before its FMAs, so several neighbour rows are in flight per thread
    constexpr int kBatch = sizeof(T) == 4 ? 4 : 2;
    if (a.split) {
      if (act) y = cmul<T>(a.diag[j], a.V[j * s + c]);
      for (int64_t k = k0; k < k1; k += kBatch) {
        int32_t col[kBatch];
        T v[kBatch];
        C2<T> x[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          const bool in = k + u < k1;
          col[u] = in ? a.colidx[k + u] : 0;
          v[u] = in ? a.offr[k + u] : T(0);
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
          x[u] = (act && k + u < k1) ? a.V[(int64_t)col[u] * s + c] : czero<T>();
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
          if (act && k + u < k1) y = cfmareal<T>(v[u], x[u], y);
      }
    } else {
      for (int64_t k = k0; k < k1; k += kBatch) {
        int32_t col[kBatch];
        C2<T> v[kBatch];
        C2<T> x[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          const bool in = k + u < k1;
          col[u] = in ? a.colidx[k + u] : 0;
          v[u] = in ? a.vals[k + u] : czero<T>();
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
          x[u] = (act && k + u < k1) ? a.V[(int64_t)col[u] * s + c] : czero<T>();
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
          if (act && k + u < k1) y = cfma<T>(v[u], x[u], y);
      }
    }
  }
  return y;
}

// STEN: the matrix-free stencil (else CSR storage)
template <typename T, int G, int NG, bool STEN>
__global__ void __launch_bounds__(kThreads) spmm_kernel(SpmmArgs<T> a, RedSet rs, const int* done) {
  if (done != nullptr && *(volatile const int*)done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int RPW = 32 / G;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = lane & (G - 1);
  const int grpbase = lane & ~(G - 1);
  const int s = a.s;
  const int64_t n = a.n;
  const int64_t rows_per_cta = (int64_t)(blockDim.x >> 5) * RPW;
  C2<T> ysc = mk<T>((T)a.ay, (T)0);
  const bool scaled = a.ys != nullptr || a.ay != 1.0;
  if (a.ys != nullptr) {
    C2<T> d = scalar_coef<T>(a.ys, a.ys_conj, a.ys_neg);
    ysc = mk<T>((T)a.ay * d.x, (T)a.ay * d.y);
  }
  const T bz = (T)a.bz;
  const StencilCoef<T> sk = stencil_coef<T>(a);
  Acc<T, G, NG> acc;
  acc_zero(acc);
  for (int64_t base = (int64_t)blockIdx.x * rows_per_cta; base < n; base += (int64_t)gridDim.x * rows_per_cta) {
    const int64_t j = base + warp * RPW + lane / G;
    const bool rowok = j < n;
    const bool act = rowok && c < s;
    C2<T> y = spmm_row<T, G, STEN ? 2 : 1>(a, sk, j, c, rowok, act);
    if (act) {
      if (scaled) y = cmul<T>(ysc, y);
      if (a.Z != nullptr) {
        const C2<T> z = a.Z[j * s + c];
        y.x = fma(bz, z.x, y.x);
        y.y = fma(bz, z.y, y.y);
      }
      if (a.Y != nullptr) a.Y[j * s + c] = y;
    }
    if (rs.nred > 0) {
#pragma unroll
      for (int ri = 0; ri < kMaxRed; ++ri) {
        if (ri < rs.nred) {
          const RedSpec& r = rs.r[ri];
          C2<T> u = czero<T>();
          if (r.kind == RED_GRAM || r.kind == RED_TRACE || r.kind == RED_CDOT) {
            // U == nullptr: reduction of the product with itself (Y^H Y)
            if (act) u = (r.U != nullptr) ? reinterpret_cast<const C2<T>*>(r.U)[j * s + c] : y;
          } else if (r.kind == RED_SUMV || r.kind == RED_GRAMV) {
            if (rowok) u = reinterpret_cast<const C2<T>*>(r.U)[j];
          }
          red_add<T, G, NG>(r, ri, acc, y, u, s, grpbase);
        }
      }
    }
  }
  if (rs.nred > 0) cta_reduce<T, G, NG>(rs, acc, s, reinterpret_cast<C2<T>*>(smem_raw));
}

// ---------------------------------------------------------------------------------------
// Row-local linear combinations with fused reductions
// ---------------------------------------------------------------------------------------
// SP: the combination has SRC_SPMM terms, products of `sp` computed row by row in this pass
template <typename T, int G, int NG, bool SP>
__device__ __forceinline__ void lincomb_rows(const LinArgs& a, const RedSet& rs, const SpmmArgs<T>& sp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int RPW = 32 / G;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = lane & (G - 1);
  const int grpbase = lane & ~(G - 1);
  const int s = a.s;
  const int64_t n = a.n;
  const int ss = s * s;
  C2<T>* Ms = reinterpret_cast<C2<T>*>(smem_raw);
  for (int m = 0; m < a.nmat; ++m) {
    const int cnt = a.mat_is_diag[m] ? s : ss;
    const bool ng = a.mat_neg[m] != 0;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      C2<T> v = from_d2<T>(a.mat[m][i]);
      if (ng) { v.x = -v.x; v.y = -v.y; }
      Ms[m * ss + i] = v;
    }
  }
  // scalar coefficients converted once per CTA (conjugation / negation applied)
  __shared__ C2<T> Sc[kMaxOut * kMaxTerm];
  if (threadIdx.x < kMaxOut * kMaxTerm) {
    const int oi = threadIdx.x / kMaxTerm, ti = threadIdx.x % kMaxTerm;
    C2<T> v = czero<T>();
    if (oi < a.nout && ti < a.o[oi].nterm && a.o[oi].t[ti].coef_kind == COEF_SCALAR)
      v = scalar_coef<T>(a.o[oi].t[ti].coef, a.o[oi].t[ti].conj, a.o[oi].t[ti].neg);
    Sc[threadIdx.x] = v;
  }
  __syncthreads();
  C2<T>* red_sm = Ms + a.nmat * ss;
  const int64_t rows_per_cta = (int64_t)(blockDim.x >> 5) * RPW;
  StencilCoef<T> sk{};
  if constexpr (SP) sk = stencil_coef<T>(sp);
  Acc<T, G, NG> acc;
  acc_zero(acc);
  for (int64_t base = (int64_t)blockIdx.x * rows_per_cta; base < n; base += (int64_t)gridDim.x * rows_per_cta) {
    const int64_t j = base + warp * RPW + lane / G;
    const bool rowok = j < n;
    const bool act = rowok && c < s;
    // the product's row, formed once (SRC_SPMM terms read it)
    C2<T> yprod = czero<T>();
    if constexpr (SP) yprod = spmm_row<T, G, 0>(sp, sk, j, c, rowok, act);
    C2<T> o[kMaxOut];
#pragma unroll
    for (int oi = 0; oi < kMaxOut; ++oi) o[oi] = czero<T>();
#pragma unroll
    for (int oi = 0; oi < kMaxOut; ++oi) {
      if (oi < a.nout) {
        const Out& out = a.o[oi];
        C2<T> val = czero<T>();
#pragma unroll
        for (int ti = 0; ti < kMaxTerm; ++ti) {
          if (ti < out.nterm) {
            const Term& t = out.t[ti];
            C2<T> x = czero<T>();
            if (t.src_kind == SRC_REG) {
              x = pick<T>(o, t.src_reg);
            } else if (t.src_kind == SRC_BLOCK) {
              if (act) x = reinterpret_cast<const C2<T>*>(t.src)[j * s + c];
            } else if (SP && t.src_kind == SRC_SPMM) {
              x = yprod;
            } else {
              if (rowok) x = reinterpret_cast<const C2<T>*>(t.src)[j];
            }
            x.y = neg_if(x.y, t.xconj);
            if (t.coef_kind == COEF_ONE) {
              x = mk<T>(neg_if(x.x, t.neg), neg_if(x.y, t.neg));
              if (ti == 0) val = x;  // leading copy: no add to zero
              else val = cadd<T>(val, x);
            } else if (t.coef_kind == COEF_REAL) {
              val = cfmareal<T>((T)t.creal, x, val);
            } else if (t.coef_kind == COEF_SCALAR) {
              val = cfma<T>(Sc[oi * kMaxTerm + ti], x, val);
            } else if (t.coef_kind == COEF_DIAG) {
              C2<T> d = (c < s) ? Ms[t.coef_idx * ss + c] : czero<T>();
              d = mk<T>(neg_if(d.x, t.neg), neg_if(d.y, (t.conj != 0) != (t.neg != 0)));
              val = cfma<T>(d, x, val);
            } else {  // COEF_MAT: val += sum_a x[j][a] * M[a][c]  (or minus)
              const C2<T>* M = Ms + t.coef_idx * ss;  // negation already folded into M
#pragma unroll
              for (int q = 0; q < G; ++q) {
                C2<T> xa = shfl<T>(x, grpbase + q);
                if (q < s && c < s) val = cfma<T>(xa, M[q * s + c], val);
              }
            }
          }
        }
        o[oi] = (out.is_vec ? rowok : act) ? val : czero<T>();
      }
    }
    if (rs.nred > 0) {
#pragma unroll
      for (int ri = 0; ri < kMaxRed; ++ri) {
        if (ri < rs.nred) {
          const RedSpec& r = rs.r[ri];
          const C2<T> y = pick<T>(o, r.ysrc);
          C2<T> u = czero<T>();
          if (r.ureg >= 0) {
            u = pick<T>(o, r.ureg);
          } else if (r.kind == RED_GRAM || r.kind == RED_TRACE || r.kind == RED_CDOT) {
            if (act) u = reinterpret_cast<const C2<T>*>(r.U)[j * s + c];
          } else if (r.kind == RED_SUMV || r.kind == RED_GRAMV) {
            if (rowok) u = reinterpret_cast<const C2<T>*>(r.U)[j];
          }
          red_add<T, G, NG>(r, ri, acc, y, u, s, grpbase);
        }
      }
    }
    // outputs are stored only after every operand of the row has been read: an output may
    // alias an operand, and with no store in between the loads can all be issued up front
#pragma unroll
    for (int oi = 0; oi < kMaxOut; ++oi) {
      if (oi < a.nout && a.o[oi].dst != nullptr) {
        if (a.o[oi].is_vec) {
          if (rowok && c == 0) reinterpret_cast<C2<T>*>(a.o[oi].dst)[j] = o[oi];
        } else if (act) {
          reinterpret_cast<C2<T>*>(a.o[oi].dst)[j * s + c] = o[oi];
        }
      }
    }
  }
  if (rs.nred > 0) cta_reduce<T, G, NG>(rs, acc, s, red_sm);
}

template <typename T, int G, int NG>
__global__ void __launch_bounds__(kThreads) lincomb_kernel(LinArgs a, RedSet rs, const int* done) {
  if (done != nullptr && *(volatile const int*)done) return;
  SpmmArgs<T> none{};
  lincomb_rows<T, G, NG, false>(a, rs, none);
}

// row-local combination whose terms include the sparse product (A V)[j] of `sp` (SRC_SPMM): the
// product's rows are formed in the same pass and never stored
template <typename T, int G, int NG>
__global__ void __launch_bounds__(kThreads) lincomb_spmm_kernel(LinArgs a, RedSet rs, SpmmArgs<T> sp,
                                                                const int* done) {
  if (done != nullptr && *(volatile const int*)done) return;
  lincomb_rows<T, G, NG, true>(a, rs, sp);
}

// ---------------------------------------------------------------------------------------
// Fixed-order sum of the CTA partial records: out[slot] = sum_p partials[p][slot] (in FP64)
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) reduce_slots_kernel(const C2<T>* partials, int nparts, int nslots,
                                                                double2* out, const int* done) {
  if (done != nullptr && *(volatile const int*)done) return;
  __shared__ double2 sm[kThreads / 32];
  const int slot = blockIdx.x;
  double2 sum = make_double2(0.0, 0.0);
  for (int p = threadIdx.x; p < nparts; p += blockDim.x) {
    const double2 v = to_d2(partials[(size_t)p * nslots + slot]);
    sum.x += v.x;
    sum.y += v.y;
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    sum.x += __shfl_down_sync(0xffffffffu, sum.x, off);
    sum.y += __shfl_down_sync(0xffffffffu, sum.y, off);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sm[warp] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 t = make_double2(0.0, 0.0);
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t.x += sm[w].x; t.y += sm[w].y; }
    out[slot] = t;
  }
}

}  // namespace kr
