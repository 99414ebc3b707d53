// Complex64 row kernels with two adjacent columns per thread.
//
// For complex64 blocks the per-element kernels are limited by instruction issue and
// memory latency rather than bandwidth: every complex column pays the index loads,
// address arithmetic and control flow of its row.  Here a thread owns the column pair
// (2p, 2p+1) of a row and moves it as one 16-byte vector, so that overhead is paid once
// per pair.  Used for even s when a launch has no s x s Gram and no s x s coefficient
// matrix (the global, economic and loop-interchanged methods); the other launches use
// the one-column kernels.
#pragma once

#include "kr_rows_impl.cuh"

namespace kr {

struct Pair {
  float2 a, b;  // columns 2p and 2p + 1
};

__device__ __forceinline__ Pair ld_pair(const float2* base, int64_t idx /* element index of column 2p */) {
  const float4 v = *reinterpret_cast<const float4*>(base + idx);
  Pair p;
  p.a = make_float2(v.x, v.y);
  p.b = make_float2(v.z, v.w);
  return p;
}
__device__ __forceinline__ void st_pair(float2* base, int64_t idx, Pair p) {
  *reinterpret_cast<float4*>(base + idx) = make_float4(p.a.x, p.a.y, p.b.x, p.b.y);
}
// Bulk prefetch of bytes [p, p + bytes) into L2 (one instruction for a whole row range;
// p and bytes multiples of 16, the range inside one allocation)
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Prefetch of bytes [lo, hi) of an allocation of `size` bytes starting at base: the range
// is widened to 16-byte boundaries but kept inside [0, size rounded down to 16).
__device__ __forceinline__ void prefetch_l2_range(const void* base, uint64_t lo, uint64_t hi, uint64_t size) {
  lo &= ~(uint64_t)15;
  hi = (hi + 15) & ~(uint64_t)15;
  const uint64_t cap = size & ~(uint64_t)15;
  if (hi > cap) hi = cap;
  if (hi > lo) prefetch_l2_bulk(reinterpret_cast<const char*>(base) + lo, (uint32_t)(hi - lo));
}

// The CSR product's operands for rows [r0, r1) into L2: row pointers, the column indices and
// values of those rows, the rows of V (the diagonal and nearby gathers), Z and of the
// reductions' memory operands.  One thread; it reads the two row pointers of the range.
__device__ __forceinline__ void prefetch_spmm_rows(const SpmmArgs<float>& a, const RedSet& rs, int64_t r0,
                                                   int64_t r1) {
  const int64_t n = a.n, s = a.s;
  prefetch_l2_range(a.rowptr, (uint64_t)r0 * 8, (uint64_t)(r1 + 1) * 8, (uint64_t)(n + 1) * 8);
  const int64_t k0 = a.rowptr[r0], k1 = a.rowptr[r1];
  const uint64_t nnz = (uint64_t)a.rowptr[n];
  prefetch_l2_range(a.colidx, (uint64_t)k0 * 4, (uint64_t)k1 * 4, nnz * 4);
  if (a.split) {
    prefetch_l2_range(a.offr, (uint64_t)k0 * 4, (uint64_t)k1 * 4, nnz * 4);
    prefetch_l2_range(a.diag, (uint64_t)r0 * 8, (uint64_t)r1 * 8, (uint64_t)n * 8);
  } else {
    prefetch_l2_range(a.vals, (uint64_t)k0 * 8, (uint64_t)k1 * 8, nnz * 8);
  }
  const uint64_t rb = (uint64_t)s * 8, total = (uint64_t)n * rb;
  prefetch_l2_range(a.V, (uint64_t)r0 * rb, (uint64_t)r1 * rb, total);
  if (a.Z != nullptr) prefetch_l2_range(a.Z, (uint64_t)r0 * rb, (uint64_t)r1 * rb, total);
#pragma unroll
  for (int ri = 0; ri < kMaxRed; ++ri)
    if (ri < rs.nred && rs.r[ri].U != nullptr && (rs.r[ri].kind == RED_TRACE || rs.r[ri].kind == RED_CDOT))
      prefetch_l2_range(rs.r[ri].U, (uint64_t)r0 * rb, (uint64_t)r1 * rb, total);
}

// The rows [r0, r0 + rows) of every block operand of a row-local launch, prefetched into L2
// by one thread; called kPrefetchAhead grid-stride iterations ahead of the rows' use.
constexpr int kPrefetchAhead = 2;

__device__ __forceinline__ void prefetch_rows(const LinArgs& a, const RedSet& rs, int64_t r0, int64_t rows) {
  if (rows <= 0) return;
  const uint32_t bytes = (uint32_t)(rows * a.s * sizeof(float2));
#pragma unroll
  for (int oi = 0; oi < kMaxOut; ++oi)
    if (oi < a.nout)
#pragma unroll
      for (int ti = 0; ti < kMaxTerm; ++ti)
        if (ti < a.o[oi].nterm && a.o[oi].t[ti].src_kind == SRC_BLOCK)
          prefetch_l2_bulk(reinterpret_cast<const float2*>(a.o[oi].t[ti].src) + r0 * a.s, bytes);
#pragma unroll
  for (int ri = 0; ri < kMaxRed; ++ri)
    if (ri < rs.nred && rs.r[ri].ureg < 0 && rs.r[ri].U != nullptr &&
        (rs.r[ri].kind == RED_TRACE || rs.r[ri].kind == RED_CDOT))
      prefetch_l2_bulk(reinterpret_cast<const float2*>(rs.r[ri].U) + r0 * a.s, bytes);
}

__device__ __forceinline__ Pair pzero() {
  Pair p;
  p.a = make_float2(0.f, 0.f);
  p.b = p.a;
  return p;
}

// accumulators of the fused reductions (kinds TRACE, SUMV, NORM2: one value; CDOT: one per column)
template <int NR = kMaxRed>
struct Acc2 {
  float2 v[NR][2];
};

template <int NR>
__device__ __forceinline__ void red2_add(const RedSpec& r, int ri, Acc2<NR>& acc, Pair y, Pair u) {
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    if (q == ri) {
      if (r.kind == RED_NORM2) {
        acc.v[q][0].x = fmaf(y.a.x, y.a.x, fmaf(y.a.y, y.a.y, acc.v[q][0].x));
        acc.v[q][0].x = fmaf(y.b.x, y.b.x, fmaf(y.b.y, y.b.y, acc.v[q][0].x));
      } else if (r.kind == RED_CDOT || r.kind == RED_GRAMV) {
        acc.v[q][0] = cfmaconj<float>(u.a, y.a, acc.v[q][0]);
        acc.v[q][1] = cfmaconj<float>(u.b, y.b, acc.v[q][1]);
      } else if (r.kind != RED_NONE) {  // TRACE, SUMV: one sum
        acc.v[q][0] = cfmaconj<float>(u.a, y.a, acc.v[q][0]);
        acc.v[q][0] = cfmaconj<float>(u.b, y.b, acc.v[q][0]);
      }
    }
  }
}

// fixed-order CTA reduction; GP threads per row (GP column pairs), s = 2 * number of pairs
template <int GP, int NR>
__device__ __forceinline__ void cta_reduce2(const RedSet& rs, Acc2<NR>& acc, int s, float2* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int ns = rs.nslots;
  const int npairs = s / 2;
#pragma unroll
  for (int ri = 0; ri < NR; ++ri) {
    if (ri < rs.nred) {
      const RedSpec& r = rs.r[ri];
      if (r.kind == RED_CDOT || r.kind == RED_GRAMV) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float2 v = acc.v[ri][h];
#pragma unroll
          for (int off = 16; off >= GP; off >>= 1) v = cadd<float>(v, shfl_down<float>(v, off));
          if (lane < npairs) sm[warp * ns + r.slot + 2 * lane + h] = v;
        }
      } else {
        float2 v = acc.v[ri][0];
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) v = cadd<float>(v, shfl_down<float>(v, off));
        if (lane == 0) sm[warp * ns + r.slot] = v;
      }
    }
  }
  __syncthreads();
  float2* out = reinterpret_cast<float2*>(rs.partials) + (size_t)blockIdx.x * ns;
  for (int t = threadIdx.x; t < ns; t += blockDim.x) {
    float2 sum = make_float2(0.f, 0.f);
    for (int w = 0; w < nw; ++w) sum = cadd<float>(sum, sm[w * ns + t]);
    out[t] = sum;
  }
}

// (A V)[j] for the column pair p of row j (e = j * s + 2p, the pair's first element), before any
// scaling: the matrix-free stencil (STENCIL) or the CSR product.  TAILBATCH: spend registers on
// loads in flight -- CSR: the last 1-3 entries of a row as one predicated batch (without it one
// entry at a time); stencil: every neighbour's load before the FMAs (without it one at a time).
template <bool STENCIL, bool TAILBATCH>
__device__ __forceinline__ Pair spmm2_row(const SpmmArgs<float>& a, const float2 stc, const float2 (&stm)[3],
                                          const float2 (&stp)[3], int64_t j, int p, int64_t e) {
  const int s = a.s;
  const int npairs = s / 2;
  Pair y = pzero();
  if constexpr (STENCIL) {
    int64_t xc[3];
    grid_coords<3>(j, a.nst, a.sdiv32, a.sdims, a.sdiv, xc);
    if constexpr (TAILBATCH) {
      // all seven loads before the FMAs (an absent neighbour loads the centre again, unused)
      bool has[6];
      int64_t off[6];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int qa = 2 - q;
        has[q] = qa < a.nst && xc[qa] > 0;
        off[q] = has[q] ? -a.sstr[qa] * s : 0;
        has[3 + q] = q < a.nst && xc[q] < a.sdims[q] - 1;
        off[3 + q] = has[3 + q] ? a.sstr[q] * s : 0;
      }
      const Pair xv = ld_pair(a.V, e);
      Pair x[6];
#pragma unroll
      for (int m = 0; m < 6; ++m) x[m] = ld_pair(a.V, e + off[m]);
      y.a = cmul<float>(stc, xv.a);
      y.b = cmul<float>(stc, xv.b);
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        if (has[m]) {
          const float2 k = m < 3 ? stm[2 - m] : stp[m - 3];
          if (a.sreal) { y.a = cfmareal<float>(k.x, x[m].a, y.a); y.b = cfmareal<float>(k.x, x[m].b, y.b); }
          else { y.a = cfma<float>(k, x[m].a, y.a); y.b = cfma<float>(k, x[m].b, y.b); }
        }
      }
    } else {
      const Pair xv = ld_pair(a.V, e);
      y.a = cmul<float>(stc, xv.a);
      y.b = cmul<float>(stc, xv.b);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int qa = 2 - q;
        if (qa < a.nst && xc[qa] > 0) {
          const Pair x = ld_pair(a.V, e - a.sstr[qa] * s);
          if (a.sreal) { y.a = cfmareal<float>(stm[qa].x, x.a, y.a); y.b = cfmareal<float>(stm[qa].x, x.b, y.b); }
          else { y.a = cfma<float>(stm[qa], x.a, y.a); y.b = cfma<float>(stm[qa], x.b, y.b); }
        }
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (q < a.nst && xc[q] < a.sdims[q] - 1) {
          const Pair x = ld_pair(a.V, e + a.sstr[q] * s);
          if (a.sreal) { y.a = cfmareal<float>(stp[q].x, x.a, y.a); y.b = cfmareal<float>(stp[q].x, x.b, y.b); }
          else { y.a = cfma<float>(stp[q], x.a, y.a); y.b = cfma<float>(stp[q], x.b, y.b); }
        }
      }
    }
  } else {
    const int64_t k0 = a.rowptr[j], k1 = a.rowptr[j + 1];
    // gathers address V as float4 (one column pair) with 32-bit column indices:
    // row c, pair p is element c * npairs + p (a 32 x 32 -> 64-bit multiply)
    const float4* Vq = reinterpret_cast<const float4*>(a.V) + p;
    const uint32_t np = (uint32_t)npairs;
    auto gather = [&](int32_t c) {
      const float4 v = Vq[(uint64_t)(uint32_t)c * np];
      Pair q;
      q.a = make_float2(v.x, v.y);
      q.b = make_float2(v.z, v.w);
      return q;
    };
    int64_t k = k0;
    if (a.split) {
      const float2 dgv = a.diag[j];
      const Pair xv = ld_pair(a.V, e);
      y.a = cmul<float>(dgv, xv.a);
      y.b = cmul<float>(dgv, xv.b);
      // full batches of four entries: indices, values and gathered pairs all in flight
      for (; k + 4 <= k1; k += 4) {
        int32_t col[4];
        float v[4];
        Pair x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) { col[u] = a.colidx[k + u]; v[u] = a.offr[k + u]; }
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = gather(col[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u) { y.a = cfmareal<float>(v[u], x[u].a, y.a); y.b = cfmareal<float>(v[u], x[u].b, y.b); }
      }
      // the last 1-3 entries as one predicated batch: their loads are in flight together
      // instead of one dependent index load and gather after another (with four
      // accumulator slots this no longer fits the 64 registers: one entry at a time)
      const int rem = (int)(k1 - k);
      if constexpr (!TAILBATCH) {
        for (; k < k1; ++k) {
          const float v = a.offr[k];
          const Pair x = gather(a.colidx[k]);
          y.a = cfmareal<float>(v, x.a, y.a);
          y.b = cfmareal<float>(v, x.b, y.b);
        }
      } else if (rem > 0) {
        int32_t col[3];
        float v[3];
        Pair x[3];
#pragma unroll
        for (int u = 0; u < 3; ++u)
          if (u < rem) { col[u] = a.colidx[k + u]; v[u] = a.offr[k + u]; }
#pragma unroll
        for (int u = 0; u < 3; ++u)
          if (u < rem) x[u] = gather(col[u]);
#pragma unroll
        for (int u = 0; u < 3; ++u)
          if (u < rem) { y.a = cfmareal<float>(v[u], x[u].a, y.a); y.b = cfmareal<float>(v[u], x[u].b, y.b); }
      }
    } else {
      for (; k + 4 <= k1; k += 4) {
        int32_t col[4];
        float2 v[4];
        Pair x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) { col[u] = a.colidx[k + u]; v[u] = a.vals[k + u]; }
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = gather(col[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u) { y.a = cfma<float>(v[u], x[u].a, y.a); y.b = cfma<float>(v[u], x[u].b, y.b); }
      }
      const int rem = (int)(k1 - k);
      if constexpr (!TAILBATCH) {
        for (; k < k1; ++k) {
          const float2 v = a.vals[k];
          const Pair x = gather(a.colidx[k]);
          y.a = cfma<float>(v, x.a, y.a);
          y.b = cfma<float>(v, x.b, y.b);
        }
      } else if (rem > 0) {
        int32_t col[3];
        float2 v[3];
        Pair x[3];
#pragma unroll
        for (int u = 0; u < 3; ++u)
          if (u < rem) { col[u] = a.colidx[k + u]; v[u] = a.vals[k + u]; }
#pragma unroll
        for (int u = 0; u < 3; ++u)
          if (u < rem) x[u] = gather(col[u]);
#pragma unroll
        for (int u = 0; u < 3; ++u)
          if (u < rem) { y.a = cfma<float>(v[u], x[u].a, y.a); y.b = cfma<float>(v[u], x[u].b, y.b); }
      }
    }
  }
  return y;
}

// ---------------------------------------------------------------------------------------
// SpMM (CSR, real-off-diagonal CSR or stencil) on column pairs
// ---------------------------------------------------------------------------------------
// STENCIL: the matrix-free stencil (a.nst > 0) or CSR; NR: accumulators for up to NR fused
// reductions (rs.nred <= NR).  Separate instantiations keep the stencil's coefficients and
// unused accumulators out of the registers of the CSR loop.
template <int GP, bool STENCIL, int NR>
__global__ void __launch_bounds__(kThreads, kCtasPerSmRows) spmm2_kernel(SpmmArgs<float> a, RedSet rs, const int* done) {
  if (done != nullptr && *(volatile const int*)done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int RPW = 32 / GP;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int p = lane & (GP - 1);  // column pair
  const int s = a.s;
  const int npairs = s / 2;
  const int64_t n = a.n;
  const int64_t rows_per_cta = (int64_t)(blockDim.x >> 5) * RPW;
  float2 ysc = make_float2((float)a.ay, 0.f);
  const bool scaled = a.ys != nullptr || a.ay != 1.0;
  if (a.ys != nullptr) {
    const float2 d = scalar_coef<float>(a.ys, a.ys_conj, a.ys_neg);
    ysc = make_float2((float)a.ay * d.x, (float)a.ay * d.y);
  }
  const float bz = (float)a.bz;
  float2 stc = make_float2(0.f, 0.f), stm[3], stp[3];
  if constexpr (STENCIL) {
    stc = make_float2((float)a.sc.x, (float)a.sc.y);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      stm[q] = make_float2((float)a.sm[q].x, (float)a.sm[q].y);
      stp[q] = make_float2((float)a.sp[q].x, (float)a.sp[q].y);
    }
  }
  Acc2<NR> acc;
#pragma unroll
  for (int q = 0; q < NR; ++q) acc.v[q][0] = acc.v[q][1] = make_float2(0.f, 0.f);
  const int64_t stride = (int64_t)gridDim.x * rows_per_cta;
  // CSR with s >= 8: the next rows' matrix entries and operands into L2 (measured: 6-9 % on the
  // fused product at s = 8-32; at s = 2 the row-pointer reads of the prefetching thread cost more)
  const bool pf = !STENCIL && s >= 8;
  if (pf && threadIdx.x == 0) {
    for (int k = 0; k < kPrefetchAhead; ++k) {
      const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta + k * stride;
      if (r0 < n) prefetch_spmm_rows(a, rs, r0, r0 + rows_per_cta < n ? r0 + rows_per_cta : n);
    }
  }
  for (int64_t base = (int64_t)blockIdx.x * rows_per_cta; base < n; base += stride) {
    if (pf && threadIdx.x == 0) {
      const int64_t r0 = base + kPrefetchAhead * stride;
      if (r0 < n) prefetch_spmm_rows(a, rs, r0, r0 + rows_per_cta < n ? r0 + rows_per_cta : n);
    }
    const int64_t j = base + warp * RPW + lane / GP;
    const bool rowok = j < n;
    const bool act = rowok && p < npairs;
    const int64_t e = j * s + 2 * p;  // element index of column 2p in row j
    Pair y = pzero();
    // CSR with at most two reductions: memory operands of the reductions loaded before the
    // product (not after the store of Y), unless the operand is Y itself
    constexpr bool kPre = !STENCIL && NR <= 2;
    Pair upre[NR];
    if constexpr (kPre) {
#pragma unroll
      for (int ri = 0; ri < NR; ++ri) {
        upre[ri] = pzero();
        if (ri < rs.nred && act && (rs.r[ri].kind == RED_TRACE || rs.r[ri].kind == RED_CDOT) &&
            rs.r[ri].U != nullptr && rs.r[ri].U != static_cast<const void*>(a.Y))
          upre[ri] = ld_pair(reinterpret_cast<const float2*>(rs.r[ri].U), e);
      }
    }
    if (act) {
      y = spmm2_row<STENCIL, (NR <= 2)>(a, stc, stm, stp, j, p, e);
      if (scaled) { y.a = cmul<float>(ysc, y.a); y.b = cmul<float>(ysc, y.b); }
      if (a.Z != nullptr) {
        const Pair z = ld_pair(a.Z, e);
        y.a.x = fmaf(bz, z.a.x, y.a.x); y.a.y = fmaf(bz, z.a.y, y.a.y);
        y.b.x = fmaf(bz, z.b.x, y.b.x); y.b.y = fmaf(bz, z.b.y, y.b.y);
      }
      if (a.Y != nullptr) st_pair(a.Y, e, y);
    }
    if (rs.nred > 0) {
#pragma unroll
      for (int ri = 0; ri < NR; ++ri) {
        if (ri < rs.nred) {
          const RedSpec& r = rs.r[ri];
          Pair u = pzero();
          if (r.kind == RED_TRACE || r.kind == RED_CDOT) {
            if (act) {
              if (r.U == nullptr) u = y;
              else if (kPre && r.U != static_cast<const void*>(a.Y)) u = upre[ri];
              else u = ld_pair(reinterpret_cast<const float2*>(r.U), e);
            }
          } else if (r.kind == RED_SUMV || r.kind == RED_GRAMV) {
            if (act) { u.a = reinterpret_cast<const float2*>(r.U)[j]; u.b = u.a; }
          }
          red2_add(r, ri, acc, y, u);
        }
      }
    }
  }
  if (rs.nred > 0) cta_reduce2<GP, NR>(rs, acc, s, reinterpret_cast<float2*>(smem_raw));
}

// ---------------------------------------------------------------------------------------
// Row-local linear combinations on column pairs (no s x s coefficient matrices)
// ---------------------------------------------------------------------------------------
// SP: the combination has SRC_SPMM terms, products of `sp` formed row by row in this pass
template <int GP, bool SP>
__device__ __forceinline__ void lincomb2_rows(const LinArgs& a, const RedSet& rs, const SpmmArgs<float>& sp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int RPW = 32 / GP;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int p = lane & (GP - 1);
  const int s = a.s;
  const int npairs = s / 2;
  const int64_t n = a.n;
  // scalar coefficients once per CTA; diagonal coefficients (per column) in shared memory
  __shared__ float2 Sc[kMaxOut * kMaxTerm];
  float2* Dg = reinterpret_cast<float2*>(smem_raw);  // nmat x s
  for (int m = 0; m < a.nmat; ++m) {
    for (int i = threadIdx.x; i < s; i += blockDim.x) {
      float2 v = from_d2<float>(a.mat[m][i]);
      if (a.mat_neg[m]) { v.x = -v.x; v.y = -v.y; }
      Dg[m * s + i] = v;
    }
  }
  if (threadIdx.x < kMaxOut * kMaxTerm) {
    const int oi = threadIdx.x / kMaxTerm, ti = threadIdx.x % kMaxTerm;
    float2 v = make_float2(0.f, 0.f);
    if (oi < a.nout && ti < a.o[oi].nterm && a.o[oi].t[ti].coef_kind == COEF_SCALAR)
      v = scalar_coef<float>(a.o[oi].t[ti].coef, a.o[oi].t[ti].conj, a.o[oi].t[ti].neg);
    Sc[threadIdx.x] = v;
  }
  __syncthreads();
  float2* red_sm = Dg + a.nmat * s;
  const int64_t rows_per_cta = (int64_t)(blockDim.x >> 5) * RPW;
  // the product's stencil coefficients, converted once (double -> float runs on the FP64 pipe)
  float2 stc = make_float2(0.f, 0.f), stm[3], stp[3];
  if constexpr (SP) {
    stc = make_float2((float)sp.sc.x, (float)sp.sc.y);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      stm[q] = make_float2((float)sp.sm[q].x, (float)sp.sm[q].y);
      stp[q] = make_float2((float)sp.sp[q].x, (float)sp.sp[q].y);
    }
  }
  Acc2<> acc;
#pragma unroll
  for (int q = 0; q < kMaxRed; ++q) acc.v[q][0] = acc.v[q][1] = make_float2(0.f, 0.f);
  const int64_t stride = (int64_t)gridDim.x * rows_per_cta;
  // prefetch only for launches streaming 3 or more blocks, read or written (measured: a
  // slight loss on a 2-block reduction, 15-20 % faster solver updates with 3-6 blocks)
  int nblk = 0;
#pragma unroll
  for (int oi = 0; oi < kMaxOut; ++oi) {
    if (oi < a.nout) {
      if (a.o[oi].dst != nullptr) ++nblk;
#pragma unroll
      for (int ti = 0; ti < kMaxTerm; ++ti)
        if (ti < a.o[oi].nterm && a.o[oi].t[ti].src_kind == SRC_BLOCK) ++nblk;
    }
  }
  const bool pf = nblk >= 3;
  if (pf && threadIdx.x == 0) {
    // the rows of the first iterations; the loop below keeps kPrefetchAhead iterations ahead
    for (int k = 0; k < kPrefetchAhead; ++k) {
      const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta + k * stride;
      if (r0 < n) prefetch_rows(a, rs, r0, r0 + rows_per_cta < n ? rows_per_cta : n - r0);
    }
  }
  for (int64_t base = (int64_t)blockIdx.x * rows_per_cta; base < n; base += stride) {
    if (pf && threadIdx.x == 0) {
      const int64_t r0 = base + kPrefetchAhead * stride;
      if (r0 < n) prefetch_rows(a, rs, r0, r0 + rows_per_cta < n ? rows_per_cta : n - r0);
    }
    const int64_t j = base + warp * RPW + lane / GP;
    const bool rowok = j < n;
    const bool act = rowok && p < npairs;
    const int64_t e = j * s + 2 * p;
    // the product's row pair, formed once (SRC_SPMM terms read it)
    Pair yprod = pzero();
    if constexpr (SP) {
      // the row's last 1-3 entries one at a time (fewer registers next to the outputs)
      if (act) yprod = sp.nst > 0 ? spmm2_row<true, false>(sp, stc, stm, stp, j, p, e)
                                  : spmm2_row<false, false>(sp, stc, stm, stp, j, p, e);
    }
    // outputs as two register arrays (columns 2p and 2p + 1), selected with constant indices
    float2 oa[kMaxOut], ob[kMaxOut];
#pragma unroll
    for (int oi = 0; oi < kMaxOut; ++oi) oa[oi] = ob[oi] = make_float2(0.f, 0.f);
#pragma unroll
    for (int oi = 0; oi < kMaxOut; ++oi) {
      if (oi < a.nout) {
        const Out& out = a.o[oi];
        Pair val = pzero();
#pragma unroll
        for (int ti = 0; ti < kMaxTerm; ++ti) {
          if (ti < out.nterm) {
            const Term& t = out.t[ti];
            Pair x = pzero();
            if (t.src_kind == SRC_REG) {
              x.a = pick<float>(oa, t.src_reg);
              x.b = pick<float>(ob, t.src_reg);
            } else if (t.src_kind == SRC_BLOCK) {
              if (act) x = ld_pair(reinterpret_cast<const float2*>(t.src), e);
            } else if (SP && t.src_kind == SRC_SPMM) {
              x = yprod;
            } else {
              if (act) { x.a = reinterpret_cast<const float2*>(t.src)[j]; x.b = x.a; }
            }
            if (t.xconj) { x.a.y = -x.a.y; x.b.y = -x.b.y; }
            if (t.coef_kind == COEF_ONE) {
              if (ti == 0) {
                val = x;
                if (t.neg) { val.a = make_float2(-x.a.x, -x.a.y); val.b = make_float2(-x.b.x, -x.b.y); }
              } else if (t.neg) {
                val.a = csub<float>(val.a, x.a); val.b = csub<float>(val.b, x.b);
              } else {
                val.a = cadd<float>(val.a, x.a); val.b = cadd<float>(val.b, x.b);
              }
            } else if (t.coef_kind == COEF_REAL) {
              val.a = cfmareal<float>((float)t.creal, x.a, val.a);
              val.b = cfmareal<float>((float)t.creal, x.b, val.b);
            } else if (t.coef_kind == COEF_SCALAR) {
              const float2 cs = Sc[oi * kMaxTerm + ti];
              val.a = cfma<float>(cs, x.a, val.a);
              val.b = cfma<float>(cs, x.b, val.b);
            } else {  // COEF_DIAG
              float2 d0 = make_float2(0.f, 0.f), d1 = d0;
              if (p < npairs) { d0 = Dg[t.coef_idx * s + 2 * p]; d1 = Dg[t.coef_idx * s + 2 * p + 1]; }
              if (t.conj) { d0.y = -d0.y; d1.y = -d1.y; }
              if (t.neg) { d0 = make_float2(-d0.x, -d0.y); d1 = make_float2(-d1.x, -d1.y); }
              val.a = cfma<float>(d0, x.a, val.a);
              val.b = cfma<float>(d1, x.b, val.b);
            }
          }
        }
        if (!act) val = pzero();
        oa[oi] = val.a;
        ob[oi] = val.b;
      }
    }
    if (rs.nred > 0) {
#pragma unroll
      for (int ri = 0; ri < kMaxRed; ++ri) {
        if (ri < rs.nred) {
          const RedSpec& r = rs.r[ri];
          Pair y, u = pzero();
          y.a = pick<float>(oa, r.ysrc);
          y.b = pick<float>(ob, r.ysrc);
          if (r.ureg >= 0) {
            u.a = pick<float>(oa, r.ureg);
            u.b = pick<float>(ob, r.ureg);
          } else if (r.kind == RED_TRACE || r.kind == RED_CDOT) {
            if (act) u = ld_pair(reinterpret_cast<const float2*>(r.U), e);
          } else if (r.kind == RED_SUMV || r.kind == RED_GRAMV) {
            if (act) { u.a = reinterpret_cast<const float2*>(r.U)[j]; u.b = u.a; }
          }
          red2_add(r, ri, acc, y, u);
        }
      }
    }
    // stores after every operand of the row has been read (an output may alias an operand)
#pragma unroll
    for (int oi = 0; oi < kMaxOut; ++oi) {
      if (oi < a.nout && a.o[oi].dst != nullptr && act) {
        Pair v;
        v.a = oa[oi];
        v.b = ob[oi];
        st_pair(reinterpret_cast<float2*>(a.o[oi].dst), e, v);
      }
    }
  }
  if (rs.nred > 0) cta_reduce2<GP, kMaxRed>(rs, acc, s, red_sm);
}

template <int GP>
__global__ void __launch_bounds__(kThreads, kCtasPerSmRows) lincomb2_kernel(LinArgs a, RedSet rs, const int* done) {
  if (done != nullptr && *(volatile const int*)done) return;
  SpmmArgs<float> none{};
  lincomb2_rows<GP, false>(a, rs, none);
}

// column-pair combination whose terms include the sparse product of `sp` (SRC_SPMM), formed in
// the same pass and never stored
template <int GP>
__global__ void __launch_bounds__(kThreads, kCtasPerSmRows) lincomb2_spmm_kernel(LinArgs a, RedSet rs,
                                                                                 SpmmArgs<float> sp,
                                                                                 const int* done) {
  if (done != nullptr && *(volatile const int*)done) return;
  lincomb2_rows<GP, true>(a, rs, sp);
}

// Can this launch run on column pairs?  Even s, 16-byte aligned blocks, no s x s Gram,
// no s x s coefficient matrix and no n-vector output (those keep the one-column kernels).
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline bool pair_ok_reds(const RedSet& rs) {
  for (int i = 0; i < rs.nred; ++i) {
    const RedSpec& r = rs.r[i];
    if (r.kind == RED_GRAM) return false;
    if ((r.kind == RED_TRACE || r.kind == RED_CDOT) && r.ureg < 0 && r.U != nullptr && !aligned16(r.U)) return false;
  }
  return true;
}
inline bool pair_ok_spmm(const SpmmArgs<float>& a, const RedSet& rs) {
  if (a.s < 2 || a.s % 2 != 0) return false;
  if (!aligned16(a.V) || !aligned16(a.Y) || !aligned16(a.Z)) return false;
  return pair_ok_reds(rs);
}
inline bool pair_ok_lin(const LinArgs& a, const RedSet& rs) {
  if (a.s < 2 || a.s % 2 != 0) return false;
  for (int m = 0; m < a.nmat; ++m)
    if (!a.mat_is_diag[m]) return false;
  for (int o = 0; o < a.nout; ++o) {
    if (a.o[o].is_vec || !aligned16(a.o[o].dst)) return false;
    for (int t = 0; t < a.o[o].nterm; ++t) {
      const Term& tm = a.o[o].t[t];
      if (tm.coef_kind == COEF_MAT) return false;
      if (tm.src_kind == SRC_BLOCK && !aligned16(tm.src)) return false;
      if (tm.src_kind == SRC_SPMM && tm.coef_kind == COEF_MAT) return false;
    }
  }
  return pair_ok_reds(rs);
}

}  // namespace kr
