// Complex64 CSR product with fused reductions, row tiles staged by TMA bulk copies.
//
// The product Y = A V of the complex64 inner solves reads the matrix once for all s columns
// (Sec. 1 of the paper).  The per-thread kernels (kr_rows_vec2.cuh) chain three dependent
// global loads per row -- row pointers, the row's indices and values, then the gathered rows
// of V -- and stay latency-bound near half of HBM; with a fused s x s Gram their s
// accumulators per thread cost occupancy as well.  Here each CTA walks row tiles of R rows:
//
//   * one thread issues 1D bulk copies (cp.async.bulk, completion on an mbarrier) of the
//     tile's row pointers, complex diagonal and the reductions' U blocks three tiles ahead (and
//     a bulk L2 prefetch of the tile's rows of V),
//     and of the tile's column indices and values one tile ahead (their range is read from
//     the row pointers already in shared memory), so only the gathers of V remain
//     synchronous loads;
//   * GP = s/2 threads per row, each owning a column pair (16-byte gathers and stores); a
//     row's entries come from shared memory and all its gathers are in flight together;
//   * fused s x s Grams U^H Y are formed after each tile from shared-memory copies of Y and U,
//     every thread owning a 2 x 2 block of entries for a subset of the tile's rows, so the
//     Gram costs neither registers in the product nor occupancy;
//   * per-row reductions (trace, column dots, norm, economic sums) accumulate as in the
//     column-pair kernel.
//
// Every output entry is computed with the operations and in the order of the other product
// kernels (diagonal first, then the stored entries in order), so Y is bitwise the same; the
// partial sums of the reductions are grouped differently and agree to FP32 rounding.  The CTA
// partial records have the layout of the other kernels (same slots), reduced by
// reduce_slots_kernel in a fixed order.
//
// Every mbarrier wait is bounded.  A wait that runs out (which correct copies never do) makes
// the CTA stop computing: all of its threads leave together at the next barrier, after waiting
// (again bounded) for the copies they issued, with NaN in the CTA's partial record and the
// device counter g_kr_wait_timeouts incremented (kr_take_device_timeouts reads it).
#pragma once

#include "kr_rows_vec2.cuh"
#include "kr_tile_c64.h"

namespace kr {

constexpr unsigned kWaitPolls = 1u << 22;  // ~1 s of polling with the back-off below

// waits that ran out (see above): counted on the device, read by kr_take_device_timeouts
static __device__ unsigned int g_kr_wait_timeouts = 0;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase of the given parity; false when the limit ran out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (unsigned i = 0; i < kWaitPolls; ++i) {
    if (mbar_test(bar, parity)) return true;
    if (i >= 32) __nanosleep(200);
  }
  return false;
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16) completing on bar
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Rings of mbarrier stages: bookkeeping packed into bits.  Parity words hold, per stage k, the
// parity of the next phase to consume (bit k); armed words hold bit 2k = stage k armed at least
// once and bit 2k + 1 = parity of its number of arms.
__device__ __forceinline__ void note_armed(uint32_t& m, int k) {
  m |= 1u << (2 * k);
  m ^= 1u << (2 * k + 1);
}
// bounded wait for the last phase armed on each of N barriers (the drain of an abort)
template <int N>
__device__ __forceinline__ void drain_stages(uint64_t* bar, uint32_t m) {
#pragma unroll
  for (int k = 0; k < N; ++k)
    if ((m >> (2 * k)) & 1u) mbar_wait(&bar[k], ((m >> (2 * k + 1)) & 1u) ^ 1u);
}
// consume the next phase of stage k: bounded wait, then flip the stage's parity bit
__device__ __forceinline__ bool take_phase(uint64_t* bar, uint32_t& par, int k) {
  const bool ok = mbar_wait(&bar[k], (par >> k) & 1u);
  par ^= 1u << k;
  return ok;
}

__device__ __forceinline__ uint32_t round16(uint64_t b) { return (uint32_t)((b + 15) & ~(uint64_t)15); }

// operator storage of a tile launch
enum TileMode : int { TILE_CSR = 0, TILE_SPLIT = 1, TILE_STENCIL = 2 };

template <int GP, int MODE>
struct TileKernel {
  static constexpr int S = 2 * GP;           // columns
  static constexpr int NB = GP * GP;         // 2 x 2 Gram blocks
  static constexpr bool SPLIT = MODE == TILE_SPLIT;
  static constexpr bool STEN = MODE == TILE_STENCIL;

  // A-stage copies of a tile into stage `sm`: row pointers and diagonal (CSR), U operands; and a
  // bulk L2 prefetch of the tile's rows of V
  static __device__ void issue_a(const SpmmArgs<float>& a, const TileLayout& L, unsigned char* sm, uint64_t* bar,
                                 int64_t r0, int rows) {
    const uint32_t brp = STEN ? 0 : round16((uint64_t)(rows + 1) * 8);
    const uint32_t bdg = SPLIT ? round16((uint64_t)rows * 8) : 0;
    const uint32_t bu = (uint32_t)rows * S * 8;  // a multiple of 16 (S even)
    mbar_arrive_expect(bar, brp + bdg + bu * L.nu);
    // the tile's own rows of V into L2 (gathered by its diagonal and by the neighbouring tiles'
    // rows, which other CTAs process at about the same time): one instruction, no completion
    prefetch_l2_bulk(reinterpret_cast<const float2*>(a.V) + r0 * S, bu);
    if (!STEN) bulk_load(sm + L.off_rp, a.rowptr + r0, brp, bar);
    if (SPLIT) bulk_load(sm + L.off_dg, a.diag + r0, bdg, bar);
    for (int u = 0; u < L.nu; ++u)
      bulk_load(sm + L.off_u + u * L.sz_u, reinterpret_cast<const float2*>(L.U[u]) + r0 * S, bu, bar);
  }

  // B-stage copies (CSR): the tile's entries [k0 & ~3, k1), read from the staged row pointers
  static __device__ void issue_b(const SpmmArgs<float>& a, const TileLayout& L, unsigned char* sm_b,
                                 const int64_t* rp, uint64_t* bar, int rows) {
    const int64_t k0 = rp[0] & ~(int64_t)3, k1 = rp[rows];
    const uint32_t bc = round16((uint64_t)(k1 - k0) * 4);
    const uint32_t bv = round16((uint64_t)(k1 - k0) * (SPLIT ? 4 : 8));
    mbar_arrive_expect(bar, bc + bv);
    if (k1 > k0) {
      bulk_load(sm_b + L.off_col, a.colidx + k0, bc, bar);
      if (SPLIT) bulk_load(sm_b + L.off_val, a.offr + k0, bv, bar);
      else bulk_load(sm_b + L.off_val, a.vals + k0, bv, bar);
    }
  }
};

// 2 x 2 block (a0..a0+1) x (c0..c0+1) of U^H Y over the rows grow, grow + RG, ... of a tile
template <int S>
__device__ __forceinline__ void gram_rows(const float2* Us, const float2* Yt, int a0, int c0, int grow, int RG,
                                          int rows, float2& x00, float2& x01, float2& x10, float2& x11) {
  for (int r = grow; r < rows; r += RG) {
    const float4 u = *reinterpret_cast<const float4*>(Us + r * S + a0);
    const float4 y = *reinterpret_cast<const float4*>(Yt + r * S + c0);
    const float2 ua = make_float2(u.x, u.y), ub = make_float2(u.z, u.w);
    const float2 ya = make_float2(y.x, y.y), yb = make_float2(y.z, y.w);
    x00 = cfmaconj<float>(ua, ya, x00);
    x01 = cfmaconj<float>(ua, yb, x01);
    x10 = cfmaconj<float>(ub, ya, x10);
    x11 = cfmaconj<float>(ub, yb, x11);
  }
}

template <int S>
__device__ __forceinline__ void gram_stage_block(float2* G, int a0, int c0, float2 x00, float2 x01, float2 x10,
                                                 float2 x11) {
  G[a0 * S + c0] = x00;
  G[a0 * S + c0 + 1] = x01;
  G[(a0 + 1) * S + c0] = x10;
  G[(a0 + 1) * S + c0 + 1] = x11;
}


// Fixed-order CTA reduction of the fused reductions into the CTA's partial record (slots as in
// the other row kernels), reusing shared memory from `sm`: per-row reductions summed over warps
// in order, Grams over row groups in order.  acc: per-thread sums of the per-row reductions (column
// pair tid % GP); g0, g1: this thread's 2 x 2 block (ga0, gc0) of each Gram over row group grow.
template <int GP, int NG>
__device__ __forceinline__ void cta_partials(unsigned char* sm, const RedSet& rs, const TileLayout& L,
                                             const Acc2<kTileRowReds>& acc, const float2 (&g0)[4],
                                             const float2 (&g1)[4], int grow, int RG, int ga0, int gc0) {
  constexpr int S = 2 * GP;
  const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5;
  float2* red = reinterpret_cast<float2*>(sm);  // [warp][compact per-row slots]
  const int nw = T >> 5;
  float2* gred = red + nw * L.ncompact;         // [gram][row group][s x s]
#pragma unroll
  for (int ri = 0; ri < kMaxRed; ++ri) {
    if (ri < rs.nred && rs.r[ri].kind != RED_GRAM) {
      const RedSpec& r = rs.r[ri];
      const int k = L.red_k[ri];
      float2* dst = red + warp * L.ncompact + L.red_c[ri];
      float2 v0 = acc.v[0][0], v1 = acc.v[0][1];
      if (k == 1) { v0 = acc.v[1][0]; v1 = acc.v[1][1]; }
      if (r.kind == RED_CDOT || r.kind == RED_GRAMV) {
#pragma unroll
        for (int off = 16; off >= GP; off >>= 1) {
          v0 = cadd<float>(v0, shfl_down<float>(v0, off));
          v1 = cadd<float>(v1, shfl_down<float>(v1, off));
        }
        if (lane < GP) { dst[2 * lane] = v0; dst[2 * lane + 1] = v1; }
      } else {
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) v0 = cadd<float>(v0, shfl_down<float>(v0, off));
        if (lane == 0) dst[0] = v0;
      }
    }
  }
  if (NG > 0 && grow < RG) {
    gram_stage_block<S>(gred + (size_t)grow * S * S, ga0, gc0, g0[0], g0[1], g0[2], g0[3]);
    if (NG > 1) gram_stage_block<S>(gred + ((size_t)RG + grow) * S * S, ga0, gc0, g1[0], g1[1], g1[2], g1[3]);
  }
  __syncthreads();
  float2* out = reinterpret_cast<float2*>(rs.partials) + (size_t)blockIdx.x * rs.nslots;
  for (int ri = 0; ri < rs.nred; ++ri) {  // per-row reductions: sum over warps in order
    const RedSpec& r = rs.r[ri];
    if (r.kind == RED_GRAM) continue;
    const int cnt = (r.kind == RED_CDOT || r.kind == RED_GRAMV) ? S : 1;
    for (int q = tid; q < cnt; q += T) {
      float2 sum = make_float2(0.f, 0.f);
      for (int w = 0; w < nw; ++w) sum = cadd<float>(sum, red[w * L.ncompact + L.red_c[ri] + q]);
      out[r.slot + q] = sum;
    }
  }
  for (int gi = 0; gi < NG; ++gi) {  // Grams: sum over row groups in order
    for (int q = tid; q < S * S; q += T) {
      float2 sum = make_float2(0.f, 0.f);
      for (int g = 0; g < RG; ++g) sum = cadd<float>(sum, gred[((size_t)gi * RG + g) * S * S + q]);
      out[L.gram_slot[gi] + q] = sum;
    }
  }
}

// A CTA that stopped on a wait that ran out marks its partial record with NaN
__device__ __forceinline__ void cta_partials_nan(const RedSet& rs) {
  if (rs.nred == 0) return;
  float2* out = reinterpret_cast<float2*>(rs.partials) + (size_t)blockIdx.x * rs.nslots;
  for (int q = threadIdx.x; q < rs.nslots; q += blockDim.x) out[q] = make_float2(__int_as_float(0x7fc00000), 0.f);
}

// y += sum over the batch's m entries of val[k + u] * x[u] (real values for the split storage)
template <bool SPLIT, int NBATCH>
__device__ __forceinline__ void tile_fma(const unsigned char* valbuf, int k, int m, const Pair (&x)[NBATCH], Pair& y) {
  if constexpr (SPLIT) {
    const float* val = reinterpret_cast<const float*>(valbuf);
#pragma unroll
    for (int u = 0; u < NBATCH; ++u)
      if (u < m) {
        y.a = cfmareal<float>(val[k + u], x[u].a, y.a);
        y.b = cfmareal<float>(val[k + u], x[u].b, y.b);
      }
  } else {
    const float2* val = reinterpret_cast<const float2*>(valbuf);
#pragma unroll
    for (int u = 0; u < NBATCH; ++u)
      if (u < m) {
        y.a = cfma<float>(val[k + u], x[u].a, y.a);
        y.b = cfma<float>(val[k + u], x[u].b, y.b);
      }
  }
}

// MODE: TileMode; NG: fused Grams (0..2); at most kTileRowReds per-row reductions.  The Grams are
// formed by the whole CTA after each tile from the shared-memory copies of Y and U.
template <int GP, int MODE, int NG>
__global__ void __launch_bounds__(kTileThreadsMax, 4) spmm_tile_kernel(SpmmArgs<float> a, RedSet rs, TileLayout L,
                                                                        const int* done) {
  if (done != nullptr && *(volatile const int*)done) return;
  using K = TileKernel<GP, MODE>;
  constexpr int S = K::S;
  constexpr int NB = K::NB;
  constexpr bool SPLIT = K::SPLIT, STEN = K::STEN;
  extern __shared__ __align__(128) unsigned char tsm[];
  __shared__ __align__(8) uint64_t barA[kTileStagesA], barB[kTileStagesB];
  __shared__ int s_abort;
  const int tid = threadIdx.x;
  const int T = blockDim.x;  // = GP * R
  const int R = L.R;
  const int64_t n = a.n;
  const int ntiles = (int)((n + R - 1) / R);
  const int p = tid % GP;   // column pair of the product phase
  const int jj = tid / GP;  // row of the tile in the product phase
  const int strideA = L.sz_rp + L.sz_dg + L.nu * L.sz_u;
  const int strideB = L.sz_col + L.sz_val;
  unsigned char* baseA = tsm;
  unsigned char* baseB = tsm + kTileStagesA * strideA;
  float2* Yt = reinterpret_cast<float2*>(tsm + L.off_y);
  // stencil coefficients, converted once (double -> float runs on the FP64 pipe)
  float2 stc = make_float2(0.f, 0.f), stm[3], stp[3];
  if constexpr (STEN) {
    stc = make_float2((float)a.sc.x, (float)a.sc.y);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      stm[q] = make_float2((float)a.sm[q].x, (float)a.sm[q].y);
      stp[q] = make_float2((float)a.sp[q].x, (float)a.sp[q].y);
    }
  }

  if (tid == 0) {
    for (int k = 0; k < kTileStagesA; ++k) mbar_init(&barA[k], 1);
    for (int k = 0; k < kTileStagesB; ++k) mbar_init(&barB[k], 1);
    s_abort = 0;
    fence_mbar_init();
    fence_async_shared();
  }
  __syncthreads();

  // accumulators: per-row reductions of the product phase, one 2 x 2 block per Gram
  Acc2<kTileRowReds> acc;
#pragma unroll
  for (int q = 0; q < kTileRowReds; ++q) acc.v[q][0] = acc.v[q][1] = make_float2(0.f, 0.f);
  float2 g0[4], g1[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) g0[e] = g1[e] = make_float2(0.f, 0.f);
  const int gb = tid % NB, grow = tid / NB, RG = T / NB;  // Gram block and row group
  const int ga0 = 2 * (gb / GP), gc0 = 2 * (gb % GP);

  // producer state (thread 0): phases armed per barrier, for the bounded drain on abort
  int armA0 = 0, armA1 = 0, armA2 = 0, armB0 = 0, armB1 = 0;
  auto arm_a = [&](int k) { if (k == 0) ++armA0; else if (k == 1) ++armA1; else ++armA2; };
  auto rows_of = [&](int t) { const int64_t r0 = (int64_t)t * R; return (int)(n - r0 < R ? n - r0 : R); };
  const int t0 = blockIdx.x, tstep = gridDim.x;
  if (tid == 0) {
    for (int k = 0; k < kTileStagesA; ++k) {
      const int t = t0 + k * tstep;
      if (t < ntiles) {
        K::issue_a(a, L, baseA + k * strideA, &barA[k], (int64_t)t * R, rows_of(t));
        arm_a(k);
      }
    }
    if constexpr (!STEN) {
      if (!mbar_wait(&barA[0], 0)) {
        s_abort = 1;
      } else {
        K::issue_b(a, L, baseB, reinterpret_cast<const int64_t*>(baseA + L.off_rp), &barB[0], rows_of(t0));
        ++armB0;
      }
    }
  }

  // stage indices and the parity each barrier's pending phase completes with
  int sa = 0, sb = 0;
  uint32_t parA = 0, parB = 0;  // bit k: parity of barrier k's next phase to consume
  for (int t = t0; t < ntiles; t += tstep) {
    unsigned char* A = baseA + sa * strideA;
    unsigned char* Bst = baseB + sb * strideB;
    const int64_t r0 = (int64_t)t * R;
    const int rows = rows_of(t);
    const int sa1 = sa == kTileStagesA - 1 ? 0 : sa + 1;
    // the producer: entries of the next tile (its row pointers were issued a tile earlier)
    if (!STEN && tid == 0 && t + tstep < ntiles && !s_abort) {
      if (!mbar_wait(&barA[sa1], (parA >> sa1) & 1u)) {
        s_abort = 1;
      } else {
        fence_async_shared();
        K::issue_b(a, L, baseB + (1 - sb) * strideB,
                   reinterpret_cast<const int64_t*>(baseA + sa1 * strideA + L.off_rp), &barB[1 - sb],
                   rows_of(t + tstep));
        if (sb == 0) ++armB1; else ++armB0;
      }
    }
    bool ok = mbar_wait(&barA[sa], (parA >> sa) & 1u);
    if (!STEN) ok = ok && mbar_wait(&barB[sb], (parB >> sb) & 1u);
    if (!ok) s_abort = 1;
    // ---- product phase: row jj, column pair p
    Pair y = pzero();
    if (ok && jj < rows) {
      const int64_t j = r0 + jj;
      const int64_t e = j * S + 2 * p;
      if constexpr (STEN) {
        y = spmm2_row<true, false>(a, stc, stm, stp, j, p, e);
      } else {
        const int64_t* rp = reinterpret_cast<const int64_t*>(A + L.off_rp);
        const int32_t* col = reinterpret_cast<const int32_t*>(Bst + L.off_col);
        const int64_t kb = rp[0] & ~(int64_t)3;
        const float4* Vq = reinterpret_cast<const float4*>(a.V) + p;
        auto gather = [&](int32_t c) {
          const float4 v = Vq[(uint64_t)(uint32_t)c * (uint32_t)GP];
          Pair q;
          q.a = make_float2(v.x, v.y);
          q.b = make_float2(v.z, v.w);
          return q;
        };
        const int k0 = (int)(rp[jj] - kb), k1 = (int)(rp[jj + 1] - kb);
        if (SPLIT) {
          const float2 dgv = reinterpret_cast<const float2*>(A + L.off_dg)[jj];
          const Pair xv = ld_pair(a.V, e);
          y.a = cmul<float>(dgv, xv.a);
          y.b = cmul<float>(dgv, xv.b);
        }
        // batches of four entries, the last 1-3 as one predicated batch: all loads of a batch in
        // flight together (a longer single batch needs more registers than 2 CTAs per SM allow)
        int k = k0;
        for (; k + 4 <= k1; k += 4) {
          Pair x[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) x[u] = gather(col[k + u]);
          tile_fma<SPLIT, 4>(Bst + L.off_val, k, 4, x, y);
        }
        const int rem = k1 - k;
        if (rem > 0) {
          Pair x[3];
#pragma unroll
          for (int u = 0; u < 3; ++u)
            if (u < rem) x[u] = gather(col[k + u]);
          tile_fma<SPLIT, 3>(Bst + L.off_val, k, rem, x, y);
        }
      }
      if (a.ys != nullptr || a.ay != 1.0) {
        float2 ysc = make_float2((float)a.ay, 0.f);
        if (a.ys != nullptr) {
          const float2 d = scalar_coef<float>(a.ys, a.ys_conj, a.ys_neg);
          ysc = make_float2((float)a.ay * d.x, (float)a.ay * d.y);
        }
        y.a = cmul<float>(ysc, y.a);
        y.b = cmul<float>(ysc, y.b);
      }
      if (a.Z != nullptr) {
        const float bz = (float)a.bz;
        const Pair z = ld_pair(a.Z, e);
        y.a.x = fmaf(bz, z.a.x, y.a.x); y.a.y = fmaf(bz, z.a.y, y.a.y);
        y.b.x = fmaf(bz, z.b.x, y.b.x); y.b.y = fmaf(bz, z.b.y, y.b.y);
      }
      if (a.Y != nullptr) st_pair(a.Y, e, y);
      // per-row reductions
#pragma unroll
      for (int ri = 0; ri < kMaxRed; ++ri) {
        if (ri < rs.nred && rs.r[ri].kind != RED_GRAM) {
          const RedSpec& r = rs.r[ri];
          Pair u = pzero();
          if (r.kind == RED_TRACE || r.kind == RED_CDOT) {
            if (L.red_u[ri] >= 0)
              u = ld_pair(reinterpret_cast<const float2*>(A + L.off_u + L.red_u[ri] * L.sz_u), (int64_t)jj * S + 2 * p);
            else
              u = y;  // the product itself (U == nullptr, or U is this launch's Y)
          } else if (r.kind == RED_SUMV || r.kind == RED_GRAMV) {
            u.a = reinterpret_cast<const float2*>(r.U)[j];
            u.b = u.a;
          }
          red2_add(r, L.red_k[ri], acc, y, u);
        }
      }
    }
    if (NG > 0) st_pair(Yt, (int64_t)jj * S + 2 * p, y);
    __syncthreads();
    // ---- Gram phase: G[a][c] += conj(U[j][a]) Y[j][c] over the tile's rows, 2 x 2 blocks
    if (NG > 0 && !s_abort && grow < RG) {
      const float2* U0 = L.gram_u[0] >= 0 ? reinterpret_cast<const float2*>(A + L.off_u + L.gram_u[0] * L.sz_u) : Yt;
      gram_rows<S>(U0, Yt, ga0, gc0, grow, RG, rows, g0[0], g0[1], g0[2], g0[3]);
      if (NG > 1) {
        const float2* U1 =
            L.gram_u[1] >= 0 ? reinterpret_cast<const float2*>(A + L.off_u + L.gram_u[1] * L.sz_u) : Yt;
        gram_rows<S>(U1, Yt, ga0, gc0, grow, RG, rows, g1[0], g1[1], g1[2], g1[3]);
      }
    }
    __syncthreads();
    if (s_abort) break;
    parA ^= 1u << sa;
    parB ^= 1u << sb;
    // the producer: row pointers, diagonal and U of the tile three ahead into the freed A-stage
    if (tid == 0) {
      const int t3 = t + kTileStagesA * tstep;
      if (t3 < ntiles) {
        fence_async_shared();
        K::issue_a(a, L, A, &barA[sa], (int64_t)t3 * R, rows_of(t3));
        arm_a(sa);
      }
    }
    sa = sa1;
    sb ^= 1;
  }

  if (s_abort) {
    // stop: wait (bounded) for the last phase armed on each barrier, mark the partial record
    if (tid == 0) {
      atomicAdd(&g_kr_wait_timeouts, 1u);
      if (armA0 > 0) mbar_wait(&barA[0], (uint32_t)((armA0 - 1) & 1));
      if (armA1 > 0) mbar_wait(&barA[1], (uint32_t)((armA1 - 1) & 1));
      if (armA2 > 0) mbar_wait(&barA[2], (uint32_t)((armA2 - 1) & 1));
      if (armB0 > 0) mbar_wait(&barB[0], (uint32_t)((armB0 - 1) & 1));
      if (armB1 > 0) mbar_wait(&barB[1], (uint32_t)((armB1 - 1) & 1));
    }
    cta_partials_nan(rs);
    return;
  }
  if (rs.nred == 0) return;
  cta_partials<GP, NG>(tsm, rs, L, acc, g0, g1, grow, RG, ga0, gc0);
}

}  // namespace kr
