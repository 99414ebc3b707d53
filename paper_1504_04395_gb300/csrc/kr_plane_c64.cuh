// Complex64 product of the matrix-free (2d+1)-point stencil (d = 2, 3) marching the planes of the
// grid through shared memory with TMA tensor copies, with fused reductions.
//
// The block product of the inner solves reads V once per neighbour; for a stencil on a
// lexicographic grid the neighbours of a tile of points are the tile itself, a one-point halo in x
// and y, and the same tile in the planes z - 1 and z + 1.  Each CTA takes a contiguous range of
// (x-y tile, plane) work units and marches along z:
//
//   * one thread loads each plane of its x-y tile once, with its halo, by a 4D TMA tensor copy
//     (cp.async.bulk.tensor, box {2s floats, tx + 2, ty + 2, 1} at (0, x0 - 1, y0 - 1, z); the
//     copy fills points outside the grid with zeros, and the product skips them) into a ring of
//     five stages: planes z - 1, z, z + 1 in use and two in flight; the reductions' U operand comes
//     the same way (box {2s, tx, ty, 1}) two planes ahead into a ring of three;
//   * GP = s/2 threads per point, one column pair each, form (A V) of their points from the three
//     planes in shared memory with the operations and in the order of the other product kernels
//     (centre, minus neighbours along axes 2, 1, 0, plus neighbours along axes 0, 1, 2), so Y is
//     bitwise the same;
//   * per-row reductions accumulate per thread; fused s x s Grams are formed by the CTA after each
//     plane from shared-memory copies of Y and U (2 x 2 blocks per thread), and the CTA's partial
//     record is written in the layout and order of the row-tile kernel.
//
// V is read from HBM about once (halos and neighbouring planes come from shared memory or L2), U
// once and Y written once: three n x s blocks per product, the stencil's algorithmic bytes.  Every
// mbarrier wait is bounded; a wait that runs out stops the CTA as in the row-tile kernel.
#pragma once

#include <cuda.h>

#include "kr_plane_c64.h"
#include "kr_tile_c64.cuh"

namespace kr {

// 4D tiled tensor copy global -> shared (the tensor map's box at coordinates c0..c3), completing on bar
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
      : "memory");
}

// c + a b componentwise as one packed FP32 FMA (fma.rn.f32x2): per component the same rounded
// FMA as fmaf, so the same result bit for bit, in half the instructions
__device__ __forceinline__ float2 fma_x2(float2 a, float2 b, float2 c) {
  unsigned long long ra, rb, rc, rd;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rc) : "f"(c.x), "f"(c.y));
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rd) : "l"(ra), "l"(rb), "l"(rc));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
  return d;
}

// neighbouring stages of a ring of N
template <int N>
__device__ __forceinline__ int next_stage(int k) { return k + 1 == N ? 0 : k + 1; }
template <int N>
__device__ __forceinline__ int prev_stage(int k) { return k == 0 ? N - 1 : k - 1; }

// IPT: (point, column pair) items per thread and plane (the tile holds at most IPT * 256 / GP points)
template <int GP, int NG, int IPT>
__global__ void __launch_bounds__(kPlaneThreads, 2)
    spmm_plane_kernel(SpmmArgs<float> a, RedSet rs, TileLayout L, PlaneGeom P,
                      const __grid_constant__ CUtensorMap tmV, const __grid_constant__ CUtensorMap tmU,
                      const int* done) {
  if (done != nullptr && *(volatile const int*)done) return;
  constexpr int S = 2 * GP;
  constexpr int NB = GP * GP;
  constexpr int NSV = kPlaneStagesV, NSU = kPlaneStagesU;
  // the tensor copies' shared-memory destinations: 128-byte aligned (the launch adds 128 bytes)
  extern __shared__ __align__(128) unsigned char psm_raw[];
  // (an offset from the array itself, so that the compiler keeps every access a shared-memory one)
  unsigned char* psm = psm_raw + ((128u - (smem_addr(psm_raw) & 127u)) & 127u);
  __shared__ __align__(8) uint64_t barV[NSV], barU[NSU];
  __shared__ int s_abort;
  const int tid = threadIdx.x;
  constexpr int T = kPlaneThreads;  // the launch's block size
  const int p = tid % GP;              // column pair
  const int q0 = tid / GP;             // first point of this thread in a plane tile
  constexpr int ppass = T / GP;        // points per pass over the tile
  const int tx = P.tx, ty = P.ty, pw = P.tx + 2;
  const int npts = tx * ty;
  const bool hasU = L.nu > 0;
  const uint32_t bytesV = (uint32_t)(pw * (ty + 2) * S * 8);
  const uint32_t bytesU = (uint32_t)(npts * S * 8);
  unsigned char* baseV = psm + P.off_v;
  unsigned char* baseU = psm + P.off_u;
  float2* Yt = reinterpret_cast<float2*>(psm + P.off_y);
  const float2 stc = make_float2((float)a.sc.x, (float)a.sc.y);
  float2 stm[3], stp[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    stm[q] = make_float2((float)a.sm[q].x, (float)a.sm[q].y);
    stp[q] = make_float2((float)a.sp[q].x, (float)a.sp[q].y);
  }

  if (tid == 0) {
    for (int k = 0; k < NSV; ++k) mbar_init(&barV[k], 1);
    for (int k = 0; k < NSU; ++k) mbar_init(&barU[k], 1);
    s_abort = 0;
    fence_mbar_init();
    fence_async_shared();
  }
  __syncthreads();

  Acc2<kTileRowReds> acc;
#pragma unroll
  for (int q = 0; q < kTileRowReds; ++q) acc.v[q][0] = acc.v[q][1] = make_float2(0.f, 0.f);
  float2 g0[4], g1[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) g0[e] = g1[e] = make_float2(0.f, 0.f);
  const int gb = tid % NB, grow = tid / NB, RG = T / NB;  // Gram block and row group
  const int ga0 = 2 * (gb / GP), gc0 = 2 * (gb % GP);

  // the product's scale (a device scalar times a real factor) and the addend's factor, converted
  // once: the same values as the per-row conversions of the other product kernels
  const bool scaled = a.ys != nullptr || a.ay != 1.0;
  float2 ysc = make_float2((float)a.ay, 0.f);
  if (a.ys != nullptr) {
    const float2 d = scalar_coef<float>(a.ys, a.ys_conj, a.ys_neg);
    ysc = make_float2((float)a.ay * d.x, (float)a.ay * d.y);
  }
  const float bz = (float)a.bz;

  // this CTA's work units: (x-y tile, plane) pairs in the order tile * nz + z
  const int64_t W = (int64_t)P.ntx * P.nty * P.nz;
  const int64_t w0 = (int64_t)blockIdx.x * W / gridDim.x, w1 = (int64_t)(blockIdx.x + 1) * W / gridDim.x;
  // stages of the next load (every thread keeps the producer's) and of the next phase to consume:
  // the loads of a ring go round its stages in order
  int kVn = 0, kUn = 0, kVc = 0, kUc = 0;
  uint32_t parV = 0, parU = 0, armV = 0, armU = 0;
  bool stop = false;
  for (int64_t w = w0; w < w1 && !stop;) {
    const int64_t xy = w / P.nz;
    const int za = (int)(w - xy * P.nz);
    const int zb = (int)(w1 - xy * P.nz < P.nz ? w1 - xy * P.nz : P.nz);
    w = xy * P.nz + zb;
    const int x0 = (int)(xy % P.ntx) * tx, y0 = (int)(xy / P.ntx) * ty;
    const int zl0 = za > 0 ? za - 1 : 0, zl1 = zb < P.nz ? zb : P.nz - 1;  // planes of V read here
    // this thread's items in the segment's tile: shared-memory offset of the point in a halo'd
    // plane, row index in plane 0, and which x-y neighbours exist (bit 0: y - 1, 1: x - 1, 2: x + 1,
    // 3: y + 1; bit 4: the point is in the grid)
    int cpt[IPT], qpt[IPT];
    uint32_t nbr[IPT];
    int64_t jxy[IPT];
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
      const int q = q0 + it * ppass;
      const int ly = q / tx, lx = q - ly * tx;
      const int gx = x0 + lx, gy = y0 + ly;
      qpt[it] = q;
      cpt[it] = ((ly + 1) * pw + lx + 1) * S + 2 * p;
      jxy[it] = (int64_t)gx + (int64_t)P.nx * gy;
      nbr[it] = (q < npts && gx < P.nx && gy < P.ny ? 16u : 0u) | (gy > 0 ? 1u : 0u) | (gx > 0 ? 2u : 0u) |
                (gx < P.nx - 1 ? 4u : 0u) | (gy < P.ny - 1 ? 8u : 0u);
    }
    const int64_t plane = (int64_t)P.nx * P.ny;
    // stages of V plane z and U plane z, advanced with z
    int sVz = za > zl0 ? next_stage<NSV>(kVn) : kVn, sUz = kUn;
    int vnext = zl0, unext = za;                  // next plane to load
    int vwait = zl0;                              // next V plane to wait for
    for (int z = za; z < zb; ++z) {
      // the producer: V planes up to z + 1 + ahead and U planes up to z + ahead, into stages that
      // the computes before this one have released (their barriers separate the reads)
      const int vlast = z + 1 + kPlaneAheadV < zl1 ? z + 1 + kPlaneAheadV : zl1;
      const int ulast = z + kPlaneAheadU < zb - 1 ? z + kPlaneAheadU : zb - 1;
      if (tid == 0) fence_async_shared();
      for (; vnext <= vlast; ++vnext, kVn = next_stage<NSV>(kVn)) {
        if (tid == 0) {
          const int k = kVn;
          mbar_arrive_expect(&barV[k], bytesV);
          tma_load_4d(baseV + k * P.stride_v, &tmV, 0, x0 - 1, y0 - 1, vnext, &barV[k]);
          note_armed(armV, k);
        }
      }
      if (hasU) {
        for (; unext <= ulast; ++unext, kUn = next_stage<NSU>(kUn)) {
          if (tid == 0) {
            const int k = kUn;
            mbar_arrive_expect(&barU[k], bytesU);
            tma_load_4d(baseU + k * P.stride_u, &tmU, 0, x0, y0, unext, &barU[k]);
            note_armed(armU, k);
          }
        }
      }
      // wait for the planes this compute needs: V up to z + 1, U of z
      bool ok = true;
      const int vneed = z + 1 < zl1 ? z + 1 : zl1;
      for (; vwait <= vneed; ++vwait, kVc = next_stage<NSV>(kVc)) ok = take_phase(barV, parV, kVc) && ok;
      if (hasU) {
        ok = take_phase(barU, parU, kUc) && ok;
        kUc = next_stage<NSU>(kUc);
      }
      if (!ok) s_abort = 1;
      const float2* Vz = reinterpret_cast<const float2*>(baseV + sVz * P.stride_v);
      const float2* Vm = reinterpret_cast<const float2*>(baseV + prev_stage<NSV>(sVz) * P.stride_v);
      const float2* Vp = reinterpret_cast<const float2*>(baseV + next_stage<NSV>(sVz) * P.stride_v);
      const float2* Us = reinterpret_cast<const float2*>(baseU + sUz * P.stride_u);
      sVz = next_stage<NSV>(sVz);
      sUz = next_stage<NSU>(sUz);
      const bool zm = z > 0, zp = z + 1 < P.nz;
      // ---- product: items (point qpt[it], pair p); first every item's loads and FMAs (independent
      // chains the compiler can interleave), then their epilogues
      const int soff[6] = {0, -pw * S, -S, S, pw * S, 0};  // neighbour offsets, same order as the masks below
      Pair yv[IPT];
#pragma unroll
      for (int it = 0; it < IPT; ++it) {
        yv[it] = pzero();
        const uint32_t m = nbr[it];
        if (ok && (m & 16u)) {
          const int c = cpt[it];
          const Pair xv = ld_pair(Vz, c);
          Pair y;
          y.a = cmul<float>(stc, xv.a);
          y.b = cmul<float>(stc, xv.b);
          // minus neighbours along axes 2, 1, 0, then plus neighbours along axes 0, 1, 2
          const bool has[6] = {zm, (m & 1u) != 0, (m & 2u) != 0, (m & 4u) != 0, (m & 8u) != 0, zp};
          const float2* src[6] = {Vm, Vz, Vz, Vz, Vz, Vp};
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            if (has[k]) {
              const Pair x = ld_pair(src[k], c + soff[k]);
              const float2 cf = k < 3 ? stm[2 - k] : stp[k - 3];
              if (a.sreal) {  // cfmareal per complex entry, packed
                const float2 rr = make_float2(cf.x, cf.x);
                y.a = fma_x2(rr, x.a, y.a);
                y.b = fma_x2(rr, x.b, y.b);
              }
              else { y.a = cfma<float>(cf, x.a, y.a); y.b = cfma<float>(cf, x.b, y.b); }
            }
          }
          yv[it] = y;
        }
      }
#pragma unroll
      for (int it = 0; it < IPT; ++it) {
        const int q = qpt[it];
        if (q >= npts) continue;
        Pair y = yv[it];
        if (ok && (nbr[it] & 16u)) {
          const int64_t j = jxy[it] + plane * z;
          const int64_t e = j * S + 2 * p;
          if (scaled) {
            y.a = cmul<float>(ysc, y.a);
            y.b = cmul<float>(ysc, y.b);
          }
          if (a.Z != nullptr) {
            const Pair zz = ld_pair(a.Z, e);
            y.a.x = fmaf(bz, zz.a.x, y.a.x); y.a.y = fmaf(bz, zz.a.y, y.a.y);
            y.b.x = fmaf(bz, zz.b.x, y.b.x); y.b.y = fmaf(bz, zz.b.y, y.b.y);
          }
          if (a.Y != nullptr) st_pair(a.Y, e, y);
#pragma unroll
          for (int ri = 0; ri < kMaxRed; ++ri) {
            if (ri < rs.nred && rs.r[ri].kind != RED_GRAM) {
              const RedSpec& r = rs.r[ri];
              Pair u = pzero();
              if (r.kind == RED_TRACE || r.kind == RED_CDOT) {
                if (L.red_u[ri] >= 0) u = ld_pair(Us, q * S + 2 * p);
                else u = y;  // the product itself (U == nullptr, or U is this launch's Y)
              } else if (r.kind == RED_SUMV || r.kind == RED_GRAMV) {
                u.a = reinterpret_cast<const float2*>(r.U)[j];
                u.b = u.a;
              }
              red2_add(r, L.red_k[ri], acc, y, u);
            }
          }
        }
        if (NG > 0) st_pair(Yt, q * S + 2 * p, y);
      }
      __syncthreads();
      // s_abort is written only before the barrier above and read between the two barriers, so
      // every thread takes the same decision
      stop = s_abort != 0;
      if (NG > 0 && !stop && grow < RG) {
        const float2* U0 = L.gram_u[0] >= 0 ? Us : Yt;
        gram_rows<S>(U0, Yt, ga0, gc0, grow, RG, npts, g0[0], g0[1], g0[2], g0[3]);
        if (NG > 1) {
          const float2* U1 = L.gram_u[1] >= 0 ? Us : Yt;
          gram_rows<S>(U1, Yt, ga0, gc0, grow, RG, npts, g1[0], g1[1], g1[2], g1[3]);
        }
      }
      __syncthreads();
      if (stop) break;
    }
  }

  if (stop) {
    if (tid == 0) {
      atomicAdd(&g_kr_wait_timeouts, 1u);
      drain_stages<NSV>(barV, armV);
      drain_stages<NSU>(barU, armU);
    }
    cta_partials_nan(rs);
    return;
  }
  if (rs.nred == 0) return;
  cta_partials<GP, NG>(psm, rs, L, acc, g0, g1, grow, RG, ga0, gc0);
}

}  // namespace kr
