// Matrix-free product with the 4D lattice operator of Example 4 (Wilson-type hopping):
//   y_x = d psi_x + sum_mu [ (I + e_f gamma_mu) U_mu(x) psi_{x+mu} + (I + e_b gamma_mu) U_mu(x-mu)^H psi_{x-mu} ]
// on a periodic lattice, rows ordered (site * 4 + spin) * 3 + colour, with the hop
// coefficient folded into the links and the projector signs in the LatHop tables.
//
// Work unit: one (site, colour) pair and one column of the block; G threads (one per
// column) handle the 4 rows (site, spin, colour) of a unit.  Per hop a thread loads the
// neighbour's 12 entries of its column, projects them onto the two independent spin
// components of the rank-2 projector (h_t = psi[rep_t] + pc_t psi[sig_t]), applies row
// `colour` of the link (U, or U^H for a backward hop) to both, and spreads the two results
// over the four output spins (rc, rsrc).  Against the CSR storage of the same operator (49
// entries per row) this reads no matrix entries (only 8 links of 9 entries per site), makes
// 12 gathers per unit and hop instead of 4 x 6, and does 2/3 of the arithmetic.  Keeping
// 4 rows per thread (not 12) and the hop loop rolled holds the kernel near 64-100
// registers.  Reductions and the epilogue (scaling, addend, store) run row by row as in
// the CSR product.
#pragma once

#include "kr_rows_impl.cuh"

namespace kr {

template <typename T, int G, int NG>
__global__ void __launch_bounds__(kThreads) lattice_kernel(SpmmArgs<T> a, RedSet rs, const int* done) {
  if (done != nullptr && *(volatile const int*)done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int UPW = 32 / G;  // units per warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = lane & (G - 1);
  const int grpbase = lane & ~(G - 1);
  const int s = a.s;
  const int64_t n = a.n;
  const int64_t sites = n / 12;
  const int64_t units = sites * 3;
  const int64_t units_per_cta = (int64_t)(blockDim.x >> 5) * UPW;
  C2<T> ysc = mk<T>((T)a.ay, (T)0);
  const bool scaled = a.ys != nullptr || a.ay != 1.0;
  if (a.ys != nullptr) {
    C2<T> d = scalar_coef<T>(a.ys, a.ys_conj, a.ys_neg);
    ysc = mk<T>((T)a.ay * d.x, (T)a.ay * d.y);
  }
  const T bz = (T)a.bz;
  // projector tables in shared memory, in the kernel's precision
  struct HopT {
    int rep[2], sig[2], rsrc[4];
    C2<T> pc[2], rc[4];
  };
  __shared__ HopT hops[8];
  if (threadIdx.x < 8) {
    const LatHop& L = a.lh[threadIdx.x];
    HopT hp;
    for (int q = 0; q < 2; ++q) {
      hp.rep[q] = L.rep[q];
      hp.sig[q] = L.sig[q];
      hp.pc[q] = from_d2<T>(L.pc[q]);
    }
    for (int q = 0; q < 4; ++q) {
      hp.rsrc[q] = L.rsrc[q];
      hp.rc[q] = from_d2<T>(L.rc[q]);
    }
    hops[threadIdx.x] = hp;
  }
  __syncthreads();
  const C2<T> dg = from_d2<T>(a.ldiag);
  Acc<T, G, NG> acc;
  acc_zero(acc);
  for (int64_t base = (int64_t)blockIdx.x * units_per_cta; base < units;
       base += (int64_t)gridDim.x * units_per_cta) {
    const int64_t unit = base + warp * UPW + lane / G;
    const bool unitok = unit < units;
    const bool act = unitok && c < s;
    const int64_t x = unit / 3;
    const int ci = (int)(unit - 3 * x);
    const C2<T>* Vc = a.V + c;
    C2<T> y[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) y[k] = czero<T>();
    if (act) {
      int64_t xc[4];
      grid_coords<4>(x, 4, a.ldiv32, a.ldims, a.ldiv, xc);
#pragma unroll
      for (int k = 0; k < 4; ++k) y[k] = cmul<T>(dg, Vc[(x * 12 + k * 3 + ci) * s]);
      // hops one after another (a rolled loop): unrolled, the compiler precomputes the
      // addresses and hoists the loads of all 8 hops (130-220 registers)
#pragma unroll 1
      for (int h = 0; h < 8; ++h) {
        const int mu = h >> 1;
        const bool fwd = (h & 1) == 0;
        // coordinate, extent and stride along mu, selected with constant indices
        const int64_t xm = mu == 0 ? xc[0] : mu == 1 ? xc[1] : mu == 2 ? xc[2] : xc[3];
        const int64_t Lm = mu == 0 ? a.ldims[0] : mu == 1 ? a.ldims[1] : mu == 2 ? a.ldims[2] : a.ldims[3];
        const int64_t sm = mu == 0 ? a.lstr[0] : mu == 1 ? a.lstr[1] : mu == 2 ? a.lstr[2] : a.lstr[3];
        // periodic neighbour x + mu (forward) or x - mu (backward)
        int64_t nb;
        if (fwd) nb = xm == Lm - 1 ? x - (Lm - 1) * sm : x + sm;
        else nb = xm == 0 ? x + (Lm - 1) * sm : x - sm;
        const HopT& L = hops[h];
        const C2<T>* Vn = Vc + nb * 12 * s;
        // spin projection onto the two independent components, all three colours
        C2<T> h0[3], h1[3];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          h0[cc] = cfma<T>(L.pc[0], Vn[(L.sig[0] * 3 + cc) * s], Vn[(L.rep[0] * 3 + cc) * s]);
          h1[cc] = cfma<T>(L.pc[1], Vn[(L.sig[1] * 3 + cc) * s], Vn[(L.rep[1] * 3 + cc) * s]);
        }
        // row ci of U (forward) or of U^H (backward)
        const C2<T>* U = a.links + ((int64_t)mu * sites + (fwd ? x : nb)) * 9;
        C2<T> g0 = czero<T>(), g1 = czero<T>();
#pragma unroll
        for (int cj = 0; cj < 3; ++cj) {
          const C2<T> u = fwd ? U[ci * 3 + cj] : cconj<T>(U[cj * 3 + ci]);
          g0 = cfma<T>(u, h0[cj], g0);
          g1 = cfma<T>(u, h1[cj], g1);
        }
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) y[sp] = cfma<T>(L.rc[sp], L.rsrc[sp] ? g1 : g0, y[sp]);
      }
    }
    // epilogue and fused reductions, row by row (all lanes of a unit group take part)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t j = x * 12 + k * 3 + ci;
      C2<T> yk = y[k];
      if (act) {
        if (scaled) yk = cmul<T>(ysc, yk);
        if (a.Z != nullptr) {
          const C2<T> z = a.Z[j * s + c];
          yk.x = fma(bz, z.x, yk.x);
          yk.y = fma(bz, z.y, yk.y);
        }
        if (a.Y != nullptr) a.Y[j * s + c] = yk;
      }
      if (rs.nred > 0) {
#pragma unroll
        for (int ri = 0; ri < kMaxRed; ++ri) {
          if (ri < rs.nred) {
            const RedSpec& r = rs.r[ri];
            C2<T> u = czero<T>();
            if (r.kind == RED_GRAM || r.kind == RED_TRACE || r.kind == RED_CDOT) {
              if (act) u = (r.U != nullptr) ? reinterpret_cast<const C2<T>*>(r.U)[j * s + c] : yk;
            } else if (r.kind == RED_SUMV || r.kind == RED_GRAMV) {
              if (unitok) u = reinterpret_cast<const C2<T>*>(r.U)[j];
            }
            red_add<T, G, NG>(r, ri, acc, yk, u, s, grpbase);
          }
        }
      }
    }
  }
  if (rs.nred > 0) cta_reduce<T, G, NG>(rs, acc, s, reinterpret_cast<C2<T>*>(smem_raw));
}

// The same product with one whole site (12 rows) per thread and column (the default): the
// neighbour's entries are loaded once per site (3x fewer gathers than the (site, colour)
// units) and the projection is not repeated per colour (2376 flops per site and column
// against 3144), at the price of 12 accumulators per thread (80 registers in complex64,
// about 160 in complex128, where the FP64 pipe, not occupancy, sets the pace).
template <typename T, int G, int NG>
__global__ void __launch_bounds__(kThreads) lattice_site_kernel(SpmmArgs<T> a, RedSet rs, const int* done) {
  if (done != nullptr && *(volatile const int*)done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int SPW = 32 / G;  // sites per warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = lane & (G - 1);
  const int grpbase = lane & ~(G - 1);
  const int s = a.s;
  const int64_t n = a.n;
  const int64_t sites = n / 12;
  const int64_t sites_per_cta = (int64_t)(blockDim.x >> 5) * SPW;
  C2<T> ysc = mk<T>((T)a.ay, (T)0);
  const bool scaled = a.ys != nullptr || a.ay != 1.0;
  if (a.ys != nullptr) {
    C2<T> d = scalar_coef<T>(a.ys, a.ys_conj, a.ys_neg);
    ysc = mk<T>((T)a.ay * d.x, (T)a.ay * d.y);
  }
  const T bz = (T)a.bz;
  struct HopT {
    int rep[2], sig[2], rsrc[4];
    C2<T> pc[2], rc[4];
  };
  __shared__ HopT hops[8];
  if (threadIdx.x < 8) {
    const LatHop& L = a.lh[threadIdx.x];
    HopT hp;
    for (int q = 0; q < 2; ++q) {
      hp.rep[q] = L.rep[q];
      hp.sig[q] = L.sig[q];
      hp.pc[q] = from_d2<T>(L.pc[q]);
    }
    for (int q = 0; q < 4; ++q) {
      hp.rsrc[q] = L.rsrc[q];
      hp.rc[q] = from_d2<T>(L.rc[q]);
    }
    hops[threadIdx.x] = hp;
  }
  __syncthreads();
  const C2<T> dg = from_d2<T>(a.ldiag);
  Acc<T, G, NG> acc;
  acc_zero(acc);
  for (int64_t base = (int64_t)blockIdx.x * sites_per_cta; base < sites;
       base += (int64_t)gridDim.x * sites_per_cta) {
    const int64_t x = base + warp * SPW + lane / G;
    const bool siteok = x < sites;
    const bool act = siteok && c < s;
    const C2<T>* Vc = a.V + c;
    C2<T> y[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) y[k] = czero<T>();
    if (act) {
      int64_t xc[4];
      grid_coords<4>(x, 4, a.ldiv32, a.ldims, a.ldiv, xc);
#pragma unroll
      for (int k = 0; k < 12; ++k) y[k] = cmul<T>(dg, Vc[(x * 12 + k) * s]);
#pragma unroll 1
      for (int h = 0; h < 8; ++h) {
        const int mu = h >> 1;
        const bool fwd = (h & 1) == 0;
        const int64_t xm = mu == 0 ? xc[0] : mu == 1 ? xc[1] : mu == 2 ? xc[2] : xc[3];
        const int64_t Lm = mu == 0 ? a.ldims[0] : mu == 1 ? a.ldims[1] : mu == 2 ? a.ldims[2] : a.ldims[3];
        const int64_t sm = mu == 0 ? a.lstr[0] : mu == 1 ? a.lstr[1] : mu == 2 ? a.lstr[2] : a.lstr[3];
        int64_t nb;
        if (fwd) nb = xm == Lm - 1 ? x - (Lm - 1) * sm : x + sm;
        else nb = xm == 0 ? x + (Lm - 1) * sm : x - sm;
        const HopT& L = hops[h];
        const C2<T>* Vn = Vc + nb * 12 * s;
        C2<T> h0[3], h1[3];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          h0[cc] = cfma<T>(L.pc[0], Vn[(L.sig[0] * 3 + cc) * s], Vn[(L.rep[0] * 3 + cc) * s]);
          h1[cc] = cfma<T>(L.pc[1], Vn[(L.sig[1] * 3 + cc) * s], Vn[(L.rep[1] * 3 + cc) * s]);
        }
        const C2<T>* U = a.links + ((int64_t)mu * sites + (fwd ? x : nb)) * 9;
#pragma unroll
        for (int ci = 0; ci < 3; ++ci) {
          C2<T> g0 = czero<T>(), g1 = czero<T>();
#pragma unroll
          for (int cj = 0; cj < 3; ++cj) {
            const C2<T> u = fwd ? U[ci * 3 + cj] : cconj<T>(U[cj * 3 + ci]);
            g0 = cfma<T>(u, h0[cj], g0);
            g1 = cfma<T>(u, h1[cj], g1);
          }
#pragma unroll
          for (int sp = 0; sp < 4; ++sp) y[sp * 3 + ci] = cfma<T>(L.rc[sp], L.rsrc[sp] ? g1 : g0, y[sp * 3 + ci]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const int64_t j = x * 12 + k;
      C2<T> yk = y[k];
      if (act) {
        if (scaled) yk = cmul<T>(ysc, yk);
        if (a.Z != nullptr) {
          const C2<T> z = a.Z[j * s + c];
          yk.x = fma(bz, z.x, yk.x);
          yk.y = fma(bz, z.y, yk.y);
        }
        if (a.Y != nullptr) a.Y[j * s + c] = yk;
      }
      if (rs.nred > 0) {
#pragma unroll
        for (int ri = 0; ri < kMaxRed; ++ri) {
          if (ri < rs.nred) {
            const RedSpec& r = rs.r[ri];
            C2<T> u = czero<T>();
            if (r.kind == RED_GRAM || r.kind == RED_TRACE || r.kind == RED_CDOT) {
              if (act) u = (r.U != nullptr) ? reinterpret_cast<const C2<T>*>(r.U)[j * s + c] : yk;
            } else if (r.kind == RED_SUMV || r.kind == RED_GRAMV) {
              if (siteok) u = reinterpret_cast<const C2<T>*>(r.U)[j];
            }
            red_add<T, G, NG>(r, ri, acc, yk, u, s, grpbase);
          }
        }
      }
    }
  }
  if (rs.nred > 0) cta_reduce<T, G, NG>(rs, acc, s, reinterpret_cast<C2<T>*>(smem_raw));
}

}  // namespace kr
