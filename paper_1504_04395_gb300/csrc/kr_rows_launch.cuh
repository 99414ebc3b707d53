// Host launchers for the row kernels, instantiated once per element type.
#pragma once

#include <atomic>
#include <unordered_map>

#include "kr_internal.h"
#include "kr_profile.h"
#include "kr_rows_impl.cuh"
#include "kr_rows_vec2.cuh"
#include "kr_lattice.cuh"
#include "kr_plane_c64.h"
#include "kr_tile_c64.h"

namespace kr {

constexpr int kMaxDynSmem = 200 * 1024;

template <typename K>
static void allow_smem(K kernel, std::atomic<uint64_t>& devices_done) {
  // the attribute belongs to the current device: set once per device (bit d of devices_done),
  // on every call for device ordinals beyond 63
  int dev = 0;
  KR_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = (dev >= 0 && dev < 64) ? (uint64_t{1} << dev) : 0;
  if (bit != 0 && (devices_done.load(std::memory_order_acquire) & bit)) return;
  KR_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem));
  if (bit != 0) devices_done.fetch_or(bit, std::memory_order_acq_rel);
}

// Clamp a grid-stride grid to the CTAs that can be resident at once (at most kCtasPerSm per SM),
// so that no CTA waits for a second wave.  Depends only on the kernel, its shared memory and the
// device, so a given launch always gets the same grid (fixed reduction order).
// The occupancy query is cached per kernel (the caller's cache), device and shared-memory size.
template <typename K>
static int resident_grid(K kernel, size_t smem, int grid, std::unordered_map<size_t, int>& cache) {
  int dev = 0;
  KR_CUDA(cudaGetDevice(&dev));
  const size_t key = smem * 256 + (size_t)dev;
  auto it = cache.find(key);
  int occ;
  if (it != cache.end()) {
    occ = it->second;
  } else {
    KR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kThreads, smem));
    if (occ < 1) occ = 1;
    if (occ > kCtasPerSm) occ = kCtasPerSm;
    cache.emplace(key, occ);
  }
  const int cap = sm_count() * occ;
  return grid < cap ? grid : cap;
}

template <typename T, int G, int NG, bool STEN>
static void spmm_go(const SpmmArgs<T>& a, const RedSet& rs, int& grid, const int* done, cudaStream_t st) {
  static std::atomic<uint64_t> attr{0};
  allow_smem(spmm_kernel<T, G, NG, STEN>, attr);
  const size_t smem = rs.nred > 0 ? (size_t)(kThreads / 32) * rs.nslots * sizeof(C2<T>) : 0;
  if (smem > (size_t)kMaxDynSmem) throw CudaError{cudaErrorInvalidValue, "spmm: too many reduction slots"};
  thread_local std::unordered_map<size_t, int> occ;
  grid = resident_grid(spmm_kernel<T, G, NG, STEN>, smem, grid, occ);
  spmm_kernel<T, G, NG, STEN><<<grid, kThreads, smem, st>>>(a, rs, done);
  KR_CUDA(cudaGetLastError());
}

template <typename T, int G, bool STEN>
static void spmm_ng(int ng, const SpmmArgs<T>& a, const RedSet& rs, int& grid, const int* done, cudaStream_t st) {
  if (ng == 0) return spmm_go<T, G, 0, STEN>(a, rs, grid, done, st);
  if constexpr (NGCap<1, G>::ok) {
    if (ng == 1) return spmm_go<T, G, 1, STEN>(a, rs, grid, done, st);
  }
  if constexpr (NGCap<2, G>::ok) {
    if (ng == 2) return spmm_go<T, G, 2, STEN>(a, rs, grid, done, st);
  }
  throw CudaError{cudaErrorInvalidValue, "spmm: fused Gram count exceeds the register budget"};
}

template <typename T, int G>
static void spmm_storage(int ng, const SpmmArgs<T>& a, const RedSet& rs, int& grid, const int* done,
                         cudaStream_t st) {
  if (a.nst > 0) return spmm_ng<T, G, true>(ng, a, rs, grid, done, st);
  return spmm_ng<T, G, false>(ng, a, rs, grid, done, st);
}

template <typename T>
static void spmm_dispatch(const SpmmArgs<T>& a, const RedSet& rs, int& grid, const int* done, cudaStream_t st) {
  const int G = threads_per_row(a.s);
  const int ng = count_grams(rs);
  switch (G) {
    case 1: return spmm_storage<T, 1>(ng, a, rs, grid, done, st);
    case 2: return spmm_storage<T, 2>(ng, a, rs, grid, done, st);
    case 4: return spmm_storage<T, 4>(ng, a, rs, grid, done, st);
    case 8: return spmm_storage<T, 8>(ng, a, rs, grid, done, st);
    case 16: return spmm_storage<T, 16>(ng, a, rs, grid, done, st);
    case 32: return spmm_storage<T, 32>(ng, a, rs, grid, done, st);
  }
  throw CudaError{cudaErrorInvalidValue, "spmm: s out of range"};
}

// matrix-free 4D lattice operator: G threads per (site, colour) unit, 4 rows per thread
template <typename T, int G, int NG>
static void lattice_go(const SpmmArgs<T>& a, const RedSet& rs, int& grid, const int* done, cudaStream_t st) {
  const size_t smem = rs.nred > 0 ? (size_t)(kThreads / 32) * rs.nslots * sizeof(C2<T>) : 0;
  if (smem > (size_t)kMaxDynSmem) throw CudaError{cudaErrorInvalidValue, "lattice: too many reduction slots"};
  const bool whole_site = lattice_rows_per_thread(sizeof(T)) == 12;
  // work units: (site, colour) with 4 rows each, or whole sites with 12 rows each
  const int64_t per_cta = (int64_t)(kThreads / 32) * (32 / G);
  const int64_t units = whole_site ? a.n / 12 : a.n / 4;
  const int64_t tiles = (units + per_cta - 1) / per_cta;
  if ((int64_t)grid > tiles) grid = (int)(tiles > 0 ? tiles : 1);
  if (whole_site) {
    static std::atomic<uint64_t> attr{0};
    allow_smem(lattice_site_kernel<T, G, NG>, attr);
    thread_local std::unordered_map<size_t, int> occ;
    grid = resident_grid(lattice_site_kernel<T, G, NG>, smem, grid, occ);
    lattice_site_kernel<T, G, NG><<<grid, kThreads, smem, st>>>(a, rs, done);
  } else {
    static std::atomic<uint64_t> attr{0};
    allow_smem(lattice_kernel<T, G, NG>, attr);
    thread_local std::unordered_map<size_t, int> occ;
    grid = resident_grid(lattice_kernel<T, G, NG>, smem, grid, occ);
    lattice_kernel<T, G, NG><<<grid, kThreads, smem, st>>>(a, rs, done);
  }
  KR_CUDA(cudaGetLastError());
}

template <typename T, int G>
static void lattice_ng(int ng, const SpmmArgs<T>& a, const RedSet& rs, int& grid, const int* done, cudaStream_t st) {
  if (ng == 0) return lattice_go<T, G, 0>(a, rs, grid, done, st);
  if constexpr (NGCap<1, G>::ok) {
    if (ng == 1) return lattice_go<T, G, 1>(a, rs, grid, done, st);
  }
  if constexpr (NGCap<2, G>::ok) {
    if (ng == 2) return lattice_go<T, G, 2>(a, rs, grid, done, st);
  }
  throw CudaError{cudaErrorInvalidValue, "lattice: fused Gram count exceeds the register budget"};
}

template <typename T>
static void lattice_dispatch(const SpmmArgs<T>& a, const RedSet& rs, int& grid, const int* done, cudaStream_t st) {
  const int ng = count_grams(rs);
  switch (threads_per_row(a.s)) {
    case 1: return lattice_ng<T, 1>(ng, a, rs, grid, done, st);
    case 2: return lattice_ng<T, 2>(ng, a, rs, grid, done, st);
    case 4: return lattice_ng<T, 4>(ng, a, rs, grid, done, st);
    case 8: return lattice_ng<T, 8>(ng, a, rs, grid, done, st);
    case 16: return lattice_ng<T, 16>(ng, a, rs, grid, done, st);
    case 32: return lattice_ng<T, 32>(ng, a, rs, grid, done, st);
  }
  throw CudaError{cudaErrorInvalidValue, "lattice: s out of range"};
}

// complex64 launches on column pairs (GP threads per row, GP = next power of two >= s/2)
template <int GP, bool STENCIL, int NR>
static void spmm2_launch(const SpmmArgs<float>& a, const RedSet& rs, int& grid, const int* done, cudaStream_t st,
                         size_t smem) {
  thread_local std::unordered_map<size_t, int> occ;
  grid = resident_grid(spmm2_kernel<GP, STENCIL, NR>, smem, grid, occ);
  spmm2_kernel<GP, STENCIL, NR><<<grid, kThreads, smem, st>>>(a, rs, done);
}

template <int GP>
static void spmm2_go(const SpmmArgs<float>& a, const RedSet& rs, int& grid, const int* done, cudaStream_t st) {
  const size_t smem = rs.nred > 0 ? (size_t)(kThreads / 32) * rs.nslots * sizeof(float2) : 0;
  if (smem > 48 * 1024) throw CudaError{cudaErrorInvalidValue, "spmm: too many reduction slots"};
  // up to two fused reductions (every product of the global, economic and Li methods but
  // the initial residual's) use the kernels with two accumulator slots
  const bool two = rs.nred <= 2;
  if (a.nst > 0) {
    if (two) spmm2_launch<GP, true, 2>(a, rs, grid, done, st, smem);
    else spmm2_launch<GP, true, kMaxRed>(a, rs, grid, done, st, smem);
  } else {
    if (two) spmm2_launch<GP, false, 2>(a, rs, grid, done, st, smem);
    else spmm2_launch<GP, false, kMaxRed>(a, rs, grid, done, st, smem);
  }
  KR_CUDA(cudaGetLastError());
}

static void spmm2_dispatch(const SpmmArgs<float>& a, const RedSet& rs, int& grid, const int* done, cudaStream_t st) {
  switch (threads_per_row(a.s / 2)) {
    case 1: return spmm2_go<1>(a, rs, grid, done, st);
    case 2: return spmm2_go<2>(a, rs, grid, done, st);
    case 4: return spmm2_go<4>(a, rs, grid, done, st);
    case 8: return spmm2_go<8>(a, rs, grid, done, st);
    case 16: return spmm2_go<16>(a, rs, grid, done, st);
  }
  throw CudaError{cudaErrorInvalidValue, "spmm: s out of range"};
}

template <int GP>
static void lin2_go(const LinArgs& a, const RedSet& rs, int& grid, const int* done, cudaStream_t st) {
  size_t smem = (size_t)a.nmat * a.s * sizeof(float2);
  if (rs.nred > 0) smem += (size_t)(kThreads / 32) * rs.nslots * sizeof(float2);
  if (smem > 48 * 1024) throw CudaError{cudaErrorInvalidValue, "lincomb: shared memory budget exceeded"};
  thread_local std::unordered_map<size_t, int> occ;
  grid = resident_grid(lincomb2_kernel<GP>, smem, grid, occ);
  lincomb2_kernel<GP><<<grid, kThreads, smem, st>>>(a, rs, done);
  KR_CUDA(cudaGetLastError());
}

static void lin2_dispatch(const LinArgs& a, const RedSet& rs, int& grid, const int* done, cudaStream_t st) {
  switch (threads_per_row(a.s / 2)) {
    case 1: return lin2_go<1>(a, rs, grid, done, st);
    case 2: return lin2_go<2>(a, rs, grid, done, st);
    case 4: return lin2_go<4>(a, rs, grid, done, st);
    case 8: return lin2_go<8>(a, rs, grid, done, st);
    case 16: return lin2_go<16>(a, rs, grid, done, st);
  }
  throw CudaError{cudaErrorInvalidValue, "lincomb: s out of range"};
}

// ---------------------------------------------------------------------------------------
// complex64 CSR product on TMA-staged row tiles (kr_tile_c64.cuh)
// ---------------------------------------------------------------------------------------
inline int round16i(int64_t b) { return (int)((b + 15) & ~(int64_t)15); }

// Reduction maps of a staged product launch (row tiles or planes): the distinct block operands U,
// the Grams' operands and slots, the per-row reductions' accumulators; false when the launch has
// more than kTileMaxU distinct operands, two Grams, kTileRowReds per-row reductions, or a U that
// is not 16-byte aligned.
static bool red_layout(const SpmmArgs<float>& a, const RedSet& rs, TileLayout& L) {
  const int s = a.s;
  L = TileLayout{};
  int ngram = 0, nc = 0, nrow = 0;
  for (int ri = 0; ri < kMaxRed; ++ri) L.red_u[ri] = -1;
  for (int ri = 0; ri < rs.nred; ++ri) {
    const RedSpec& r = rs.r[ri];
    if (r.ureg >= 0) return false;
    const bool block_u = r.kind == RED_GRAM || r.kind == RED_TRACE || r.kind == RED_CDOT;
    int ui = -1;
    if (block_u && r.U != nullptr && r.U != static_cast<const void*>(a.Y)) {
      if (!aligned16(r.U)) return false;
      for (int u = 0; u < L.nu; ++u)
        if (L.U[u] == r.U) ui = u;
      if (ui < 0) {
        if (L.nu == kTileMaxU) return false;
        ui = L.nu;
        L.U[L.nu++] = r.U;
      }
    }
    if (r.kind == RED_GRAM) {
      if (ngram == 2) return false;
      L.gram_u[ngram] = ui;
      L.gram_slot[ngram] = r.slot;
      ++ngram;
    } else {
      if (nrow == kTileRowReds) return false;
      L.red_u[ri] = ui;
      L.red_c[ri] = nc;
      L.red_k[ri] = nrow++;
      nc += (r.kind == RED_CDOT || r.kind == RED_GRAMV) ? s : 1;
    }
  }
  L.ngram = ngram;
  L.ystage = ngram > 0 ? 1 : 0;
  L.ncompact = nc;
  return true;
}

// Shared-memory layout and reduction maps of a tile launch; false when the launch does not fit
// the tile kernel (then the other kernels run it).
static bool tile_layout(const SpmmArgs<float>& a, const RedSet& rs, TileLayout& L) {
  if (a.lat) return false;
  const bool sten = a.nst > 0;
  const int s = a.s;
  if (s != 4 && s != 8 && s != 16 && s != 32) return false;
  const int GP = s / 2;
  const int R = std::min(128, kTileThreadsMax / GP);
  if (!sten && (int64_t)R * a.maxrow > kTileEcap) return false;
  if (!aligned16(a.V) || !aligned16(a.Y) || !aligned16(a.Z)) return false;
  if (rs.nred > kMaxRed) return false;
  if (!red_layout(a, rs, L)) return false;
  L.R = R;
  const int ngram = L.ngram, nc = L.ncompact;
  const bool split = !sten && a.split != 0;
  L.mode = sten ? 2 : (split ? 1 : 0);
  L.off_rp = 0;
  L.sz_rp = sten ? 0 : round16i((int64_t)(R + 2) * 8);
  L.off_dg = L.sz_rp;
  L.sz_dg = split ? R * 8 : 0;
  L.off_u = L.sz_rp + L.sz_dg;
  L.sz_u = R * s * 8;
  L.off_col = 0;
  L.sz_col = sten ? 0 : round16i((int64_t)(kTileEcap + 8) * 4);
  L.off_val = L.sz_col;
  L.sz_val = sten ? 0 : round16i((int64_t)(kTileEcap + 8) * (split ? 4 : 8));
  const int strideA = L.sz_rp + L.sz_dg + L.nu * L.sz_u, strideB = L.sz_col + L.sz_val;
  L.off_y = kTileStagesA * strideA + kTileStagesB * strideB;
  const int staged = L.off_y + (L.ystage ? R * s * 8 : 0);
  const int T = GP * R;
  const int final_red = (T / 32) * nc * 8 + ngram * (T / (GP * GP)) * s * s * 8;
  L.total = std::max(staged, final_red);
  return L.total <= kMaxDynSmem;
}

// Geometry, shared-memory layout and reduction maps of a plane launch (kr_plane_c64.cuh); false when
// the launch does not qualify (then the row-tile or per-row kernels run it).  The x-y tile is the
// largest of the candidates whose stages fit two CTAs per SM (else one).
static bool plane_layout(const SpmmArgs<float>& a, const RedSet& rs, TileLayout& L, PlaneGeom& P) {
  if (a.lat || a.nst < 2 || a.nst > 3) return false;
  const int s = a.s;
  if (s != 2 && s != 4 && s != 8 && s != 16 && s != 32) return false;
  if (!aligned16(a.V) || !aligned16(a.Y) || !aligned16(a.Z)) return false;
  if (rs.nred > kMaxRed) return false;
  const int64_t nx = a.sdims[0], ny = a.sdims[1], nz = a.nst == 3 ? a.sdims[2] : 1;
  if (a.sstr[0] != 1 || a.sstr[1] != nx || (a.nst == 3 && a.sstr[2] != nx * ny)) return false;
  if (nx * ny * nz != a.n || a.n > 0x7fffffffLL) return false;
  if (!red_layout(a, rs, L) || L.nu > 1) return false;
  const int GP = s / 2;
  const int T = kPlaneThreads;
  auto r128 = [](int64_t b) { return (int)((b + 127) & ~(int64_t)127); };
  static const int cand[][2] = {{32, 8}, {32, 4}, {32, 2}, {16, 4}, {16, 2}, {32, 1}, {16, 1}, {8, 1}};
  const int final_red = (T / 32) * L.ncompact * 8 + L.ngram * (T / (GP * GP)) * s * s * 8;
  for (int pass = 0; pass < 2; ++pass) {
    const int cap = (pass == 0 ? 110 * 1024 : kMaxDynSmem) - 128;  // the launch adds 128 bytes of alignment
    for (const auto& c : cand) {
      const int tx = (int)std::min<int64_t>(c[0], nx), ty = (int)std::min<int64_t>(c[1], ny);
      PlaneGeom g{};
      g.nx = (int)nx; g.ny = (int)ny; g.nz = (int)nz;
      g.tx = tx; g.ty = ty;
      g.ntx = (int)((nx + tx - 1) / tx);
      g.nty = (int)((ny + ty - 1) / ty);
      g.ipt = (tx * ty * GP + T - 1) / T;
      if (g.ipt > kPlaneMaxIpt) continue;
      g.off_v = 0;
      g.stride_v = r128((int64_t)(tx + 2) * (ty + 2) * s * 8);
      g.off_u = kPlaneStagesV * g.stride_v;
      g.stride_u = L.nu > 0 ? r128((int64_t)tx * ty * s * 8) : 0;
      g.off_y = g.off_u + kPlaneStagesU * g.stride_u;
      const int staged = g.off_y + (L.ngram > 0 ? r128((int64_t)tx * ty * s * 8) : 0);
      g.total = std::max(staged, final_red);
      if (g.total <= cap) {
        P = g;
        return true;
      }
    }
  }
  return false;
}

template <typename T>
int launch_spmm(const SpmmArgs<T>& a, const RedSet& rs, int grid, const int* done, cudaStream_t st) {
  ProfToken tk = prof_begin(sizeof(T) == 4 ? KC_SPMM32 : KC_SPMM, st);
  bool done_launch = false;
  if (a.lat) {
    lattice_dispatch<T>(a, rs, grid, done, st);
    done_launch = true;
  }
  if constexpr (sizeof(T) == 4) {
    TileLayout L;
    PlaneGeom P;
    if (!done_launch && tile_kernels_enabled() && plane_layout(a, rs, L, P) && plane_kernels_available()) {
      grid = launch_spmm_plane(a, rs, L, P, done, st);
      done_launch = true;
    }
    if (!done_launch && tile_kernels_enabled() && tile_layout(a, rs, L)) {
      grid = launch_spmm_tile(a, rs, L, grid, done, st);
      done_launch = true;
    }
    if (!done_launch && pair_kernels_enabled() && pair_ok_spmm(a, rs)) {
      spmm2_dispatch(a, rs, grid, done, st);
      done_launch = true;
    }
  }
  if (!done_launch) spmm_dispatch<T>(a, rs, grid, done, st);
  const double E = sizeof(C2<T>);
  const double n = (double)a.n, s = (double)a.s, nnz = (double)a.nnz;
  double f = a.split ? s * (4.0 * nnz + 6.0 * n) : s * 8.0 * nnz;
  // per site and column: diagonal (12 complex products) + 8 hops x (6 projection + 18 link + 12
  // reconstruction complex multiply-adds) for whole sites; with (site, colour) units the
  // projection is repeated per colour: 3 x 8 x (6 + 6 + 4)
  if (a.lat) {
    if (lattice_rows_per_thread(sizeof(T)) == 12) f = s * (n / 12.0) * (6.0 * 12 + 8 * (6 + 18 + 12) * 8);
    else f = s * (n / 12.0) * (6.0 * 12 + 3.0 * 8 * (6 + 6 + 4) * 8);
  }
  if (a.ys != nullptr || a.ay != 1.0) f += 6.0 * s * n;
  if (a.Z != nullptr) f += 4.0 * s * n;
  f += red_flops(rs, a.n, a.s);
  double b = a.nst > 0 ? 0.0 : 8.0 * (n + 1) + 4.0 * nnz + (a.split ? sizeof(T) * nnz + E * n : E * nnz);
  if (a.lat) b = 4.0 * (n / 12.0) * 9.0 * E;  // the links
  if (a.nst > 0 && !a.sreal) f = s * 8.0 * (nnz + n);
  b += E * n * s;
  if (a.Y != nullptr) b += E * n * s;
  if (a.Z != nullptr) b += E * n * s;
  const void* counted[3] = {a.V, a.Y, a.Z};
  b += red_bytes(rs, a.n, a.s, E, counted, 3);
  prof_end(tk, st, f, b);
  return grid;
}

template <typename T, int G, int NG>
static void lin_go(const LinArgs& a, const RedSet& rs, int& grid, const int* done, cudaStream_t st) {
  static std::atomic<uint64_t> attr{0};
  allow_smem(lincomb_kernel<T, G, NG>, attr);
  size_t smem = (size_t)a.nmat * a.s * a.s * sizeof(C2<T>);
  if (rs.nred > 0) smem += (size_t)(kThreads / 32) * rs.nslots * sizeof(C2<T>);
  if (smem > (size_t)kMaxDynSmem) throw CudaError{cudaErrorInvalidValue, "lincomb: shared memory budget exceeded"};
  thread_local std::unordered_map<size_t, int> occ;
  grid = resident_grid(lincomb_kernel<T, G, NG>, smem, grid, occ);
  lincomb_kernel<T, G, NG><<<grid, kThreads, smem, st>>>(a, rs, done);
  KR_CUDA(cudaGetLastError());
}

template <typename T, int G>
static void lin_ng(int ng, const LinArgs& a, const RedSet& rs, int& grid, const int* done, cudaStream_t st) {
  if (ng == 0) return lin_go<T, G, 0>(a, rs, grid, done, st);
  if constexpr (NGCap<1, G>::ok) {
    if (ng == 1) return lin_go<T, G, 1>(a, rs, grid, done, st);
  }
  if constexpr (NGCap<2, G>::ok) {
    if (ng == 2) return lin_go<T, G, 2>(a, rs, grid, done, st);
  }
  throw CudaError{cudaErrorInvalidValue, "lincomb: fused Gram count exceeds the register budget"};
}

template <typename T>
static void lin_dispatch(const LinArgs& a, const RedSet& rs, int& grid, const int* done, cudaStream_t st);

// profile accounting of a row-local launch (flops, bytes), shared by both launchers
static void lin_account(const LinArgs& a, const RedSet& rs, double E, double& f, double& b) {
  const double n = (double)a.n, s = (double)a.s;
  f = 0.0;
  b = 0.0;
  const void* counted[kMaxOut * kMaxTerm + kMaxOut];
  int nc = 0;
  for (int o = 0; o < a.nout; ++o) {
    const Out& q = a.o[o];
    const double cnt = q.is_vec ? n : n * s;
    for (int t = 0; t < q.nterm; ++t) {
      const Term& tm = q.t[t];
      switch (tm.coef_kind) {
        case COEF_ONE: f += (t == 0 ? 0.0 : 2.0) * cnt; break;  // a leading copy is not arithmetic
        case COEF_REAL: f += 4.0 * cnt; break;
        case COEF_MAT: f += 8.0 * s * cnt; break;
        default: f += 8.0 * cnt; break;
      }
      if (tm.src_kind == SRC_BLOCK || tm.src_kind == SRC_VEC) {
        bool seen = false;
        for (int k = 0; k < nc; ++k) seen = seen || counted[k] == tm.src;
        if (!seen) {
          counted[nc++] = tm.src;
          b += E * (tm.src_kind == SRC_VEC ? n : n * s);
        }
      }
    }
    if (q.dst != nullptr) b += E * cnt;
  }
  f += red_flops(rs, a.n, a.s);
  b += red_bytes(rs, a.n, a.s, E, counted, nc);
}

template <typename T>
int launch_lincomb(const LinArgs& a_in, const RedSet& rs_in, int grid, const int* done, cudaStream_t st) {
  LinArgs a = a_in;
  RedSet rs = rs_in;
  if (!resolve_sources(a, rs)) throw CudaError{cudaErrorInvalidValue, "lincomb: too many distinct operands"};
  ProfToken tk = prof_begin(sizeof(T) == 4 ? KC_LINCOMB32 : KC_LINCOMB, st);
  if (sizeof(T) == 4 && pair_kernels_enabled() && pair_ok_lin(a, rs)) lin2_dispatch(a, rs, grid, done, st);
  else lin_dispatch<T>(a, rs, grid, done, st);
  double f = 0.0, b = 0.0;
  lin_account(a, rs, sizeof(C2<T>), f, b);
  prof_end(tk, st, f, b);
  return grid;
}

template <typename T>
static void lin_dispatch(const LinArgs& a, const RedSet& rs, int& grid, const int* done, cudaStream_t st) {
  const int G = threads_per_row(a.s);
  const int ng = count_grams(rs);
  switch (G) {
    case 1: return lin_ng<T, 1>(ng, a, rs, grid, done, st);
    case 2: return lin_ng<T, 2>(ng, a, rs, grid, done, st);
    case 4: return lin_ng<T, 4>(ng, a, rs, grid, done, st);
    case 8: return lin_ng<T, 8>(ng, a, rs, grid, done, st);
    case 16: return lin_ng<T, 16>(ng, a, rs, grid, done, st);
    case 32: return lin_ng<T, 32>(ng, a, rs, grid, done, st);
  }
  throw CudaError{cudaErrorInvalidValue, "lincomb: s out of range"};
}

template <typename T>
void launch_reduce(const void* partials, int nparts, int nslots, double2* out, const int* done, cudaStream_t st) {
  if (nslots <= 0) return;
  ProfToken tk = prof_begin(KC_REDUCE, st);
  reduce_slots_kernel<T><<<nslots, kThreads, 0, st>>>(reinterpret_cast<const C2<T>*>(partials), nparts, nslots,
                                                       out, done);
  KR_CUDA(cudaGetLastError());
  prof_end(tk, st, 2.0 * nparts * nslots, (double)sizeof(C2<T>) * nparts * nslots + 16.0 * nslots);
}

// products and reductions in one unit, row-local combinations in another (parallel build)
#define KR_INSTANTIATE_ROWS(T)                                                                               \
  template int launch_spmm<T>(const SpmmArgs<T>&, const RedSet&, int, const int*, cudaStream_t);            \
  template void launch_reduce<T>(const void*, int, int, double2*, const int*, cudaStream_t);
#define KR_INSTANTIATE_LIN(T) \
  template int launch_lincomb<T>(const LinArgs&, const RedSet&, int, const int*, cudaStream_t);

}  // namespace kr
