// Host-side interface of the complex64 row-tile product (kr_tile_c64.cuh, kr_tile_f32.cu).
#pragma once

#include "kr_internal.h"

namespace kr {

constexpr int kTileEcap = 1024;        // stored entries per tile held in shared memory
constexpr int kTileStagesA = 3;        // row pointers / diagonal / U blocks: tiles in flight
constexpr int kTileStagesB = 2;        // indices / values: tiles in flight
constexpr int kTileMaxU = 2;           // distinct block operands of the reductions
constexpr int kTileThreadsMax = 256;
constexpr int kTileRowReds = 2;        // per-row reductions (trace, column dots, norm, sums)

// Shared-memory layout of one launch (byte offsets, all multiples of 16) and the reduction maps,
// computed on the host.
struct TileLayout {
  int R;          // rows per tile (GP * R threads)
  int mode;       // 0: CSR, 1: CSR with real off-diagonal entries and complex diagonal, 2: stencil
  int nu;         // distinct block operands U staged per tile (0..2)
  int ngram;      // fused Grams (0..2)
  int ystage;     // Y kept in shared memory for the Grams
  int gram_u[2];  // per Gram: staged operand index, or -1 for Y itself (Y^H Y)
  int gram_slot[2];       // per Gram: first slot of its s x s record
  int red_u[kMaxRed];     // per-row reductions: staged operand index, or -1 (Y itself / n-vector)
  int red_c[kMaxRed];     // per-row reductions: offset in the compact per-warp record
  int red_k[kMaxRed];     // per-row reductions: accumulator index (0 or 1)
  int ncompact;           // slots of the per-row reductions
  int off_rp, sz_rp;      // per A-stage: row pointers (R + 2 int64)
  int off_dg, sz_dg;      // per A-stage: complex diagonal (split storage)
  int off_u, sz_u;        // per A-stage and operand: U rows (R x s complex64)
  int off_col, sz_col;    // per B-stage: column indices
  int off_val, sz_val;    // per B-stage: values (float or float2)
  int off_y;              // R x s complex64
  int total;
  const void* U[kTileMaxU];  // the staged operands
};

// Launch the tile product (layout from tile_layout); returns the grid launched.
int launch_spmm_tile(const SpmmArgs<float>& a, const RedSet& rs, const TileLayout& L, int grid, const int* done,
                     cudaStream_t st);

}  // namespace kr
