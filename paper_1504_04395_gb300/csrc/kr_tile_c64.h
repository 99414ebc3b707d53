// Host-side interface of the complex64 row-tile product (kr_tile_c64.cuh, kr_tile_f32.cu).
#pragma once

#include "kr_internal.h"

namespace kr {

constexpr int kTileThreads = 256;      // threads per CTA: GP = s/2 per row, R = 256 / GP rows per tile
// pipeline stages (buffers in tile order) and how many tiles ahead of the consumed one each is filled
constexpr int kTileStagesA1 = 6;       // row pointers, issued 5 tiles ahead
constexpr int kTileStagesB = 4;        // column indices and values, issued 3 tiles ahead
constexpr int kTileStagesA2 = 3;       // diagonal and U blocks, issued 3 tiles ahead (after the tile is freed)
constexpr int kTileStagesG = 2;        // gathered rows of V, issued 1 tile ahead
constexpr int kTileMaxU = 2;           // distinct block operands of the reductions
constexpr int kTileRowReds = 2;        // per-row reductions (trace, column dots, norm, sums)
constexpr int kTileStencilSlots = 7;   // gathered rows per row of the (2d+1)-point stencil, d <= 3

// Shared-memory layout of one launch (byte offsets, all multiples of 16) and the reduction maps,
// computed on the host.
struct TileLayout {
  int R;          // rows per tile (GP * R = kTileThreads threads)
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
  int ecap;               // stored entries per tile held in shared memory (CSR)
  int sz_rp;              // per A1-stage: row pointers (R + 2 int64)
  int off_dg, sz_dg;      // per A2-stage: complex diagonal (split storage)
  int off_u, sz_u;        // per A2-stage and operand: U rows (R x s complex64)
  int off_col, sz_col;    // per B-stage: column indices
  int off_val, sz_val;    // per B-stage: values (float or float2)
  int off_ge;             // per G-stage: first gathered entry (after R diagonal rows, split storage)
  int stride_a1, stride_a2, stride_b, stride_g;  // bytes per stage
  int off_a2, off_b, off_g;  // first A2-, B- and G-stage (the A1-stages start at 0)
  int off_y;              // R x s complex64
  int total;
  const void* U[kTileMaxU];  // the staged operands
};

// Launch the tile product (layout from tile_layout); returns the grid launched.
int launch_spmm_tile(const SpmmArgs<float>& a, const RedSet& rs, const TileLayout& L, int grid, const int* done,
                     cudaStream_t st);

}  // namespace kr
