// Host-side interface of the complex64 plane-marching stencil product (kr_plane_c64.cuh,
// kr_tile_f32.cu).
#pragma once

#include "kr_tile_c64.h"

namespace kr {

constexpr int kPlaneThreads = 256;
constexpr int kPlaneStagesV = 5;  // halo'd planes of V: z-1, z, z+1 in use, two more in flight
constexpr int kPlaneStagesU = 3;  // planes of U: the current one, two more in flight
constexpr int kPlaneAheadV = 2;   // V planes loaded ahead of the ones in use
constexpr int kPlaneAheadU = 2;   // U planes loaded ahead of the current one
constexpr int kPlaneMaxIpt = 2;   // (point, column pair) items per thread and plane

// Geometry and shared-memory layout of one launch (byte offsets, multiples of 128).
struct PlaneGeom {
  int nx, ny, nz;        // grid extents (nz = 1 for a 2D stencil)
  int tx, ty;            // tile extents in x and y
  int ntx, nty;          // tiles per plane along x and y
  int ipt;               // (point, column pair) items per thread and plane
  int off_v, stride_v;   // first V stage; bytes per V stage ((ty + 2) x (tx + 2) points)
  int off_u, stride_u;   // first U stage; bytes per U stage (ty x tx points)
  int off_y;             // the plane tile's Y (fused Grams)
  int total;
};

// Whether the driver provides the tensor-map encoder the plane product needs (else the other
// complex64 product kernels run its launches).
bool plane_kernels_available();

// Launch the plane product (geometry and reduction maps from plane_layout in kr_rows_launch.cuh);
// returns the grid launched.
int launch_spmm_plane(const SpmmArgs<float>& a, const RedSet& rs, const TileLayout& L, const PlaneGeom& P,
                      const int* done, cudaStream_t st);

}  // namespace kr
