// Skewed-tile task geometry shared by the Gauss-Seidel and temporal Jacobi
// schedulers (host and device).
//
// The interior is cut into tiles W x H x D.  A task (I, J, K, p) performs the
// ns = min(nt, nsweeps - p*nt) sweeps of pass p on tile (I, J, K); at the
// pass-local sweep s (0 <= s < ns) the tile is shifted by -s in x, y and z:
//     x in [I*W - s, (I+1)*W - s)   (likewise y with H, z with D),
// clipped to the interior.  Shifting each sweep back by one cell makes every
// neighbour a task reads either its own earlier sweep or a task of lower
// level, so the in-place grid itself serves as the boundary store between
// tiles (Sec. 4: "no additional computations are necessary for the
// boundary treatment").  Tasks are ordered by the level
//     L = I + J + K + c*p,  c = 2 if nt == 1, else 4,
// and all tasks of one level are independent.  Tile counts cover the shifted
// tiles: NI = ceil((nx + nt - 1) / W).  The shift of a pass (nt - 1 cells)
// must stay below every tile extent, nt <= min(W, H, D): then a task's box
// meets only tiles one step away and tasks of one level never touch the same
// site (with nt = min + 1 the result already depends on the order of the
// tasks within a level).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace stn {

struct TileGeom {
  int W, H, D;       // tile extents
  int nt;            // sweeps per pass
  int NI, NJ, NK;    // tiles per dimension
  int npass;         // passes
  int nsweeps;       // total sweeps
  int cstride;       // level distance between passes
  int sigma_max;     // NI + NJ + NK - 3
  int nlevels;       // sigma_max + cstride*(npass-1) + 1
};

__host__ __device__ inline uint64_t pack_tile(int I, int J, int K) {
  return (uint64_t)I | ((uint64_t)J << 21) | ((uint64_t)K << 42);
}
__host__ __device__ inline void unpack_tile(uint64_t t, int* I, int* J, int* K) {
  *I = (int)(t & 0x1FFFFF);
  *J = (int)((t >> 21) & 0x1FFFFF);
  *K = (int)((t >> 42) & 0x1FFFFF);
}

// Intra-tile site entry: tile-local (ii, jj, kk) at pass-local sweep s.
__host__ __device__ inline uint32_t pack_site(int ii, int jj, int kk, int s) {
  return (uint32_t)ii | ((uint32_t)jj << 8) | ((uint32_t)kk << 16) | ((uint32_t)s << 24);
}

}  // namespace stn

struct stencil_ctx;
namespace stn {
struct Geom;
// host helpers (gs.cu): task geometry, the (I,J,K)-by-sigma slice table cached
// in the context, and the number of tasks of one level
TileGeom make_tile_geom(const Geom& g, int W, int H, int D, int nt, int nsweeps);
int ensure_slices(stencil_ctx* ctx, const TileGeom& tg, cudaStream_t st);
int tasks_at_level(const stencil_ctx* ctx, const TileGeom& tg, int L);
const uint64_t* slices_ptr(stencil_ctx* ctx);
const int* slice_off_ptr(stencil_ctx* ctx);

// Device: the task (I, J, K, p) that CTA `blockIdx.x` of level `level` runs;
// false if the index is beyond the level (not for a correctly sized launch).
__device__ __forceinline__ bool find_task(const TileGeom& tg, const uint64_t* __restrict__ slices,
                                          const int* __restrict__ slice_off, int level, int* I, int* J, int* K,
                                          int* p) {
  int b = blockIdx.x;
  int pp = level / tg.cstride;
  if (pp > tg.npass - 1) pp = tg.npass - 1;
  int sigma = level - tg.cstride * pp;
  for (;;) {
    int cnt = (sigma <= tg.sigma_max) ? slice_off[sigma + 1] - slice_off[sigma] : 0;
    if (b < cnt) break;
    b -= cnt;
    --pp;
    sigma += tg.cstride;
    if (pp < 0) return false;
  }
  unpack_tile(slices[slice_off[sigma] + b], I, J, K);
  *p = pp;
  return true;
}
}  // namespace stn
