// The 2.5D z-march of the Jacobi sweep (jacobi.cu), shared by the one-sweep
// kernel and the in-place slab kernel (jacobi_inplace.cu).
//
// A CTA of 32 x BY threads owns a 32 x BY tile of (x, y) columns and a range
// of z-planes.  Each thread keeps its own column's planes k-1, k, k+1 in
// registers (the paper's "three planes in cache" of Fig. stencil_mapping,
// here in the register file), the current plane is staged in shared memory
// (double-buffered, one __syncthreads per plane) for the four in-plane
// neighbours, and halo columns/rows of the tile are loaded by the edge
// threads.
#pragma once

#include "internal.h"

namespace stn {

// The march of the CTA's tile (bx, by) (columns bx*32.., rows by*BY..) over
// planes [z0, z1) of g (z0 < z1, the same for the whole CTA): src -> dst, sm
// the CTA's plane buffers.
template <typename T, class Ar, bool HAS_F, bool WEIGHTED, int BY>
__device__ __forceinline__ void zmarch_body(const T* __restrict__ src, T* __restrict__ dst, const T* __restrict__ f,
                                            const Geom g, int z0, int z1, const Coef<T> c,
                                            T (&sm)[2][BY + 2][32 + 2], int bx, int by) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x = bx * 32 + tx;
  const int y = by * BY + ty;
  const bool inside = (x <= g.nx) && (y <= g.ny);  // own column lies in the interior or the +1 halo
  const bool active = (x < g.nx) && (y < g.ny);    // own column is an interior column
  // halo duties (each at most one extra column or row)
  const bool hw = (tx == 0) && (y <= g.ny);                     // column x-1 (>= -1)
  const bool he = (tx == 31) && (x + 1 <= g.nx) && (y <= g.ny);  // column x+1
  const bool hs = (ty == 0) && (x <= g.nx);                     // row y-1 (>= -1)
  const bool hn = (ty == BY - 1) && (y + 1 <= g.ny) && (x <= g.nx);
  const int64_t sy = g.sy;
  // pointers at plane z (advanced by one plane per step; dereferenced only when in range)
  const int64_t o0 = (int64_t)(z0 + 1) * sy;
  const T* pc = src + (inside ? g.at(x, y, -1) : 0) + o0;
  const T* pw = src + (hw ? g.at(x - 1, y, -1) : 0) + o0;
  const T* pe = src + (he ? g.at(x + 1, y, -1) : 0) + o0;
  const T* ps = src + (hs ? g.at(x, y - 1, -1) : 0) + o0;
  const T* pn = src + (hn ? g.at(x, y + 1, -1) : 0) + o0;
  const int64_t od = (inside ? g.at(x, y, -1) : 0) + o0;
  T* pd = dst + od;
  const T* pf = HAS_F ? f + od : nullptr;
  T below = inside ? pc[-sy] : T(0);
  T cur = inside ? pc[0] : T(0);
  T above = inside ? pc[sy] : T(0);
  auto step = [&](int z, int bf) {
    sm[bf][ty + 1][tx + 1] = cur;
    if (hw) sm[bf][ty + 1][0] = *pw;
    if (he) sm[bf][ty + 1][33] = *pe;
    if (hs) sm[bf][0][tx + 1] = *ps;
    if (hn) sm[bf][BY + 1][tx + 1] = *pn;
    // prefetch plane z+2 (exists up to the top halo plane nz)
    const T next = (inside && z + 2 <= g.nz) ? pc[2 * sy] : T(0);
    T fv = T(0);
    if (HAS_F && active) fv = *pf;
    __syncthreads();
    if constexpr (AdaptOf<Ar>::on) {  // the whole warp votes (its lanes are converged here)
      const T v = site_update_warp<T, Ar, HAS_F, WEIGHTED>(active, sm[bf][ty + 1][tx], sm[bf][ty + 1][tx + 2],
                                                           sm[bf][ty][tx + 1], sm[bf][ty + 2][tx + 1], below,
                                                           above, fv, cur, c);
      if (active) *pd = v;
    } else if (active) {
      *pd = site_update<T, Ar, HAS_F, WEIGHTED>(sm[bf][ty + 1][tx], sm[bf][ty + 1][tx + 2], sm[bf][ty][tx + 1],
                                                sm[bf][ty + 2][tx + 1], below, above, fv, cur, c);
    }
    below = cur;
    cur = above;
    above = next;
    pc += sy;
    pw += sy;
    pe += sy;
    ps += sy;
    pn += sy;
    pd += sy;
    if (HAS_F) pf += sy;
  };
  int z = z0;
  for (; z + 1 < z1; z += 2) {  // two planes per trip: the buffer index is a constant
    step(z, 0);
    step(z + 1, 1);
  }
  if (z < z1) step(z, 0);
}

}  // namespace stn
