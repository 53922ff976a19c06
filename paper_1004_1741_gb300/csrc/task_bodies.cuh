// Per-task bodies of the skewed-tile schedules (tiles.h), shared by the
// level-launch kernels (one CTA per task of a level) and the persistent
// dataflow kernel (CTAs pull tasks from a queue).  A body is executed by all
// threads of a CTA and ends with a __syncthreads.
#pragma once

#include "common.cuh"
#include "tiles.h"

struct stencil_ctx;

namespace stn {

constexpr int GS_THREADS = 256;
constexpr int GS_MAXPOS = 2048 / GS_THREADS;  // box-plane positions per thread: (W+nt+1)(H+nt+1) <= 2048
constexpr int GS_MAXLEVELS = 128;  // tile-local levels W+H+D-3+ns <= 128

// Site table of the tile-local levels (built on the host, see ensure_sites).
struct SiteTable {
  const uint32_t* coords;  // packed (ii, jj, kk, s)
  const uint16_t* lis;     // shared-memory index of the site inside the staged box
  const int* off;          // level offsets, per ns one block of W+H+D-2+ns entries
  const int* base;         // base[ns]: first entry of ns's block in off
  const int* goff;         // per site: grid offset from the tile origin for one grid shape, or nullptr
};

// Gauss-Seidel task (I, J, K, p) updated in place through the L1 cache: the
// tile-local levels ii+jj+kk-s run one after the other, all sites of a level
// in parallel, listed compactly in the site table so that warp lanes are
// packed.  A site written at level lv is read at level lv+1 by threads of the
// same CTA after the barrier; everything written by other tasks was
// published before this task started.  s_off: shared int[GS_MAXLEVELS+1].
template <typename T, class Ar, bool HAS_F, int W, int H, int D>
__device__ __forceinline__ void gs_task_body(T* u, const T* __restrict__ f, const Geom& g, const Coef<T>& c,
                                             const SiteTable& tb, const TileGeom& tg, int I, int J, int K, int p,
                                             int* s_off) {
  const int tid = threadIdx.x;
  const int X0 = I * W, Y0 = J * H, Z0 = K * D;
  const int ns = min(tg.nt, tg.nsweeps - p * tg.nt);
  const int nlv = W + H + D - 3 + ns;
  const int* so = tb.off + tb.base[ns];
  for (int l = tid; l <= nlv; l += GS_THREADS) s_off[l] = so[l];
  const bool full = (X0 - ns + 1 >= 0) && (Y0 - ns + 1 >= 0) && (Z0 - ns + 1 >= 0) && (X0 + W <= g.nx) &&
                    (Y0 + H <= g.ny) && (Z0 + D <= g.nz);
  const int64_t sx = g.sx, sy = g.sy;
  T* ut = u + g.at(X0, Y0, Z0);  // site (ii, jj, kk) of sweep s at ut[(kk-s)*sy + (jj-s)*sx + (ii-s)]
  __syncthreads();
  for (int lv = 0; lv < nlv; ++lv) {
    const int beg = s_off[lv], end = s_off[lv + 1];
    int t = tid - (((int)blockIdx.x + lv) & (GS_THREADS / 32 - 1)) * 32;
    if (t < 0) t += GS_THREADS;
    if (full && tb.goff) {
      // interior task: the site's offset comes precomputed from the table
      for (int e = beg + t; e < end; e += GS_THREADS) {
        T* q = ut + tb.goff[e];
        T fv = T(0);
        if (HAS_F) fv = f[q - u];
        *q = site_update<T, Ar, HAS_F, false>(q[-1], q[1], q[-sx], q[sx], q[-sy], q[sy], fv, T(0), c);
      }
    } else {
      for (int e = beg + t; e < end; e += GS_THREADS) {
        const uint32_t s = tb.coords[e];
        const int sw = (int)(s >> 24);
        const int dx = (int)(s & 0xFF) - sw, dy = (int)((s >> 8) & 0xFF) - sw, dz = (int)((s >> 16) & 0xFF) - sw;
        if (!full && (X0 + dx < 0 || X0 + dx >= g.nx || Y0 + dy < 0 || Y0 + dy >= g.ny || Z0 + dz < 0 ||
                      Z0 + dz >= g.nz))
          continue;
        T* q = ut + ((int64_t)dz * sy + (int64_t)dy * sx + dx);
        T fv = T(0);
        if (HAS_F) fv = f[q - u];
        *q = site_update<T, Ar, HAS_F, false>(q[-1], q[1], q[-sx], q[sx], q[-sy], q[sy], fv, T(0), c);
      }
    }
    __syncthreads();
  }
}

// Jacobi task (I, J, K, p): the ns sweeps of pass p on the shifted tile, level
// v read from the grid of v's parity, level v+1 written to the other grid.
template <typename T, class Ar, bool HAS_F, bool WEIGHTED, int W, int H, int D>
__device__ __forceinline__ void jacobi_task_body(T* g_even, T* g_odd, const T* __restrict__ f, const Geom& g,
                                                 const Coef<T>& c, const TileGeom& tg, int I, int J, int K, int p) {
  const int ns = min(tg.nt, tg.nsweeps - p * tg.nt);
  const int X0 = I * W, Y0 = J * H, Z0 = K * D;
  const bool full = (X0 - ns + 1 >= 0) && (Y0 - ns + 1 >= 0) && (Z0 - ns + 1 >= 0) && (X0 + W <= g.nx) &&
                    (Y0 + H <= g.ny) && (Z0 + D <= g.nz);
  const int64_t sx = g.sx, sy = g.sy;
  const int64_t base = g.at(X0, Y0, Z0);
  constexpr int NSITE = W * H * D;
  static_assert(NSITE % 32 == 0, "whole warps of sites");
  for (int s = 0; s < ns; ++s) {
    const int v = p * tg.nt + s;
    const T* src = (v & 1) ? g_odd : g_even;
    T* dst = (v & 1) ? g_even : g_odd;
    const int64_t sb = base - (int64_t)s * (sy + sx + 1);
#pragma unroll 2
    for (int q = threadIdx.x; q < NSITE; q += GS_THREADS) {  // the same trip count for every lane of a warp
      const int ii = q % W, jj = (q / W) % H, kk = q / (W * H);
      bool act = true;
      if (!full) {
        const int x = X0 - s + ii, y = Y0 - s + jj, z = Z0 - s + kk;
        act = !(x < 0 || x >= g.nx || y < 0 || y >= g.ny || z < 0 || z >= g.nz);
      }
      // a lane whose site lies outside the grid reads the first interior site instead (result discarded), so
      // that the whole warp takes part in the adaptive arithmetic's vote
      const int64_t o = act ? sb + (int64_t)kk * sy + (int64_t)jj * sx + ii : g.at(0, 0, 0);
      T fv = T(0);
      if (HAS_F) fv = f[o];
      const T val = site_update_warp<T, Ar, HAS_F, WEIGHTED>(act, src[o - 1], src[o + 1], src[o - sx], src[o + sx],
                                                            src[o - sy], src[o + sy], fv, WEIGHTED ? src[o] : T(0), c);
      if (act) dst[o] = val;
    }
    __syncthreads();
  }
}

struct TileGeom;
// host (gs.cu): the site table for tiles W x H x D and ns = 1..nt, cached in the context
int ensure_sites(stencil_ctx* ctx, const TileGeom& tg, cudaStream_t st);
SiteTable site_table(stencil_ctx* ctx, const TileGeom& tg);

}  // namespace stn
