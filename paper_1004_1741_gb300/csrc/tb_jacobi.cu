// Temporally blocked Jacobi (Sec. 4): nt sweeps per pass over memory on the
// skewed-tile task schedule of tiles.h, without redundant computation.
//
// Two grids hold alternate time levels (level v in grid v % 2, as the paper's
// out-of-place Jacobi holds src and dst).  A task runs the ns sweeps of its
// pass one after the other on its tile, shifted back by one cell per sweep,
// reading level v and writing level v+1.  Because of the shift, a tile stops
// updating its last column before it would overwrite the level-v value the
// next tile still reads, so the two grids alone carry every value exchanged
// between tiles: they play the part of the paper's boundary array, and no
// site is computed twice.  Within a sweep all sites of the tile are
// independent; the tile is updated in place through the L1 cache, so the
// values of the nt sweeps stay on chip (L1/L2) between the pass's single read
// of level p*nt and its single write of level (p+1)*nt.
#include "internal.h"
#include "tiles.h"

namespace stn {

constexpr int TBJ_THREADS = 256;

template <typename T, class Ar, bool HAS_F, bool WEIGHTED, int W, int H, int D>
__global__ void __launch_bounds__(TBJ_THREADS) jacobi_task_kernel(T* g_even, T* g_odd, const T* __restrict__ f,
                                                                   Geom g, Coef<T> c,
                                                                   const uint64_t* __restrict__ slices,
                                                                   const int* __restrict__ slice_off, TileGeom tg,
                                                                   int level) {
  int I, J, K, p;
  if (!find_task(tg, slices, slice_off, level, &I, &J, &K, &p)) return;
  const int ns = min(tg.nt, tg.nsweeps - p * tg.nt);
  const int X0 = I * W, Y0 = J * H, Z0 = K * D;
  const bool full = (X0 - ns + 1 >= 0) && (Y0 - ns + 1 >= 0) && (Z0 - ns + 1 >= 0) && (X0 + W <= g.nx) &&
                    (Y0 + H <= g.ny) && (Z0 + D <= g.nz);
  const int64_t sx = g.sx, sy = g.sy;
  const int64_t base = g.at(X0, Y0, Z0);
  constexpr int NSITE = W * H * D;
  for (int s = 0; s < ns; ++s) {
    const int v = p * tg.nt + s;
    const T* src = (v & 1) ? g_odd : g_even;
    T* dst = (v & 1) ? g_even : g_odd;
    const int64_t sb = base - (int64_t)s * (sy + sx + 1);
#pragma unroll 2
    for (int q = threadIdx.x; q < NSITE; q += TBJ_THREADS) {
      const int ii = q % W, jj = (q / W) % H, kk = q / (W * H);
      if (!full) {
        const int x = X0 - s + ii, y = Y0 - s + jj, z = Z0 - s + kk;
        if (x < 0 || x >= g.nx || y < 0 || y >= g.ny || z < 0 || z >= g.nz) continue;
      }
      const int64_t o = sb + (int64_t)kk * sy + (int64_t)jj * sx + ii;
      T fv = T(0);
      if (HAS_F) fv = f[o];
      dst[o] = site_update<T, Ar, HAS_F, WEIGHTED>(src[o - 1], src[o + 1], src[o - sx], src[o + sx], src[o - sy],
                                                   src[o + sy], fv, WEIGHTED ? src[o] : T(0), c);
    }
    __syncthreads();
  }
}

template <typename T, class Ar, bool HAS_F, bool WEIGHTED, int W, int H, int D>
static int tbj_levels(stencil_ctx* ctx, T* g_even, T* g_odd, const T* f, const Geom& g, Coef<T> c,
                      const TileGeom& tg, cudaStream_t st) {
  auto kern = jacobi_task_kernel<T, Ar, HAS_F, WEIGHTED, W, H, D>;
  const uint64_t* slices = slices_ptr(ctx);
  const int* soff = slice_off_ptr(ctx);
  for (int L = 0; L < tg.nlevels; ++L) {
    int n = tasks_at_level(ctx, tg, L);
    if (n == 0) continue;
    kern<<<n, TBJ_THREADS, 0, st>>>(g_even, g_odd, f, g, c, slices, soff, tg, L);
    ctx->launches++;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(ctx, e, "jacobi_task_kernel launch");
  return STENCIL_OK;
}

template <typename T, int W, int H, int D>
static int tbj_dispatch(stencil_ctx* ctx, T* g_even, T* g_odd, const T* f, const Geom& g, Coef<T> c,
                        const TileGeom& tg, bool weighted, cudaStream_t st) {
  using Ar = typename DefaultArith<T>::type;
  if (f)
    return weighted ? tbj_levels<T, Ar, true, true, W, H, D>(ctx, g_even, g_odd, f, g, c, tg, st)
                    : tbj_levels<T, Ar, true, false, W, H, D>(ctx, g_even, g_odd, f, g, c, tg, st);
  return weighted ? tbj_levels<T, Ar, false, true, W, H, D>(ctx, g_even, g_odd, f, g, c, tg, st)
                  : tbj_levels<T, Ar, false, false, W, H, D>(ctx, g_even, g_odd, f, g, c, tg, st);
}

template <typename T>
int tb_jacobi_run(stencil_ctx* ctx, T* u, T* tmp, const T* f, const Geom& g, double h, int nsweeps,
                  const stencil_params* p, cudaStream_t st) {
  const int nt = p->nt;
  // default tile: 32x8x8, or 32x16x16 when the skew of nt-1 cells needs it
  const bool big = nt > 8;
  const int tx = p->tile_x ? p->tile_x : 32;
  const int ty = p->tile_y ? p->tile_y : (big ? 16 : 8);
  const int tz = p->tile_z ? p->tile_z : (big ? 16 : 8);
  if (nt > tx || nt > ty || nt > tz)
    return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "nt = %d needs every tile extent >= nt (tile %dx%dx%d)", nt, tx, ty,
                   tz);
  Coef<T> c;
  c.a = (T)p->a;
  c.b = (T)(p->b != 0.0 ? p->b : 1.0 / 6.0);
  c.hh = (T)(h * h);
  const bool weighted = p->a != 0.0;
  // level nsweeps must land in u: with an odd count, level 0 starts in the workspace
  const size_t bytes = (size_t)g.sy * (size_t)(g.nz + 2) * sizeof(T);
  cudaError_t e = cudaMemcpyAsync(tmp, u, bytes, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaMemcpyAsync(jacobi halo)");
  T* g_even = (nsweeps % 2) ? tmp : u;
  T* g_odd = (nsweeps % 2) ? u : tmp;
  int rc;
#define TBJ_TILE(WW, HH, DD)                                                              \
  if (tx == WW && ty == HH && tz == DD) {                                                 \
    TileGeom tg = make_tile_geom(g, WW, HH, DD, nt, nsweeps);                             \
    if ((rc = ensure_slices(ctx, tg, st)) != STENCIL_OK) return rc;                       \
    return tbj_dispatch<T, WW, HH, DD>(ctx, g_even, g_odd, f, g, c, tg, weighted, st);    \
  }
  TBJ_TILE(32, 8, 8)
  TBJ_TILE(32, 16, 8)
  TBJ_TILE(32, 16, 16)
  TBJ_TILE(16, 16, 16)
  TBJ_TILE(64, 8, 8)
#undef TBJ_TILE
  return set_err(ctx, STENCIL_ERR_UNSUPPORTED,
                 "temporal Jacobi tile %dx%dx%d (supported 32x8x8, 32x16x8, 32x16x16, 16^3, 64x8x8)", tx, ty, tz);
}

template int tb_jacobi_run<double>(stencil_ctx*, double*, double*, const double*, const Geom&, double, int,
                                   const stencil_params*, cudaStream_t);
template int tb_jacobi_run<float>(stencil_ctx*, float*, float*, const float*, const Geom&, double, int,
                                  const stencil_params*, cudaStream_t);

}  // namespace stn
