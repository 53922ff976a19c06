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
#include "task_bodies.cuh"

namespace stn {

constexpr int TBJ_THREADS = GS_THREADS;

template <typename T, class Ar, bool HAS_F, bool WEIGHTED, int W, int H, int D>
__global__ void __launch_bounds__(TBJ_THREADS) jacobi_task_kernel(T* g_even, T* g_odd, const T* __restrict__ f,
                                                                   Geom g, Coef<T> c,
                                                                   const uint64_t* __restrict__ slices,
                                                                   const int* __restrict__ slice_off, TileGeom tg,
                                                                   int level) {
  int I, J, K, p;
  if (!find_task(tg, slices, slice_off, level, &I, &J, &K, &p)) return;
  jacobi_task_body<T, Ar, HAS_F, WEIGHTED, W, H, D>(g_even, g_odd, f, g, c, tg, I, J, K, p);
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

template <typename T, class Ar, int W, int H, int D>
static int tbj_arith(stencil_ctx* ctx, T* g_even, T* g_odd, const T* f, const Geom& g, Coef<T> c,
                     const TileGeom& tg, bool weighted, cudaStream_t st) {
  if (f)
    return weighted ? tbj_levels<T, Ar, true, true, W, H, D>(ctx, g_even, g_odd, f, g, c, tg, st)
                    : tbj_levels<T, Ar, true, false, W, H, D>(ctx, g_even, g_odd, f, g, c, tg, st);
  return weighted ? tbj_levels<T, Ar, false, true, W, H, D>(ctx, g_even, g_odd, f, g, c, tg, st)
                  : tbj_levels<T, Ar, false, false, W, H, D>(ctx, g_even, g_odd, f, g, c, tg, st);
}

// FP64: the z-march's integer-pipe forms -- the adaptive arithmetic by default (3 of 5 additions on the
// integer pipes for non-negative neighbourhoods, else the multiplication in integer arithmetic), int_adds 3
// the fixed 3-addition form; int_adds 0..2, 4, 5 every operation on the FP64 pipe.  Same bits either way.
template <typename T, int W, int H, int D>
static int tbj_dispatch(stencil_ctx* ctx, T* g_even, T* g_odd, const T* f, const Geom& g, Coef<T> c,
                        const TileGeom& tg, bool weighted, int int_adds, cudaStream_t st) {
  if constexpr (sizeof(T) == 8) {
    if (int_adds < 0 || int_adds == kIntAddsAdaptive)
      return tbj_arith<T, AdaptJacobi, W, H, D>(ctx, g_even, g_odd, f, g, c, tg, weighted, st);
    if (int_adds == 3)
      return tbj_arith<T, ArithF64Mix<0x12u>, W, H, D>(ctx, g_even, g_odd, f, g, c, tg, weighted, st);
  }
  return tbj_arith<T, typename DefaultArith<T>::type, W, H, D>(ctx, g_even, g_odd, f, g, c, tg, weighted, st);
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
  if (p->variant == 3) {
    if (weighted) return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "weighted Jacobi on the dataflow variant");
    T* const a[1] = {g_even};
    T* const b[1] = {g_odd};
    const T* const fs[1] = {f};
    const int ns[1] = {nsweeps};
    const double hs[1] = {h};
    return dataflow_run<T>(ctx, STENCIL_JACOBI, 1, a, b, fs, &g, ns, hs, tx, ty, tz, nt, ctx->df_timeout_ns,
                           ctx->df_poison, st);
  }
#define TBJ_TILE(WW, HH, DD)                                                              \
  if (tx == WW && ty == HH && tz == DD) {                                                 \
    TileGeom tg = make_tile_geom(g, WW, HH, DD, nt, nsweeps);                             \
    if ((rc = ensure_slices(ctx, tg, st)) != STENCIL_OK) return rc;                       \
    return tbj_dispatch<T, WW, HH, DD>(ctx, g_even, g_odd, f, g, c, tg, weighted, p->int_adds, st); \
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
