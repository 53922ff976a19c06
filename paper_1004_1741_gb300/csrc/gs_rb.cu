// Red-black Gauss-Seidel (Sec. 3 names it as the common parallel alternative
// to the lexicographic sweep): first every site with (i+j+k) even, then every
// site with (i+j+k) odd, in place (0-based interior coordinates).  All updates
// of one colour read only the other colour, so each colour is one fully
// parallel launch and any order within it gives the same bits.
#include <cmath>
#include <type_traits>

#include "internal.h"

namespace stn {

constexpr int RB_BY = 8, RB_ZCHUNK = 16;

template <typename T, class Ar, bool HAS_F>
__global__ void __launch_bounds__(32 * RB_BY) gs_rb_kernel(T* u, const T* __restrict__ f, Geom g, Coef<T> c,
                                                           int colour) {
  const int xi = blockIdx.x * 32 + threadIdx.x;  // index among the row's sites of this colour
  const int y = blockIdx.y * RB_BY + threadIdx.y;
  if (y >= g.ny) return;
  const int z0 = blockIdx.z * RB_ZCHUNK, z1 = min(g.nz, z0 + RB_ZCHUNK);
  const int64_t sx = g.sx, sy = g.sy;
  for (int z = z0; z < z1; ++z) {
    // a warp is one row: every lane takes part in the adaptive arithmetic's vote; lanes past the row's
    // last site of this colour read the last site's neighbours and store nothing
    const int x = 2 * xi + ((y + z + colour) & 1);
    const bool act = x < g.nx;
    T* q = u + g.at(act ? x : g.nx - 1, y, z);
    T fv = T(0);
    if (HAS_F) fv = f[q - u];
    const T v = site_update_warp<T, Ar, HAS_F, false>(act, q[-1], q[1], q[-sx], q[sx], q[-sy], q[sy], fv, T(0), c);
    if (act) *q = v;
  }
}

template <typename T>
int gs_rb_run(stencil_ctx* ctx, T* u, const T* f, const Geom& g, double h, int nsweeps, const stencil_params* p,
              cudaStream_t st) {
  if (nsweeps == 0 || g.nx == 0 || g.ny == 0 || g.nz == 0) return STENCIL_OK;
  Coef<T> c;
  c.a = T(0);
  c.b = (T)((p && p->b != 0.0) ? p->b : 1.0 / 6.0);
  c.hh = (T)(h * h);
  // FP64: the adaptive arithmetic (per warp: three integer-pipe additions for non-negative neighbourhoods,
  // else the multiplication in integer arithmetic; the same bits)
  using Ar = typename std::conditional<sizeof(T) == 8, AdaptJacobi, typename DefaultArith<T>::type>::type;
  dim3 block(32, RB_BY);
  dim3 grid((g.nx / 2 + 1 + 31) / 32, (g.ny + RB_BY - 1) / RB_BY, (g.nz + RB_ZCHUNK - 1) / RB_ZCHUNK);
  for (int s = 0; s < nsweeps; ++s)
    for (int colour = 0; colour < 2; ++colour) {
      if (f)
        gs_rb_kernel<T, Ar, true><<<grid, block, 0, st>>>(u, f, g, c, colour);
      else
        gs_rb_kernel<T, Ar, false><<<grid, block, 0, st>>>(u, f, g, c, colour);
      ctx->launches++;
    }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(ctx, e, "gs_rb_kernel launch");
  return STENCIL_OK;
}

template int gs_rb_run<double>(stencil_ctx*, double*, const double*, const Geom&, double, int, const stencil_params*,
                               cudaStream_t);
template int gs_rb_run<float>(stencil_ctx*, float*, const float*, const Geom&, double, int, const stencil_params*,
                              cudaStream_t);

static int rb_checks(stencil_ctx* ctx, const void* u, const int64_t dims[3], double h, int nsweeps,
                     const stencil_params* p, Geom* g) {
  if (!ctx) return STENCIL_ERR_ARG;
  ctx->err.clear();
  int rc = check_dims(ctx, dims, g);
  if (rc) return rc;
  if (!u) return set_err(ctx, STENCIL_ERR_ARG, "u is NULL");
  if (nsweeps < 0) return set_err(ctx, STENCIL_ERR_ARG, "nsweeps < 0");
  if (!(h > 0.0) || !std::isfinite(h)) return set_err(ctx, STENCIL_ERR_ARG, "h must be finite and > 0");
  if (p && p->a != 0.0) return set_err(ctx, STENCIL_ERR_ARG, "a != 0 is only accepted by Jacobi");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  return STENCIL_OK;
}

}  // namespace stn

using namespace stn;

extern "C" {

int stencil_gs_rb(stencil_ctx* ctx, double* u, const double* f, const int64_t dims[3], double h, int nsweeps,
                  const stencil_params* params, void* stream) {
  Geom g;
  int rc = rb_checks(ctx, u, dims, h, nsweeps, params, &g);
  if (rc) return rc;
  return gs_rb_run<double>(ctx, u, f, g, h, nsweeps, params, (cudaStream_t)stream);
}

int stencil_gs_rb_f32(stencil_ctx* ctx, float* u, const float* f, const int64_t dims[3], double h, int nsweeps,
                      const stencil_params* params, void* stream) {
  Geom g;
  int rc = rb_checks(ctx, u, dims, h, nsweeps, params, &g);
  if (rc) return rc;
  return gs_rb_run<float>(ctx, u, f, g, h, nsweeps, params, (cudaStream_t)stream);
}

}  // extern "C"
