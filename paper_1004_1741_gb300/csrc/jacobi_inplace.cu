// Jacobi in place, without a second grid (stencil_params variant 6).
//
// The paper keeps a ring of a few new planes and writes each back once no
// sweep-old value of it is read any more (Sec. 4).  Here the ring holds
// z-slabs: slab s (S planes) is computed from u into ring buffer s % 3 by the
// z-march (zmarch.cuh) run on a sub-geometry whose pointers start at the
// slab; the same launch copies slab s-2 back from its buffer into u.  That is
// safe: slab s reads u's planes from the last plane of slab s-1 to the first
// of slab s+1, none of slab s-2; and slab s-1, the last reader of slab s-2's
// old values, ran before.  Three buffers keep the buffer a launch copies out
// apart from the one it fills.  After the last slab of a sweep the two slabs
// still in the ring are copied back by plain copy launches, so every sweep
// starts from a complete u.  Workspace: 3 S planes instead of a grid.
#include <algorithm>

#include "internal.h"
#include "zmarch.cuh"

namespace stn {

// u (interior) of planes [k0, k0+planes) <- a slab buffer (plane z of the slab at z * sy)
template <typename T>
__global__ void __launch_bounds__(256) slab_copy_back_kernel(T* __restrict__ u, const T* __restrict__ slab, Geom g,
                                                             int k0, int planes) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 8 + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int64_t o = (int64_t)(y + 1) * g.sx + (x + 1);
  for (int z = blockIdx.z; z < planes; z += gridDim.z) u[g.at(x, y, k0 + z)] = slab[(int64_t)z * g.sy + o];
}

// The march of one slab (sub-geometry gs, one z-chunk per CTA) into its buffer, and -- when cb is not
// null -- the copy-back of an earlier slab (planes [cb_k0, cb_k0 + cb_planes) of u) for this CTA's columns.
template <typename T, class Ar, bool HAS_F, bool WEIGHTED, int BY>
__global__ void __launch_bounds__(32 * BY) jacobi_slab_kernel(const T* __restrict__ src, T* __restrict__ dst,
                                                              const T* __restrict__ f, Geom gs, Coef<T> c,
                                                              T* __restrict__ u, const T* __restrict__ cb, int cb_k0,
                                                              int cb_planes) {
  __shared__ T sm[2][BY + 2][32 + 2];
  if (cb) {
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * BY + threadIdx.y;
    if (x < gs.nx && y < gs.ny) {
      const int64_t o = (int64_t)(y + 1) * gs.sx + (x + 1);
      for (int z = 0; z < cb_planes; ++z) u[gs.at(x, y, cb_k0 + z)] = cb[(int64_t)z * gs.sy + o];
    }
  }
  zmarch_body<T, Ar, HAS_F, WEIGHTED, BY>(src, dst, f, gs, 0, gs.nz, c, sm, blockIdx.x, blockIdx.y);
}

template <typename T, class Ar, int BY>
static cudaError_t slab_launch(const T* src, T* dst, const T* f, const Geom& gs, const Coef<T>& c, bool weighted,
                               T* u, const T* cb, int cb_k0, int cb_planes, cudaStream_t st) {
  const dim3 grid((gs.nx + 31) / 32, (gs.ny + BY - 1) / BY, 1), block(32, BY);
#define SLAB_GO(HF, WT) \
  jacobi_slab_kernel<T, Ar, HF, WT, BY><<<grid, block, 0, st>>>(src, dst, f, gs, c, u, cb, cb_k0, cb_planes)
  if (f) {
    if (weighted) SLAB_GO(true, true);
    else SLAB_GO(true, false);
  } else {
    if (weighted) SLAB_GO(false, true);
    else SLAB_GO(false, false);
  }
#undef SLAB_GO
  return cudaGetLastError();
}

template <typename T, class Ar>
static cudaError_t slab_by(int by, const T* src, T* dst, const T* f, const Geom& gs, const Coef<T>& c, bool weighted,
                           T* u, const T* cb, int cb_k0, int cb_planes, cudaStream_t st) {
  if (by == 4) return slab_launch<T, Ar, 4>(src, dst, f, gs, c, weighted, u, cb, cb_k0, cb_planes, st);
  return slab_launch<T, Ar, 8>(src, dst, f, gs, c, weighted, u, cb, cb_k0, cb_planes, st);
}

template <typename T>
static cudaError_t slab_step(int int_adds, int by, const T* src, T* dst, const T* f, const Geom& gs,
                             const Coef<T>& c, bool weighted, T* u, const T* cb, int cb_k0, int cb_planes,
                             cudaStream_t st) {
  if constexpr (sizeof(T) == 8) {
    switch (int_adds) {
      case 1: return slab_by<T, ArithF64Mix<0x1Du>>(by, src, dst, f, gs, c, weighted, u, cb, cb_k0, cb_planes, st);
      case 2: return slab_by<T, ArithF64Mix<0x15u>>(by, src, dst, f, gs, c, weighted, u, cb, cb_k0, cb_planes, st);
      case 3: return slab_by<T, ArithF64Mix<0x12u>>(by, src, dst, f, gs, c, weighted, u, cb, cb_k0, cb_planes, st);
      case 4: return slab_by<T, ArithF64Mix<0x10u>>(by, src, dst, f, gs, c, weighted, u, cb, cb_k0, cb_planes, st);
      case 5: return slab_by<T, ArithF64Mix<0x00u>>(by, src, dst, f, gs, c, weighted, u, cb, cb_k0, cb_planes, st);
      case kIntAddsAdaptive:
        return slab_by<T, AdaptJacobi>(by, src, dst, f, gs, c, weighted, u, cb, cb_k0, cb_planes, st);
      default: break;
    }
  }
  return slab_by<T, typename DefaultArith<T>::type>(by, src, dst, f, gs, c, weighted, u, cb, cb_k0, cb_planes, st);
}

template <typename T>
int jacobi_inplace_run(stencil_ctx* ctx, T* u, const T* f, const Geom& g, double h, int nsweeps,
                       const stencil_params* p, cudaStream_t st) {
  const int nt = (p && p->nt > 0) ? p->nt : 1;
  if (nt != 1) return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "in-place Jacobi runs nt = 1 only");
  const int S = std::min((p && p->tile_z > 0) ? p->tile_z : 32, g.nz);
  const int by = (p && p->tile_y) ? p->tile_y : (sizeof(T) == 8 ? 4 : 8);
  if (by != 4 && by != 8) return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "in-place Jacobi tile_y = %d (4 or 8)", by);
  if (p && p->tile_x && p->tile_x != 32)
    return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "Jacobi tile_x = %d (supported 32)", p->tile_x);
  const int int_adds = (p && p->int_adds >= 0) ? p->int_adds : kDefaultIntAddsJacobi;
  if (int_adds < 0 || int_adds > kIntAddsAdaptive)
    return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "int_adds = %d (supported 0..6)", int_adds);
  int status = STENCIL_OK;
  const size_t slab_elems = (size_t)S * (size_t)g.sy;
  T* ring = (T*)ws_get(ctx, SLOT_JACOBI_SLABS, 3 * slab_elems * sizeof(T), &status);
  if (!ring) return status;
  Coef<T> c;
  c.a = (T)(p ? p->a : 0.0);
  c.b = (T)((p && p->b != 0.0) ? p->b : 1.0 / 6.0);
  c.hh = (T)(h * h);
  const bool weighted = p && p->a != 0.0;
  const int nslab = (g.nz + S - 1) / S;
  auto buf = [&](int s) { return ring + (size_t)(s % 3) * slab_elems; };
  auto planes_of = [&](int s) { return std::min(S, g.nz - s * S); };
  const dim3 cgrid((g.nx + 31) / 32, (g.ny + 7) / 8, (unsigned)std::min(S, 64));
  for (int sw = 0; sw < nsweeps; ++sw) {
    for (int s = 0; s < nslab; ++s) {
      Geom gs = g;
      gs.nz = planes_of(s);
      // gs.at(x, y, z) = (z+1)*sy + ...: u and f from the slab's first plane, the buffer from its own
      const int64_t off = (int64_t)s * S * g.sy;
      const bool copy = s >= 2;
      cudaError_t e = slab_step<T>(int_adds, by, u + off, buf(s) - g.sy, f ? f + off : nullptr, gs, c, weighted, u,
                                   copy ? buf(s - 2) : nullptr, (s - 2) * S, copy ? planes_of(s - 2) : 0, st);
      ctx->launches++;
      if (e != cudaSuccess) return cuda_err(ctx, e, "jacobi_slab_kernel launch");
    }
    for (int s = std::max(0, nslab - 2); s < nslab; ++s) {  // the slabs still in the ring
      slab_copy_back_kernel<T><<<cgrid, dim3(32, 8), 0, st>>>(u, buf(s), g, s * S, planes_of(s));
      ctx->launches++;
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_err(ctx, e, "slab copy-back");
    }
  }
  return STENCIL_OK;
}

template int jacobi_inplace_run<double>(stencil_ctx*, double*, const double*, const Geom&, double, int,
                                        const stencil_params*, cudaStream_t);
template int jacobi_inplace_run<float>(stencil_ctx*, float*, const float*, const Geom&, double, int,
                                       const stencil_params*, cudaStream_t);

}  // namespace stn
