// residual_norm_noalloc: the residual norm without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need the
// residual: code that owns every byte of the GPU through its own allocator,
// loops that must not stall on cudaMalloc or fragment the heap, or callers
// that are about to record the work into a CUDA graph.  For them this entry
// point takes its reduction scratch from a fixed array that is part of the
// library image on each device instead of from a context workspace.
//
// The kernels are residual_norm's own (residual_kernels.cuh), launched with
// the same shape, so both entry points give the same bits.  The scratch holds
// NA_MAX_BLOCKS partial-sum pairs (512 KiB) plus the two final sums.  Each
// call overwrites exactly the partials it later reads, so nothing has to be
// cleared between calls; calls that overlap on the GPU (different streams, or
// different host threads on one device) share the one array and race.
#include <cmath>

#include "internal.h"
#include "residual_kernels.cuh"

namespace stn {

constexpr int64_t NA_MAX_BLOCKS = 32768;

// [0, 2*NA_MAX_BLOCKS): per-CTA partial sums (r^2, f^2); then the two totals.
static __device__ __align__(256) double na_scratch[2 * NA_MAX_BLOCKS + 2];

// The device address of na_scratch in the calling thread's current context.
// The symbol's address belongs to a context, so it is looked up on every call
// (a cheap lookup) instead of being cached.
static int na_scratch_address(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, na_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return set_err(nullptr, STENCIL_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
  }
  *out = (double*)p;
  return STENCIL_OK;
}

// STENCIL_OK if p is device (or managed) memory that the current device can
// address as its own; a host pointer or another device's memory is rejected
// before any kernel is launched.
static int na_check_on_device(const void* p, int dev, const char* name) {
  if (!p) return STENCIL_OK;
  cudaPointerAttributes a{};
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(nullptr, STENCIL_ERR_ARG, "%s is not a CUDA pointer (%s)", name, cudaGetErrorString(e));
  }
  if (a.type == cudaMemoryTypeManaged) return STENCIL_OK;
  if (a.type != cudaMemoryTypeDevice)
    return set_err(nullptr, STENCIL_ERR_ARG, "%s is not device memory (pointer type %d)", name, (int)a.type);
  if (a.device != dev)
    return set_err(nullptr, STENCIL_ERR_ARG, "%s lives on device %d, the current device is %d", name, a.device, dev);
  return STENCIL_OK;
}

}  // namespace stn

using namespace stn;

extern "C" int residual_norm_noalloc(const double* u, const double* f, const int64_t dims[3], double h, double* r_out,
                                     double* out_abs, double* out_rel, void* stream) {
  set_err(nullptr, STENCIL_OK, "");  // no stale message from an earlier call
  Geom g;
  int rc = check_dims(nullptr, dims, &g);
  if (rc) return rc;
  if (!u) return set_err(nullptr, STENCIL_ERR_ARG, "u is NULL");
  if (!out_abs) return set_err(nullptr, STENCIL_ERR_ARG, "out_abs is NULL");
  if (!(h > 0.0) || !std::isfinite(h)) return set_err(nullptr, STENCIL_ERR_ARG, "h must be finite and > 0");
  const dim3 block(RES_BX, RES_BY);
  const dim3 grid = residual_grid(g);
  const int64_t nblk = (int64_t)grid.x * grid.y * grid.z;
  if (nblk > NA_MAX_BLOCKS)
    return set_err(nullptr, STENCIL_ERR_ARG,
                   "grid %lldx%lldx%lld needs %lld partial sums; the fixed scratch holds %lld "
                   "(ceil(nx/32)*ceil(ny/8)*ceil(nz/32) must be <= %lld)",
                   (long long)dims[0], (long long)dims[1], (long long)dims[2], (long long)nblk,
                   (long long)NA_MAX_BLOCKS, (long long)NA_MAX_BLOCKS);
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_err(nullptr, STENCIL_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if ((rc = na_check_on_device(u, dev, "u")) || (rc = na_check_on_device(f, dev, "f")) ||
      (rc = na_check_on_device(r_out, dev, "r_out")))
    return rc;
  double* scratch = nullptr;
  if ((rc = na_scratch_address(&scratch))) return rc;
  double* totals = scratch + 2 * NA_MAX_BLOCKS;
  cudaStream_t st = (cudaStream_t)stream;
  const double ih2 = 1.0 / (h * h);
  if (nblk > 0) {
    if (f && r_out) residual_kernel<true, true, false, true><<<grid, block, 0, st>>>(u, f, r_out, nullptr, g, ih2, scratch);
    else if (f) residual_kernel<true, false, false, true><<<grid, block, 0, st>>>(u, f, r_out, nullptr, g, ih2, scratch);
    else if (r_out) residual_kernel<false, true, false, true><<<grid, block, 0, st>>>(u, f, r_out, nullptr, g, ih2, scratch);
    else residual_kernel<false, false, false, true><<<grid, block, 0, st>>>(u, f, r_out, nullptr, g, ih2, scratch);
  }
  reduce_pairs_kernel<1024><<<1, 1024, 0, st>>>(scratch, nblk, totals);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_err(nullptr, STENCIL_ERR_CUDA, "residual_norm_noalloc launch: %s", cudaGetErrorString(e));
  double sums[2];
  e = cudaMemcpyAsync(sums, totals, sizeof(sums), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_err(nullptr, STENCIL_ERR_CUDA, "residual_norm_noalloc: %s", cudaGetErrorString(e));
  const double rn = std::sqrt(sums[0]), fn = std::sqrt(sums[1]);
  *out_abs = rn;
  if (out_rel) *out_rel = fn > 0.0 ? rn / fn : rn;
  return STENCIL_OK;
}
