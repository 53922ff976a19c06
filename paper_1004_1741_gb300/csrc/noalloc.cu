// residual_norm_noalloc: the residual norm without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need the
// residual: code that owns every byte of the GPU through its own allocator,
// loops that must not stall on cudaMalloc or fragment the heap, or callers
// that are about to record the work into a CUDA graph.  For them this entry
// point takes its reduction scratch from a fixed array that is part of the
// library image on each device instead of from a context workspace.
//
// The scratch holds NA_MAX_BLOCKS partial-sum pairs (512 KiB) plus the two
// final sums.  Each call overwrites exactly the partials it later reads, so
// nothing has to be cleared between calls; calls that overlap on the GPU
// (different streams, or different host threads on one device) share the one
// array and race.
#include <mutex>

#include "internal.h"

namespace stn {

constexpr int NA_BX = 32, NA_BY = 8, NA_ZCHUNK = 32;
constexpr int64_t NA_MAX_BLOCKS = 32768;
constexpr int NA_MAX_DEVICES = 64;

// [0, 2*NA_MAX_BLOCKS): per-CTA partial sums (r^2, f^2); then the two totals.
static __device__ __align__(256) double na_scratch[2 * NA_MAX_BLOCKS + 2];

template <bool HAS_F, bool WANT_R>
__global__ void __launch_bounds__(NA_BX* NA_BY) na_residual_kernel(const double* __restrict__ u,
                                                                    const double* __restrict__ f, double* r_out,
                                                                    Geom g, double ih2, double* __restrict__ partials) {
  using Ar = ArithF64;
  const int x = blockIdx.x * NA_BX + threadIdx.x;
  const int y = blockIdx.y * NA_BY + threadIdx.y;
  const int z0 = blockIdx.z * NA_ZCHUNK;
  const int z1 = min(g.nz, z0 + NA_ZCHUNK);
  double rr = 0.0, ff = 0.0;
  if (x < g.nx && y < g.ny) {
    for (int z = z0; z < z1; ++z) {
      const int64_t c = g.at(x, y, z);
      double s = Ar::add(u[c - 1], u[c + 1]);
      s = Ar::add(s, u[c - g.sx]);
      s = Ar::add(s, u[c + g.sx]);
      s = Ar::add(s, u[c - g.sy]);
      s = Ar::add(s, u[c + g.sy]);
      const double au = __dmul_rn(__dsub_rn(__dmul_rn(6.0, u[c]), s), ih2);
      const double fv = HAS_F ? f[c] : 0.0;
      const double r = __dsub_rn(fv, au);
      if (WANT_R) r_out[c] = r;
      rr = __fma_rn(r, r, rr);
      if (HAS_F) ff = __fma_rn(fv, fv, ff);
    }
  }
  __shared__ double wr[NA_BY], wf[NA_BY];
  for (int o = 16; o > 0; o >>= 1) {
    rr = __dadd_rn(rr, __shfl_down_sync(0xffffffffu, rr, o));
    ff = __dadd_rn(ff, __shfl_down_sync(0xffffffffu, ff, o));
  }
  if (threadIdx.x == 0) {
    wr[threadIdx.y] = rr;
    wf[threadIdx.y] = ff;
  }
  __syncthreads();
  if (threadIdx.y == 0 && threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < NA_BY; ++w) {
      a = __dadd_rn(a, wr[w]);
      b = __dadd_rn(b, wf[w]);
    }
    const int64_t bid = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    partials[2 * bid] = a;
    partials[2 * bid + 1] = b;
  }
}

__global__ void __launch_bounds__(1024) na_reduce_kernel(const double* __restrict__ partials, int64_t n,
                                                         double* __restrict__ out) {
  __shared__ double sa[1024], sb[1024];
  double a = 0.0, b = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 1024) {
    a = __dadd_rn(a, partials[2 * i]);
    b = __dadd_rn(b, partials[2 * i + 1]);
  }
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int s = 512; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      sa[threadIdx.x] = __dadd_rn(sa[threadIdx.x], sa[threadIdx.x + s]);
      sb[threadIdx.x] = __dadd_rn(sb[threadIdx.x], sb[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sa[0];
    out[1] = sb[0];
  }
}

// Device address of na_scratch on each device, looked up once per device (with
// that device current) on the first call made there.
static double* na_addr[NA_MAX_DEVICES];
static std::mutex na_mu;

static int na_scratch_for_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_err(nullptr, STENCIL_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= NA_MAX_DEVICES)
    return set_err(nullptr, STENCIL_ERR_UNSUPPORTED, "device %d beyond the %d devices supported", dev, NA_MAX_DEVICES);
  std::lock_guard<std::mutex> lock(na_mu);
  if (!na_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, na_scratch);
    if (e != cudaSuccess || !p)
      return set_err(nullptr, STENCIL_ERR_CUDA, "cudaGetSymbolAddress(scratch) on device %d: %s", dev,
                     cudaGetErrorString(e));
    na_addr[dev] = (double*)p;
  }
  *out = na_addr[dev];
  return STENCIL_OK;
}

}  // namespace stn

using namespace stn;

extern "C" int residual_norm_noalloc(const double* u, const double* f, const int64_t dims[3], double h, double* r_out,
                                     double* out_abs, double* out_rel, void* stream) {
  Geom g;
  int rc = check_dims(nullptr, dims, &g);
  if (rc) return rc;
  if (!u) return set_err(nullptr, STENCIL_ERR_ARG, "u is NULL");
  if (!out_abs) return set_err(nullptr, STENCIL_ERR_ARG, "out_abs is NULL");
  if (!(h > 0.0) || !(h < 1e300)) return set_err(nullptr, STENCIL_ERR_ARG, "h must be finite and > 0");
  dim3 block(NA_BX, NA_BY);
  dim3 grid((g.nx + NA_BX - 1) / NA_BX, (g.ny + NA_BY - 1) / NA_BY, (g.nz + NA_ZCHUNK - 1) / NA_ZCHUNK);
  const int64_t nblk = (int64_t)grid.x * grid.y * grid.z;
  if (nblk > NA_MAX_BLOCKS)
    return set_err(nullptr, STENCIL_ERR_ARG,
                   "grid %lldx%lldx%lld needs %lld partial sums; the fixed scratch holds %lld "
                   "(ceil(nx/32)*ceil(ny/8)*ceil(nz/32) must be <= %lld)",
                   (long long)dims[0], (long long)dims[1], (long long)dims[2], (long long)nblk,
                   (long long)NA_MAX_BLOCKS, (long long)NA_MAX_BLOCKS);
  double* scratch = nullptr;
  if ((rc = na_scratch_for_current_device(&scratch))) return rc;
  double* totals = scratch + 2 * NA_MAX_BLOCKS;
  cudaStream_t st = (cudaStream_t)stream;
  const double ih2 = 1.0 / (h * h);
  if (nblk > 0) {
    if (f && r_out) na_residual_kernel<true, true><<<grid, block, 0, st>>>(u, f, r_out, g, ih2, scratch);
    else if (f) na_residual_kernel<true, false><<<grid, block, 0, st>>>(u, f, r_out, g, ih2, scratch);
    else if (r_out) na_residual_kernel<false, true><<<grid, block, 0, st>>>(u, f, r_out, g, ih2, scratch);
    else na_residual_kernel<false, false><<<grid, block, 0, st>>>(u, f, r_out, g, ih2, scratch);
  }
  na_reduce_kernel<<<1, 1024, 0, st>>>(scratch, nblk, totals);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_err(nullptr, STENCIL_ERR_CUDA, "residual_norm_noalloc launch: %s", cudaGetErrorString(e));
  double sums[2];
  e = cudaMemcpyAsync(sums, totals, sizeof(sums), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_err(nullptr, STENCIL_ERR_CUDA, "residual_norm_noalloc: %s", cudaGetErrorString(e));
  const double rn = sqrt(sums[0]), fn = sqrt(sums[1]);
  *out_abs = rn;
  if (out_rel) *out_rel = fn > 0.0 ? rn / fn : rn;
  return STENCIL_OK;
}
