// Batched Jacobi, one sweep per pass: one launch per sweep over the tile
// columns of every grid of the batch that still has sweeps to do.
//
// An out-of-place Jacobi sweep has no dependencies inside itself, so every
// (grid, tile column, z-chunk) of a sweep can run in the same launch: the
// CTAs of all grids are numbered one after the other, a CTA finds its grid
// by binary search over the grids' first CTA indices and runs the z-march of
// zmarch.cuh on its tile.  Each grid alternates between its own array and a
// workspace copy (which carries the same halo) so that the last of its
// nsweeps sweeps lands in its own array, as in the single-grid call.
#include <algorithm>
#include <vector>

#include "internal.h"
#include "zmarch.cuh"

namespace stn {

template <typename T>
struct BJGrid {
  const T* src;
  T* dst;
  const T* f;
  Geom g;
  Coef<T> c;
  int tiles_x, tiles_y, zchunk;
  long long cta0;  // first CTA of this grid in the launch
};

template <typename T, class Ar, int BY>
__global__ void __launch_bounds__(32 * BY) batched_jacobi_kernel(const BJGrid<T>* __restrict__ grids, int n) {
  __shared__ T sm[2][BY + 2][32 + 2];
  __shared__ int s_gi;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    int lo = 0, hi = n - 1;  // last grid whose first CTA is <= blockIdx.x
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (grids[mid].cta0 <= (long long)blockIdx.x) lo = mid;
      else hi = mid - 1;
    }
    s_gi = lo;
  }
  __syncthreads();
  const BJGrid<T> d = grids[s_gi];
  const long long local = (long long)blockIdx.x - d.cta0;
  const int bx = (int)(local % d.tiles_x);
  const long long rest = local / d.tiles_x;
  const int by = (int)(rest % d.tiles_y);
  const int bz = (int)(rest / d.tiles_y);
  const int z0 = bz * d.zchunk, z1 = min(d.g.nz, z0 + d.zchunk);
  if (z0 >= z1) return;  // uniform over the CTA
  if (d.f)
    zmarch_body<T, Ar, true, false, BY>(d.src, d.dst, d.f, d.g, z0, z1, d.c, sm, bx, by);
  else
    zmarch_body<T, Ar, false, false, BY>(d.src, d.dst, nullptr, d.g, z0, z1, d.c, sm, bx, by);
}

template <typename T, class Ar>
static cudaError_t bj_launch(int by, const BJGrid<T>* grids, int n, long long ctas, cudaStream_t st) {
  if (by == 4) batched_jacobi_kernel<T, Ar, 4><<<(unsigned)ctas, dim3(32, 4), 0, st>>>(grids, n);
  else batched_jacobi_kernel<T, Ar, 8><<<(unsigned)ctas, dim3(32, 8), 0, st>>>(grids, n);
  return cudaGetLastError();
}

// pre: the grids' f arrays hold hh*f already (ArithPreF)
template <typename T, template <class> class W>
static cudaError_t bj_dispatch_w(int int_adds, int by, const BJGrid<T>* grids, int n, long long ctas,
                                 cudaStream_t st) {
  if constexpr (sizeof(T) == 8) {
    switch (int_adds) {
      case 1: return bj_launch<T, W<ArithF64Mix<0x1Du>>>(by, grids, n, ctas, st);
      case 2: return bj_launch<T, W<ArithF64Mix<0x15u>>>(by, grids, n, ctas, st);
      case 3: return bj_launch<T, W<ArithF64Mix<0x12u>>>(by, grids, n, ctas, st);
      case 4: return bj_launch<T, W<ArithF64Mix<0x10u>>>(by, grids, n, ctas, st);
      case 5: return bj_launch<T, W<ArithF64Mix<0x00u>>>(by, grids, n, ctas, st);
      case kIntAddsAdaptive:
        return bj_launch<T, ArithAdaptive<W<ArithF64Mix<0x12u>>, W<ArithF64Mix<0x1Fu, true>>>>(by, grids, n, ctas, st);
      default: break;
    }
  }
  return bj_launch<T, W<typename DefaultArith<T>::type>>(by, grids, n, ctas, st);
}

template <class A>
using Plain = A;

template <typename T>
static cudaError_t bj_dispatch(bool pre, int int_adds, int by, const BJGrid<T>* grids, int n, long long ctas,
                               cudaStream_t st) {
  if constexpr (sizeof(T) == 8) {
    if (pre) return bj_dispatch_w<T, ArithPreF>(int_adds, by, grids, n, ctas, st);
  }
  return bj_dispatch_w<T, Plain>(int_adds, by, grids, n, ctas, st);
}

template <typename T>
int batched_jacobi_zmarch(stencil_ctx* ctx, int n, T* const* u, const T* const* f, const Geom* geoms,
                          const double* h, const int* nsweeps, double bco, int int_adds, int by, int zchunk,
                          cudaStream_t st) {
  if (int_adds < 0 || int_adds > kIntAddsAdaptive)
    return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "int_adds = %d (supported 0..6)", int_adds);
  if (by == 0) by = sizeof(T) == 8 ? 4 : 8;
  if (by != 4 && by != 8) return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "batched Jacobi tile_y = %d (4 or 8)", by);
  if (zchunk < 0) return set_err(ctx, STENCIL_ERR_ARG, "tile_z < 0");
  // second arrays: one workspace copy per grid, carrying its halo
  size_t total = 0;
  for (int i = 0; i < n; ++i) total += (size_t)geoms[i].sy * (size_t)(geoms[i].nz + 2);
  int status;
  T* tmp = (T*)ws_get(ctx, SLOT_BATCH_TMP, total * sizeof(T), &status);
  if (!tmp) return status;
  std::vector<T*> first((size_t)n), second((size_t)n);
  int max_ns = 0;
  size_t off = 0;
  for (int i = 0; i < n; ++i) {
    const size_t cnt = (size_t)geoms[i].sy * (size_t)(geoms[i].nz + 2);
    T* ti = tmp + off;
    off += cnt;
    max_ns = std::max(max_ns, nsweeps[i]);
    if (nsweeps[i] == 0 || geoms[i].nx == 0 || geoms[i].ny == 0 || geoms[i].nz == 0) continue;
    cudaError_t e = cudaMemcpyAsync(ti, u[i], cnt * sizeof(T), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_err(ctx, e, "batched halo copy");
    const bool odd = nsweeps[i] % 2;  // the last sweep must land in u[i]
    first[(size_t)i] = odd ? ti : u[i];
    second[(size_t)i] = odd ? u[i] : ti;
  }
  // FP64 with f over several sweeps: hh*f once per grid into workspace laid out like the second grids
  // (one FP64 multiplication per site and sweep fewer); skipped when the budget has no room for it
  std::vector<const T*> fuse((size_t)n);
  for (int i = 0; i < n; ++i) fuse[(size_t)i] = f ? f[i] : nullptr;
  bool pre = false;
  if constexpr (sizeof(T) == 8) {
    bool want = false;
    for (int i = 0; i < n; ++i) want = want || (f && f[i] && nsweeps[i] >= 2);
    double* w = want ? (double*)ws_try(ctx, SLOT_F_SCALED, total * sizeof(double)) : nullptr;
    if (w) {
      pre = true;
      size_t o = 0;
      for (int i = 0; i < n; ++i) {
        const size_t cnt = (size_t)geoms[i].sy * (size_t)(geoms[i].nz + 2);
        if (f && f[i] && nsweeps[i] > 0) {
          cudaError_t e = prescale_f(f[i], w + o, cnt, h[i] * h[i], ctx->sm_count, st);
          ctx->launches++;
          if (e != cudaSuccess) return cuda_err(ctx, e, "prescale_f launch");
          fuse[(size_t)i] = w + o;
        }
        o += cnt;
      }
    }
  }
  // descriptors of every sweep's launch, uploaded once
  std::vector<BJGrid<T>> desc;
  std::vector<size_t> start((size_t)max_ns + 1, 0);
  std::vector<long long> ctas((size_t)max_ns, 0);
  for (int s = 0; s < max_ns; ++s) {
    start[(size_t)s] = desc.size();
    long long cta = 0;
    for (int i = 0; i < n; ++i) {
      const Geom& g = geoms[i];
      if (s >= nsweeps[i] || g.nx == 0 || g.ny == 0 || g.nz == 0) continue;
      BJGrid<T> d;
      d.src = (s % 2 == 0) ? first[(size_t)i] : second[(size_t)i];
      d.dst = (s % 2 == 0) ? second[(size_t)i] : first[(size_t)i];
      d.f = fuse[(size_t)i];
      d.g = g;
      d.c.a = T(0);
      d.c.b = (T)bco;
      d.c.hh = (T)(h[i] * h[i]);
      d.tiles_x = (g.nx + 31) / 32;
      d.tiles_y = (g.ny + by - 1) / by;
      d.zchunk = zchunk ? std::min(zchunk, g.nz) : (g.nz <= 256 ? g.nz : 128);  // default: whole columns
      d.cta0 = cta;
      cta += (long long)d.tiles_x * d.tiles_y * ((g.nz + d.zchunk - 1) / d.zchunk);
      desc.push_back(d);
    }
    ctas[(size_t)s] = cta;
  }
  start[(size_t)max_ns] = desc.size();
  if (desc.empty()) return STENCIL_OK;
  BJGrid<T>* ddesc = (BJGrid<T>*)ws_get(ctx, SLOT_BATCH_DESC, desc.size() * sizeof(BJGrid<T>), &status);
  if (!ddesc) return status;
  cudaError_t e = cudaMemcpyAsync(ddesc, desc.data(), desc.size() * sizeof(BJGrid<T>), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // `desc` goes out of scope
  if (e != cudaSuccess) return cuda_err(ctx, e, "batched descriptors");
  for (int s = 0; s < max_ns; ++s) {
    const int cnt = (int)(start[(size_t)s + 1] - start[(size_t)s]);
    if (cnt == 0 || ctas[(size_t)s] == 0) continue;
    if (ctas[(size_t)s] > 0x7FFFFFFFLL) return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "batch too large for one launch");
    e = bj_dispatch<T>(pre, int_adds, by, ddesc + start[(size_t)s], cnt, ctas[(size_t)s], st);
    ctx->launches++;
    if (e != cudaSuccess) return cuda_err(ctx, e, "batched_jacobi_kernel launch");
  }
  e = cudaStreamSynchronize(st);  // blocking, like the persistent batched launch
  return e == cudaSuccess ? STENCIL_OK : cuda_err(ctx, e, "batched Jacobi");
}

template int batched_jacobi_zmarch<double>(stencil_ctx*, int, double* const*, const double* const*, const Geom*,
                                           const double*, const int*, double, int, int, int, cudaStream_t);
template int batched_jacobi_zmarch<float>(stencil_ctx*, int, float* const*, const float* const*, const Geom*,
                                          const double*, const int*, double, int, int, int, cudaStream_t);

}  // namespace stn
