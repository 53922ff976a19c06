// Jacobi smoother (Sec. 3, first listing): one sweep per pass over memory.
//
// Kernel: a 2.5D z-march.  A CTA of 32 x BY threads owns a 32 x BY tile of
// (x, y) columns and a chunk of z-planes.  Each thread keeps its own column's
// planes k-1, k, k+1 in registers (the paper's "three planes in cache" of
// Fig. stencil_mapping, here in the register file), the current plane is
// staged in shared memory (double-buffered, one __syncthreads per plane) for
// the four in-plane neighbours, and halo columns/rows of the tile are loaded
// by the edge threads.  Every lane of every warp produces an output site, so
// the FP64 pipe executes exactly the 6 (Laplace) or 8 (Poisson) operations
// of a site update per lattice update and nothing else.
//
// Temporal blocking (nt > 1 sweeps per pass) is implemented by the
// skewed-tile task scheduler in tb_jacobi.cu and, for FP32, on chip in
// tb_zmarch.cu; the in-place form without a second grid (variant 6) runs the
// same z-march slab by slab.
#include <algorithm>

#include "internal.h"
#include "zmarch.cuh"

namespace stn {

template <typename T, class Ar, bool HAS_F, bool WEIGHTED, int BY>
__global__ void __launch_bounds__(32 * BY) jacobi_zmarch_kernel(const T* __restrict__ src, T* __restrict__ dst,
                                                                const T* __restrict__ f, Geom g, int zchunk,
                                                                Coef<T> c) {
  __shared__ T sm[2][BY + 2][32 + 2];
  const int z0 = blockIdx.z * zchunk;
  const int z1 = min(g.nz, z0 + zchunk);
  if (z0 >= z1) return;  // uniform over the block
  zmarch_body<T, Ar, HAS_F, WEIGHTED, BY>(src, dst, f, g, z0, z1, c, sm, blockIdx.x, blockIdx.y);
}

// Pipelined variant: the same 2.5D z-march, but planes arrive in shared
// memory through asynchronous copies (cp.async) issued PF = S-4 planes ahead
// into a ring of S plane buffers, so each CTA keeps several planes of loads
// in flight.  Bandwidth-bound FP32 sweeps need that memory-level parallelism;
// the FP64 sweep is FP64-pipe-bound either way.  One barrier per plane: the
// buffer a new copy fills was last read two iterations earlier.

template <typename T, class Ar, bool HAS_F, bool WEIGHTED, int BY, int S>
__global__ void __launch_bounds__(32 * BY) jacobi_pipe_kernel(const T* __restrict__ src, T* __restrict__ dst,
                                                              const T* __restrict__ f, Geom g, int zchunk, Coef<T> c) {
  constexpr int PF = S - 4;
  static_assert(PF >= 1, "ring too small");
  __shared__ T ring[S][BY + 2][32 + 2];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x = blockIdx.x * 32 + tx;
  const int y = blockIdx.y * BY + ty;
  const int z0 = blockIdx.z * zchunk;
  const int z1 = min(g.nz, z0 + zchunk);
  if (z0 >= z1) return;
  const bool inside = (x <= g.nx) && (y <= g.ny);
  const bool active = (x < g.nx) && (y < g.ny);
  const bool hw = (tx == 0) && (y <= g.ny);
  const bool he = (tx == 31) && (x + 1 <= g.nx) && (y <= g.ny);
  const bool hs = (ty == 0) && (x <= g.nx);
  const bool hn = (ty == BY - 1) && (y + 1 <= g.ny) && (x <= g.nx);
  const int64_t sy = g.sy;
  const int64_t col = inside ? g.at(x, y, -1) : 0;
  const int64_t colw = hw ? g.at(x - 1, y, -1) : 0;
  const int64_t cole = he ? g.at(x + 1, y, -1) : 0;
  const int64_t cols = hs ? g.at(x, y - 1, -1) : 0;
  const int64_t coln = hn ? g.at(x, y + 1, -1) : 0;
  // plane q (interior index, -1..nz) lives in ring[(q - z0 + 1) % S]
  auto issue = [&](int q) {
    if (q <= z1) {
      const int sl = (q - z0 + 1) % S;
      const int64_t pz = (int64_t)(q + 1) * sy;
      if (inside) cp_async_elem(&ring[sl][ty + 1][tx + 1], src + col + pz);
      if (hw) cp_async_elem(&ring[sl][ty + 1][0], src + colw + pz);
      if (he) cp_async_elem(&ring[sl][ty + 1][33], src + cole + pz);
      if (hs) cp_async_elem(&ring[sl][0][tx + 1], src + cols + pz);
      if (hn) cp_async_elem(&ring[sl][BY + 1][tx + 1], src + coln + pz);
    }
    cp_async_commit();
  };
  for (int q = z0 - 1; q <= z0 + PF; ++q) issue(q);
  for (int z = z0; z < z1; ++z) {
    issue(z + 1 + PF);
    cp_async_wait<PF>();
    __syncthreads();
    if (active) {
      const int sb = (z - z0) % S, sc = (z - z0 + 1) % S, st = (z - z0 + 2) % S;
      T fv = T(0);
      if (HAS_F) fv = f[col + (int64_t)(z + 1) * sy];
      const T v = site_update<T, Ar, HAS_F, WEIGHTED>(ring[sc][ty + 1][tx], ring[sc][ty + 1][tx + 2],
                                                      ring[sc][ty][tx + 1], ring[sc][ty + 2][tx + 1],
                                                      ring[sb][ty + 1][tx + 1], ring[st][ty + 1][tx + 1], fv,
                                                      ring[sc][ty + 1][tx + 1], c);
      dst[col + (int64_t)(z + 1) * sy] = v;
    }
  }
  cp_async_wait<0>();
}

template <typename T>
struct JacobiLaunch {
  template <class Ar, bool HAS_F, bool WEIGHTED, int BY>
  static cudaError_t go(const T* src, T* dst, const T* f, const Geom& g, int zchunk, Coef<T> c, bool pipe,
                        cudaStream_t st) {
    dim3 block(32, BY);
    dim3 grid((g.nx + 31) / 32, (g.ny + BY - 1) / BY, (g.nz + zchunk - 1) / zchunk);
    if constexpr (!AdaptOf<Ar>::on) {  // the copy-ahead variant has no adaptive form (it runs Pos)
      if (pipe) {
        jacobi_pipe_kernel<T, Ar, HAS_F, WEIGHTED, BY, 8><<<grid, block, 0, st>>>(src, dst, f, g, zchunk, c);
        return cudaGetLastError();
      }
    } else if (pipe) {
      jacobi_pipe_kernel<T, typename Ar::Pos, HAS_F, WEIGHTED, BY, 8><<<grid, block, 0, st>>>(src, dst, f, g, zchunk,
                                                                                               c);
      return cudaGetLastError();
    }
    jacobi_zmarch_kernel<T, Ar, HAS_F, WEIGHTED, BY><<<grid, block, 0, st>>>(src, dst, f, g, zchunk, c);
    return cudaGetLastError();
  }
  template <class Ar, int BY>
  static cudaError_t pick(const T* src, T* dst, const T* f, const Geom& g, int zchunk, Coef<T> c, bool weighted,
                          bool pipe, cudaStream_t st) {
    if (f) {
      return weighted ? go<Ar, true, true, BY>(src, dst, f, g, zchunk, c, pipe, st)
                      : go<Ar, true, false, BY>(src, dst, f, g, zchunk, c, pipe, st);
    }
    return weighted ? go<Ar, false, true, BY>(src, dst, f, g, zchunk, c, pipe, st)
                    : go<Ar, false, false, BY>(src, dst, f, g, zchunk, c, pipe, st);
  }
};

// One sweep src -> dst (both hold the same Dirichlet halo).
template <typename T, class Ar>
static cudaError_t jacobi_sweep_ar(const T* src, T* dst, const T* f, const Geom& g, int by, int zchunk, Coef<T> c,
                                   bool weighted, bool pipe, cudaStream_t st) {
  switch (by) {
    case 4: return JacobiLaunch<T>::template pick<Ar, 4>(src, dst, f, g, zchunk, c, weighted, pipe, st);
    case 16: return JacobiLaunch<T>::template pick<Ar, 16>(src, dst, f, g, zchunk, c, weighted, pipe, st);
    default: return JacobiLaunch<T>::template pick<Ar, 8>(src, dst, f, g, zchunk, c, weighted, pipe, st);
  }
}

// int_adds: additions of the neighbour sum done on the integer pipes (FP64 only; 0, 3, 4 or 5).
template <typename T>
cudaError_t jacobi_sweep(const T* src, T* dst, const T* f, const Geom& g, int by, int zchunk, Coef<T> c,
                         bool weighted, bool pipe, int int_adds, cudaStream_t st) {
  if constexpr (sizeof(T) == 8) {
    switch (int_adds) {
      case 1: return jacobi_sweep_ar<T, ArithF64Mix<0x1Du>>(src, dst, f, g, by, zchunk, c, weighted, pipe, st);
      case 2: return jacobi_sweep_ar<T, ArithF64Mix<0x15u>>(src, dst, f, g, by, zchunk, c, weighted, pipe, st);
      case 3: return jacobi_sweep_ar<T, ArithF64Mix<0x12u>>(src, dst, f, g, by, zchunk, c, weighted, pipe, st);
      case 4: return jacobi_sweep_ar<T, ArithF64Mix<0x10u>>(src, dst, f, g, by, zchunk, c, weighted, pipe, st);
      case 5: return jacobi_sweep_ar<T, ArithF64Mix<0x00u>>(src, dst, f, g, by, zchunk, c, weighted, pipe, st);
      case kIntAddsAdaptive: return jacobi_sweep_ar<T, AdaptJacobi>(src, dst, f, g, by, zchunk, c, weighted, pipe, st);
      default: break;
    }
  }
  return jacobi_sweep_ar<T, typename DefaultArith<T>::type>(src, dst, f, g, by, zchunk, c, weighted, pipe, st);
}

__global__ void __launch_bounds__(256) prescale_f_kernel(const double* __restrict__ f, double* __restrict__ g,
                                                         double hh, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    g[i] = ArithF64Fma::mul(hh, f[i]);
}

cudaError_t prescale_f(const double* f, double* g, size_t n, double hh, int sm_count, cudaStream_t st) {
  const size_t want = (n + 255) / 256;
  const unsigned blocks = (unsigned)std::max<size_t>(1, std::min<size_t>(want, (size_t)sm_count * 8));
  prescale_f_kernel<<<blocks, 256, 0, st>>>(f, g, hh, n);
  return cudaGetLastError();
}

// One unweighted FP64 z-march sweep whose f holds hh*f already (tile height 4 or 8); Ar is an ArithPreF
// arithmetic (or an ArithAdaptive of two).
template <class Ar>
static cudaError_t jacobi_sweep_pre_ar(const double* src, double* dst, const double* gf, const Geom& g, int by,
                                       int zchunk, Coef<double> c, cudaStream_t st) {
  dim3 grid((g.nx + 31) / 32, (g.ny + by - 1) / by, (g.nz + zchunk - 1) / zchunk);
  if (by == 4)
    jacobi_zmarch_kernel<double, Ar, true, false, 4><<<grid, dim3(32, 4), 0, st>>>(src, dst, gf, g, zchunk, c);
  else
    jacobi_zmarch_kernel<double, Ar, true, false, 8><<<grid, dim3(32, 8), 0, st>>>(src, dst, gf, g, zchunk, c);
  return cudaGetLastError();
}

static cudaError_t jacobi_sweep_pre(const double* src, double* dst, const double* gf, const Geom& g, int by,
                                    int zchunk, Coef<double> c, int int_adds, cudaStream_t st) {
  switch (int_adds) {
    case 1: return jacobi_sweep_pre_ar<ArithPreF<ArithF64Mix<0x1Du>>>(src, dst, gf, g, by, zchunk, c, st);
    case 2: return jacobi_sweep_pre_ar<ArithPreF<ArithF64Mix<0x15u>>>(src, dst, gf, g, by, zchunk, c, st);
    case 3: return jacobi_sweep_pre_ar<ArithPreF<ArithF64Mix<0x12u>>>(src, dst, gf, g, by, zchunk, c, st);
    case 4: return jacobi_sweep_pre_ar<ArithPreF<ArithF64Mix<0x10u>>>(src, dst, gf, g, by, zchunk, c, st);
    case 5: return jacobi_sweep_pre_ar<ArithPreF<ArithF64Mix<0x00u>>>(src, dst, gf, g, by, zchunk, c, st);
    case kIntAddsAdaptive: return jacobi_sweep_pre_ar<AdaptJacobiPre>(src, dst, gf, g, by, zchunk, c, st);
    default: return jacobi_sweep_pre_ar<ArithPreF<ArithF64Fma>>(src, dst, gf, g, by, zchunk, c, st);
  }
}

template <typename T>
int tb_jacobi_run(stencil_ctx* ctx, T* u, T* tmp, const T* f, const Geom& g, double h, int nsweeps,
                  const stencil_params* p, cudaStream_t st);
cudaError_t jacobi_tbz_pass(const float* src, float* dst, const float* f, const Geom& g, int levels, int by,
                            int zchunk, Coef<float> c, cudaStream_t st);

// FP32 temporal blocking on chip (tb_zmarch.cu): passes of up to nt <= 4 sweeps.
template <typename T>
static int tbz_run(stencil_ctx* ctx, T* u, T* tmp, const T* f, const Geom& g, double h, int nsweeps, int nt,
                   const stencil_params* p, cudaStream_t st) {
  if (sizeof(T) != 4) return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "on-chip temporal blocking is FP32 only");
  const int by = (p && p->tile_y) ? p->tile_y : 32;
  if (by != 16 && by != 32) return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "tile_y = %d (16 or 32)", by);
  if (nt > 4) return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "on-chip temporal blocking: nt = %d > 4", nt);
  int zchunk = (p && p->tile_z) ? p->tile_z : 0;
  if (zchunk <= 0) {
    const long long cols = (long long)((g.nx + 63 - 2 * nt) / (64 - 2 * nt)) * ((g.ny + by - 1 - 2 * nt) / (by - 2 * nt));
    const long long want = (long long)ctx->sm_count * 4;
    const long long chunks = (want + cols - 1) / cols;
    zchunk = (int)((g.nz + chunks - 1) / chunks);
    if (zchunk < 32) zchunk = 32;
  }
  Coef<float> c;
  c.a = 0.f;
  c.b = (float)((p && p->b != 0.0) ? p->b : 1.0 / 6.0);
  c.hh = (float)(h * h);
  const int npass = (nsweeps + nt - 1) / nt;
  T* a = (npass % 2) ? tmp : u;
  T* b = (npass % 2) ? u : tmp;
  int left = nsweeps;
  for (int k = 0; k < npass; ++k) {
    const int lv = left < nt ? left : nt;
    cudaError_t e = jacobi_tbz_pass((const float*)a, (float*)b, (const float*)f, g, lv, by, zchunk, c, st);
    if (e != cudaSuccess) return cuda_err(ctx, e, "jacobi_tbz_kernel launch");
    ctx->launches++;
    left -= lv;
    T* sw = a; a = b; b = sw;
  }
  return STENCIL_OK;
}

template <typename T>
static Coef<T> make_coef(double h, const stencil_params* p) {
  Coef<T> c;
  double b = (p && p->b != 0.0) ? p->b : 1.0 / 6.0;
  c.a = (T)(p ? p->a : 0.0);
  c.b = (T)b;
  c.hh = (T)(h * h);
  return c;
}

template <typename T>
int jacobi_run(stencil_ctx* ctx, T* u, const T* f, const Geom& g, double h, int nsweeps, const stencil_params* p,
               cudaStream_t st) {
  if (nsweeps == 0 || g.nx == 0 || g.ny == 0 || g.nz == 0) return STENCIL_OK;
  if (p && p->variant == 6) return jacobi_inplace_run<T>(ctx, u, f, g, h, nsweeps, p, st);
  const size_t bytes = (size_t)g.sy * (size_t)(g.nz + 2) * sizeof(T);
  int status = STENCIL_OK;
  T* tmp = (T*)ws_get(ctx, SLOT_JACOBI_TMP, bytes, &status);
  if (!tmp) return status;
  const int nt = (p && p->nt > 0) ? p->nt : 1;
  const bool weighted0 = p && p->a != 0.0;
  // FP32 with 1..4 sweeps per pass: the on-chip kernel is the default (two columns per thread and
  // overlapped tiles beat the one-column z-march even at one sweep per pass); at one sweep per pass
  // an explicit tile_y keeps the z-march it was chosen for
  const bool tbz_default = sizeof(T) == 4 && (!p || p->variant == 0) && nt >= 1 && nt <= 4 && !weighted0 &&
                           (nt > 1 || !p || p->tile_y == 0);
  if (tbz_default) {
    cudaError_t e0 = cudaMemcpyAsync(tmp, u, bytes, cudaMemcpyDeviceToDevice, st);
    if (e0 != cudaSuccess) return cuda_err(ctx, e0, "cudaMemcpyAsync(jacobi halo)");
    stencil_params q = p ? *p : stencil_params{};
    if (!q.tile_y) q.tile_y = nt == 1 ? 16 : 32;
    if (!q.tile_z) q.tile_z = 64;
    return tbz_run<T>(ctx, u, tmp, f, g, h, nsweeps, nt, &q, st);
  }
  if (p && p->variant == 4) {
    if (weighted0) return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "weighted sweeps on variant 4");
    cudaError_t e0 = cudaMemcpyAsync(tmp, u, bytes, cudaMemcpyDeviceToDevice, st);
    if (e0 != cudaSuccess) return cuda_err(ctx, e0, "cudaMemcpyAsync(jacobi halo)");
    return tbz_run<T>(ctx, u, tmp, f, g, h, nsweeps, nt, p, st);
  }
  if (nt > 1 || (p && p->variant == 3)) {
    stencil_params q = *p;
    q.nt = nt;
    return tb_jacobi_run<T>(ctx, u, tmp, f, g, h, nsweeps, &q, st);
  }
  const bool weighted = p && p->a != 0.0;
  // variant 1: plain z-march (default), 2: z-march with asynchronous plane copies
  const int variant = p ? p->variant : 0;
  if (variant < 0 || variant > 4) return set_err(ctx, STENCIL_ERR_ARG, "variant = %d", variant);
  const bool pipe = variant == 2;
  const int int_adds = (p && p->int_adds >= 0) ? p->int_adds : kDefaultIntAddsJacobi;
  if (int_adds < 0 || int_adds > kIntAddsAdaptive)
    return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "int_adds = %d (supported 0..6)", int_adds);
  Coef<T> c = make_coef<T>(h, p);
  int by = (p && p->tile_y) ? p->tile_y : (sizeof(T) == 8 ? 4 : 8);  // FP64: 32x4 measured fastest
  if (by != 4 && by != 8 && by != 16)
    return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "Jacobi tile_y = %d (supported 4, 8, 16)", by);
  if (p && p->tile_x && p->tile_x != 32)
    return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "Jacobi tile_x = %d (supported 32)", p->tile_x);
  int zchunk = (p && p->tile_z) ? p->tile_z : 0;
  if (zchunk <= 0) {
    // enough CTAs for ~8 waves of resident CTAs, chunks of at least 16 planes
    long long cols = (long long)((g.nx + 31) / 32) * ((g.ny + by - 1) / by);
    long long want = (long long)ctx->sm_count * (2048 / (32 * by)) * 8;
    long long chunks = (want + cols - 1) / cols;
    zchunk = (int)((g.nz + chunks - 1) / chunks);
    if (zchunk < 16) zchunk = 16;
  }
  // the workspace grid carries the same halo as u
  cudaError_t e = cudaMemcpyAsync(tmp, u, bytes, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaMemcpyAsync(jacobi halo)");
  // FP64 with f over several sweeps: hh*f once into workspace, the sweeps add it as it is (one FP64
  // multiplication per site fewer; skipped when the workspace budget has no room for it)
  const double* gf = nullptr;
  if (sizeof(T) == 8 && f && nsweeps >= 2 && !weighted && !pipe && (by == 4 || by == 8)) {
    const size_t n = (size_t)g.sy * (size_t)(g.nz + 2);
    double* w = (double*)ws_try(ctx, SLOT_F_SCALED, n * sizeof(double));
    if (w) {
      e = prescale_f((const double*)f, w, n, (double)c.hh, ctx->sm_count, st);
      ctx->launches++;
      if (e != cudaSuccess) return cuda_err(ctx, e, "prescale_f launch");
      gf = w;
    }
  }
  // ping-pong; with an odd count the first sweep reads the copy so the last lands in u
  T* a = (nsweeps % 2) ? tmp : u;
  T* b = (nsweeps % 2) ? u : tmp;
  for (int s = 0; s < nsweeps; ++s) {
    if constexpr (sizeof(T) == 8) {
      if (gf) e = jacobi_sweep_pre((const double*)a, (double*)b, gf, g, by, zchunk, c, int_adds, st);
      else e = jacobi_sweep<T>(a, b, f, g, by, zchunk, c, weighted, pipe, int_adds, st);
    } else {
      e = jacobi_sweep<T>(a, b, f, g, by, zchunk, c, weighted, pipe, int_adds, st);
    }
    ctx->launches++;
    if (e != cudaSuccess) return cuda_err(ctx, e, "jacobi_zmarch_kernel launch");
    T* sw = a; a = b; b = sw;
  }
  return STENCIL_OK;
}

template int jacobi_run<double>(stencil_ctx*, double*, const double*, const Geom&, double, int,
                                const stencil_params*, cudaStream_t);
template int jacobi_run<float>(stencil_ctx*, float*, const float*, const Geom&, double, int, const stencil_params*,
                               cudaStream_t);
template cudaError_t jacobi_sweep<double>(const double*, double*, const double*, const Geom&, int, int, Coef<double>,
                                          bool, bool, int, cudaStream_t);
template cudaError_t jacobi_sweep<float>(const float*, float*, const float*, const Geom&, int, int, Coef<float>, bool,
                                         bool, int, cudaStream_t);

}  // namespace stn
