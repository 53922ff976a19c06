// Residual kernels shared by residual_norm (residual.cu) and
// residual_norm_noalloc (noalloc.cu): both entry points instantiate these
// templates, so their sums come from the same code in the same order.
//
// r = f - (6 u - S) * (1/(h*h)) on the interior, with S the six neighbours
// added in the site update's order.  With NORM, each CTA reduces its sums of
// r^2 and f^2 in a fixed tree (warp shuffles, then warp 0 over the warp sums)
// into partials[2*bid], partials[2*bid+1]; reduce_pairs_kernel then adds the
// per-CTA pairs in a fixed order, so a given grid shape always gives the same
// bits.
#pragma once

#include "common.cuh"

namespace stn {

constexpr int RES_BX = 32, RES_BY = 8, RES_ZCHUNK = 32;

// Launch shape of residual_kernel for a grid: (ceil(nx/32), ceil(ny/8), ceil(nz/32)) CTAs of 32 x 8.
inline dim3 residual_grid(const Geom& g) {
  return dim3((g.nx + RES_BX - 1) / RES_BX, (g.ny + RES_BY - 1) / RES_BY, (g.nz + RES_ZCHUNK - 1) / RES_ZCHUNK);
}

// The neighbour sum takes three of its five additions on the integer pipes
// (common.cuh; the same bits as the FP64 pipe).
template <bool HAS_F, bool WANT_R, bool WANT_R32, bool NORM>
__global__ void __launch_bounds__(RES_BX* RES_BY) residual_kernel(const double* __restrict__ u,
                                                                  const double* __restrict__ f, double* r_out,
                                                                  float* r32_out, Geom g, double ih2,
                                                                  double* __restrict__ partials) {
  using Ar = ArithF64Mix<0x12u>;
  const int x = blockIdx.x * RES_BX + threadIdx.x;
  const int y = blockIdx.y * RES_BY + threadIdx.y;
  const int z0 = blockIdx.z * RES_ZCHUNK;
  const int z1 = min(g.nz, z0 + RES_ZCHUNK);
  double rr = 0.0, ff = 0.0;
  if (x < g.nx && y < g.ny) {
    for (int z = z0; z < z1; ++z) {
      const int64_t c = g.at(x, y, z);
      double s = Ar::template add_k<0>(u[c - 1], u[c + 1]);
      s = Ar::template add_k<1>(s, u[c - g.sx]);
      s = Ar::template add_k<2>(s, u[c + g.sx]);
      s = Ar::template add_k<3>(s, u[c - g.sy]);
      s = Ar::template add_k<4>(s, u[c + g.sy]);
      const double au = __dmul_rn(__dsub_rn(__dmul_rn(6.0, u[c]), s), ih2);
      const double fv = HAS_F ? f[c] : 0.0;
      const double r = __dsub_rn(fv, au);
      if (WANT_R) r_out[c] = r;
      if (WANT_R32) r32_out[c] = __double2float_rn(r);
      if (NORM) {
        rr = __fma_rn(r, r, rr);
        if (HAS_F) ff = __fma_rn(fv, fv, ff);
      }
    }
  }
  if (!NORM) return;
  // fixed-order block reduction: warp tree, then warp 0 over the warp sums
  __shared__ double wr[RES_BY], wf[RES_BY];
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
    double a = 0.0, bsum = 0.0;
    for (int w = 0; w < RES_BY; ++w) {
      a = __dadd_rn(a, wr[w]);
      bsum = __dadd_rn(bsum, wf[w]);
    }
    const int64_t bid = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    partials[2 * bid] = a;
    partials[2 * bid + 1] = bsum;
  }
}

// One CTA of 1024 threads: sums partials[2*i] and partials[2*i+1] over i < n
// in a fixed order (strided running sums, then a shared-memory tree).
template <int NT = 1024>
__global__ void __launch_bounds__(NT) reduce_pairs_kernel(const double* __restrict__ partials, int64_t n,
                                                          double* __restrict__ out) {
  __shared__ double sa[NT], sb[NT];
  double a = 0.0, b = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += NT) {
    a = __dadd_rn(a, partials[2 * i]);
    b = __dadd_rn(b, partials[2 * i + 1]);
  }
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int s = NT / 2; s > 0; s >>= 1) {
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

}  // namespace stn

namespace stn {

// FP32 residual r = f - (6u - S) * ih2 (every operation in binary32, ih2 =
// (float)(1/(h*h))) on the interior, for the FP32 multigrid levels; no norm.
template <bool HAS_F>
__global__ void __launch_bounds__(RES_BX* RES_BY) residual_f32_kernel(const float* __restrict__ u,
                                                                      const float* __restrict__ f,
                                                                      float* __restrict__ r_out, Geom g, float ih2) {
  using Ar = ArithF32;
  const int x = blockIdx.x * RES_BX + threadIdx.x;
  const int y = blockIdx.y * RES_BY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int z0 = blockIdx.z * RES_ZCHUNK;
  const int z1 = min(g.nz, z0 + RES_ZCHUNK);
  for (int z = z0; z < z1; ++z) {
    const int64_t c = g.at(x, y, z);
    float s = Ar::add(u[c - 1], u[c + 1]);
    s = Ar::add(s, u[c - g.sx]);
    s = Ar::add(s, u[c + g.sx]);
    s = Ar::add(s, u[c - g.sy]);
    s = Ar::add(s, u[c + g.sy]);
    const float au = __fmul_rn(__fsub_rn(__fmul_rn(6.0f, u[c]), s), ih2);
    const float fv = HAS_F ? f[c] : 0.0f;
    r_out[c] = __fsub_rn(fv, au);
  }
}

}  // namespace stn
