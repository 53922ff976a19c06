// Temporal blocking on chip for bandwidth-bound (FP32) Jacobi: nt sweeps per
// pass over memory in one 2.5D z-march (Sec. 4's wavefront of time levels,
// restated for a CTA).
//
// A CTA of 32 x BY threads owns a 64 x BY tile of (x, y) columns (two columns
// per thread, 32 apart); the tile overlaps its neighbours by NT columns on
// each side.  Marching up in z, at step q the CTA loads plane q of level 0 and
// computes level l at plane q-l for l = 1..NT: a time level trails the one
// below by one plane.  Each column keeps the three newest planes of every
// level in registers (the paper's "three planes in cache"), and the newest
// plane of each level below NT is published in shared memory (double
// buffered, one barrier per step) for the in-plane neighbours.  Level NT is
// written out for the tile's central (64 - 2NT) x (BY - 2NT) columns; the
// outer ring is recomputed by the neighbouring tile.  That recomputation
// costs ALU work, which FP32 has plenty of, and buys a single read and a
// single write of the grid per NT sweeps.  (The FP64 pipe has no such slack:
// FP64 uses the no-recomputation skewed-tile schedule instead.)
#include <type_traits>

#include "internal.h"

namespace stn {

template <typename T, class Ar, bool HAS_F, int NT, int BY>
__global__ void __launch_bounds__(32 * BY) jacobi_tbz_kernel(const T* __restrict__ src, T* __restrict__ dst,
                                                             const T* __restrict__ f, Geom g, int zchunk, Coef<T> c) {
  constexpr int TW = 64;  // tile width in x
  extern __shared__ __align__(16) unsigned char tbz_raw[];
  // sm(l, buf, row, col): newest plane of level l, double buffered
  T* smb = reinterpret_cast<T*>(tbz_raw);
#define SM(l, bb, r, cc) smb[(((l)*2 + (bb)) * BY + (r)) * TW + (cc)]
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int z0 = blockIdx.z * zchunk;
  const int z1 = min(g.nz, z0 + zchunk);
  if (z0 >= z1) return;
  const int y = (int)blockIdx.y * (BY - 2 * NT) - NT + ty;
  int x[2];
  bool valid[2], interior[2], out[2];
  int64_t col[2];
  for (int k = 0; k < 2; ++k) {
    x[k] = (int)blockIdx.x * (TW - 2 * NT) - NT + tx + 32 * k;
    valid[k] = x[k] >= -1 && x[k] <= g.nx && y >= -1 && y <= g.ny;  // grid or halo column
    interior[k] = x[k] >= 0 && x[k] < g.nx && y >= 0 && y < g.ny;
    const int tc = tx + 32 * k;
    out[k] = interior[k] && tc >= NT && tc < TW - NT && ty >= NT && ty < BY - NT;
    col[k] = valid[k] ? g.at(x[k], y, -1) : 0;  // padded offset of the column at plane -1
  }
  // neighbour indices in the tile (clamped at the tile edge: those lanes feed no output)
  const int ym = ty > 0 ? ty - 1 : ty, yp = ty < BY - 1 ? ty + 1 : ty;
  int xm[2], xp[2];
  for (int k = 0; k < 2; ++k) {
    const int tc = tx + 32 * k;
    xm[k] = tc > 0 ? tc - 1 : tc;
    xp[k] = tc < TW - 1 ? tc + 1 : tc;
  }
  const int zs = max(z0 - NT, -1);         // first level-0 plane
  const int ze = min(z1 + NT - 1, g.nz);   // last level-0 plane
  T P[2][NT], C[2][NT], N[2][NT];         // planes p-1, p, p+1 of level l, p = q-l-1 after step q
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int l = 0; l < NT; ++l) P[k][l] = C[k][l] = N[k][l] = T(0);
  const int64_t sy = g.sy;
  // level-0 planes are loaded PF steps before they are used (register queue)
  constexpr int PF = 4;
  T qv[2][PF];
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int i = 0; i < PF; ++i)
      qv[k][i] = (valid[k] && zs + i <= ze) ? src[col[k] + (int64_t)(zs + i + 1) * sy] : T(0);
  // per-column pointers at the plane each one serves after step q = zs; advanced by one plane per step
  // and dereferenced only when that plane exists
  const T* pq[2];   // level-0 load: plane q + PF
  const T* pfq[2];  // right-hand side at plane q (level l reads plane q - l)
  T* pd[2];         // output: plane q - NT
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    pq[k] = src + col[k] + (int64_t)(zs + PF + 1) * sy;
    pfq[k] = HAS_F ? f + col[k] + (int64_t)(zs + 1) * sy : nullptr;
    pd[k] = dst + col[k] + (int64_t)(zs - NT + 1) * sy;
  }
  auto step = [&](int q, auto bc) {
    constexpr int b = decltype(bc)::value, bp = b ^ 1;
    // level 0: plane q
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const T v = qv[k][0];
#pragma unroll
      for (int i = 0; i + 1 < PF; ++i) qv[k][i] = qv[k][i + 1];
      qv[k][PF - 1] = (valid[k] && q + PF <= ze) ? *pq[k] : T(0);
      P[k][0] = C[k][0];
      C[k][0] = N[k][0];
      N[k][0] = v;
      SM(0, b, ty, tx + 32 * k) = v;
    }
    // levels 1..NT: level l at plane q-l
#pragma unroll
    for (int l = 1; l <= NT; ++l) {
      const int p = q - l;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int tc = tx + 32 * k;
        T v;
        if (interior[k] && p >= 0 && p < g.nz) {
          T fv = T(0);
          if (HAS_F) fv = pfq[k][-(int64_t)l * sy];
          v = site_update<T, Ar, HAS_F, false>(SM(l - 1, bp, ty, xm[k]), SM(l - 1, bp, ty, xp[k]),
                                               SM(l - 1, bp, ym, tc), SM(l - 1, bp, yp, tc), P[k][l - 1],
                                               N[k][l - 1], fv, T(0), c);
        } else {
          v = C[k][l - 1];  // halo column or halo plane: the Dirichlet value, at every level
        }
        if (l < NT) {
          P[k][l] = C[k][l];
          C[k][l] = N[k][l];
          N[k][l] = v;
          SM(l, b, ty, tc) = v;
        } else if (out[k] && p >= z0 && p < z1) {
          *pd[k] = v;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      pq[k] += sy;
      if (HAS_F) pfq[k] += sy;
      pd[k] += sy;
    }
    __syncthreads();
  };
  // the buffer index of step q is q & 1; two steps per trip keep it a constant
  const int qe = z1 - 1 + NT;
  int q = zs;
  if (q & 1) step(q++, std::integral_constant<int, 1>{});
  for (; q + 1 <= qe; q += 2) {
    step(q, std::integral_constant<int, 0>{});
    step(q + 1, std::integral_constant<int, 1>{});
  }
  if (q <= qe) step(q, std::integral_constant<int, 0>{});
#undef SM
}

template <typename T, int NT, int BY>
static cudaError_t tbz_launch(const T* src, T* dst, const T* f, const Geom& g, int zchunk, Coef<T> c,
                              cudaStream_t st) {
  using Ar = typename DefaultArith<T>::type;
  const int smem = NT * 2 * BY * 64 * (int)sizeof(T);
  auto k0 = jacobi_tbz_kernel<T, Ar, false, NT, BY>;
  auto k1 = jacobi_tbz_kernel<T, Ar, true, NT, BY>;
  cudaError_t e = cudaFuncSetAttribute(f ? k1 : k0, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  dim3 block(32, BY);
  dim3 grid((g.nx + (64 - 2 * NT) - 1) / (64 - 2 * NT), (g.ny + (BY - 2 * NT) - 1) / (BY - 2 * NT),
            (g.nz + zchunk - 1) / zchunk);
  if (f)
    k1<<<grid, block, smem, st>>>(src, dst, f, g, zchunk, c);
  else
    k0<<<grid, block, smem, st>>>(src, dst, f, g, zchunk, c);
  return cudaGetLastError();
}

// One pass of `levels` sweeps src -> dst (levels in {1, 2, 3, 4}); by: CTA rows (16 or 32).
cudaError_t jacobi_tbz_pass(const float* src, float* dst, const float* f, const Geom& g, int levels, int by,
                            int zchunk, Coef<float> c, cudaStream_t st) {
  switch (levels * 100 + by) {
    case 116: return tbz_launch<float, 1, 16>(src, dst, f, g, zchunk, c, st);
    case 132: return tbz_launch<float, 1, 32>(src, dst, f, g, zchunk, c, st);
    case 216: return tbz_launch<float, 2, 16>(src, dst, f, g, zchunk, c, st);
    case 232: return tbz_launch<float, 2, 32>(src, dst, f, g, zchunk, c, st);
    case 316: return tbz_launch<float, 3, 16>(src, dst, f, g, zchunk, c, st);
    case 332: return tbz_launch<float, 3, 32>(src, dst, f, g, zchunk, c, st);
    case 416: return tbz_launch<float, 4, 16>(src, dst, f, g, zchunk, c, st);
    case 432: return tbz_launch<float, 4, 32>(src, dst, f, g, zchunk, c, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace stn
