// Shared device helpers of the GB300 stencil library (product path only).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace stn {

// ---------------------------------------------------------------------------
// Arithmetic.  Every operation of the site update is one IEEE-754
// round-to-nearest operation that the compiler may not fuse or reorder
// (__dadd_rn / __dmul_rn and friends are never contracted), so the GPU result
// is bit-identical to the serial loops of Sec. 3.
//
// FP64 has two encodings of the same operations: plain DADD/DMUL, or the FMA
// pipe form add(a,b) = fma(a, 1, b) and mul(a,b) = fma(a, b, -0).  Both round
// exactly once to the same value (a*1 is exact; adding -0 leaves every
// product, a signed zero included, unchanged), so they are interchangeable
// bit for bit.  The FMA form is issued through inline PTX so that it cannot
// be folded back into DADD/DMUL.
// ---------------------------------------------------------------------------
struct ArithF64 {
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
};

struct ArithF64Fma {
  static __device__ __forceinline__ double add(double a, double b) {
    double r;
    asm("fma.rn.f64 %0, %1, 0d3FF0000000000000, %2;" : "=d"(r) : "d"(a), "d"(b));
    return r;
  }
  static __device__ __forceinline__ double mul(double a, double b) {
    double r;
    asm("fma.rn.f64 %0, %1, %2, 0d8000000000000000;" : "=d"(r) : "d"(a), "d"(b));
    return r;
  }
};

struct ArithF32 {
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
};

template <typename T>
struct DefaultArith;
template <>
struct DefaultArith<double> {
  using type = ArithF64Fma;
};
template <>
struct DefaultArith<float> {
  using type = ArithF32;
};

// Coefficients of one smoother call in the working precision.
template <typename T>
struct Coef {
  T a;   // weight of the old value (weighted Jacobi); used only when WEIGHTED
  T b;   // weight of the bracket, 1/6 by default
  T hh;  // h*h, used only when f != NULL
};

// The site update u' = [a*u +] b*(((((W+E)+S)+N)+B)+T [+ hh*f]).
template <typename T, class Ar, bool HAS_F, bool WEIGHTED>
__device__ __forceinline__ T site_update(T w, T e, T s, T n, T bo, T t, T fv, T uc, const Coef<T>& c) {
  T acc = Ar::add(w, e);
  acc = Ar::add(acc, s);
  acc = Ar::add(acc, n);
  acc = Ar::add(acc, bo);
  acc = Ar::add(acc, t);
  if (HAS_F) acc = Ar::add(acc, Ar::mul(c.hh, fv));
  T v = Ar::mul(c.b, acc);
  if (WEIGHTED) v = Ar::add(Ar::mul(c.a, uc), v);
  return v;
}

// Padded-grid geometry: interior (nx, ny, nz), element (x, y, z) of the
// interior (x in [-1, nx] etc. reaching the halo) at
// ((z+1)*(ny+2) + (y+1))*(nx+2) + (x+1).
struct Geom {
  int nx, ny, nz;
  int64_t sx;  // nx + 2
  int64_t sy;  // (nx+2)*(ny+2)
  __host__ __device__ __forceinline__ int64_t at(int x, int y, int z) const {
    return (int64_t)(z + 1) * sy + (int64_t)(y + 1) * sx + (x + 1);
  }
};

inline Geom make_geom(int nx, int ny, int nz) {
  Geom g;
  g.nx = nx; g.ny = ny; g.nz = nz;
  g.sx = (int64_t)nx + 2;
  g.sy = ((int64_t)nx + 2) * ((int64_t)ny + 2);
  return g;
}

}  // namespace stn
