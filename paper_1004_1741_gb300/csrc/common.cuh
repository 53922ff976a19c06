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
  template <int K>
  static __device__ __forceinline__ double add_k(double a, double b) { return add(a, b); }
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
  template <int K>
  static __device__ __forceinline__ double add_k(double a, double b) { return add(a, b); }
};

struct ArithF32 {
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  template <int K>
  static __device__ __forceinline__ float add_k(float a, float b) { return add(a, b); }
};

// Binary64 addition carried out on the integer pipes.
//
// The FP64 pipe of a GB300 SM retires ~1.6 lanes per clock, while its
// integer pipes issue 128 lanes per clock, so an FP64-bound kernel leaves
// most issue slots idle.  int_add_f64 computes the IEEE-754 round-to-nearest-
// even sum of two doubles with 64-bit integer arithmetic when both are
// non-negative, the larger is normal and at most 2^1022, and the smaller is
// +0 or normal with an exponent at most 31 below (the common case for
// smoothed fields); otherwise it reports failure and the caller uses the
// FP64 pipe.  Method: align the significands (53 bits, implicit bit at bit
// 62, ten guard bits) with the bits shifted out OR-ed into the lowest bit,
// add, renormalise by at most one bit (again keeping the sticky bit), round
// to 53 bits to nearest, ties to even, and let a carry of the rounding ripple
// into the exponent field.
__device__ __forceinline__ bool int_add_f64(double a, double b, double* out) {
  const unsigned long long A = (unsigned long long)__double_as_longlong(a);
  const unsigned long long B = (unsigned long long)__double_as_longlong(b);
  const unsigned long long H = A > B ? A : B;  // a negative operand ends up here and fails the exponent test
  const unsigned long long L = A > B ? B : A;
  const unsigned eh = (unsigned)(H >> 52), el = (unsigned)(L >> 52);
  const unsigned d = eh - el;
  const bool lzero = L == 0ull;
  if (!((eh - 1u) < 2045u && (lzero || (el >= 1u && d < 32u)))) return false;
  const unsigned long long FRAC = 0xFFFFFFFFFFFFFull;
  const unsigned long long MH = ((H & FRAC) << 10) | (1ull << 62);
  const unsigned long long ML = ((L & FRAC) << 10) | (1ull << 62);
  const unsigned dd = lzero ? 0u : d;
  unsigned long long Ms = ML >> dd;
  Ms |= (unsigned long long)((((unsigned)ML) & ((1u << dd) - 1u)) != 0u);  // sticky
  unsigned long long S = MH + Ms;                                            // < 2^64
  const unsigned c = (unsigned)(S >> 63);
  S = (S >> c) | (S & (unsigned long long)c);
  unsigned long long M = S >> 10;
  const unsigned rem = (unsigned)S & 1023u;
  M += (unsigned long long)((rem > 512u) | ((rem == 512u) & ((unsigned)M & 1u)));
  const unsigned long long R = ((unsigned long long)(eh + c - 1u) << 52) + M;
  *out = __longlong_as_double((long long)(lzero ? H : R));
  return true;
}

// FP64 arithmetic that splits the additions of a site update between the
// integer pipes (int_add_f64) and the FP64 pipe: the additions whose bit is
// set in NATIVE_MASK (0 = first, 4 = last of the neighbour sum) and every
// multiplication go to the FP64 pipe.  Same bits as ArithF64 either way.
template <unsigned NATIVE_MASK>
struct ArithF64Mix {
  static __device__ __forceinline__ double add(double a, double b) { return ArithF64Fma::add(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return ArithF64Fma::mul(a, b); }
  template <int K>
  static __device__ __forceinline__ double add_k(double a, double b) {
    if (NATIVE_MASK & (1u << K)) return ArithF64Fma::add(a, b);
    double r;
    if (int_add_f64(a, b, &r)) return r;
    return ArithF64Fma::add(a, b);
  }
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
  T acc = Ar::template add_k<0>(w, e);
  acc = Ar::template add_k<1>(acc, s);
  acc = Ar::template add_k<2>(acc, n);
  acc = Ar::template add_k<3>(acc, bo);
  acc = Ar::template add_k<4>(acc, t);
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
