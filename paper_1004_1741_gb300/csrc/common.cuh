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
// integer pipes issue far more, so an FP64-bound kernel leaves most issue
// slots idle.  int_add_f64 computes the IEEE-754 round-to-nearest-even sum of
// two doubles with 64-bit integer arithmetic when both are non-negative, the
// larger is normal and below 2^1022, and the smaller is +0 or normal at most
// 10 binades below it (the common case for neighbouring values of a smoothed
// field); otherwise it reports failure and the caller uses the FP64 pipe.
// Method: the significands (implicit bit at bit 62) are aligned within ten
// guard bits, so no bit is shifted out and no sticky bit is needed; the sum is
// rounded to 53 bits, to nearest with ties to even, by adding
// 2^(k-1) - 1 + (bit k of the sum) before the shift by k = 10 or 11 (one more
// when the addition carried into bit 63); a carry out of the rounding ripples
// into the exponent field.
__device__ __forceinline__ bool int_add_f64(double a, double b, double* out) {
  const unsigned long long A = (unsigned long long)__double_as_longlong(a);
  const unsigned long long B = (unsigned long long)__double_as_longlong(b);
  const unsigned ea = (unsigned)(A >> 52), eb = (unsigned)(B >> 52);  // sign bit included: negatives fail below
  const bool sw = eb > ea;
  const unsigned long long H = sw ? B : A, L = sw ? A : B;
  const unsigned eh = sw ? eb : ea, el = sw ? ea : eb;
  const unsigned d = eh - el;
  const bool lzero = L == 0ull;
  if (!((eh - 1u) < 2045u && (lzero || (el >= 1u && d <= 10u)))) return false;
  const unsigned long long FRAC = 0xFFFFFFFFFFFFFull, ONE = 1ull << 52;
  const unsigned long long MH = ((H & FRAC) | ONE) << 10;
  const unsigned long long ML = lzero ? 0ull : ((((L & FRAC) | ONE) << 10) >> d);
  const unsigned long long S = MH + ML;  // < 2^64
  const unsigned c = (unsigned)(S >> 63);
  const unsigned k = 10u + c;
  const unsigned long long M = (S + ((1ull << (k - 1u)) - 1ull + ((S >> k) & 1ull))) >> k;
  *out = __longlong_as_double((long long)(((unsigned long long)(eh + c - 1u) << 52) + M));
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

// Asynchronous element copy global -> shared (cp.async, through L1) and its
// group bookkeeping: wait until at most N of this thread's groups are pending.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem_dst, const T* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
  if (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
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
