// Shared device helpers of the GB300 stencil library (product path only).
#pragma once
#include <type_traits>

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
  static __device__ __forceinline__ double mul_b(double b, double s) { return mul(b, s); }
  static __device__ __forceinline__ double f_term(double hh, double fv) { return mul(hh, fv); }
  template <int K>
  static __device__ __forceinline__ double add_k(double a, double b) { return add(a, b); }
  static __device__ __forceinline__ double add_f(double a, double b) { return add(a, b); }
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
  static __device__ __forceinline__ double f_term(double hh, double fv) { return mul(hh, fv); }
  static __device__ __forceinline__ double mul_b(double b, double s) { return mul(b, s); }
  template <int K>
  static __device__ __forceinline__ double add_k(double a, double b) { return add(a, b); }
  static __device__ __forceinline__ double add_f(double a, double b) { return add(a, b); }
};

struct ArithF32 {
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float mul_b(float b, float s) { return mul(b, s); }
  static __device__ __forceinline__ float f_term(float hh, float fv) { return mul(hh, fv); }
  template <int K>
  static __device__ __forceinline__ float add_k(float a, float b) { return add(a, b); }
  static __device__ __forceinline__ float add_f(float a, float b) { return add(a, b); }
};

// Binary64 addition carried out on the integer pipes.
//
// The FP64 pipe of a GB300 SM retires ~1.6 lanes per clock, while its
// integer pipes issue far more, so an FP64-bound kernel leaves most issue
// slots idle.  int_add_f64 computes the IEEE-754 round-to-nearest-even sum of
// two doubles with 32-bit integer arithmetic when both are positive and
// normal, the larger has exponent field 11..2045 and the smaller lies at most
// 10 binades below it (the common case for neighbouring values of a smoothed
// field; the exponent bound makes the smaller operand normal whenever the gap
// is at most 10); otherwise it reports failure and the caller uses the FP64
// pipe.  Method: with ten guard bits the larger significand (implicit bit at
// 62) and the smaller one, shifted by 10 - gap, add exactly in 64 bits.  A
// carry into bit 63 is folded back by one right shift that ORs the dropped
// bit into bit 0 (it only matters as a sticky bit), so the sum always rounds
// at bit 10: to nearest with ties to even, by adding 2^9 - 1 + (bit 10)
// before the shift; a carry out of the rounding ripples into the exponent.
__device__ __forceinline__ bool int_add_f64(double a, double b, double* out) {
  const unsigned ahi = (unsigned)__double2hiint(a), alo = (unsigned)__double2loint(a);
  const unsigned bhi = (unsigned)__double2hiint(b), blo = (unsigned)__double2loint(b);
  const bool sw = (bhi >> 20) > (ahi >> 20);  // sign bit included: negatives fail below
  const unsigned hhi = sw ? bhi : ahi, hlo = sw ? blo : alo;
  const unsigned lhi = sw ? ahi : bhi, llo = sw ? alo : blo;
  const unsigned eh = hhi >> 20;
  const unsigned d = eh - (lhi >> 20);
  if (!((eh - 11u) < 2035u && d <= 10u)) return false;
  const unsigned mh = (hhi & 0xFFFFFu) | 0x100000u, ml = (lhi & 0xFFFFFu) | 0x100000u;
  const unsigned sh = 10u - d;
  const unsigned long long MH = ((unsigned long long)__funnelshift_l(hlo, mh, 10) << 32) | (hlo << 10);
  const unsigned long long ML = ((unsigned long long)__funnelshift_l(llo, ml, sh) << 32) | (llo << sh);
  const unsigned long long S = MH + ML;  // < 2^64
  const unsigned shi = (unsigned)(S >> 32), slo = (unsigned)S;
  const unsigned c = shi >> 31;
  const unsigned s2lo = __funnelshift_r(slo, shi, c) | (slo & c), s2hi = shi >> c;
  const unsigned long long R = (((unsigned long long)s2hi << 32) | s2lo) + (0x1FFu + ((s2lo >> 10) & 1u));
  const unsigned rlo = (unsigned)R, rhi = (unsigned)(R >> 32);
  const unsigned mlo = __funnelshift_r(rlo, rhi, 10), mhi = (rhi >> 10) + ((eh + c - 1u) << 20);
  *out = __hiloint2double((int)mhi, (int)mlo);
  return true;
}

// The same addition for an ordered pair: the fast path needs the exponent of a
// at least that of b (and at most 10 above it), so no swap is needed; every
// other pair, including a with the smaller exponent, goes to the FP64 pipe.
// In the neighbour sum every addition after the first adds one neighbour to a
// running sum of two to five positive values, which almost always satisfies it.
__device__ __forceinline__ bool int_add_f64_ge(double a, double b, double* out) {
  const unsigned hhi = (unsigned)__double2hiint(a), hlo = (unsigned)__double2loint(a);
  const unsigned lhi = (unsigned)__double2hiint(b), llo = (unsigned)__double2loint(b);
  const unsigned eh = hhi >> 20;  // sign bit included: negatives fail below
  const unsigned d = eh - (lhi >> 20);
  if (!((eh - 11u) < 2035u && d <= 10u)) return false;  // also fails when b's exponent is larger (d wraps)
  const unsigned mh = (hhi & 0xFFFFFu) | 0x100000u, ml = (lhi & 0xFFFFFu) | 0x100000u;
  const unsigned sh = 10u - d;
  const unsigned long long MH = ((unsigned long long)__funnelshift_l(hlo, mh, 10) << 32) | (hlo << 10);
  const unsigned long long ML = ((unsigned long long)__funnelshift_l(llo, ml, sh) << 32) | (llo << sh);
  const unsigned long long S = MH + ML;
  const unsigned shi = (unsigned)(S >> 32), slo = (unsigned)S;
  const unsigned c = shi >> 31;
  const unsigned s2lo = __funnelshift_r(slo, shi, c) | (slo & c), s2hi = shi >> c;
  const unsigned long long R = (((unsigned long long)s2hi << 32) | s2lo) + (0x1FFu + ((s2lo >> 10) & 1u));
  const unsigned rlo = (unsigned)R, rhi = (unsigned)(R >> 32);
  const unsigned mlo = __funnelshift_r(rlo, rhi, 10), mhi = (rhi >> 10) + ((eh + c - 1u) << 20);
  *out = __hiloint2double((int)mhi, (int)mlo);
  return true;
}

// Binary64 addition of operands of any signs on the integer pipes: the
// IEEE-754 round-to-nearest-even sum whenever the operand of larger magnitude
// has exponent field 1..2045 and the sum is zero or normal (both operands zero
// included); otherwise it reports failure and the caller uses the FP64 pipe.
// Method: order the operands by magnitude; the larger significand (implicit
// bit at 62) and the smaller one, shifted right by the exponent gap with the
// bits shifted out ORed into bit 0 (a sticky bit), are added or subtracted in
// 64 bits.  The ten bits below the rounding position keep the result on the
// right side of every rounding boundary: the sticky bit makes the computed
// value odd and off the true one by less than one unit of bit 0, while every
// boundary (and every tie) is a multiple of 2^8 there; a subtraction with a gap
// of two or more normalises by at most one bit, and one with a gap of at most
// one loses no bit at all.  The result is normalised to bit 62 (a carry into
// bit 63 folds back by one right shift, the dropped bit ORed into bit 0) and
// rounded at bit 10 as in int_add_f64; an exact zero difference is +0.
__device__ __forceinline__ bool int_add_f64_any(double a, double b, double* out) {
  const unsigned long long A = (unsigned long long)__double_as_longlong(a);
  const unsigned long long B = (unsigned long long)__double_as_longlong(b);
  const unsigned long long MAG = 0x7FFFFFFFFFFFFFFFull, FRAC = 0xFFFFFFFFFFFFFull;
  const bool sw = (B & MAG) > (A & MAG);
  const unsigned long long H = sw ? B : A, L = sw ? A : B;
  const unsigned eh = (unsigned)(H >> 52) & 0x7FFu, el = (unsigned)(L >> 52) & 0x7FFu;
  if (eh - 1u >= 2045u) {  // the larger operand is zero, subnormal or too large
    if ((H & MAG) != 0ull) return false;
    *out = __longlong_as_double((long long)(A & B));  // two zeros: -0 only when both are -0
    return true;
  }
  const unsigned long long MH = ((H & FRAC) | (1ull << 52)) << 10;
  const unsigned long long ML0 = ((L & FRAC) | (el ? (1ull << 52) : 0ull)) << 10;  // a subnormal has no implicit bit
  const unsigned d = min(eh - max(el, 1u), 63u);                                   // ... and exponent 1
  const unsigned long long ML = (ML0 >> d) | (unsigned long long)((ML0 & ((1ull << d) - 1ull)) != 0ull);
  const unsigned long long D = ((A ^ B) >> 63) ? MH - ML : MH + ML;
  if (D == 0ull) {
    *out = 0.0;
    return true;
  }
  const int lz = __clzll((long long)D);
  const int e = (int)eh + 1 - lz;  // exponent field of the normalised sum
  if (e < 1) return false;
  const unsigned long long D2 = lz == 0 ? (D >> 1) | (D & 1ull) : D << (lz - 1);
  const unsigned long long R = D2 + (0x1FFull + ((D2 >> 10) & 1ull));
  const unsigned long long res = (R >> 10) + ((unsigned long long)(e - 1) << 52);
  *out = __longlong_as_double((long long)(res | (H & ~MAG)));
  return true;
}

// Binary64 multiplication carried out in integer arithmetic (the 64-bit
// products on the integer multiply-add path, the rest on the ALU pipe): the
// IEEE round-to-nearest-even product when both operands are normal and the
// product's exponent stays in the normal range; otherwise it reports failure
// and the caller uses the FP64 pipe.  Method: the significands (implicit bit
// set, 53 bits) give a 106-bit product P in [2^104, 2^106); with one operand
// pre-shifted by 11, the high 64 bits of the 128-bit product are P / 2^53 and
// the low 64 bits hold P's remaining 53 bits at the top.  A product of two or
// more keeps the high word as its significand, a smaller one takes the next
// bit from the low word; the first dropped bit and the OR of the rest round to
// nearest with ties to even; a carry out of the rounding ripples into the
// exponent (a carry into the exponent's all-ones code reports failure).
__device__ __forceinline__ bool int_mul_f64(double a, double b, double* out) {
  const unsigned long long A = (unsigned long long)__double_as_longlong(a);
  const unsigned long long B = (unsigned long long)__double_as_longlong(b);
  const unsigned ea = (unsigned)(A >> 52) & 0x7FFu, eb = (unsigned)(B >> 52) & 0x7FFu;
  const int e = (int)ea + (int)eb - 1023;  // exponent field of a product in [1, 2)
  if (ea - 1u >= 2046u || eb - 1u >= 2046u || (unsigned)(e - 1) >= 2045u) return false;
  const unsigned long long FRAC = 0xFFFFFFFFFFFFFull, IMPL = 1ull << 52;
  const unsigned long long ma = ((A & FRAC) | IMPL) << 11, mb = (B & FRAC) | IMPL;
  const unsigned long long hi = __umul64hi(ma, mb), lo = ma * mb;
  const unsigned c = (unsigned)(hi >> 52);  // 1: the product is at least 2
  const unsigned long long mant = c ? hi : (hi << 1) | (lo >> 63);
  const unsigned long long rb = c ? (lo >> 63) : ((lo >> 62) & 1ull);
  const unsigned long long sticky = (c ? (lo << 1) : (lo << 2)) != 0ull;
  const unsigned long long m2 = mant + (rb & (sticky | (mant & 1ull)));
  const unsigned long long res = m2 + ((unsigned long long)(e + (int)c - 1) << 52);
  if (((res >> 52) & 0x7FFull) == 0x7FFull) return false;
  *out = __longlong_as_double((long long)(res | ((A ^ B) & (1ull << 63))));
  return true;
}

// FP64 arithmetic that splits the additions of a site update between the
// integer pipes (int_add_f64) and the FP64 pipe: the additions whose bit is
// set in NATIVE_MASK (0 = first, 4 = last of the neighbour sum) and every
// multiplication go to the FP64 pipe.  Same bits as ArithF64 either way.
template <unsigned NATIVE_MASK, bool INT_MUL = false>
struct ArithF64Mix {
  static __device__ __forceinline__ double add(double a, double b) { return ArithF64Fma::add(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return ArithF64Fma::mul(a, b); }
  // the bracket's weight times the bracket, on the integer path when INT_MUL
  static __device__ __forceinline__ double mul_b(double b, double s) {
    double r;
    if (INT_MUL && int_mul_f64(b, s, &r)) return r;
    return ArithF64Fma::mul(b, s);
  }
  static __device__ __forceinline__ double f_term(double hh, double fv) { return mul(hh, fv); }
  template <int K>
  static __device__ __forceinline__ double add_k(double a, double b) {
    if (NATIVE_MASK & (1u << K)) return ArithF64Fma::add(a, b);
    double r;
    // the first addition (W + E) has no preferred order; later ones add a neighbour to the running sum
    if (K == 0 ? int_add_f64(a, b, &r) : int_add_f64_ge(a, b, &r)) return r;
    return ArithF64Fma::add(a, b);
  }
  static __device__ __forceinline__ double add_f(double a, double b) { return add(a, b); }
};

// The arithmetic A for a sweep whose f array already holds the products
// hh*f (prescale_f: the same multiplication, once per call instead of once
// per sweep): the site update adds f as it is.  Same bits.
template <class A>
struct ArithPreF : A {
  template <typename T>
  static __device__ __forceinline__ T f_term(T, T fv) { return fv; }
};

// Data-dependent choice per warp and update: POS for neighbourhoods that are
// all non-negative (integer-pipe additions apply), MIXED otherwise (additions
// on the FP64 pipe, the multiplication on the integer path).  The kernel body
// takes the vote (site_update_adaptive); every other operation uses POS.
template <class POS, class MIXED>
struct ArithAdaptive : POS {
  using Pos = POS;
  using Mixed = MIXED;
};

template <class Ar>
struct AdaptOf {
  static constexpr bool on = false;
};
template <class P, class M>
struct AdaptOf<ArithAdaptive<P, M>> {
  static constexpr bool on = true;
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
  if (HAS_F) acc = Ar::add_f(acc, Ar::f_term(c.hh, fv));
  T v = Ar::mul_b(c.b, acc);
  if (WEIGHTED) v = Ar::add(Ar::mul(c.a, uc), v);
  return v;
}

// site_update for the whole warp (every lane must call it; `active` lanes
// get their update): with an ArithAdaptive the warp takes POS when every
// active lane's six neighbours have their sign bit clear, else MIXED.
template <typename T, class Ar, bool HAS_F, bool WEIGHTED>
__device__ __forceinline__ T site_update_warp(bool active, T w, T e, T s, T n, T bo, T t, T fv, T uc,
                                              const Coef<T>& c) {
  if constexpr (AdaptOf<Ar>::on && sizeof(T) == 8) {
    const int sg = __double2hiint(w) | __double2hiint(e) | __double2hiint(s) | __double2hiint(n) |
                   __double2hiint(bo) | __double2hiint(t);
    if (__all_sync(0xFFFFFFFFu, !active || sg >= 0))
      return active ? site_update<T, typename Ar::Pos, HAS_F, WEIGHTED>(w, e, s, n, bo, t, fv, uc, c) : T(0);
    return active ? site_update<T, typename Ar::Mixed, HAS_F, WEIGHTED>(w, e, s, n, bo, t, fv, uc, c) : T(0);
  } else {
    return active ? site_update<T, Ar, HAS_F, WEIGHTED>(w, e, s, n, bo, t, fv, uc, c) : T(0);
  }
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
