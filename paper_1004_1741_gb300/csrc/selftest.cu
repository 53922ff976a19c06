// Self-check of the integer-pipe binary64 additions (common.cuh int_add_f64,
// its ordered form int_add_f64_ge and the any-sign form int_add_f64_any) and
// of the integer-arithmetic multiplication (int_mul_f64) against the FP64
// pipe on generated operand pairs.
#include "internal.h"

namespace stn {

// splitmix64: a counter-based generator (Steele, Lea, Flood 2014)
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double gen_operand(unsigned long long r, unsigned long long r2, int kind) {
  switch (kind) {
    case 0: {  // uniform significand, exponent near 0
      const unsigned long long e = 1023ull - 40ull + (r2 % 80ull);
      return __longlong_as_double((long long)((e << 52) | (r & 0xFFFFFFFFFFFFFull)));
    }
    case 1: {  // operands close to each other (ties and carries are frequent)
      const unsigned long long e = 1023ull + (r2 % 3ull);
      return __longlong_as_double((long long)((e << 52) | (r & 0xFFFFFFFFFFFFFull)));
    }
    case 2: {  // any bit pattern (specials, subnormals, signs)
      return __longlong_as_double((long long)r);
    }
    default: {  // small integers scaled (exact ties)
      return (double)(long long)(r % 4096ull) * 0x1p-12;
    }
  }
}

__global__ void selftest_int_add_kernel(unsigned long long n, unsigned long long seed,
                                        unsigned long long* __restrict__ counts) {
  unsigned long long mism = 0, fast = 0, fast_any = 0;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long r0 = mix64(seed ^ (4 * i)), r1 = mix64(seed ^ (4 * i + 1));
    const unsigned long long r2 = mix64(seed ^ (4 * i + 2)), r3 = mix64(seed ^ (4 * i + 3));
    const int kind = (int)(r3 & 3ull);
    const int kind2 = (int)((r3 >> 2) & 3ull);
    double a = gen_operand(r0, r2, kind);
    double b = gen_operand(r1, r2 >> 7, kind2);
    if ((r3 >> 8) & 1ull) b = __longlong_as_double(__double_as_longlong(a) + (long long)((r3 >> 9) & 15ull) - 8);
    if (((r3 >> 13) & 15ull) == 0) b = 0.0;
    const double ref = __dadd_rn(a, b);
    double em;
    if (int_add_f64(a, b, &em)) {
      ++fast;
      if (__double_as_longlong(em) != __double_as_longlong(ref)) ++mism;
    }
    // the ordered form, in both argument orders
    if (int_add_f64_ge(a, b, &em) && __double_as_longlong(em) != __double_as_longlong(ref)) ++mism;
    if (int_add_f64_ge(b, a, &em) && __double_as_longlong(em) != __double_as_longlong(__dadd_rn(b, a))) ++mism;
    // the integer-path multiplication, on the same pair with independent random signs
    const double sa = ((r3 >> 17) & 1ull) ? -a : a, sb = ((r3 >> 18) & 1ull) ? -b : b;
    // the any-sign addition, on the pair with those signs, in both argument orders
    if (int_add_f64_any(sa, sb, &em)) {
      ++fast_any;
      if (__double_as_longlong(em) != __double_as_longlong(__dadd_rn(sa, sb))) ++mism;
    }
    if (int_add_f64_any(sb, sa, &em) && __double_as_longlong(em) != __double_as_longlong(__dadd_rn(sb, sa))) ++mism;
    if (int_mul_f64(sa, sb, &em) && __double_as_longlong(em) != __double_as_longlong(__dmul_rn(sa, sb))) ++mism;
    if (int_mul_f64(sb, sa, &em) && __double_as_longlong(em) != __double_as_longlong(__dmul_rn(sb, sa))) ++mism;
  }
  atomicAdd(counts, mism);
  atomicAdd(counts + 1, fast);
  atomicAdd(counts + 2, fast_any);
}

}  // namespace stn

using namespace stn;

extern "C" int stencil_selftest_int_add(stencil_ctx* ctx, uint64_t n, uint64_t seed, uint64_t* out_mismatch,
                                        uint64_t* out_fast, uint64_t* out_fast_any) {
  if (!ctx || !out_mismatch || !out_fast) return STENCIL_ERR_ARG;
  ctx->err.clear();
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  int status;
  unsigned long long* d = (unsigned long long*)ws_get(ctx, SLOT_RED_RESULT, 4 * sizeof(double), &status);
  if (!d) return status;
  unsigned long long h[3] = {0, 0, 0};
  e = cudaMemset(d, 0, sizeof(h));
  if (e == cudaSuccess) {
    selftest_int_add_kernel<<<ctx->sm_count * 8, 256>>>((unsigned long long)n, (unsigned long long)seed, d);
    ctx->launches++;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_err(ctx, e, "selftest_int_add");
  *out_mismatch = h[0];
  *out_fast = h[1];
  if (out_fast_any) *out_fast_any = h[2];
  return STENCIL_OK;
}
