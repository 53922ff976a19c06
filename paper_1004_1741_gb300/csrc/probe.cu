// Throughput probes of the pipes the smoothers run on: FP64 and FP32
// additions, 32-bit integer ALU instructions, the binary64 addition carried
// out on the integer pipes (common.cuh int_add_f64_ge), and a copy kernel's
// DRAM bandwidth.  They give the denominators of the roofline the benchmark
// reports, measured on the GPU at hand instead of taken from unit counts and
// nominal clocks.
//
// Every arithmetic probe runs CH independent dependency chains per thread in
// a grid of 32 warps per SM (enough chains to cover the pipes' latency), for
// ITER iterations, and stores a value derived from every chain so that
// nothing is dead code; it is launched once to warm up and once timed with
// CUDA events.  Rates are whole-GPU operations per second.
#include "internal.h"

namespace stn {

constexpr int PROBE_CH = 8;
constexpr int PROBE_THREADS = 256;

__global__ void __launch_bounds__(PROBE_THREADS) probe_fp64_kernel(int iters, double* __restrict__ out) {
  double v[PROBE_CH];
  const double inc = 1.0 + 1e-9 * threadIdx.x;
#pragma unroll
  for (int c = 0; c < PROBE_CH; ++c) v[c] = 0.5 + 1e-3 * (c + blockIdx.x);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < PROBE_CH; ++c) v[c] = ArithF64Fma::add(v[c], inc);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < PROBE_CH; ++c) s = __dadd_rn(s, v[c]);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_THREADS) probe_fp32_kernel(int iters, float* __restrict__ out) {
  float v[PROBE_CH];
  const float inc = 1.0f + 1e-6f * threadIdx.x;
#pragma unroll
  for (int c = 0; c < PROBE_CH; ++c) v[c] = 0.5f + 1e-3f * (c + blockIdx.x);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < PROBE_CH; ++c) v[c] = __fadd_rn(v[c], inc);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < PROBE_CH; ++c) s = __fadd_rn(s, v[c]);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// One 32-bit ALU instruction per chain step: a three-input logic operation
// (lop3) that the compiler cannot fold across iterations.
__global__ void __launch_bounds__(PROBE_THREADS) probe_alu_kernel(int iters, unsigned* __restrict__ out) {
  unsigned v[PROBE_CH];
  const unsigned k = 0x9E3779B9u * (threadIdx.x + 1);
#pragma unroll
  for (int c = 0; c < PROBE_CH; ++c) v[c] = k + c * 0x85EBCA6Bu + blockIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < PROBE_CH; ++c) {
      unsigned r;
      asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(v[c]), "r"(k), "r"((unsigned)it));
      v[c] = r;
    }
  }
  unsigned s = 0;
#pragma unroll
  for (int c = 0; c < PROBE_CH; ++c) s ^= v[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Binary64 additions on the integer pipes: each chain adds a small positive
// value to a running value of about 1 and then clears the result's lowest
// significand bits back to the start, so the operands stay in the fast path
// (same exponent range) while every addition depends on the previous one.
// The count of additions that took the fast path is returned in out_fast.
__global__ void __launch_bounds__(PROBE_THREADS) probe_int_add_kernel(int iters, double* __restrict__ out,
                                                                      unsigned long long* __restrict__ out_fast) {
  double v[PROBE_CH];
  const double b = 0.001 * (1.0 + threadIdx.x * 1e-3);
#pragma unroll
  for (int c = 0; c < PROBE_CH; ++c) v[c] = 1.0 + 1e-3 * c;
  unsigned fast = 0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < PROBE_CH; ++c) {
      double r;
      if (int_add_f64_ge(v[c], b, &r)) ++fast;
      else r = ArithF64Fma::add(v[c], b);
      // back to [1, 2): keep the sum's low 32 significand bits, reset the exponent and high bits
      v[c] = __hiloint2double(0x3FF00000, __double2loint(r));
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < PROBE_CH; ++c) s = __dadd_rn(s, v[c]);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  atomicAdd(out_fast, (unsigned long long)fast);
}

// The any-sign integer-pipe addition (common.cuh int_add_f64_any) on pairs of
// unlike signs: each chain adds a small value of alternating sign to a running
// value of about 1 and resets the exponent as above, so every addition is a
// true subtraction or addition of magnitudes and none leaves the fast path.
__global__ void __launch_bounds__(PROBE_THREADS) probe_int_add_any_kernel(int iters, double* __restrict__ out) {
  double v[PROBE_CH];
  const double b = 0.001 * (1.0 + threadIdx.x * 1e-3);
#pragma unroll
  for (int c = 0; c < PROBE_CH; ++c) v[c] = (c & 1) ? -(1.0 + 1e-3 * c) : 1.0 + 1e-3 * c;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < PROBE_CH; ++c) {
      const double bb = (it & 1) ? b : -b;
      double r;
      if (!int_add_f64_any(v[c], bb, &r)) r = ArithF64Fma::add(v[c], bb);
      v[c] = __hiloint2double((__double2hiint(r) & 0x80000000) | 0x3FF00000, __double2loint(r));
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < PROBE_CH; ++c) s = __dadd_rn(s, v[c]);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Device-to-device copy of n 16-byte vectors (grid-stride): DRAM read + write bandwidth.
__global__ void __launch_bounds__(PROBE_THREADS) probe_copy_kernel(const double2* __restrict__ src,
                                                                   double2* __restrict__ dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

}  // namespace stn

using namespace stn;

extern "C" int stencil_probe_throughput(stencil_ctx* ctx, size_t copy_bytes, stencil_probe_result* out) {
  if (!ctx || !out) return STENCIL_ERR_ARG;
  ctx->err.clear();
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  *out = stencil_probe_result{};
  int clk = 0;
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, ctx->device);
  out->sm_count = ctx->sm_count;
  out->clock_khz = clk;
  const int blocks = ctx->sm_count * (2048 / PROBE_THREADS);  // 32 warps per SM
  const size_t nthr = (size_t)blocks * PROBE_THREADS;
  int status;
  unsigned char* scratch = (unsigned char*)ws_get(ctx, SLOT_TUNE_GRID, nthr * sizeof(double) + 64, &status);
  if (!scratch) return status;
  unsigned long long* d_fast = (unsigned long long*)(scratch + nthr * sizeof(double));
  cudaEvent_t e0, e1;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return cuda_err(ctx, e, "cudaEventCreate");
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_err(ctx, e, "cudaEventCreate");
  }
  const int iters = 4096;
  const double ops = (double)nthr * PROBE_CH * iters;
  auto timed = [&](auto launch) -> double {
    launch();  // warm-up
    cudaEventRecord(e0, 0);
    launch();
    cudaEventRecord(e1, 0);
    if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ctx->launches += 2;
    return ms * 1e-3;
  };
  double t = timed([&] { probe_fp64_kernel<<<blocks, PROBE_THREADS>>>(iters, (double*)scratch); });
  out->fp64_ops_per_s = t > 0 ? ops / t : 0.0;
  t = timed([&] { probe_fp32_kernel<<<blocks, PROBE_THREADS>>>(iters, (float*)scratch); });
  out->fp32_ops_per_s = t > 0 ? ops / t : 0.0;
  t = timed([&] { probe_alu_kernel<<<blocks, PROBE_THREADS>>>(iters, (unsigned*)scratch); });
  out->alu_ops_per_s = t > 0 ? ops / t : 0.0;
  const int iters_add = 512;
  e = cudaMemset(d_fast, 0, sizeof(unsigned long long));
  if (e == cudaSuccess)
    t = timed([&] { probe_int_add_kernel<<<blocks, PROBE_THREADS>>>(iters_add, (double*)scratch, d_fast); });
  unsigned long long fast = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&fast, d_fast, sizeof(fast), cudaMemcpyDeviceToHost);
  const double adds = (double)nthr * PROBE_CH * iters_add;
  out->int_add_f64_per_s = t > 0 ? adds / t : 0.0;
  out->int_add_fast_fraction = fast / (2.0 * adds);  // warm-up and timed launch both counted
  if (e == cudaSuccess) {
    t = timed([&] { probe_int_add_any_kernel<<<blocks, PROBE_THREADS>>>(iters_add, (double*)scratch); });
    out->int_add_any_f64_per_s = t > 0 ? adds / t : 0.0;
  }
  if (e == cudaSuccess && copy_bytes >= 32) {
    const size_t n = copy_bytes / 2 / sizeof(double2);
    double2* buf = (double2*)ws_get(ctx, SLOT_JACOBI_TMP, 2 * n * sizeof(double2), &status);
    if (!buf) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return status;
    }
    e = cudaMemset(buf, 0, 2 * n * sizeof(double2));
    const int cblocks = ctx->sm_count * 8;
    t = timed([&] { probe_copy_kernel<<<cblocks, PROBE_THREADS>>>(buf, buf + n, n); });
    out->copy_bytes_per_s = t > 0 ? 2.0 * n * sizeof(double2) / t : 0.0;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(ctx, e, "throughput probes");
  return STENCIL_OK;
}
