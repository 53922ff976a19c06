// Device side of the persistent dataflow execution (dataflow.cu): grid
// descriptors, the task queue, completion flags with release/acquire
// ordering, and the bounded wait of a task for its dependencies.
#pragma once

#include "internal.h"
#include "tiles.h"

namespace stn {

struct DFGridDesc {
  void* a;        // Gauss-Seidel: the grid; Jacobi: grid of even levels
  void* b;        // Jacobi: grid of odd levels
  const void* f;  // right-hand side or nullptr
  Geom g;
  TileGeom tg;
  double bco, hh;
  long long flag_base;
};

struct DFRun {
  const DFGridDesc* grids;
  const int4* tasks;  // x = grid, y = I, z = J | K << 16, w = p
  long long ntasks;
  unsigned int* flags;
  unsigned long long* counter;
  int* error;  // [0] status (0 or STENCIL_ERR_TIMEOUT), [1] queue index that gave up
  long long timeout_ns;
  long long poison;  // queue index whose completion is never published (failure tests), -1 = none
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ long long df_flag(const DFGridDesc& d, int I, int J, int K, int p) {
  const TileGeom& t = d.tg;
  return d.flag_base + (((long long)p * t.NK + K) * t.NJ + J) * t.NI + I;
}

// Thread 0: wait until every dependency of the task is published; false on timeout/error.
__device__ inline bool df_wait(const DFRun& run, const DFGridDesc& d, int I, int J, int K, int p, long long qi) {
  long long deps[11];
  int n = 0;
  if (I > 0) deps[n++] = df_flag(d, I - 1, J, K, p);
  if (J > 0) deps[n++] = df_flag(d, I, J - 1, K, p);
  if (K > 0) deps[n++] = df_flag(d, I, J, K - 1, p);
  if (p > 0) {
    const TileGeom& t = d.tg;
    if (t.nt == 1) {
      deps[n++] = df_flag(d, I, J, K, p - 1);
      if (I + 1 < t.NI) deps[n++] = df_flag(d, I + 1, J, K, p - 1);
      if (J + 1 < t.NJ) deps[n++] = df_flag(d, I, J + 1, K, p - 1);
      if (K + 1 < t.NK) deps[n++] = df_flag(d, I, J, K + 1, p - 1);
    } else {
      for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
          for (int a = 0; a < 2; ++a)
            if (I + a < t.NI && J + b < t.NJ && K + c < t.NK) deps[n++] = df_flag(d, I + a, J + b, K + c, p - 1);
    }
  }
  const long long t0 = global_ns();
  for (int i = 0; i < n; ++i) {
    const unsigned* fl = run.flags + deps[i];
    unsigned spins = 0;
    while (ld_acquire(fl) == 0u) {
      if ((++spins & 63u) == 0u) {
        if (*(volatile int*)run.error != 0) return false;
        if (global_ns() - t0 > run.timeout_ns) {
          if (atomicCAS(run.error, 0, STENCIL_ERR_TIMEOUT) == 0) run.error[1] = (int)qi;
          return false;
        }
      }
      __nanosleep(64);
    }
  }
  return true;
}

}  // namespace stn
