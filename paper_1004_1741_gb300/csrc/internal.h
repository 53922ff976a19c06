// Internal interfaces between the translation units of the stencil library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "stencil.h"
#include "common.cuh"

namespace stn {

// One device allocation owned by the context, reused across calls.
struct Slot {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// Slots of the workspace (one buffer per purpose).
enum SlotId {
  SLOT_JACOBI_TMP = 0,   // second grid of the out-of-place Jacobi sweep
  SLOT_RED_PARTIALS,     // per-block partial sums of reductions
  SLOT_RED_RESULT,       // final reduction results (a few doubles)
  SLOT_MIX_E32,          // FP32 correction e of the mixed solve
  SLOT_MIX_R32,          // FP32 residual of the mixed solve
  SLOT_MIX_TMP32,        // FP32 second grid for inner Jacobi sweeps
  SLOT_GS_SLICES,        // Gauss-Seidel tile slices (I,J,K by I+J+K)
  SLOT_GS_SITES,         // Gauss-Seidel intra-tile site table
  SLOT_BATCH_DESC,       // batched-launch descriptors
  SLOT_DF_QUEUE,         // dataflow run: grid descriptors, task queue, completion flags
  SLOT_BATCH_TMP,        // batched Jacobi: second grids
  SLOT_TUNE_GRID,        // autotuner: copy of the caller's grid
  SLOT_GS_GOFF,          // Gauss-Seidel site offsets for one grid shape
  SLOT_MG_LEVELS,        // multigrid: correction and right-hand side of every coarse level
  SLOT_MG_R,             // multigrid: residual of the level being restricted
  SLOT_JACOBI_SLABS,     // in-place Jacobi: ring of three z-slabs of new values
  SLOT_F_SCALED,         // FP64 sweeps with f: the products hh*f, computed once per call
  SLOT_MG32_LEVELS,      // mixed multigrid: FP32 correction and right-hand side of every coarse level
  SLOT_MG32_R,           // mixed multigrid: FP32 residual of the level being restricted
  SLOT_COUNT
};

}  // namespace stn

namespace stn {
// A multigrid V-cycle captured as a CUDA graph, for the arguments and workspace in `key`.
struct MGGraph {
  std::vector<int64_t> key;
  cudaGraphExec_t exec = nullptr;
  unsigned long long nlaunch = 0;  // kernels one replay launches
  unsigned long long last_use = 0;
  int uses = 0;                    // calls seen; -1: capture failed, always launch directly
};
// One tile-slice table (tiles (I,J,K) grouped by I+J+K) on the device, for one tile-count shape.
struct SliceEntry {
  int NI = 0, NJ = 0, NK = 0;
  void* dev = nullptr;
  size_t bytes = 0;
  std::vector<int> off;  // host copy of the prefix offsets
  unsigned long long last_use = 0;
};
}  // namespace stn

struct stencil_ctx {
  int device = 0;
  size_t budget = 0;  // 0 = unlimited
  size_t held = 0;
  std::string err;
  stn::Slot slots[stn::SLOT_COUNT];
  // Gauss-Seidel geometry cache key of what SLOT_GS_SITES holds (entries 3..7)
  int64_t gs_key[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  // tile-slice tables of the recently used tile-count shapes (the levels of a multigrid cycle each have
  // their own); `slice_cur` is the one ensure_slices made current
  std::vector<stn::SliceEntry> slices;
  int slice_cur = -1;
  unsigned long long slice_clock = 0;
  // device buffers a captured graph may refer to change only when this counter moves (a workspace slot
  // reallocated, a slice table evicted); multigrid cycles captured as graphs, keyed by it
  unsigned long long ws_gen = 0;
  std::vector<stn::MGGraph> mg_graphs;
  unsigned long long mg_clock = 0;
  cudaStream_t cstream = nullptr;  // stream for capturing multigrid cycles
  int64_t goff_key[6] = {0, 0, 0, 0, 0, 0};  // (W, H, D, nt, sx, sy) of SLOT_GS_GOFF
  int sm_count = 0;
  unsigned long long launches = 0;  // kernels this context has launched
  void* pinned = nullptr;           // small pinned host buffer for status words
  long long df_timeout_ns = 10000000000LL;  // bound on every dataflow wait
  long long df_poison = -1;                 // failure tests: queue index never published
  void* df_plans = nullptr;                 // cached dataflow plans (dataflow.cu)
  unsigned long long df_clock = 0;
  cudaStream_t gstream = nullptr;           // stream for graph capture and replay
  bool df_direct_first = false;             // dataflow plans: launch a shape's first call without a graph
  cudaEvent_t ev = nullptr;
};

namespace stn {

int set_err(stencil_ctx* ctx, int code, const char* fmt, ...);
int cuda_err(stencil_ctx* ctx, cudaError_t e, const char* where);
// Returns a device buffer of at least `bytes` for slot `id` (growing it if
// needed within the budget), or nullptr with ctx->err set.
void* ws_get(stencil_ctx* ctx, SlotId id, size_t bytes, int* status);
// The same for optional workspace: nullptr, and no error recorded, when the
// budget or the device has no room (the caller then takes a path without it).
void* ws_try(stencil_ctx* ctx, SlotId id, size_t bytes);
int check_dims(stencil_ctx* ctx, const int64_t dims[3], Geom* g);

// --- launchers (return STENCIL_* status) ---
template <typename T>
int jacobi_run(stencil_ctx* ctx, T* u, const T* f, const Geom& g, double h, int nsweeps,
               const stencil_params* p, cudaStream_t st);
template <typename T>
int gs_run(stencil_ctx* ctx, T* u, const T* f, const Geom& g, double h, int nsweeps,
           const stencil_params* p, cudaStream_t st);
// red-black Gauss-Seidel sweeps (gs_rb.cu; params: b only)
template <typename T>
int gs_rb_run(stencil_ctx* ctx, T* u, const T* f, const Geom& g, double h, int nsweeps, const stencil_params* p,
              cudaStream_t st);
// g[i] = hh * f[i] over n elements, with the site update's multiplication (ArithPreF sweeps then add g as
// it is and give the same bits); one grid-stride launch on st.
cudaError_t prescale_f(const double* f, double* g, size_t n, double hh, int sm_count, cudaStream_t st);

// Batched Jacobi, one sweep per pass: one launch per sweep over all grids (batched_jacobi.cu)
template <typename T>
int batched_jacobi_zmarch(stencil_ctx* ctx, int n, T* const* u, const T* const* f, const Geom* geoms,
                          const double* h, const int* nsweeps, double bco, int int_adds, int by, int zchunk,
                          cudaStream_t st);
// Jacobi in place without a second grid (jacobi_inplace.cu; stencil_params variant 6)
template <typename T>
int jacobi_inplace_run(stencil_ctx* ctx, T* u, const T* f, const Geom& g, double h, int nsweeps,
                       const stencil_params* p, cudaStream_t st);
// column-march Gauss-Seidel, one sweep per task (gs_column.cu); zero tile extents: defaults; pre_f: f holds
// hh*f (Ar is then an ArithPreF, and the persistent form takes int_adds 0 or 2)
template <typename T, class Ar>
int gs_column_run(stencil_ctx* ctx, T* u, const T* f, const Geom& g, Coef<T> c, int tx, int ty, int tz,
                  int nsweeps, bool persistent, int int_adds, double h, cudaStream_t st, bool pre_f = false);

// Residual r = f - A u; optional FP64 r and/or FP32 r32 on the interior;
// sums of r^2 and f^2 into the context's result slot (device) when `norm`
// (else FP64 r only, no sums); returns status.  `result` receives the device
// pointer of the two sums.
int residual_launch(stencil_ctx* ctx, const double* u, const double* f, const Geom& g, double h,
                    double* r_out, float* r32_out, double** result, cudaStream_t st, bool norm = true);
// FP32 residual r = f - A u on the interior (every operation in binary32), no norm: the FP32 multigrid levels
int residual32_launch(stencil_ctx* ctx, const float* u, const float* f, const Geom& g, double h, float* r_out,
                      cudaStream_t st);
// copies the two sums of residual_launch to the host (blocking)
int read_sums(stencil_ctx* ctx, const double* dres, double* sums, cudaStream_t st);
// u[interior] += (double) e[interior]
int correct_launch(stencil_ctx* ctx, double* u, const float* e, const Geom& g, cudaStream_t st);

constexpr int STENCIL_UNSUPPORTED_TILE = 1;
// default number of FP64 neighbour-sum additions done on the integer pipes,
// the balance of the FP64 pipe against the (half-rate) integer ALU pipe
// measured at 400^3, 100 sweeps: Jacobi z-march (32x4) 81 GLUP/s at 0, 121 at
// 2, 148 at 3, 129 at 4; Gauss-Seidel column march (8x8, persistent) 105 at 2,
// 103 at 3; Gauss-Seidel tile tasks 66 at 0, 71 at 1, 70.5 at 2
constexpr int kDefaultIntAdds = 1;
// int_adds = 6: the adaptive form (ArithAdaptive): per warp and update, 3 (Jacobi z-march) or 2
// (column march) integer-pipe additions when the neighbours are non-negative, else the additions on
// the FP64 pipe and the multiplication on the integer path; the FP64 default of both families
constexpr int kIntAddsAdaptive = 6;
constexpr int kDefaultIntAddsJacobi = kIntAddsAdaptive;
constexpr int kDefaultIntAddsColumn = kIntAddsAdaptive;
using AdaptJacobi = ArithAdaptive<ArithF64Mix<0x12u>, ArithF64Mix<0x1Fu, true>>;
using AdaptJacobiPre = ArithAdaptive<ArithPreF<ArithF64Mix<0x12u>>, ArithPreF<ArithF64Mix<0x1Fu, true>>>;
using AdaptColumn = ArithAdaptive<ArithF64Mix<0x15u>, ArithF64Mix<0x1Fu, true>>;
using AdaptColumnPre = ArithAdaptive<ArithPreF<ArithF64Mix<0x15u>>, ArithPreF<ArithF64Mix<0x1Fu, true>>>;
void dataflow_release(stencil_ctx* ctx);  // internal: no kernel instantiated for a tile shape

// Persistent dataflow run of the skewed-tile schedule over n grids (dataflow.cu).
template <typename T>
int dataflow_run(stencil_ctx* ctx, int kind, int n, T* const* a, T* const* b, const T* const* f, const Geom* geoms,
                 const int* nsweeps, const double* h, int W, int H, int D, int nt, long long timeout_ns,
                 long long poison, cudaStream_t st, double bco = 1.0 / 6.0, int int_adds = 0,
                 bool pre_f = false);
// task kind of dataflow_run beside STENCIL_JACOBI / STENCIL_GS: the column-march
// Gauss-Seidel task (gs_column.cu; nt = 1, tile W x H columns x D planes)
constexpr int DF_KIND_GS_COLUMN = 16;
struct DFRun;
// launch of the persistent column-march kernel for one dataflow run (gs_column.cu); pre_f: the grids' f
// arrays hold hh*f (offered at int_adds 0, 2 and 6); nt > 1: tasks of nt sweeps each (gs_column_ns.cuh)
template <typename T>
int df_column_launch(stencil_ctx* ctx, const DFRun& run, int tx, int ty, int nt, int int_adds, bool any_f, bool pre_f,
                     cudaStream_t st);

// Column march with NS = 2..4 sweeps per task (gs_column_ns.cuh; instantiated per NS in gs_column_ns<NS>.cu):
// level launches or one persistent dataflow launch; tiles 8x8 and 16x8
template <typename T, class Ar, int NS>
int gs_column_ns_run(stencil_ctx* ctx, T* u, const T* f, const Geom& g, Coef<T> c, int tx, int ty, int tz,
                     int nsweeps, bool persistent, int int_adds, double h, cudaStream_t st, bool pre_f);
template <typename T, int NS>
int df_column_ns_launch(stencil_ctx* ctx, const DFRun& run, int tx, int ty, int int_adds, bool any_f, bool pre_f,
                        cudaStream_t st);

}  // namespace stn
