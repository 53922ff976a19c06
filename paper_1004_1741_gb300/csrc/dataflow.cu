// Persistent dataflow execution of the skewed-tile schedule (tiles.h) for one
// or many grids in a single launch.
//
// The tasks of all grids are listed in one queue in order of their level
// (tasks of equal level from all grids side by side), which is a topological
// order of their dependencies.  Each CTA of a persistent grid takes the next
// task from an atomic counter, waits until the tasks it depends on have
// published their completion flags, runs the task body (task_bodies.cuh) and
// publishes its own flag.  A task only waits on tasks earlier in the queue,
// which some running CTA has already taken, so the wait always ends; it is
// nevertheless bounded by a time limit, after which the kernel records
// STENCIL_ERR_TIMEOUT in an error word and every CTA leaves.
//
// Dependencies of task (I, J, K, p): its three backward face neighbours of
// pass p and, of pass p-1, itself and its three forward face neighbours
// (nt = 1) or the eight tiles (I+a, J+b, K+c), a, b, c in {0, 1}, whose
// shifted tiles end inside its box (nt > 1).  Any execution order that
// respects them reproduces the serial sweeps bit for bit (checked on the CPU
// over random orders).  Compared with one kernel launch per level this removes
// the launch boundaries and the idle tail of every level.
#include <algorithm>
#include <numeric>
#include <type_traits>
#include <vector>

#include "dataflow.cuh"
#include "internal.h"
#include "task_bodies.cuh"
#include "tiles.h"

namespace stn {

template <typename T, int KIND, int W, int H, int D>
__global__ void __launch_bounds__(GS_THREADS) dataflow_kernel(DFRun run, SiteTable tb) {
  // FP64 Jacobi tasks: the adaptive integer-pipe arithmetic, as the tile tasks of the level launches
  using Ar = typename std::conditional<KIND == STENCIL_JACOBI && sizeof(T) == 8, AdaptJacobi,
                                       typename DefaultArith<T>::type>::type;
  __shared__ long long s_q;
  __shared__ int s_off[GS_MAXLEVELS + 1];
  for (;;) {
    if (threadIdx.x == 0) {
      long long q = -1;
      if (*(volatile int*)run.error == 0) {
        const unsigned long long got = atomicAdd(run.counter, 1ULL);
        if ((long long)got < run.ntasks) q = (long long)got;
      }
      if (q >= 0) {
        const int4 tk = run.tasks[q];
        if (!df_wait(run, run.grids[tk.x], tk.y, tk.z & 0xFFFF, tk.z >> 16, tk.w, q)) q = -1;
      }
      s_q = q;
    }
    __syncthreads();
    const long long q = s_q;
    if (q < 0) return;
    const int4 tk = run.tasks[q];
    const DFGridDesc& d = run.grids[tk.x];
    const int I = tk.y, J = tk.z & 0xFFFF, K = tk.z >> 16, p = tk.w;
    Coef<T> c;
    c.a = T(0);
    c.b = (T)d.bco;
    c.hh = (T)d.hh;
    const T* f = (const T*)d.f;
    if constexpr (KIND == STENCIL_GS) {
      if (f)
        gs_task_body<T, Ar, true, W, H, D>((T*)d.a, f, d.g, c, tb, d.tg, I, J, K, p, s_off);
      else
        gs_task_body<T, Ar, false, W, H, D>((T*)d.a, f, d.g, c, tb, d.tg, I, J, K, p, s_off);
    } else {
      if (f)
        jacobi_task_body<T, Ar, true, false, W, H, D>((T*)d.a, (T*)d.b, f, d.g, c, d.tg, I, J, K, p);
      else
        jacobi_task_body<T, Ar, false, false, W, H, D>((T*)d.a, (T*)d.b, f, d.g, c, d.tg, I, J, K, p);
    }
    // the body ended with a barrier: all of the task's writes precede the release
    if (threadIdx.x == 0 && q != run.poison) st_release(run.flags + df_flag(d, I, J, K, p), 1u);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename T, int KIND, int W, int H, int D>
static int df_launch(stencil_ctx* ctx, const DFRun& run, const SiteTable& tb, cudaStream_t st) {
  auto kern = dataflow_kernel<T, KIND, W, H, D>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, GS_THREADS, 0);
  if (e != cudaSuccess || per_sm < 1) per_sm = 1;
  long long blocks = (long long)ctx->sm_count * per_sm;
  if (blocks > run.ntasks) blocks = run.ntasks > 0 ? run.ntasks : 1;
  kern<<<(unsigned)blocks, GS_THREADS, 0, st>>>(run, tb);
  ctx->launches++;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(ctx, e, "dataflow_kernel launch");
  return STENCIL_OK;
}

// A plan: the task queue of one batch shape, resident on the device (taken
// from the stream-ordered allocator), plus, once the shape recurs, the CUDA
// graph that resets the flags and runs the persistent kernel.  The grid
// descriptors (pointers, coefficients) are re-uploaded on every call, so the
// same plan and graph serve any grids of the same shapes.
struct DFPlan {
  std::vector<long long> key;
  long long exec_timeout = 0, exec_poison = -2;
  const void* exec_tb = nullptr;
  unsigned char* dev = nullptr;
  size_t bytes = 0;
  size_t b_desc = 0, b_task = 0, b_flag = 0;
  long long ntasks = 0, nflags = 0;
  int n = 0;
  DFRun run{};
  cudaGraphExec_t exec = nullptr;
  unsigned long long last_use = 0;
  unsigned long long uses = 0;  // calls made with this plan
};

static std::vector<DFPlan*>& plans_of(stencil_ctx* ctx) {
  if (!ctx->df_plans) ctx->df_plans = new std::vector<DFPlan*>();
  return *(std::vector<DFPlan*>*)ctx->df_plans;
}

static void plan_free(stencil_ctx* ctx, DFPlan* pl) {
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->dev) {
    cudaFreeAsync(pl->dev, ctx->gstream);  // the plan's work on that stream has completed (its calls block)
    ctx->held -= pl->bytes;
  }
  delete pl;
}

void dataflow_release(stencil_ctx* ctx) {
  if (!ctx->df_plans) return;
  for (DFPlan* pl : plans_of(ctx)) plan_free(ctx, pl);
  delete (std::vector<DFPlan*>*)ctx->df_plans;
  ctx->df_plans = nullptr;
  if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
  ctx->gstream = nullptr;
}

template <typename T>
static int plan_build(stencil_ctx* ctx, DFPlan* pl, int kind, int n, const Geom* geoms, const int* nsweeps, int W,
                      int H, int D, int nt, cudaStream_t st) {
  std::vector<TileGeom> tgs((size_t)n);
  std::vector<long long> lvl_count;
  long long nflags = 0;
  for (int i = 0; i < n; ++i) {
    TileGeom t = make_tile_geom(geoms[i], W, H, D, nt, nsweeps[i]);
    if (nsweeps[i] == 0 || geoms[i].nx == 0 || geoms[i].ny == 0 || geoms[i].nz == 0) t.npass = 0;
    if (t.NI > 0xFFFF || t.NJ > 0xFFFF || t.NK > 0x7FFF)
      return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "grid %d has too many tiles for the task queue", i);
    nflags += (long long)t.NI * t.NJ * t.NK * t.npass;
    if (t.npass > 0 && (long long)lvl_count.size() < t.nlevels) lvl_count.resize((size_t)t.nlevels, 0);
    tgs[(size_t)i] = t;
  }
  for (int i = 0; i < n; ++i) {
    const TileGeom& t = tgs[(size_t)i];
    for (int pp = 0; pp < t.npass; ++pp)
      for (int K = 0; K < t.NK; ++K)
        for (int J = 0; J < t.NJ; ++J)
          for (int I = 0; I < t.NI; ++I) lvl_count[(size_t)(I + J + K + t.cstride * pp)]++;
  }
  std::vector<long long> start(lvl_count.size() + 1, 0);
  for (size_t l = 0; l < lvl_count.size(); ++l) start[l + 1] = start[l] + lvl_count[l];
  const long long ntasks = start.back();
  std::vector<int4> tasks((size_t)ntasks);
  for (int i = 0; i < n; ++i) {
    const TileGeom& t = tgs[(size_t)i];
    for (int pp = 0; pp < t.npass; ++pp)
      for (int K = 0; K < t.NK; ++K)
        for (int J = 0; J < t.NJ; ++J)
          for (int I = 0; I < t.NI; ++I)
            tasks[(size_t)start[(size_t)(I + J + K + t.cstride * pp)]++] = make_int4(i, I, J | (K << 16), pp);
  }
  pl->b_desc = ((size_t)n * sizeof(DFGridDesc) + 255) / 256 * 256;
  pl->b_task = ((size_t)ntasks * sizeof(int4) + 255) / 256 * 256;
  pl->b_flag = ((size_t)nflags * sizeof(unsigned) + 255) / 256 * 256;
  pl->bytes = pl->b_desc + pl->b_task + pl->b_flag + 256;
  if (ctx->budget && ctx->held + pl->bytes > ctx->budget)
    return set_err(ctx, STENCIL_ERR_OOM, "task queue needs %zu bytes; %zu held, budget %zu", pl->bytes, ctx->held,
                   ctx->budget);
  cudaError_t e = cudaMallocAsync(&pl->dev, pl->bytes, st);  // stream-ordered: no device-wide synchronisation
  if (e != cudaSuccess) {
    cudaGetLastError();
    pl->dev = nullptr;
    return set_err(ctx, STENCIL_ERR_OOM, "cudaMalloc(%zu) for the task queue: %s", pl->bytes, cudaGetErrorString(e));
  }
  ctx->held += pl->bytes;
  pl->ntasks = ntasks;
  pl->nflags = nflags;
  pl->n = n;
  e = cudaMemcpyAsync(pl->dev + pl->b_desc, tasks.data(), (size_t)ntasks * sizeof(int4), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // `tasks` goes out of scope
  if (e != cudaSuccess) return cuda_err(ctx, e, "task queue upload");
  DFRun& run = pl->run;
  run.grids = (const DFGridDesc*)pl->dev;
  run.tasks = (const int4*)(pl->dev + pl->b_desc);
  run.ntasks = ntasks;
  run.flags = (unsigned*)(pl->dev + pl->b_desc + pl->b_task);
  run.counter = (unsigned long long*)(pl->dev + pl->b_desc + pl->b_task + pl->b_flag);
  run.error = (int*)(pl->dev + pl->b_desc + pl->b_task + pl->b_flag + 64);
  return STENCIL_OK;
}

// The plan's launch: reset the flags and counters, run the persistent kernel.  capture: record it into
// the plan's CUDA graph (replayed by later calls of the same shape); otherwise launch it directly on the
// context's graph stream (a plan's first call: shapes that never recur pay no capture).
template <typename T>
static int plan_capture(stencil_ctx* ctx, DFPlan* pl, int kind, int W, int H, int D, int nt, const SiteTable& tb,
                        int int_adds, bool any_f, bool pre_f, bool capture = true) {
  cudaStream_t gs = ctx->gstream;
  cudaError_t e = capture ? cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal) : cudaSuccess;
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaStreamBeginCapture");
  int rc = STENCIL_OK;
  e = cudaMemsetAsync(pl->dev + pl->b_desc + pl->b_task, 0, pl->b_flag + 256, gs);
  if (e == cudaSuccess && kind == DF_KIND_GS_COLUMN) {
    rc = df_column_launch<T>(ctx, pl->run, W, H, nt, int_adds, any_f, pre_f, gs);
  } else if (e == cudaSuccess) {
    rc = STENCIL_UNSUPPORTED_TILE;
#define DF_TILE(WW, HH, DD)                                                                          \
  if (W == WW && H == HH && D == DD)                                                                 \
    rc = kind == STENCIL_GS ? df_launch<T, STENCIL_GS, WW, HH, DD>(ctx, pl->run, tb, gs)             \
                            : df_launch<T, STENCIL_JACOBI, WW, HH, DD>(ctx, pl->run, tb, gs);
    DF_TILE(16, 16, 16)
    DF_TILE(32, 8, 8)
    DF_TILE(8, 8, 8)
    DF_TILE(32, 16, 16)
#undef DF_TILE
  }
  if (!capture) {
    if (e != cudaSuccess) return cuda_err(ctx, e, "flag reset");
    if (rc == STENCIL_UNSUPPORTED_TILE)
      return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "dataflow tile %dx%dx%d (supported 16^3, 32x8x8, 8^3, 32x16x16)",
                     W, H, D);
    return rc;
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(gs, &graph);
  if (e != cudaSuccess) return cuda_err(ctx, e, "memset in capture");
  if (rc == STENCIL_UNSUPPORTED_TILE)
    rc = set_err(ctx, STENCIL_ERR_UNSUPPORTED, "dataflow tile %dx%dx%d (supported 16^3, 32x8x8, 8^3, 32x16x16)", W, H,
                 D);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e2 != cudaSuccess) return cuda_err(ctx, e2, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&pl->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaGraphInstantiate");
  ctx->launches--;  // the capture did not launch; each replay counts below
  return STENCIL_OK;
}

// One dataflow run over n grids of one dtype and smoother.  a[i]: the grid
// (GS) or the even-level grid (Jacobi); b[i]: the odd-level grid (Jacobi).
// All grids share the tile and nt; nsweeps, h, f and extents are per grid.
// Ordered after the work already in `st`; blocking: returns once the run is
// done, with its status.
template <typename T>
int dataflow_run(stencil_ctx* ctx, int kind, int n, T* const* a, T* const* b, const T* const* f, const Geom* geoms,
                 const int* nsweeps, const double* h, int W, int H, int D, int nt, long long timeout_ns,
                 long long poison, cudaStream_t st, double bco, int int_adds, bool pre_f) {
  cudaError_t e;
  if (!ctx->gstream) {
    e = cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_err(ctx, e, "cudaStreamCreate");
  }
  if (!ctx->ev) {
    e = cudaEventCreateWithFlags(&ctx->ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_err(ctx, e, "cudaEventCreate");
  }
  if (!ctx->pinned) {
    e = cudaMallocHost(&ctx->pinned, 64);
    if (e != cudaSuccess) return cuda_err(ctx, e, "cudaMallocHost(status word)");
  }
  // ---- find or build the plan of this shape
  bool any_f = false;
  for (int i = 0; f && i < n; ++i) any_f = any_f || f[i] != nullptr;
  // the column-march kernel's shared memory holds an f ring only when some grid has f
  std::vector<long long> key = {(long long)sizeof(T), kind, n, W, H, D, nt, int_adds, any_f ? 1 : 0, pre_f ? 1 : 0};
  for (int i = 0; i < n; ++i) {
    key.push_back(geoms[i].nx);
    key.push_back(geoms[i].ny);
    key.push_back(geoms[i].nz);
    key.push_back(nsweeps[i]);
  }
  std::vector<DFPlan*>& plans = plans_of(ctx);
  DFPlan* pl = nullptr;
  for (DFPlan* c : plans)
    if (c->key == key) pl = c;
  if (!pl) {
    if (plans.size() >= 4) {  // keep the four most recently used
      auto it = std::min_element(plans.begin(), plans.end(),
                                 [](const DFPlan* x, const DFPlan* y) { return x->last_use < y->last_use; });
      plan_free(ctx, *it);
      plans.erase(it);
    }
    pl = new DFPlan();
    pl->key = key;
    int rc = plan_build<T>(ctx, pl, kind, n, geoms, nsweeps, W, H, D, nt, ctx->gstream);
    if (rc) {
      plan_free(ctx, pl);
      return rc;
    }
    plans.push_back(pl);
  }
  pl->last_use = ++ctx->df_clock;
  if (pl->ntasks == 0) return STENCIL_OK;
  SiteTable tb{};
  if (kind == STENCIL_GS) {
    TileGeom tg0 = make_tile_geom(geoms[0], W, H, D, nt, 1);
    int rc = ensure_sites(ctx, tg0, ctx->gstream);
    if (rc) return rc;
    tb = site_table(ctx, tg0);
  }
  pl->run.timeout_ns = timeout_ns;
  pl->run.poison = poison;
  // a plan is captured into a graph at its first call and replayed; with ctx->df_direct_first (the
  // server, whose batch shapes rarely recur) its first call launches directly and a second call captures
  bool direct = false;
  if (!pl->exec || pl->exec_timeout != timeout_ns || pl->exec_poison != poison || pl->exec_tb != tb.coords) {
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    pl->exec = nullptr;
    if (pl->uses == 0 && ctx->df_direct_first) {
      direct = true;
    } else {
      int rc = plan_capture<T>(ctx, pl, kind, W, H, D, nt, tb, int_adds, any_f, pre_f);
      if (rc) return rc;
      pl->exec_timeout = timeout_ns;
      pl->exec_poison = poison;
      pl->exec_tb = tb.coords;
    }
  }
  pl->uses++;
  // ---- descriptors of this call's grids
  std::vector<DFGridDesc> gd((size_t)n);
  long long fbase = 0;
  for (int i = 0; i < n; ++i) {
    DFGridDesc& d = gd[(size_t)i];
    d.a = a[i];
    d.b = b ? b[i] : nullptr;
    d.f = f ? f[i] : nullptr;
    d.g = geoms[i];
    d.tg = make_tile_geom(geoms[i], W, H, D, nt, nsweeps[i]);
    if (nsweeps[i] == 0 || geoms[i].nx == 0 || geoms[i].ny == 0 || geoms[i].nz == 0) d.tg.npass = 0;
    d.bco = bco;
    d.hh = h[i] * h[i];
    d.flag_base = fbase;
    fbase += (long long)d.tg.NI * d.tg.NJ * d.tg.NK * d.tg.npass;
  }
  // order after the caller's stream, upload, replay the graph, read the status
  e = cudaEventRecord(ctx->ev, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->gstream, ctx->ev, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(pl->dev, gd.data(), (size_t)n * sizeof(DFGridDesc), cudaMemcpyHostToDevice, ctx->gstream);
  if (e != cudaSuccess) return cuda_err(ctx, e, "dataflow descriptors");
  if (direct) {
    int rc = plan_capture<T>(ctx, pl, kind, W, H, D, nt, tb, int_adds, any_f, pre_f, false);
    if (rc) return rc;
  } else {
    e = cudaGraphLaunch(pl->exec, ctx->gstream);
    ctx->launches++;
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->pinned, pl->run.error, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->gstream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->gstream);
  if (e != cudaSuccess) return cuda_err(ctx, e, "dataflow run");
  const int* hs = (const int*)ctx->pinned;
  if (hs[0] != 0)
    return set_err(ctx, STENCIL_ERR_TIMEOUT, "dataflow wait timed out (queue index %d of %lld)", hs[1], pl->ntasks);
  return STENCIL_OK;
}

template int dataflow_run<double>(stencil_ctx*, int, int, double* const*, double* const*, const double* const*,
                                  const Geom*, const int*, const double*, int, int, int, int, long long, long long,
                                  cudaStream_t, double, int, bool);
template int dataflow_run<float>(stencil_ctx*, int, int, float* const*, float* const*, const float* const*,
                                 const Geom*, const int*, const double*, int, int, int, int, long long, long long,
                                 cudaStream_t, double, int, bool);

}  // namespace stn
