/*
 * stencil.h - C ABI of the GB300 library for the 3D 7-point Jacobi and
 * lexicographic Gauss-Seidel smoothers with temporal blocking.
 *
 * The operations follow Treibig, Wellein, Hager, "Efficient multicore-aware
 * parallelization strategies for iterative stencil computations" (2010):
 * the Jacobi sweep of Sec. 3 (first listing), the lexicographic Gauss-Seidel
 * sweep of Sec. 3 (second listing), temporal blocking that applies several
 * sweeps per pass over memory (Sec. 4) and the pipeline-parallel Gauss-Seidel
 * that keeps the serial update order (Sec. 3, Fig. pipeline_gs).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  Grid layout.  A grid with interior extents dims = {nx, ny, nz} is stored as
 *  (nz+2)*(ny+2)*(nx+2) contiguous elements in C order, element (i, j, k) of
 *  the padded array at offset (k*(ny+2) + j)*(nx+2) + i, i fastest (the
 *  paper's src[k][j][i]).  Padded index 0 and n+1 in each dimension form a
 *  one-cell Dirichlet halo that is read and never written.  The halo's edges
 *  and corners are never read.  Extents may be 0 (nothing to do); each must
 *  be <= 2^20 and the padded element count < 2^40.
 *
 *  Site update.  With S = ((((W + E) + S_) + N) + B) + T the six neighbours
 *  added left to right in the listing's order (W = i-1, E = i+1, S_ = j-1,
 *  N = j+1, B = k-1, T = k+1):
 *      Laplace (f == NULL):  u' = b * S
 *      Poisson (f != NULL):  u' = b * (S + hh * f)        hh = h*h
 *      weighted Jacobi:      u' = a * u + b * (...)       (a != 0 only)
 *  b = 1/6 rounded to the working precision unless given.  Poisson means
 *  -Lap_h u = f.  Every + and * is one IEEE-754 round-to-nearest operation,
 *  never contracted, so results are bit-identical to the serial loops.
 *
 *  Pointers.  u and f are DEVICE pointers (cudaMalloc'd or equivalent) owned
 *  by the caller; the library never frees them.  Host pointers are named
 *  out_* or say "host".
 *
 *  Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy
 *  default stream).  Calls are stream-ordered and asynchronous unless they
 *  return a value through a host out-parameter, in which case they
 *  synchronise the stream before returning.  A context's workspace (second
 *  grids, h^2 f products, task tables) is shared by its calls: calls on one
 *  context must be ordered with each other (one stream, or streams the
 *  caller orders with events); concurrent streams take a context each.
 *
 *  Errors.  Every int-returning call returns STENCIL_OK (0) or a negative
 *  STENCIL_ERR_* code; stencil_last_error(ctx) then describes the failure.
 *  Argument errors are detected on the host before anything is enqueued.
 *  After STENCIL_ERR_CUDA the caller's arrays may be partially updated.
 *
 *  Threads.  A context may be used by one host thread at a time.
 */
#ifndef STENCIL_H_
#define STENCIL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define STENCIL_OK 0
#define STENCIL_ERR_ARG (-1)           /* invalid argument (NULL, negative size, bad enum)  */
#define STENCIL_ERR_OOM (-2)           /* workspace would exceed the budget, or cudaMalloc  */
#define STENCIL_ERR_CUDA (-3)          /* a CUDA runtime call or kernel launch failed       */
#define STENCIL_ERR_TIMEOUT (-4)       /* a bounded device-side wait expired                */
#define STENCIL_ERR_NOT_CONVERGED (-5) /* a solve stopped at its cap; outputs still valid   */
#define STENCIL_ERR_UNSUPPORTED (-6)   /* valid request the library does not implement     */
#define STENCIL_ERR_CANCELLED (-7)     /* a served request was cancelled before admission   */

#define STENCIL_JACOBI 0
#define STENCIL_GS 1
#define STENCIL_GS_RB 2 /* red-black Gauss-Seidel: multigrid smoother only */

#define STENCIL_F64 0
#define STENCIL_F32 1

typedef struct stencil_ctx stencil_ctx;

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the device
 * memory the context itself allocates (workspace, task tables); 0 = no cap.
 * *out receives the context.  Fails with STENCIL_ERR_CUDA if the device
 * cannot be used, STENCIL_ERR_ARG if out is NULL. */
int stencil_create(stencil_ctx** out, int device, size_t hbm_budget_bytes);

/* Release the context and its device memory (synchronises the device).
 * NULL is ignored. */
void stencil_destroy(stencil_ctx* ctx);

/* Text of the last error on this context; never NULL; valid until the next
 * call on the context.  With ctx == NULL, the last error of stencil_create
 * or residual_norm_noalloc on the calling thread. */
const char* stencil_last_error(const stencil_ctx* ctx);

/* Bytes the context currently holds on the device. */
size_t stencil_workspace_bytes(const stencil_ctx* ctx);

/* Number of CUDA kernels this context has launched so far (a counter for
 * benchmarks: every kernel launch of every entry point adds one). */
unsigned long long stencil_kernel_launches(const stencil_ctx* ctx);

/* Tuning of one smoother call (fields 0 = library default, except int_adds,
 * where 0 puts every addition on the FP64 pipe and -1 is the default: set it
 * to -1 in a zero-initialised struct).
 *  nt      sweeps applied per pass over device memory (temporal blocking,
 *          Sec. 4); 1 = one sweep per pass.  Range 1..16.
 *  tile_x, tile_y, tile_z
 *          tile extents (Jacobi: thread-block tile in x, y; z chunk length.
 *          Gauss-Seidel: task tile W, H, D).  Must be supported by the build,
 *          else STENCIL_ERR_UNSUPPORTED.
 *  a, b    weights of the site update; b == 0 means 1/6.  a != 0 is only
 *          accepted by Jacobi (weighted Jacobi, a = 1 - omega, b = omega/6).
 *  variant kernel variant: 0 = default; Gauss-Seidel 1 = tile staged in
 *          shared memory, 2 = tile updated in place through the L1 cache
 *          (one launch per tile level), 4 = column march: tasks of
 *          tile_x x tile_y columns x tile_z planes, one thread per column
 *          marching up the tile-local wavefront through a shared-memory ring
 *          (one launch per task level); nt = 1: tiles 8x8, 8x16, 16x8;
 *          nt = 2..4: tiles 8x8, 16x8, every task applying its nt sweeps in
 *          one march (sweep s on the tile shifted by -s, two steps behind
 *          sweep s-1; FP64 int_adds 0, 2 or 6);
 *          5 = the column march as one persistent dataflow launch over the
 *          tasks (blocking, like 3; no launch boundary between levels);
 *          Gauss-Seidel default: variant 4 at nt = 1..4 without a tile (8x8
 *          for FP64, 16x8 for FP32, chunks of at most 100 planes, 16 for
 *          calls of fewer than 8 sweeps), variant 2 otherwise (up to
 *          nt = 16; variant 1 takes FP64 up to nt = 8);
 *          3 (both smoothers) = one persistent
 *          dataflow launch over a dependency-ordered task queue (blocking);
 *          Jacobi 1 = z-march, 2 = z-march with asynchronous plane copies,
 *          4 = FP32 temporal blocking on chip (nt <= 4, tile_y 16 or 32),
 *          6 = in place without a second grid (nt = 1, tile_y 4 or 8):
 *          z-slabs of tile_z planes (default 32) are computed into a ring
 *          of three slab buffers and copied back two slabs behind
 *          (workspace 3 tile_z planes instead of a whole grid).
 *          Jacobi default: FP32 unweighted sweeps with nt <= 4 run variant 4
 *          (at nt = 1 only when tile_y is 0); FP64, weighted and the rest
 *          run the z-march at nt = 1 and skewed tiles at nt > 1.
 *          Every variant gives the same bits.
 *  int_adds FP64 only: how many of the five additions of the neighbour sum
 *          are computed on the integer pipes (exact binary64 addition in
 *          integer arithmetic for positive operands, falling back to the
 *          FP64 pipe for operands it does not cover): 0 = all on the FP64
 *          pipe ... 5 = all five on the integer pipes; 6 = adaptive: per warp
 *          and update, 3 (Jacobi z-march) or 2 (column march) integer-pipe
 *          additions when every neighbour is non-negative, else the additions
 *          on the FP64 pipe and the multiplication by b in exact integer
 *          arithmetic (Poisson iterates take both signs); -1 = the library
 *          default: 6 on the Jacobi z-march (also in place and batched), the
 *          Jacobi skewed-tile tasks (nt > 1; they take 6 or -1 as adaptive,
 *          3 as the fixed 3-addition form, any other value as all on the
 *          FP64 pipe) and the Gauss-Seidel column march, 1 on the other
 *          Gauss-Seidel paths (which take 6 as 1).  Same bits whatever the
 *          value.
 *  FP64 calls with f != NULL and at least two sweeps compute h^2 f once into
 *  a further grid of workspace when the budget has room for it (Jacobi on the
 *  z-march; Gauss-Seidel on the column march at int_adds 0, 2 or 6; batched
 *  calls alike) and add it as it is in every sweep: the same products, one
 *  FP64 multiplication per site and sweep fewer. */
typedef struct stencil_params {
  int nt;
  int tile_x, tile_y, tile_z;
  double a, b;
  int variant;
  int int_adds;
} stencil_params;

/* Jacobi smoother (Sec. 3, first listing; temporal blocking Sec. 4).
 * Applies nsweeps >= 0 sweeps to u in place: after the call u holds the
 * nsweeps-th Jacobi iterate (whatever the parity of nsweeps).  The second
 * array of the out-of-place sweep comes from the context's workspace
 * (one grid's size, or three slabs with variant 6; STENCIL_ERR_OOM beyond the
 * budget).  f: device pointer of
 * the same padded shape, or NULL for f = 0.  h > 0 (used only when f != NULL).
 * params may be NULL. */
int stencil_jacobi(stencil_ctx* ctx, double* u, const double* f, const int64_t dims[3], double h,
                   int nsweeps, void* stream);
int stencil_jacobi_ex(stencil_ctx* ctx, double* u, const double* f, const int64_t dims[3], double h,
                      int nsweeps, const stencil_params* params, void* stream);
int stencil_jacobi_f32(stencil_ctx* ctx, float* u, const float* f, const int64_t dims[3], double h,
                       int nsweeps, const stencil_params* params, void* stream);

/* Lexicographic Gauss-Seidel (Sec. 3, second listing; wavefront temporal
 * blocking Sec. 4).  In place on u, nsweeps >= 0.  Each sweep visits sites in
 * (k, j, i) ascending order: at the moment of an update the i-1, j-1, k-1
 * neighbours hold this sweep's values and i+1, j+1, k+1 the previous
 * sweep's.  The parallel schedule reproduces the serial result bit for bit.
 * The context keeps a task table per (dims, tile, nt, nsweeps) shape (a few
 * KB to MB of device memory).  params->a must be 0. */
int stencil_gs_lex(stencil_ctx* ctx, double* u, const double* f, const int64_t dims[3], double h,
                   int nsweeps, void* stream);
int stencil_gs_lex_ex(stencil_ctx* ctx, double* u, const double* f, const int64_t dims[3], double h,
                      int nsweeps, const stencil_params* params, void* stream);
int stencil_gs_lex_f32(stencil_ctx* ctx, float* u, const float* f, const int64_t dims[3], double h,
                       int nsweeps, const stencil_params* params, void* stream);

/* Red-black Gauss-Seidel (Sec. 3 names it as the usual parallel alternative
 * to the lexicographic order): each sweep updates all sites with (i+j+k)
 * even, then all with (i+j+k) odd (0-based interior coordinates), in place,
 * with the same site update.  u, f, dims, h, nsweeps as stencil_gs_lex;
 * params may be NULL (only b is used).  Two launches per sweep. */
int stencil_gs_rb(stencil_ctx* ctx, double* u, const double* f, const int64_t dims[3], double h, int nsweeps,
                  const stencil_params* params, void* stream);
int stencil_gs_rb_f32(stencil_ctx* ctx, float* u, const float* f, const int64_t dims[3], double h, int nsweeps,
                      const stencil_params* params, void* stream);

/* Residual r = f - A u, A u = (6 u - S) * (1/(h*h)), on the interior (not in
 * the paper; the defect of -Lap_h u = f).  f may be NULL (f = 0).
 * r_out (device, same padded shape, may be NULL): receives r on the
 * interior; its halo is not written.
 * out_abs (host, required): ||r||_2 over the interior, FP64.
 * out_rel (host, may be NULL): ||r||_2 / ||f||_2 (or ||r||_2 when f is NULL
 * or zero).  Blocking: synchronises `stream`.  The reduction has a fixed
 * order for a given dims, so repeated calls give identical bits. */
int residual_norm(stencil_ctx* ctx, const double* u, const double* f, const int64_t dims[3], double h,
                  double* r_out, double* out_abs, double* out_rel, void* stream);

/* Batched smoothing of n independent grids of uneven sizes (not in the
 * paper): Gauss-Seidel, and Jacobi at nt > 1 or variant 1..3, run in ONE
 * persistent kernel launch replayed from a CUDA graph (the tasks of all grids
 * share one dependency-ordered work queue, so small grids fill the GPU
 * together); Jacobi at nt = 1 (variant 0) runs one z-march launch per sweep
 * over the tile columns of every grid that still has sweeps to do.
 * u[i], f[i]: device pointers of grid i (f may be NULL, or f[i] NULL, for
 * f = 0); dims[3i..3i+2] its interior extents; h[i], nsweeps[i] (host
 * arrays).  smoother: STENCIL_JACOBI or STENCIL_GS; dtype: STENCIL_F64 or
 * STENCIL_F32 (u and f are double* or float* accordingly).  Every grid ends
 * exactly as after stencil_jacobi / stencil_gs_lex with the same arguments.
 * params (may be NULL): nt, tile, b and int_adds shared by all grids
 * (defaults nt = 1; Gauss-Seidel at nt = 1, and at nt = 2..4 without a
 * tile or with variant 4/5: column-march tasks of 8x8 columns (16x8 for
 * FP32) x 100 + nt - 1 planes, each task applying its nt sweeps, unless
 * variant is 1..3; else 16^3 tile tasks; Jacobi 32x4 (FP64) or 32x8 (FP32)
 * z-march columns at nt = 1, else 32x8x8 tile tasks; FP64 int_adds: the
 * adaptive form); a must be 0.
 * Jacobi takes a workspace of the total size of the batch, FP64 with f a
 * further one for h^2 f when the budget has room.  Blocking: returns when the
 * batch is done; STENCIL_ERR_TIMEOUT if a bounded device wait expired (the
 * grids are then undefined, the context stays usable). */
int stencil_batched(stencil_ctx* ctx, int n, void* const* u, const void* const* f, const int64_t* dims,
                    const double* h, const int* nsweeps, int smoother, int dtype, const stencil_params* params,
                    void* stream);

/* Multigrid V-cycle solve of -Lap_h u = f (the paper's smoothers inside the
 * solver that Sec. 1 and Sec. 3 name as their setting; the cycle itself is not
 * in the paper and follows the textbook form).  FP64, in place on u (device),
 * f device or NULL (f = 0), dims interior extents, h > 0.
 *  Levels: level 0 is u's grid; while fewer than max_levels (1..32) levels
 *    exist and every extent of the last is odd and >= 3, the next level has
 *    extents (n-1)/2 and spacing 2h (coarse site I on fine site 2I+1).
 *  Cycle: nu1 sweeps of the smoother, r = f - A u, full-weighting
 *    restriction (weights 1/4, 1/2, 1/4 per axis; x, then y, then z), the
 *    coarse correction from zero with zero Dirichlet values (one cycle deeper),
 *    trilinear prolongation added to u (x, then y, then z), nu2 sweeps;
 *    ncoarse sweeps on the coarsest level.
 *  smoother: STENCIL_JACOBI = weighted Jacobi, omega = 6/7 (a = b = 1/7);
 *    STENCIL_GS = lexicographic Gauss-Seidel (b = 1/6); STENCIL_GS_RB =
 *    red-black Gauss-Seidel (b = 1/6, red = (i+j+k) even first).
 *  Runs cycles while ||r||/||f|| (||r0|| if f = 0) > rtol and fewer than
 *  max_cycles ran; *out_rel, *out_cycles (host, may be NULL) get the last
 *  relative residual and the cycles run.  Returns STENCIL_OK or
 *  STENCIL_ERR_NOT_CONVERGED (u holds the last iterate either way).
 *  Workspace: the coarse levels (about 2/7 of u's size) and one residual grid
 *  of u's size, plus the smoothers' own.  Blocking (reads the residual after
 *  every cycle).  Same bits as the serial definition. */
int stencil_mg_solve(stencil_ctx* ctx, double* u, const double* f, const int64_t dims[3], double h, int smoother,
                     int nu1, int nu2, int ncoarse, int max_levels, double rtol, int max_cycles, double* out_rel,
                     int* out_cycles, void* stream);

/* Mixed-precision multigrid solve of -Lap_h u = f (not in the paper: the
 * smoothers of Sec. 3 inside the multigrid solver Sec. 1 and Sec. 3 name,
 * with the bulk of the work on binary32 storage).  Defect correction:
 *   r = f - A u in FP64 (its norm gives the stopping test), r32 = (float) r;
 *   e = 0; inner_cycles V-cycles on A e = r32 entirely in FP32 (the
 *   stencil_mg_solve cycle with every operation in binary32: FP32 residual
 *   r = f - (6u - S) * (float)(1/(h*h)), FP32 smoothers, the same transfers
 *   with float weights); u += (double) e in FP64;
 * until ||r||/||f|| <= rtol (||r0|| if f = 0) or max_outer iterations.
 * u (device, FP64) in place; f device or NULL; dims, h, smoother, nu1, nu2,
 * ncoarse, max_levels as stencil_mg_solve.  *out_rel, *out_iters (host, may
 * be NULL) get the last relative residual and the outer iterations done.
 * Returns STENCIL_OK or STENCIL_ERR_NOT_CONVERGED (u holds the last iterate
 * either way).  Workspace: two FP32 grids of u's size (r32, e), the FP32
 * coarse levels (about 2/7 of an FP32 grid) and one FP32 residual grid, plus
 * the FP32 smoothers' own.  Blocking (reads the residual after every outer
 * iteration).  Same bits as the serial definition. */
int stencil_solve_mixed_mg(stencil_ctx* ctx, double* u, const double* f, const int64_t dims[3], double h,
                           int smoother, int nu1, int nu2, int ncoarse, int max_levels, double rtol, int max_outer,
                           int inner_cycles, double* out_rel, int* out_iters, void* stream);

/* Bound on every device-side wait of the persistent kernels (default 10 s).
 * never_publish >= 0 makes the task at that queue index never publish its
 * completion, so that a test can watch the bound expire and the error come
 * back (STENCIL_ERR_TIMEOUT); pass -1 for normal operation. */
int stencil_set_wait_limit(stencil_ctx* ctx, long long timeout_ns, long long never_publish);

/* Autotuner (not in the paper): times candidate kernel variants, temporal
 * depths nt, tiles and (FP64, one sweep per pass) the integer-pipe form --
 * the adaptive default or the fixed form fastest on non-negative data -- for
 * `smoother` on a copy of the caller's grid u (device, dtype STENCIL_F64/F32;
 * f may be NULL) for nsweeps sweeps and writes the fastest, int_adds
 * included, into *out (and its GLUP/s into *out_glups if not NULL).  u is not
 * modified.  Blocking. */
int stencil_autotune(stencil_ctx* ctx, int smoother, int dtype, const void* u, const void* f, const int64_t dims[3],
                     double h, int nsweeps, stencil_params* out, double* out_glups, void* stream);

/* Autotuner for a batch (not in the paper): times the batched paths' candidate
 * kernel forms, temporal depths nt, tiles and (FP64) integer-pipe forms on
 * copies of the caller's n grids (device u[i], dtype STENCIL_F64/F32; f[i] may
 * be NULL) with their sweep counts, exactly as stencil_batched would run them,
 * and writes the fastest into *out (its whole-batch GLUP/s into *out_glups if
 * not NULL).  The grids are not modified.  Workspace: one copy of the batch.
 * Blocking. */
int stencil_autotune_batched(stencil_ctx* ctx, int n, const void* const* u, const void* const* f, const int64_t* dims,
                             const double* h, const int* nsweeps, int smoother, int dtype, stencil_params* out,
                             double* out_glups, void* stream);

/* ---------------------------------------------------------------------------
 * Continuous-batching server (not in the paper).
 *
 * Two worker threads own one GPU.  A copy thread admits waiting requests in
 * arrival order while their device memory fits hbm_budget_bytes (0 = no cap)
 * and fewer than max_active requests are admitted (0 = no slot limit), takes
 * their grids from a stream-ordered memory pool of the server (no cudaMalloc
 * or cudaFree per request) and copies them to the device on a stream of its
 * own, where they stay until completion, and copies finished grids back.  A
 * compute thread runs rounds over the requests on the device: up to
 * sweeps_per_round sweeps (0 = 10) of every smoothing request -- all requests
 * of one (smoother, dtype) class in ONE batched persistent launch -- and up
 * to sweeps_per_round / 4 multigrid cycles (at least one) of every solve
 * request.  Requests that arrive meanwhile are
 * admitted as memory and slots free up; their copies overlap the rounds'
 * kernels.  A request's result is the same alone and in any mix.
 * ------------------------------------------------------------------------- */
#define STENCIL_PENDING 1 /* poll/wait: the request has not finished yet */

#define STENCIL_REQ_JACOBI 0 /* nsweeps Jacobi sweeps */
#define STENCIL_REQ_GS 1     /* nsweeps Gauss-Seidel sweeps */
#define STENCIL_REQ_SOLVE 2  /* solve until ||f-Au||/||f|| <= rtol (FP64 only): multigrid V(2,2) cycles with the
                              * red-black Gauss-Seidel smoother (stencil_mg_solve, sweeps_per_round sweeps on the
                              * coarsest level) when every extent is odd and >= 3, else lexicographic Gauss-Seidel
                              * sweeps; nsweeps caps the fine-grid sweeps, a cycle counting 4; the residual is
                              * tested after each cycle or round of sweeps */
#define STENCIL_REQ_SOLVE_MIXED 3 /* the same solve with FP32 multigrid V(2,2) cycles (red-black) inside FP64
                                   * defect correction (stencil_solve_mixed_mg, one FP32 cycle per outer
                                   * iteration, the FP64 residual after each) when every extent is odd and
                                   * >= 3, else as STENCIL_REQ_SOLVE; an outer iteration counts 4 sweeps */

typedef struct stencil_server stencil_server;

typedef struct stencil_request {
  int kind;          /* STENCIL_REQ_* */
  int dtype;         /* STENCIL_F64 or STENCIL_F32 (solves: F64) */
  int64_t dims[3];   /* interior extents, each >= 1 */
  double h;          /* mesh width > 0 */
  int nsweeps;       /* sweeps, or the sweep cap of a solve */
  double rtol;       /* solve only */
  const void* u_in;  /* HOST padded grid, read at admission; must stay valid until then */
  const void* f_in;  /* HOST right-hand side or NULL (f = 0) */
  void* u_out;       /* HOST buffer for the result or NULL; written before completion is reported */
} stencil_request;

typedef struct stencil_result {
  int status;          /* STENCIL_OK, STENCIL_ERR_NOT_CONVERGED (solve capped), _CANCELLED, _OOM, ... */
  int sweeps_done;
  double rel_residual; /* solve: final relative residual; else -1 */
  double queue_s;      /* submit -> admission */
  double latency_s;    /* submit -> completion */
} stencil_result;

typedef struct stencil_server_stats {
  uint64_t submitted, admitted, completed, cancelled, launches;
  double p50_s, p99_s, mean_s; /* latency of completed requests */
  double lup_total;            /* lattice-site updates performed */
  double busy_s;               /* wall time of rounds */
  double glups;                /* lup_total / busy_s / 1e9 */
  size_t hbm_in_use, hbm_peak; /* request memory on the device */
  int queue_depth, active;
  double smooth_lup, smooth_s; /* smoothing requests: updates and seconds of their batched launches */
  double solve_cycles, solve_s; /* solve requests: multigrid cycles (mixed: outer iterations; one level: rounds
                                 * of sweeps) and their seconds */
  double copy_bytes, copy_s;    /* bytes copied in and out by the copy thread and the seconds it spent copying */
} stencil_server_stats;

int stencil_server_create(stencil_server** out, int device, size_t hbm_budget_bytes, int sweeps_per_round,
                          int max_active);
/* Enqueue a request (copies the descriptor, not the grids); *ticket identifies it. */
int stencil_server_submit(stencil_server* srv, const stencil_request* req, uint64_t* ticket);
/* STENCIL_OK and *out filled if finished, STENCIL_PENDING if not. */
int stencil_server_poll(stencil_server* srv, uint64_t ticket, stencil_result* out);
/* Blocks up to timeout_s seconds; STENCIL_OK or STENCIL_PENDING. */
int stencil_server_wait(stencil_server* srv, uint64_t ticket, double timeout_s, stencil_result* out);
/* Cancels a request not yet admitted (its result: STENCIL_ERR_CANCELLED); STENCIL_ERR_ARG otherwise. */
int stencil_server_cancel(stencil_server* srv, uint64_t ticket);
int stencil_server_stats_get(stencil_server* srv, stencil_server_stats* out);
/* Stops the worker after the current round and frees everything. */
void stencil_server_destroy(stencil_server* srv);

/* Self-check of the integer-arithmetic binary64 addition and multiplication:
 * n pairs drawn from a counter-based generator seeded by `seed` (random
 * magnitudes, ties, carries, zeros, signs), each summed on the integer pipes
 * (the symmetric form, the ordered form in both argument orders, and the
 * any-sign form in both orders with random signs) and multiplied in integer
 * arithmetic (both orders, random signs), against the FP64 pipe.
 * *out_mismatch (host) receives the number of results whose bits differ (must
 * be 0), *out_fast the number of pairs the symmetric addition handled and,
 * when out_fast_any is not NULL, *out_fast_any the number the any-sign
 * addition handled.  Blocking. */
int stencil_selftest_int_add(stencil_ctx* ctx, uint64_t n, uint64_t seed, uint64_t* out_mismatch,
                             uint64_t* out_fast, uint64_t* out_fast_any);

/* Throughput probes (not in the paper; they measure the roofline's
 * denominators on the GPU at hand): whole-GPU rates of FP64 additions (the
 * smoothers' FMA-form addition, one rounding each), FP32 additions, 32-bit
 * integer ALU instructions (lop3), binary64 additions carried out on the
 * integer pipes (the smoothers' ordered integer-pipe addition on operands in
 * its fast path; int_add_fast_fraction must be 1), the any-sign integer-pipe
 * addition on operands of unlike signs, each from 8 independent dependency
 * chains per thread at 32 warps per SM; and, when copy_bytes >= 32,
 * the DRAM bandwidth of a 16-byte-vector copy kernel over copy_bytes of
 * workspace (read + write bytes per second).  sm_count and clock_khz are the
 * device's (cudaDevAttrClockRate: the maximum SM clock).  Blocking; changes
 * no device setting. */
typedef struct stencil_probe_result {
  double fp64_ops_per_s;
  double fp32_ops_per_s;
  double alu_ops_per_s;
  double int_add_f64_per_s;
  double int_add_fast_fraction;
  double int_add_any_f64_per_s;
  double copy_bytes_per_s;
  int sm_count;
  int clock_khz;
} stencil_probe_result;

int stencil_probe_throughput(stencil_ctx* ctx, size_t copy_bytes, stencil_probe_result* out);

/* residual_norm without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc when they
 * need a residual (an application that owns all device memory through its
 * own allocator, a time-critical loop that must not stall or fragment the
 * heap).  Same arguments,
 * results and reduction order as residual_norm (the same kernels), but no
 * context: the work runs on the calling thread's current CUDA device, and u,
 * f and r_out must be device (or managed) memory of that device; anything
 * else (a host pointer, another device's memory) returns STENCIL_ERR_ARG
 * before any kernel is launched.  The reduction scratch is a fixed array
 * inside the library (512 KiB + 16 B on every device that loads it, held
 * until the process exits), so the grid must satisfy
 *     ceil(nx/32) * ceil(ny/8) * ceil(nz/32) <= 32768
 * (e.g. up to 640^3); larger grids return STENCIL_ERR_ARG with the limit in
 * stencil_last_error(NULL).  Each call looks up the array's address in the
 * current context.  Every call reuses the same array: calls that overlap on
 * the GPU (two streams, two host threads on one device) race and must be
 * serialised by the caller.  Blocking: synchronises `stream`.  Errors are
 * reported through stencil_last_error(NULL), which each call clears first. */
int residual_norm_noalloc(const double* u, const double* f, const int64_t dims[3], double h, double* r_out,
                          double* out_abs, double* out_rel, void* stream);

/* Mixed-precision Poisson solve by defect correction (not in the paper):
 *   repeat: r = f - A u (FP64); e = 0; inner_sweeps FP32 sweeps of
 *   `smoother` (STENCIL_JACOBI or STENCIL_GS) on A e = (float) r;
 *   u += (double) e;  until ||r||/||f|| <= rtol or max_outer iterations.
 * u (device, FP64) is updated in place; f (device, FP64) required.
 * Workspace: one FP64 and two FP32 grids.  out_rel / out_iters (host, may be
 * NULL) receive the final relative residual and the outer iterations done.
 * Returns STENCIL_ERR_NOT_CONVERGED (outputs valid) if rtol was not reached.
 * Blocking. */
int stencil_solve_mixed(stencil_ctx* ctx, double* u, const double* f, const int64_t dims[3], double h,
                        int smoother, double rtol, int max_outer, int inner_sweeps,
                        double* out_rel, int* out_iters, void* stream);

/* FP64-only solve by plain sweeps of `smoother` for comparison: the residual
 * is checked every check_every sweeps until rel <= rtol or max_sweeps.
 * out_sweeps (host, may be NULL) receives the sweeps done.  Blocking. */
int stencil_solve_f64(stencil_ctx* ctx, double* u, const double* f, const int64_t dims[3], double h,
                      int smoother, double rtol, int max_sweeps, int check_every, const stencil_params* params,
                      double* out_rel, int* out_sweeps, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* STENCIL_H_ */
