// Lexicographic Gauss-Seidel, one sweep per task, as a column march
// (Sec. 3's pipelined wavefront with every thread owning one (x, y) column).
//
// Tasks are the nt = 1 tiles of tiles.h: box tiles TX x TY columns x D planes,
// task (I, J, K, p) = sweep p of tile (I, J, K), level I+J+K+2p, one launch
// per level; tasks of one level never share a face, so they run in parallel.
// Inside a task the sites of the tile-local wavefront i+j+k = t are exactly
// "column (i, j) at plane t-i-j": thread (i, j) marches up its column, one
// plane per step, i+j steps behind the tile's corner column.
//
// The tile lives in a shared-memory ring of R plane slots, each holding the
// tile's TY rows plus the two neighbouring rows, each row the TX columns plus
// the two neighbouring columns.  Cell (i, j, k) (tile column i, row j, local
// plane k; -1 and TX / TY for the neighbours) is stored in slot (k+i+j) mod R,
// the step at which it is updated: at step t every thread reads slot t-1 (W,
// S, B, all updated one step earlier), slot t+1 (E, N, T, not yet updated)
// and writes slot t, the same three slots for the whole CTA.  Row y of plane
// z enters the ring as one coalesced line (cp.async, at least PF+1 steps
// before its first reader), sites are updated in place, and a finished row
// leaves as one coalesced line after its last reader.  In-place updating is
// exact for the same reason as in the grid.  Neighbour rows, columns and
// planes outside the tile belong to tiles one level below (W, S, B: swept)
// or above (E, N, T: not yet swept): they are loaded like the tile's own
// lines and never written back.
#include <type_traits>

#include "dataflow.cuh"
#include "internal.h"
#include "tiles.h"

namespace stn {

constexpr int kColPF = 2;  // steps of copies in flight ahead of their first reader
// Ring depth: a cell's slot is refilled only after its row has been written
// back: a row line lives from its copy (PF+1 steps before its first reader)
// to its write-back (TX+2 steps after), so R = TX + PF + 4 slots.
__host__ __device__ constexpr int col_ring_slots(int tx) { return tx + kColPF + 4; }
// Row pitch: the TX columns and their two neighbours.  (In 8-wide tiles a
// half-warp's two rows then share some 8-byte banks; layouts that avoid it
// measured slower or equal, and the smaller ring keeps more CTAs resident.)
__host__ __device__ constexpr int col_row_pitch(int tx) { return tx + 2; }
// Shared memory of one task: the ring of u (halo rows and columns included)
// and, with a right-hand side, a ring of f (interior cells only, same slots).
template <typename T, int TX, int TY>
constexpr size_t col_smem_bytes(bool has_f) {
  return (size_t)col_ring_slots(TX) * ((TY + 2) * col_row_pitch(TX) + (has_f ? TX * TY : 0)) * sizeof(T);
}

// The task (I, J, K, p): sweep p of tile (I, J, K) in place on u; all threads
// of the CTA (TX x TY) take part; ring: col_smem_bytes(HAS_F) of shared memory.
// Returns after a barrier, with all of the task's global writes issued.
template <typename T, class Ar, bool HAS_F, int TX, int TY>
__device__ __forceinline__ void gs_column_body(T* u, const T* __restrict__ f, const Geom& g, const Coef<T>& c,
                                               const TileGeom& tg, int I, int J, int K, T* ring) {
  static_assert(TX >= 2 && TY >= 2, "tile of at least 2 x 2 columns");
  constexpr int PF = kColPF;
  constexpr int R = col_ring_slots(TX);
  constexpr int RW = col_row_pitch(TX), RH = TY + 2;
  constexpr int PL = RW * RH;  // cells per slot
  constexpr int FPL = TX * TY;  // cells per slot of the f ring
  const int i = threadIdx.x, j = threadIdx.y;
  const int x0 = I * TX, y0 = J * TY;
  const int x = x0 + i, y = y0 + j;
  const int z0 = K * tg.D;
  const int nzl = min(g.nz - z0, tg.D);
  const bool comp = x < g.nx && y < g.ny;
  // copies (only elements of the padded grid): own row line (column i+1); the
  // W / E column on the first / last lane (TX >= 2: never both); the S / N
  // row on the first / last row (TY >= 2: never both)
  const bool ldo = x <= g.nx && y <= g.ny;
  const bool ldx = (i == 0 && y <= g.ny) || (i == TX - 1 && x0 + TX <= g.nx && y <= g.ny);
  const bool ldy = (j == 0 && x <= g.nx) || (j == TY - 1 && y0 + TY <= g.ny && x <= g.nx);
  const int64_t sy = g.sy;
  // At step t: own-row and column copies of plane ql = t - j + 2 + PF into
  // slot t + 2 + PF + i (column W: t + 1 + PF, column E: t + 2 + PF + TX);
  // S row of plane t + 3 + PF and N row of plane t - TY + 2 + PF, both into
  // slot t + 2 + PF + i; update of plane kk = t - i - j in slot t; write-back
  // of plane qw = t - TX - j - 1 from slot t - TX - 1 + i.
  const int ts = -3 - PF;            // first copies: plane -1 of row 0, plane 0 of the S row
  const int te = nzl + TX + TY - 1;  // last write-back
  // step windows (inclusive) of each duty
  const int lo_l = j - 3 - PF, hi_l = j - 2 - PF + nzl;  // own row / columns, planes -1..nzl
  const int lo_y = j == 0 ? -3 - PF : TY - 2 - PF;       // S / N row, planes 0..nzl-1
  const int hi_y = lo_y + nzl - 1;
  const int lo_c = i + j, hi_c = i + j + nzl - 1;        // update
  const int lo_w = TX + j + 1, hi_w = TX + j + nzl;      // write-back, planes 0..nzl-1
  const int lo_f = j - 2 - PF, hi_f = j - 3 - PF + nzl;  // own row of f, planes 0..nzl-1
  auto inwin = [](int t, int lo, int hi) { return (unsigned)(t - lo) <= (unsigned)(hi - lo); };
  auto mod = [](int q) { return ((q % R) + R) % R; };
  // per-thread ring cells (slot 0) and the running slots of copies, update and write-back
  T* const cell = ring + (j + 1) * RW + (i + 1);
  T* const xcell = ring + (j + 1) * RW + (i == 0 ? 0 : TX + 1);
  T* const ycell = ring + (j == 0 ? 0 : TY + 1) * RW + (i + 1);
  T* const fcell = ring + R * PL + j * TX + i;  // f ring: cell (i, j, k) in slot (k+i+j) mod R, like u
  const int xoff = i == 0 ? 1 + PF : 2 + PF + TX;  // column slot - t
  int sl = mod(ts + 2 + PF + i), sx = mod(ts + xoff), sw = mod(ts - TX - 1 + i), st = mod(ts);
  // global pointers at the plane of step ts
  const T* go = u + (ldo ? g.at(x, y, z0) : 0) + (int64_t)(ts - j + 2 + PF) * sy;
  const T* gx = u + (ldx ? g.at(i == 0 ? x0 - 1 : x0 + TX, y, z0) : 0) + (int64_t)(ts - j + 2 + PF) * sy;
  const T* gy = u + (ldy ? g.at(x, j == 0 ? y0 - 1 : y0 + TY, z0) : 0) +
                (int64_t)(j == 0 ? ts + 3 + PF : ts - TY + 2 + PF) * sy;
  T* gw = u + (comp ? g.at(x, y, z0) : 0) + (int64_t)(ts - TX - j - 1) * sy;
  // f: copied with the own row (plane t - j + 2 + PF, same slot), read at the update
  const T* gf = HAS_F ? f + (comp ? g.at(x, y, z0) : 0) + (int64_t)(ts - j + 2 + PF) * sy : nullptr;
  auto wrap = [](int s) { return s == R - 1 ? 0 : s + 1; };
  for (int t = ts; t <= te; ++t) {
    const bool wl = inwin(t, lo_l, hi_l);
    if (ldo && wl) cp_async_elem(cell + sl * PL, go);
    if (ldx && wl) cp_async_elem(xcell + sx * PL, gx);
    if (ldy && inwin(t, lo_y, hi_y)) cp_async_elem(ycell + sl * PL, gy);
    if (HAS_F && comp && inwin(t, lo_f, hi_f)) cp_async_elem(fcell + sl * FPL, gf);
    cp_async_commit();
    if constexpr (AdaptOf<Ar>::on) {  // the whole warp votes (t is uniform; every ring read stays in the ring)
      const bool upd = comp && inwin(t, lo_c, hi_c);
      const int sm1 = st == 0 ? R - 1 : st - 1, sp1 = wrap(st);
      const T* pm = cell + sm1 * PL;
      const T* pp = cell + sp1 * PL;
      const T fv = HAS_F ? fcell[st * FPL] : T(0);
      const T v = site_update_warp<T, Ar, HAS_F, false>(upd, pm[-1], pp[1], pm[-RW], pp[RW], pm[0], pp[0], fv, T(0),
                                                        c);
      if (upd) cell[st * PL] = v;
    } else if (comp && inwin(t, lo_c, hi_c)) {
      const int sm1 = st == 0 ? R - 1 : st - 1, sp1 = wrap(st);
      const T* pm = cell + sm1 * PL;
      const T* pp = cell + sp1 * PL;
      const T fv = HAS_F ? fcell[st * FPL] : T(0);
      const T v = site_update<T, Ar, HAS_F, false>(pm[-1], pp[1], pm[-RW], pp[RW], pm[0], pp[0], fv, T(0), c);
      cell[st * PL] = v;
    }
    if (comp && inwin(t, lo_w, hi_w)) *gw = cell[sw * PL];
    if (HAS_F) gf += sy;
    cp_async_wait<PF>();
    __syncthreads();
    sl = wrap(sl); sx = wrap(sx); sw = wrap(sw); st = wrap(st);
    go += sy; gx += sy; gy += sy; gw += sy;
  }
  cp_async_wait<0>();
  __syncthreads();
}

// One launch per task level (find_task: CTA -> task of the level).
template <typename T, class Ar, bool HAS_F, int TX, int TY>
__global__ void __launch_bounds__(TX * TY) gs_column_kernel(T* u, const T* __restrict__ f, Geom g, Coef<T> c,
                                                            const uint64_t* __restrict__ slices,
                                                            const int* __restrict__ slice_off, TileGeom tg,
                                                            int level) {
  extern __shared__ __align__(16) unsigned char gsc_raw[];
  int I, J, K, p;
  if (!find_task(tg, slices, slice_off, level, &I, &J, &K, &p)) return;
  gs_column_body<T, Ar, HAS_F, TX, TY>(u, f, g, c, tg, I, J, K, reinterpret_cast<T*>(gsc_raw));
}

// Persistent form: each CTA takes the next task of the level-ordered queue,
// waits (bounded) for the tasks it depends on, runs the column march and
// publishes its completion (dataflow.cuh).  No launch boundaries, no idle tail
// per level.
template <typename T, class Ar, int TX, int TY>
__global__ void __launch_bounds__(TX * TY) dataflow_column_kernel(DFRun run) {
  extern __shared__ __align__(16) unsigned char gsc_raw[];
  T* ring = reinterpret_cast<T*>(gsc_raw);
  __shared__ long long s_q;
  const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
  for (;;) {
    if (lead) {
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
    if (d.f)
      gs_column_body<T, Ar, true, TX, TY>((T*)d.a, (const T*)d.f, d.g, c, d.tg, I, J, K, ring);
    else
      gs_column_body<T, Ar, false, TX, TY>((T*)d.a, nullptr, d.g, c, d.tg, I, J, K, ring);
    // the body ended with a barrier after its last writes: they precede the release
    if (lead && q != run.poison) {
      __threadfence();
      st_release(run.flags + df_flag(d, I, J, K, p), 1u);
    }
  }
}

template <typename T, class Ar, bool HAS_F, int TX, int TY>
static int gs_column_levels(stencil_ctx* ctx, T* u, const T* f, const Geom& g, Coef<T> c, int tz, int nsweeps,
                            cudaStream_t st) {
  const TileGeom tg = make_tile_geom(g, TX, TY, tz, 1, nsweeps);
  int rc = ensure_slices(ctx, tg, st);
  if (rc) return rc;
  const uint64_t* slices = slices_ptr(ctx);
  const int* soff = slice_off_ptr(ctx);
  auto kern = gs_column_kernel<T, Ar, HAS_F, TX, TY>;
  const size_t smem = col_smem_bytes<T, TX, TY>(HAS_F);
  cudaError_t e0 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e0 != cudaSuccess) return cuda_err(ctx, e0, "gs_column_kernel shared memory");
  for (int L = 0; L < tg.nlevels; ++L) {
    const int n = tasks_at_level(ctx, tg, L);
    if (n == 0) continue;
    kern<<<n, dim3(TX, TY), smem, st>>>(u, f, g, c, slices, soff, tg, L);
    ctx->launches++;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(ctx, e, "gs_column_kernel launch");
  return STENCIL_OK;
}

template <typename T, class Ar, int TX, int TY>
static int df_column_launch_t(stencil_ctx* ctx, const DFRun& run, bool any_f, cudaStream_t st) {
  auto kern = dataflow_column_kernel<T, Ar, TX, TY>;
  const size_t smem = col_smem_bytes<T, TX, TY>(any_f);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_err(ctx, e, "dataflow_column_kernel shared memory");
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TX * TY, smem);
  if (e != cudaSuccess || per_sm < 1) per_sm = 1;
  long long blocks = (long long)ctx->sm_count * per_sm;
  if (blocks > run.ntasks) blocks = run.ntasks > 0 ? run.ntasks : 1;
  kern<<<(unsigned)blocks, dim3(TX, TY), smem, st>>>(run);
  ctx->launches++;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(ctx, e, "dataflow_column_kernel launch");
  return STENCIL_OK;
}

template <typename T, class Ar>
static int df_column_tile(stencil_ctx* ctx, const DFRun& run, int tx, int ty, bool any_f, cudaStream_t st) {
  if (tx == 8 && ty == 8) return df_column_launch_t<T, Ar, 8, 8>(ctx, run, any_f, st);
  if (tx == 8 && ty == 16) return df_column_launch_t<T, Ar, 8, 16>(ctx, run, any_f, st);
  if (tx == 16 && ty == 8) return df_column_launch_t<T, Ar, 16, 8>(ctx, run, any_f, st);
  return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "column-march Gauss-Seidel tile %dx%d (supported 8x8, 8x16, 16x8)",
                 tx, ty);
}

template <typename T>
int df_column_launch(stencil_ctx* ctx, const DFRun& run, int tx, int ty, int nt, int int_adds, bool any_f, bool pre_f,
                     cudaStream_t st) {
  if (nt == 2) return df_column_ns_launch<T, 2>(ctx, run, tx, ty, int_adds, any_f, pre_f, st);
  if (nt == 3) return df_column_ns_launch<T, 3>(ctx, run, tx, ty, int_adds, any_f, pre_f, st);
  if (nt == 4) return df_column_ns_launch<T, 4>(ctx, run, tx, ty, int_adds, any_f, pre_f, st);
  if (nt != 1) return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "column march with %d sweeps per task (1..4)", nt);
  if constexpr (sizeof(T) == 8) {
    if (pre_f) {  // f holds hh*f
      if (int_adds == kIntAddsAdaptive) return df_column_tile<T, AdaptColumnPre>(ctx, run, tx, ty, any_f, st);
      if (int_adds == 2) return df_column_tile<T, ArithPreF<ArithF64Mix<0x15u>>>(ctx, run, tx, ty, any_f, st);
      if (int_adds == 0) return df_column_tile<T, ArithPreF<ArithF64Fma>>(ctx, run, tx, ty, any_f, st);
      return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "prescaled f with int_adds = %d (0, 2 or 6)", int_adds);
    }
    if (int_adds == kIntAddsAdaptive) return df_column_tile<T, AdaptColumn>(ctx, run, tx, ty, any_f, st);
    if (int_adds == 1) return df_column_tile<T, ArithF64Mix<0x1Du>>(ctx, run, tx, ty, any_f, st);
    if (int_adds == 2) return df_column_tile<T, ArithF64Mix<0x15u>>(ctx, run, tx, ty, any_f, st);
    if (int_adds == 3) return df_column_tile<T, ArithF64Mix<0x12u>>(ctx, run, tx, ty, any_f, st);
    if (int_adds == 4) return df_column_tile<T, ArithF64Mix<0x10u>>(ctx, run, tx, ty, any_f, st);
    if (int_adds == 5) return df_column_tile<T, ArithF64Mix<0x00u>>(ctx, run, tx, ty, any_f, st);
  }
  return df_column_tile<T, typename DefaultArith<T>::type>(ctx, run, tx, ty, any_f, st);
}
template int df_column_launch<double>(stencil_ctx*, const DFRun&, int, int, int, int, bool, bool, cudaStream_t);
template int df_column_launch<float>(stencil_ctx*, const DFRun&, int, int, int, int, bool, bool, cudaStream_t);

// Column-march Gauss-Seidel: tiles tx x ty columns (8x8, 8x16, 16x8; default 8x8 for FP64, whose FP64
// pipe favours the short ramp of narrow tiles, 16x8 for FP32) x tz planes (default: equal chunks of at
// most 100 planes -- 16 when the call runs fewer than 8 sweeps --, enough tasks per level to fill the
// GPU while the march's ramp of tx + ty steps stays short against the chunk).  persistent: one dataflow launch (blocking) instead of one launch per level.
template <typename T, class Ar>
int gs_column_run(stencil_ctx* ctx, T* u, const T* f, const Geom& g, Coef<T> c, int tx, int ty, int tz,
                  int nsweeps, bool persistent, int int_adds, double h, cudaStream_t st, bool pre_f) {
  if (tx == 0) tx = sizeof(T) == 8 ? 8 : 16;
  if (ty == 0) ty = 8;
  if (tz <= 0) {
    // a call of few sweeps is bound by the fill and drain of the task wavefront (levels x task length):
    // short chunks shorten it; many sweeps keep the GPU full and favour long chunks (short ramp per plane)
    const int cap = nsweeps < 8 ? 16 : 100;
    const int chunks = (g.nz + cap - 1) / cap;
    tz = (g.nz + chunks - 1) / chunks;
  }
  if (persistent) {
    if (!((tx == 8 && (ty == 8 || ty == 16)) || (tx == 16 && ty == 8)))
      return set_err(ctx, STENCIL_ERR_UNSUPPORTED,
                     "column-march Gauss-Seidel tile %dx%d (supported 8x8, 8x16, 16x8)", tx, ty);
    T* const a[1] = {u};
    const T* const fs[1] = {f};
    const int ns[1] = {nsweeps};
    const double hs[1] = {h};
    return dataflow_run<T>(ctx, DF_KIND_GS_COLUMN, 1, a, nullptr, fs, &g, ns, hs, tx, ty, tz, 1, ctx->df_timeout_ns,
                           ctx->df_poison, st, (double)c.b, int_adds, pre_f);
  }
#define GS_COL(TXX, TYY)                                                                     \
  if (tx == TXX && ty == TYY)                                                                \
    return f ? gs_column_levels<T, Ar, true, TXX, TYY>(ctx, u, f, g, c, tz, nsweeps, st)     \
             : gs_column_levels<T, Ar, false, TXX, TYY>(ctx, u, f, g, c, tz, nsweeps, st);
  GS_COL(8, 8)
  GS_COL(8, 16)
  GS_COL(16, 8)
#undef GS_COL
  return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "column-march Gauss-Seidel tile %dx%d (supported 8x8, 8x16, 16x8)",
                 tx, ty);
}

template int gs_column_run<double, ArithF64Fma>(stencil_ctx*, double*, const double*, const Geom&, Coef<double>, int, int,
                                  int, int, bool, int, double, cudaStream_t, bool);
template int gs_column_run<double, ArithF64Mix<0x1Du>>(stencil_ctx*, double*, const double*, const Geom&, Coef<double>, int, int,
                                  int, int, bool, int, double, cudaStream_t, bool);
template int gs_column_run<double, ArithF64Mix<0x15u>>(stencil_ctx*, double*, const double*, const Geom&, Coef<double>, int, int,
                                  int, int, bool, int, double, cudaStream_t, bool);
template int gs_column_run<double, ArithF64Mix<0x12u>>(stencil_ctx*, double*, const double*, const Geom&, Coef<double>, int, int,
                                  int, int, bool, int, double, cudaStream_t, bool);
template int gs_column_run<double, ArithF64Mix<0x10u>>(stencil_ctx*, double*, const double*, const Geom&, Coef<double>, int, int,
                                  int, int, bool, int, double, cudaStream_t, bool);
template int gs_column_run<double, ArithF64Mix<0x00u>>(stencil_ctx*, double*, const double*, const Geom&, Coef<double>, int, int,
                                  int, int, bool, int, double, cudaStream_t, bool);
template int gs_column_run<double, AdaptColumn>(stencil_ctx*, double*, const double*, const Geom&,
                                  Coef<double>, int, int, int, int, bool, int, double, cudaStream_t, bool);
template int gs_column_run<double, AdaptColumnPre>(stencil_ctx*, double*, const double*, const Geom&,
                                  Coef<double>, int, int, int, int, bool, int, double, cudaStream_t, bool);
template int gs_column_run<double, ArithPreF<ArithF64Fma>>(stencil_ctx*, double*, const double*, const Geom&,
                                  Coef<double>, int, int, int, int, bool, int, double, cudaStream_t, bool);
template int gs_column_run<double, ArithPreF<ArithF64Mix<0x15u>>>(stencil_ctx*, double*, const double*, const Geom&,
                                  Coef<double>, int, int, int, int, bool, int, double, cudaStream_t, bool);
template int gs_column_run<float, ArithF32>(stencil_ctx*, float*, const float*, const Geom&, Coef<float>, int, int,
                                  int, int, bool, int, double, cudaStream_t, bool);

}  // namespace stn
