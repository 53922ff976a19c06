// Lexicographic Gauss-Seidel as a column march with NS sweeps per task: the
// wavefront temporal blocking of Sec. 4 inside one tile.
//
// Tasks are the skewed tiles of tiles.h with nt = NS: task (I, J, K, p)
// applies the ns = min(NS, nsweeps - p NS) sweeps of pass p to tile (I, J, K),
// sweep s on the tile's box shifted by -s in x, y and z, so that every value a
// sweep reads outside its box is final in the grid (lower levels) or not yet
// touched (higher levels).  Inside the task, thread (i, j) of a TX x TY CTA
// updates at step t, for every sweep s < ns, the site (i - s, j - s, k) with
// k = t - i - j: sweep s trails sweep s - 1 by two steps, the "distance of
// two" between successive time levels of the paper's wavefront, so the NS
// updates of one step are independent and the CTA pays one barrier for NS
// site updates.
//
// The tile lives in a shared-memory ring of R = TX + NS + PF + 2 plane slots;
// a slot holds rows -NS..TY and columns -NS..TX of one plane (tile-local
// coordinates), cell (i, j, k) in slot (i + j + k) mod R.  At step t sweep s
// reads slots t - 2s - 1 (W, S, B: its own values) and t - 2s + 1 (E, N, T:
// sweep s - 1's) and writes slot t - 2s; reads are at odd and writes at even
// distances from t, so no cell is read and written in one step.  Row line
// (j, k) enters by cp.async at step j + k - 2 - PF (as one coalesced line of
// the padded grid) and lands before its first reader (step j + k - 1); the
// cells of the row that this task updates leave at step j + k + TX + NS - 1,
// one step after their last update; the slot is refilled from step
// j + k + R - 2 - PF on.  The copies, updates and write-backs of a step are
// spread over the CTA's threads as flat lists of cells ("duties"), each with
// the window of steps in which its plane is in range.  A right-hand side f
// travels in a second ring with the same slots (rows and columns
// -NS+1..TY-1 / TX-1: the cells some sweep updates).  The whole schedule is
// modelled cell by cell on the CPU (tests/_column_ring_ns.py), where R - 1
// slots fail.
#pragma once

#include "internal.h"
#include "tiles.h"

namespace stn {

template <int TX, int TY, int NS, int PF>
struct ColNS {
  static constexpr int R = TX + NS + PF + 2;      // ring slots
  static constexpr int RW = TX + NS + 1;          // columns -NS..TX
  static constexpr int RH = TY + NS + 1;          // rows -NS..TY
  static constexpr int PL = RW * RH;              // cells per slot of u
  static constexpr int FW = TX + NS - 1;          // columns -NS+1..TX-1
  static constexpr int FH = TY + NS - 1;          // rows -NS+1..TY-1
  static constexpr int FPL = FW * FH;             // cells per slot of f (and per step of write-backs)
  static constexpr int NT = TX * TY;              // threads
  static constexpr int LD = (PL + NT - 1) / NT;   // copy duties of u per thread
  static constexpr int FD = (FPL + NT - 1) / NT;  // copy duties of f, and write-back duties, per thread
};

constexpr int kColNsPF = 2;

template <typename T, int TX, int TY, int NS>
constexpr size_t col_ns_smem_bytes(bool has_f) {
  using C = ColNS<TX, TY, NS, kColNsPF>;
  return (size_t)C::R * (C::PL + (has_f ? C::FPL : 0)) * sizeof(T);
}

// A step window [lo, lo + span]; an empty one never matches.
struct StepWin {
  int lo, span;
  __device__ __forceinline__ bool in(int t) const { return (unsigned)(t - lo) <= (unsigned)span; }
  __device__ __forceinline__ void set(int a, int b) {
    if (a <= b) {
      lo = a;
      span = b - a;
    } else {
      lo = 0x40000000;
      span = 0;
    }
  }
};

template <int R>
__device__ __forceinline__ int ring_mod(int q) {
  q %= R;
  return q < 0 ? q + R : q;
}

// Task (I, J, K, p): the ns sweeps of pass p on tile (I, J, K) (tg.nt == NS),
// in place on u; every thread of the TX x TY CTA takes part; ring:
// col_ns_smem_bytes(HAS_F) of shared memory.  Returns after a barrier, with all
// of the task's global writes issued.
template <typename T, class Ar, bool HAS_F, int TX, int TY, int NS>
__device__ __forceinline__ void gs_column_ns_body(T* u, const T* __restrict__ f, const Geom& g, const Coef<T>& c,
                                                  const TileGeom& tg, int I, int J, int K, int p, T* ring) {
  constexpr int PF = kColNsPF;
  using C = ColNS<TX, TY, NS, PF>;
  constexpr int R = C::R, RW = C::RW, PL = C::PL, FW = C::FW, FPL = C::FPL, NT = C::NT;
  static_assert(NS >= 1 && NS <= TX && NS <= TY, "NS sweeps need tiles of at least NS columns and rows");
  const int i = threadIdx.x, j = threadIdx.y;
  const int tid = j * TX + i;
  const int D = tg.D;
  const int nse = min(NS, tg.nsweeps - p * NS);
  const int x0 = I * TX, y0 = J * TY, z0 = K * D;
  const int64_t sy = g.sy;
  const int64_t tbase = g.at(x0, y0, z0);  // offset of the tile's local (0, 0, 0)
  T* const fring = ring + R * PL;
  const int ts = -2 * NS - 2 - PF;
  const int te = TX + TY + D + NS - 3;

  // copies of u: cell e = (row jj + NS) * RW + (column ii + NS) of every plane k in [-NS, D] that lies in
  // the padded grid; row (jj, k) is copied at step jj + k - 2 - PF into slot (ii + jj + k) mod R
  int ld_cell[C::LD], ld_slot[C::LD];
  int64_t ld_off[C::LD];
  StepWin ld_win[C::LD];
#pragma unroll
  for (int m = 0; m < C::LD; ++m) {
    const int e = tid + m * NT;
    const int jj = e / RW - NS, ii = e % RW - NS;
    const int x = x0 + ii, y = y0 + jj;
    const bool ok = e < PL && x >= -1 && x <= g.nx && y >= -1 && y <= g.ny;
    const int klo = max(-NS, -1 - z0), khi = min(D, g.nz - z0);
    ld_win[m].set(ok ? klo + jj - 2 - PF : 1, ok ? khi + jj - 2 - PF : 0);
    ld_cell[m] = e;
    ld_slot[m] = ring_mod<R>(ii + ts + 2 + PF);
    ld_off[m] = tbase + (int64_t)jj * g.sx + ii + (int64_t)(ts + 2 + PF - jj) * sy;
  }
  // copies of f and write-backs of u share the cell list e = (jj + NS - 1) * FW + (ii + NS - 1),
  // rows and columns -NS+1..TY-1 / TX-1
  int fd_cell[C::FD], fd_wpos[C::FD], fd_fslot[C::FD], fd_wslot[C::FD];
  int64_t fd_foff[C::FD], fd_woff[C::FD];
  StepWin fd_fwin[C::FD], fd_wwin[C::FD];
#pragma unroll
  for (int m = 0; m < C::FD; ++m) {
    const int e = tid + m * NT;
    const int jj = e / FW - NS + 1, ii = e % FW - NS + 1;
    const int x = x0 + ii, y = y0 + jj;
    const bool ok = e < FPL && x >= 0 && x < g.nx && y >= 0 && y < g.ny;
    // f of the interior planes in [-NS+1, D-1], copied with its row of u
    const int fklo = max(-NS + 1, -z0), fkhi = min(D - 1, g.nz - 1 - z0);
    fd_fwin[m].set(ok && HAS_F ? fklo + jj - 2 - PF : 1, ok && HAS_F ? fkhi + jj - 2 - PF : 0);
    fd_fslot[m] = ring_mod<R>(ii + ts + 2 + PF);
    fd_foff[m] = tbase + (int64_t)jj * g.sx + ii + (int64_t)(ts + 2 + PF - jj) * sy;
    // write-back of the planes in which some sweep s < nse updates the cell:
    // max(0, -ii, -jj, -k) <= s <= min(nse - 1, TX-1-ii, TY-1-jj, D-1-k)
    const int a = max(0, max(-ii, -jj)), b = min(nse - 1, min(TX - 1 - ii, TY - 1 - jj));
    const int wklo = max(-b, -z0), wkhi = min(D - 1 - a, g.nz - 1 - z0);
    const int wdel = TX + NS - 1 + jj;  // write-back step - k
    fd_wwin[m].set(ok && a <= b ? wklo + wdel : 1, ok && a <= b ? wkhi + wdel : 0);
    fd_wslot[m] = ring_mod<R>(ii + ts - (TX + NS - 1));
    fd_woff[m] = tbase + (int64_t)jj * g.sx + ii + (int64_t)(ts - wdel) * sy;
    fd_cell[m] = e;
    fd_wpos[m] = (jj + NS) * RW + (ii + NS);  // the cell's place in a slot of u
  }
  // updates: sweep s of thread (i, j) is site (i - s, j - s, t - i - j), in its box and in the interior
  int up_pos[NS], up_fpos[NS];
  StepWin up_win[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const bool ok = s < nse && x0 + i - s >= 0 && x0 + i - s < g.nx && y0 + j - s >= 0 && y0 + j - s < g.ny;
    const int klo = max(-s, -z0), khi = min(D - 1 - s, g.nz - 1 - z0);
    up_win[s].set(ok ? klo + i + j : 1, ok ? khi + i + j : 0);
    up_pos[s] = (j - s + NS) * RW + (i - s + NS);
    up_fpos[s] = (j - s + NS - 1) * FW + (i - s + NS - 1);
  }
  int st = ring_mod<R>(ts);  // slot of step t
  auto wrap = [](int q) { return q == R - 1 ? 0 : q + 1; };
  for (int t = ts; t <= te; ++t) {
#pragma unroll
    for (int m = 0; m < C::LD; ++m) {
      if (ld_win[m].in(t)) cp_async_elem(ring + ld_slot[m] * PL + ld_cell[m], u + ld_off[m]);
      ld_slot[m] = wrap(ld_slot[m]);
      ld_off[m] += sy;
    }
    if (HAS_F) {
#pragma unroll
      for (int m = 0; m < C::FD; ++m) {
        if (fd_fwin[m].in(t)) cp_async_elem(fring + fd_fslot[m] * FPL + fd_cell[m], f + fd_foff[m]);
        fd_fslot[m] = wrap(fd_fslot[m]);
        fd_foff[m] += sy;
      }
    }
    cp_async_commit();
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const bool act = up_win[s].in(t);
      int q = st - 2 * s;
      if (q < 0) q += R;
      const int qm = q == 0 ? R - 1 : q - 1, qp = wrap(q);
      const int pos = up_pos[s];
      const T* pm = ring + qm * PL + pos;
      const T* pp = ring + qp * PL + pos;
      if constexpr (AdaptOf<Ar>::on) {  // the warp votes; every lane reads inside the ring
        const T fv = HAS_F ? fring[q * FPL + up_fpos[s]] : T(0);
        const T v = site_update_warp<T, Ar, HAS_F, false>(act, pm[-1], pp[1], pm[-RW], pp[RW], pm[0], pp[0], fv,
                                                          T(0), c);
        if (act) ring[q * PL + pos] = v;
      } else if (act) {
        const T fv = HAS_F ? fring[q * FPL + up_fpos[s]] : T(0);
        ring[q * PL + pos] =
            site_update<T, Ar, HAS_F, false>(pm[-1], pp[1], pm[-RW], pp[RW], pm[0], pp[0], fv, T(0), c);
      }
    }
#pragma unroll
    for (int m = 0; m < C::FD; ++m) {
      if (fd_wwin[m].in(t)) u[fd_woff[m]] = ring[fd_wslot[m] * PL + fd_wpos[m]];
      fd_wslot[m] = wrap(fd_wslot[m]);
      fd_woff[m] += sy;
    }
    cp_async_wait<PF>();
    __syncthreads();
    st = wrap(st);
  }
  cp_async_wait<0>();
  __syncthreads();
}

// One launch per task level (find_task: CTA -> task of the level).
template <typename T, class Ar, bool HAS_F, int TX, int TY, int NS>
__global__ void __launch_bounds__(TX * TY) gs_column_ns_kernel(T* u, const T* __restrict__ f, Geom g, Coef<T> c,
                                                               const uint64_t* __restrict__ slices,
                                                               const int* __restrict__ slice_off, TileGeom tg,
                                                               int level) {
  extern __shared__ __align__(16) unsigned char gsn_raw[];
  int I, J, K, p;
  if (!find_task(tg, slices, slice_off, level, &I, &J, &K, &p)) return;
  gs_column_ns_body<T, Ar, HAS_F, TX, TY, NS>(u, f, g, c, tg, I, J, K, p, reinterpret_cast<T*>(gsn_raw));
}

}  // namespace stn

// ---------------------------------------------------------------------------
// Persistent form and host runners (instantiated per NS in gs_column_ns<NS>.cu)
// ---------------------------------------------------------------------------
#include "dataflow.cuh"

namespace stn {

// Each CTA takes the next task of the level-ordered queue, waits (bounded) for
// its dependencies -- the three backward faces of its pass and the 2 x 2 x 2
// tiles ahead of the previous pass --, runs the march and publishes its flag.
template <typename T, class Ar, int TX, int TY, int NS>
__global__ void __launch_bounds__(TX * TY, 14 * 64 / (TX * TY)) dataflow_column_ns_kernel(DFRun run) {
  extern __shared__ __align__(16) unsigned char gsn_raw[];
  T* ring = reinterpret_cast<T*>(gsn_raw);
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
      gs_column_ns_body<T, Ar, true, TX, TY, NS>((T*)d.a, (const T*)d.f, d.g, c, d.tg, I, J, K, p, ring);
    else
      gs_column_ns_body<T, Ar, false, TX, TY, NS>((T*)d.a, nullptr, d.g, c, d.tg, I, J, K, p, ring);
    // the body ended with a barrier after its last writes: they precede the release
    if (lead && q != run.poison) {
      __threadfence();
      st_release(run.flags + df_flag(d, I, J, K, p), 1u);
    }
  }
}

template <typename T, class Ar, bool HAS_F, int TX, int TY, int NS>
static int gs_column_ns_levels(stencil_ctx* ctx, T* u, const T* f, const Geom& g, Coef<T> c, int tz, int nsweeps,
                               cudaStream_t st) {
  const TileGeom tg = make_tile_geom(g, TX, TY, tz, NS, nsweeps);
  int rc = ensure_slices(ctx, tg, st);
  if (rc) return rc;
  const uint64_t* slices = slices_ptr(ctx);
  const int* soff = slice_off_ptr(ctx);
  auto kern = gs_column_ns_kernel<T, Ar, HAS_F, TX, TY, NS>;
  const size_t smem = col_ns_smem_bytes<T, TX, TY, NS>(HAS_F);
  cudaError_t e0 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e0 != cudaSuccess) return cuda_err(ctx, e0, "gs_column_ns_kernel shared memory");
  for (int L = 0; L < tg.nlevels; ++L) {
    const int n = tasks_at_level(ctx, tg, L);
    if (n == 0) continue;
    kern<<<n, dim3(TX, TY), smem, st>>>(u, f, g, c, slices, soff, tg, L);
    ctx->launches++;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(ctx, e, "gs_column_ns_kernel launch");
  return STENCIL_OK;
}

template <typename T, class Ar, int TX, int TY, int NS>
static int df_column_ns_launch_t(stencil_ctx* ctx, const DFRun& run, bool any_f, cudaStream_t st) {
  auto kern = dataflow_column_ns_kernel<T, Ar, TX, TY, NS>;
  const size_t smem = col_ns_smem_bytes<T, TX, TY, NS>(any_f);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_err(ctx, e, "dataflow_column_ns_kernel shared memory");
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TX * TY, smem);
  if (e != cudaSuccess || per_sm < 1) per_sm = 1;
  long long blocks = (long long)ctx->sm_count * per_sm;
  if (blocks > run.ntasks) blocks = run.ntasks > 0 ? run.ntasks : 1;
  kern<<<(unsigned)blocks, dim3(TX, TY), smem, st>>>(run);
  ctx->launches++;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(ctx, e, "dataflow_column_ns_kernel launch");
  return STENCIL_OK;
}

template <typename T, class Ar, int NS>
static int df_column_ns_tile(stencil_ctx* ctx, const DFRun& run, int tx, int ty, bool any_f, cudaStream_t st) {
  if (tx == 8 && ty == 8) return df_column_ns_launch_t<T, Ar, 8, 8, NS>(ctx, run, any_f, st);
  if (tx == 16 && ty == 8) return df_column_ns_launch_t<T, Ar, 16, 8, NS>(ctx, run, any_f, st);
  return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "column-march Gauss-Seidel with %d sweeps per task: tile %dx%d "
                 "(supported 8x8, 16x8)", NS, tx, ty);
}

// The persistent launch of a dataflow run whose tasks are column marches of NS sweeps.
template <typename T, int NS>
int df_column_ns_launch(stencil_ctx* ctx, const DFRun& run, int tx, int ty, int int_adds, bool any_f, bool pre_f,
                        cudaStream_t st) {
  if constexpr (sizeof(T) == 8) {
    if (pre_f) {
      if (int_adds == kIntAddsAdaptive) return df_column_ns_tile<T, AdaptColumnPre, NS>(ctx, run, tx, ty, any_f, st);
      if (int_adds == 2) return df_column_ns_tile<T, ArithPreF<ArithF64Mix<0x15u>>, NS>(ctx, run, tx, ty, any_f, st);
      if (int_adds == 0) return df_column_ns_tile<T, ArithPreF<ArithF64Fma>, NS>(ctx, run, tx, ty, any_f, st);
      return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "prescaled f with int_adds = %d (0, 2 or 6)", int_adds);
    }
    if (int_adds == kIntAddsAdaptive) return df_column_ns_tile<T, AdaptColumn, NS>(ctx, run, tx, ty, any_f, st);
    if (int_adds == 2) return df_column_ns_tile<T, ArithF64Mix<0x15u>, NS>(ctx, run, tx, ty, any_f, st);
    if (int_adds != 0)
      return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "column march with %d sweeps per task: int_adds = %d (0, 2 or 6)",
                     NS, int_adds);
  }
  return df_column_ns_tile<T, typename DefaultArith<T>::type, NS>(ctx, run, tx, ty, any_f, st);
}

// Column march with NS sweeps per task: level launches, or one persistent dataflow launch.
template <typename T, class Ar, int NS>
int gs_column_ns_run(stencil_ctx* ctx, T* u, const T* f, const Geom& g, Coef<T> c, int tx, int ty, int tz,
                     int nsweeps, bool persistent, int int_adds, double h, cudaStream_t st, bool pre_f) {
  if (persistent) {
    T* const a[1] = {u};
    const T* const fs[1] = {f};
    const int ns[1] = {nsweeps};
    const double hs[1] = {h};
    return dataflow_run<T>(ctx, DF_KIND_GS_COLUMN, 1, a, nullptr, fs, &g, ns, hs, tx, ty, tz, NS, ctx->df_timeout_ns,
                           ctx->df_poison, st, (double)c.b, int_adds, pre_f);
  }
#define GS_COLNS(TXX, TYY)                                                                        \
  if (tx == TXX && ty == TYY)                                                                     \
    return f ? gs_column_ns_levels<T, Ar, true, TXX, TYY, NS>(ctx, u, f, g, c, tz, nsweeps, st)   \
             : gs_column_ns_levels<T, Ar, false, TXX, TYY, NS>(ctx, u, f, g, c, tz, nsweeps, st);
  GS_COLNS(8, 8)
  GS_COLNS(16, 8)
#undef GS_COLNS
  return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "column-march Gauss-Seidel with %d sweeps per task: tile %dx%d "
                 "(supported 8x8, 16x8)", NS, tx, ty);
}

}  // namespace stn

// Explicit instantiations of one NS (used by gs_column_ns<NS>.cu).
#define STN_COLUMN_NS_INSTANTIATE(NS)                                                                                 \
  namespace stn {                                                                                                     \
  template int df_column_ns_launch<double, NS>(stencil_ctx*, const DFRun&, int, int, int, bool, bool, cudaStream_t); \
  template int df_column_ns_launch<float, NS>(stencil_ctx*, const DFRun&, int, int, int, bool, bool, cudaStream_t);  \
  template int gs_column_ns_run<double, ArithF64Fma, NS>(stencil_ctx*, double*, const double*, const Geom&,          \
                                                         Coef<double>, int, int, int, int, bool, int, double,        \
                                                         cudaStream_t, bool);                                        \
  template int gs_column_ns_run<double, ArithF64Mix<0x15u>, NS>(stencil_ctx*, double*, const double*, const Geom&,   \
                                                                Coef<double>, int, int, int, int, bool, int, double, \
                                                                cudaStream_t, bool);                                 \
  template int gs_column_ns_run<double, AdaptColumn, NS>(stencil_ctx*, double*, const double*, const Geom&,          \
                                                         Coef<double>, int, int, int, int, bool, int, double,        \
                                                         cudaStream_t, bool);                                        \
  template int gs_column_ns_run<double, AdaptColumnPre, NS>(stencil_ctx*, double*, const double*, const Geom&,       \
                                                            Coef<double>, int, int, int, int, bool, int, double,     \
                                                            cudaStream_t, bool);                                     \
  template int gs_column_ns_run<double, ArithPreF<ArithF64Fma>, NS>(stencil_ctx*, double*, const double*,            \
                                                                    const Geom&, Coef<double>, int, int, int, int,   \
                                                                    bool, int, double, cudaStream_t, bool);          \
  template int gs_column_ns_run<double, ArithPreF<ArithF64Mix<0x15u>>, NS>(stencil_ctx*, double*, const double*,     \
                                                                           const Geom&, Coef<double>, int, int, int, \
                                                                           int, bool, int, double, cudaStream_t,     \
                                                                           bool);                                    \
  template int gs_column_ns_run<float, ArithF32, NS>(stencil_ctx*, float*, const float*, const Geom&, Coef<float>,   \
                                                     int, int, int, int, bool, int, double, cudaStream_t, bool);     \
  }
