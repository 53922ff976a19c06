// Lexicographic Gauss-Seidel (Sec. 3, second listing) with the pipelined,
// temporally blocked schedule of Sec. 3 / Sec. 4 restated for a GPU.
//
// Exactness.  A site (i, j, k) of sweep t reads the i-1, j-1, k-1 neighbours
// of sweep t and the i+1, j+1, k+1 neighbours of sweep t-1.  Every such read
// refers to a site update of level i+j+k+2t - 1 when the update itself has
// level i+j+k+2t, so all updates of one level are independent and any
// level-ordered execution reproduces the serial loops bit for bit (the
// pipeline-parallel claim of Sec. 3 and Fig. pipeline_gs).
//
// Schedule.  The same rule at tile granularity (tiles.h): tasks of equal
// level I+J+K+c*p run as one kernel launch, one CTA per task.  A CTA stages
// its tile plus a one-cell halo (for nt > 1 the union of the nt shifted
// tiles) in shared memory, runs the tile-local levels ii+jj+kk-s one after
// the other (all sites of a level in parallel, listed compactly in a site
// table so that every warp lane has a site), and writes back exactly the
// sites it updated.  nt sweeps per task is the paper's wavefront temporal
// blocking: the tile stays on chip for nt sweeps and the grid is read and
// written once per nt sweeps.
//
// With one sweep per pass and no explicit tile the column march of
// gs_column.cu (variants 4 and 5) runs instead: the same nt = 1 task order,
// a thread per column inside each task.
#include <algorithm>
#include <vector>

#include "internal.h"
#include "tiles.h"
#include "task_bodies.cuh"

namespace stn {

template <typename T, class Ar, bool HAS_F, int W, int H, int D>
__global__ void __launch_bounds__(GS_THREADS) gs_task_kernel(T* __restrict__ u, const T* __restrict__ f, Geom g,
                                                              Coef<T> c, const uint64_t* __restrict__ slices,
                                                              const int* __restrict__ slice_off, SiteTable tb,
                                                              TileGeom tg, int level) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  __shared__ int s_off[GS_MAXLEVELS + 1];
  const int tid = threadIdx.x;

  int I, J, K, p;
  if (!find_task(tg, slices, slice_off, level, &I, &J, &K, &p)) return;
  const int ns = min(tg.nt, tg.nsweeps - p * tg.nt);
  const int X0 = I * W, Y0 = J * H, Z0 = K * D;

  // ---- the staged box [X0-ns, X0+W] x [Y0-ns, Y0+H] x [Z0-ns, Z0+D]
  const int bw = W + ns + 1, bh = H + ns + 1, bd = D + ns + 1;
  const int plane = bw * bh;
  const int bx0 = X0 - ns, by0 = Y0 - ns, bz0 = Z0 - ns;
  const int nlv = W + H + D - 3 + ns;
  const int* so = tb.off + tb.base[ns];
  for (int l = tid; l <= nlv; l += GS_THREADS) s_off[l] = so[l];
  // every site this task updates is an interior site: no bounds checks per site
  const bool full = (X0 - ns + 1 >= 0) && (Y0 - ns + 1 >= 0) && (Z0 - ns + 1 >= 0) && (X0 + W <= g.nx) &&
                    (Y0 + H <= g.ny) && (Z0 + D <= g.nz);

  // stage: each thread owns fixed (x, y) positions of the box plane and walks z
  const int zlo = max(0, -1 - bz0), zhi = min(bd - 1, g.nz - bz0);  // box planes inside [-1, nz]
#pragma unroll
  for (int r = 0; r < GS_MAXPOS; ++r) {
    const int e = tid + r * GS_THREADS;
    if (e >= plane) break;
    const int ly = e / bw, lx = e - ly * bw;
    const int x = bx0 + lx, y = by0 + ly;
    if (x < -1 || x > g.nx || y < -1 || y > g.ny) continue;
    if (zlo > zhi) continue;
    const T* src = u + g.at(x, y, bz0 + zlo);
    T* dst = sm + e + zlo * plane;
#pragma unroll 4
    for (int lz = 0; lz <= zhi - zlo; ++lz) dst[lz * plane] = src[(int64_t)lz * g.sy];
  }
  __syncthreads();

  // ---- tile-local levels ii+jj+kk-s, from -(ns-1) to W+H+D-3
  for (int lv = 0; lv < nlv; ++lv) {
    const int beg = s_off[lv], end = s_off[lv + 1];
    // A level's sites go to consecutive threads starting at a warp that rotates
    // with the level and the CTA, so small levels do not all land on warp 0 and
    // thereby on one SM sub-partition's FP64 pipe.
    int t = tid - (((int)blockIdx.x + lv) & (GS_THREADS / 32 - 1)) * 32;
    if (t < 0) t += GS_THREADS;
    for (int e = beg + t; e < end; e += GS_THREADS) {
      const int li = tb.lis[e];
      T fv = T(0);
      if (!full || HAS_F) {
        const uint32_t s = tb.coords[e];
        const int sw = (int)(s >> 24);
        const int x = X0 - sw + (int)(s & 0xFF);
        const int y = Y0 - sw + (int)((s >> 8) & 0xFF);
        const int z = Z0 - sw + (int)((s >> 16) & 0xFF);
        if (!full && (x < 0 || x >= g.nx || y < 0 || y >= g.ny || z < 0 || z >= g.nz)) continue;
        if (HAS_F) fv = f[g.at(x, y, z)];
      }
      sm[li] = site_update<T, Ar, HAS_F, false>(sm[li - 1], sm[li + 1], sm[li - bw], sm[li + bw], sm[li - plane],
                                                sm[li + plane], fv, T(0), c);
    }
    __syncthreads();
  }

  // ---- write back every site this task updated (its last value here).  Site
  // (x, y, z) is updated at the pass-local sweeps s with X0-s <= x < X0+W-s (same
  // in y, z) and 0 <= s < ns; the xy part of that range is fixed per position.
#pragma unroll
  for (int r = 0; r < GS_MAXPOS; ++r) {
    const int e = tid + r * GS_THREADS;
    if (e >= plane) break;
    const int ly = e / bw, lx = e - ly * bw;
    const int x = bx0 + lx, y = by0 + ly;
    if (x < 0 || x >= g.nx || y < 0 || y >= g.ny) continue;
    const int a = max(max(X0 - x, Y0 - y), 0);
    const int bb = min(min(X0 + W - x, Y0 + H - y), ns);
    if (a >= bb) continue;
    // z with max(a, Z0-z) < min(bb, Z0+D-z): Z0-bb < z < Z0+D-a, inside the interior
    const int z_lo = max(Z0 - bb + 1, 0), z_hi = min(Z0 + D - a - 1, g.nz - 1);
    T* dst = u + g.at(x, y, 0);
    const T* src = sm + e;
#pragma unroll 4
    for (int z = z_lo; z <= z_hi; ++z) dst[(int64_t)z * g.sy] = src[(z - bz0) * plane];
  }
}

// Direct variant (variant 2; the default for nt > 1 or an explicit tile): the
// task body of task_bodies.cuh, one CTA per task
// of the level.
template <typename T, class Ar, bool HAS_F, int W, int H, int D>
__global__ void __launch_bounds__(GS_THREADS) gs_direct_kernel(T* u, const T* __restrict__ f, Geom g, Coef<T> c,
                                                                const uint64_t* __restrict__ slices,
                                                                const int* __restrict__ slice_off, SiteTable tb,
                                                                TileGeom tg, int level) {
  __shared__ int s_off[GS_MAXLEVELS + 1];
  int I, J, K, p;
  if (!find_task(tg, slices, slice_off, level, &I, &J, &K, &p)) return;
  gs_task_body<T, Ar, HAS_F, W, H, D>(u, f, g, c, tb, tg, I, J, K, p, s_off);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
TileGeom make_tile_geom(const Geom& g, int W, int H, int D, int nt, int nsweeps) {
  TileGeom t;
  t.W = W; t.H = H; t.D = D; t.nt = nt; t.nsweeps = nsweeps;
  t.NI = (g.nx + nt - 1 + W - 1) / W;
  t.NJ = (g.ny + nt - 1 + H - 1) / H;
  t.NK = (g.nz + nt - 1 + D - 1) / D;
  t.npass = (nsweeps + nt - 1) / nt;
  t.cstride = nt == 1 ? 2 : 4;
  t.sigma_max = t.NI + t.NJ + t.NK - 3;
  t.nlevels = t.sigma_max + t.cstride * (t.npass - 1) + 1;
  return t;
}

// Slices: all tiles (I, J, K) grouped by sigma = I+J+K; cached per (NI, NJ, NK).
// Slices: all tiles (I, J, K) grouped by sigma = I+J+K; one table per (NI, NJ, NK), the 32 most recently
// used kept on the device, so that calls alternating between shapes (the levels of a multigrid cycle)
// upload each table once.
int ensure_slices(stencil_ctx* ctx, const TileGeom& tg, cudaStream_t st) {
  for (size_t i = 0; i < ctx->slices.size(); ++i) {
    SliceEntry& en = ctx->slices[i];
    if (en.NI == tg.NI && en.NJ == tg.NJ && en.NK == tg.NK) {
      en.last_use = ++ctx->slice_clock;
      ctx->slice_cur = (int)i;
      return STENCIL_OK;
    }
  }
  const int nsig = tg.sigma_max + 1;
  std::vector<int> off(nsig + 1, 0);
  for (int K = 0; K < tg.NK; ++K)
    for (int J = 0; J < tg.NJ; ++J)
      for (int I = 0; I < tg.NI; ++I) off[I + J + K + 1]++;
  for (int s = 0; s < nsig; ++s) off[s + 1] += off[s];
  std::vector<uint64_t> tiles((size_t)off[nsig]);
  std::vector<int> fill(off.begin(), off.end() - 1);
  for (int K = 0; K < tg.NK; ++K)
    for (int J = 0; J < tg.NJ; ++J)
      for (int I = 0; I < tg.NI; ++I) tiles[(size_t)fill[I + J + K]++] = pack_tile(I, J, K);
  const size_t bytes = tiles.size() * sizeof(uint64_t) + off.size() * sizeof(int) + 64;
  // room: evict the least recently used table when 32 are held
  if (ctx->slices.size() >= 32) {
    size_t lru = 0;
    for (size_t i = 1; i < ctx->slices.size(); ++i)
      if (ctx->slices[i].last_use < ctx->slices[lru].last_use) lru = i;
    cudaError_t e0 = cudaStreamSynchronize(st);  // launches of this stream may still read it
    if (e0 != cudaSuccess) return cuda_err(ctx, e0, "slice table eviction");
    cudaFree(ctx->slices[lru].dev);
    ctx->held -= ctx->slices[lru].bytes;
    ctx->slices.erase(ctx->slices.begin() + (long)lru);
    ctx->ws_gen++;
  }
  if (ctx->budget && ctx->held + bytes > ctx->budget)
    return set_err(ctx, STENCIL_ERR_OOM, "tile-slice table needs %zu bytes; %zu held, budget %zu", bytes, ctx->held,
                   ctx->budget);
  void* d = nullptr;
  cudaError_t e = cudaMalloc(&d, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, STENCIL_ERR_OOM, "cudaMalloc(%zu) for a tile-slice table: %s", bytes, cudaGetErrorString(e));
  }
  e = cudaMemcpyAsync(d, tiles.data(), tiles.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((unsigned char*)d + tiles.size() * sizeof(uint64_t), off.data(), off.size() * sizeof(int),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host vectors go out of scope
  if (e != cudaSuccess) {
    cudaFree(d);
    return cuda_err(ctx, e, "upload of tile slices");
  }
  SliceEntry en;
  en.NI = tg.NI;
  en.NJ = tg.NJ;
  en.NK = tg.NK;
  en.dev = d;
  en.bytes = bytes;
  en.off = std::move(off);
  en.last_use = ++ctx->slice_clock;
  ctx->held += bytes;
  ctx->slices.push_back(std::move(en));
  ctx->slice_cur = (int)ctx->slices.size() - 1;
  return STENCIL_OK;
}

const uint64_t* slices_ptr(stencil_ctx* ctx) { return (const uint64_t*)ctx->slices[(size_t)ctx->slice_cur].dev; }
const int* slice_off_ptr(stencil_ctx* ctx) {
  const SliceEntry& en = ctx->slices[(size_t)ctx->slice_cur];
  const size_t ntiles = (size_t)en.off.back();
  return (const int*)((const unsigned char*)en.dev + ntiles * sizeof(uint64_t));
}

// Number of tasks of level L.
int tasks_at_level(const stencil_ctx* ctx, const TileGeom& tg, int L) {
  int n = 0;
  for (int p = std::min(tg.npass - 1, L / tg.cstride); p >= 0; --p) {
    int sigma = L - tg.cstride * p;
    if (sigma > tg.sigma_max) break;
    n += ctx->slices[(size_t)ctx->slice_cur].off[sigma + 1] - ctx->slices[(size_t)ctx->slice_cur].off[sigma];
  }
  return n;
}

// Site tables of the tile-local levels ii+jj+kk-s for ns = 1..nt, cached per
// (W, H, D, nt).  Layout in the slot: coords (u32) | lis (u16) | off (int) | base (int).
int ensure_sites(stencil_ctx* ctx, const TileGeom& tg, cudaStream_t st) {
  if (ctx->gs_key[3] == tg.W && ctx->gs_key[4] == tg.H && ctx->gs_key[5] == tg.D && ctx->gs_key[6] == tg.nt &&
      ctx->slots[SLOT_GS_SITES].ptr)
    return STENCIL_OK;
  std::vector<uint32_t> sites;
  std::vector<uint16_t> lis;
  std::vector<int> off;
  std::vector<int> base(tg.nt + 1, 0);
  for (int ns = 1; ns <= tg.nt; ++ns) {
    base[ns] = (int)off.size();
    const int bw = tg.W + ns + 1, bh = tg.H + ns + 1;
    const int lo = -(ns - 1), hi = tg.W + tg.H + tg.D - 3;
    for (int lv = lo; lv <= hi; ++lv) {
      off.push_back((int)sites.size());
      for (int s = 0; s < ns; ++s)
        for (int kk = 0; kk < tg.D; ++kk)
          for (int jj = 0; jj < tg.H; ++jj) {
            int ii = lv + s - kk - jj;
            if (ii < 0 || ii >= tg.W) continue;
            sites.push_back(pack_site(ii, jj, kk, s));
            lis.push_back((uint16_t)(((kk + ns - s) * bh + (jj + ns - s)) * bw + (ii + ns - s)));
          }
    }
    off.push_back((int)sites.size());
  }
  const size_t b_sites = sites.size() * sizeof(uint32_t);
  const size_t b_lis = (lis.size() * sizeof(uint16_t) + 15) / 16 * 16;
  const size_t b_off = off.size() * sizeof(int);
  const size_t b_base = base.size() * sizeof(int);
  int status;
  unsigned char* d = (unsigned char*)ws_get(ctx, SLOT_GS_SITES, b_sites + b_lis + b_off + b_base + 64, &status);
  if (!d) return status;
  cudaError_t e = cudaMemcpyAsync(d, sites.data(), b_sites, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d + b_sites, lis.data(), lis.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d + b_sites + b_lis, off.data(), b_off, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d + b_sites + b_lis + b_off, base.data(), b_base, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(ctx, e, "upload of site table");
  ctx->gs_key[3] = tg.W; ctx->gs_key[4] = tg.H; ctx->gs_key[5] = tg.D; ctx->gs_key[6] = tg.nt;
  ctx->gs_key[7] = (int64_t)sites.size();
  return STENCIL_OK;
}

SiteTable site_table(stencil_ctx* ctx, const TileGeom& tg) {
  const unsigned char* sb = (const unsigned char*)ctx->slots[SLOT_GS_SITES].ptr;
  const size_t nsites = (size_t)ctx->gs_key[7];
  const size_t b_sites = nsites * sizeof(uint32_t);
  const size_t b_lis = (nsites * sizeof(uint16_t) + 15) / 16 * 16;
  size_t noff = 0;
  for (int ns = 1; ns <= tg.nt; ++ns) noff += (size_t)(tg.W + tg.H + tg.D - 2 + ns);
  SiteTable t;
  t.goff = nullptr;
  t.coords = (const uint32_t*)sb;
  t.lis = (const uint16_t*)(sb + b_sites);
  t.off = (const int*)(sb + b_sites + b_lis);
  t.base = t.off + noff;
  return t;
}

// Per-site grid offsets (relative to the tile origin) for one grid shape, so
// that interior tasks skip the coordinate decoding; cached per (tile, nt, sx, sy).
static int ensure_goff(stencil_ctx* ctx, const TileGeom& tg, const Geom& g, cudaStream_t st, const int** out) {
  *out = nullptr;
  const int64_t key[6] = {tg.W, tg.H, tg.D, tg.nt, g.sx, g.sy};
  if ((double)g.sy * (tg.D + tg.nt) >= 2147483647.0) return STENCIL_OK;  // offsets would not fit int32
  bool same = ctx->slots[SLOT_GS_GOFF].ptr != nullptr;
  for (int i = 0; i < 6; ++i) same = same && ctx->goff_key[i] == key[i];
  if (!same) {
    // rebuild from the packed coordinates (same order as the site table)
    std::vector<int> goff;
    for (int ns = 1; ns <= tg.nt; ++ns) {
      const int lo = -(ns - 1), hi = tg.W + tg.H + tg.D - 3;
      for (int lv = lo; lv <= hi; ++lv)
        for (int s = 0; s < ns; ++s)
          for (int kk = 0; kk < tg.D; ++kk)
            for (int jj = 0; jj < tg.H; ++jj) {
              int ii = lv + s - kk - jj;
              if (ii < 0 || ii >= tg.W) continue;
              goff.push_back((int)((int64_t)(kk - s) * g.sy + (int64_t)(jj - s) * g.sx + (ii - s)));
            }
    }
    int status;
    int* d = (int*)ws_get(ctx, SLOT_GS_GOFF, goff.size() * sizeof(int), &status);
    if (!d) return status;
    cudaError_t e = cudaMemcpyAsync(d, goff.data(), goff.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_err(ctx, e, "upload of site offsets");
    for (int i = 0; i < 6; ++i) ctx->goff_key[i] = key[i];
  }
  *out = (const int*)ctx->slots[SLOT_GS_GOFF].ptr;
  return STENCIL_OK;
}

template <typename T, class Ar, bool HAS_F, int W, int H, int D>
static int gs_levels(stencil_ctx* ctx, T* u, const T* f, const Geom& g, Coef<T> c, const TileGeom& tg,
                     bool direct, cudaStream_t st) {
  size_t smem = (size_t)(W + tg.nt + 1) * (H + tg.nt + 1) * (D + tg.nt + 1) * sizeof(T);
  auto kern = gs_task_kernel<T, Ar, HAS_F, W, H, D>;
  cudaError_t e = cudaSuccess;
  if (direct) {
    kern = gs_direct_kernel<T, Ar, HAS_F, W, H, D>;
    smem = 0;
  } else {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  if (e != cudaSuccess) return cuda_err(ctx, e, "gs smem attribute");
  SiteTable tb = site_table(ctx, tg);
  if (direct) {
    int rc = ensure_goff(ctx, tg, g, st, &tb.goff);
    if (rc) return rc;
  }
  const uint64_t* slices = slices_ptr(ctx);
  const int* soff = slice_off_ptr(ctx);
  for (int L = 0; L < tg.nlevels; ++L) {
    int n = tasks_at_level(ctx, tg, L);
    if (n == 0) continue;
    kern<<<n, GS_THREADS, smem, st>>>(u, f, g, c, slices, soff, tb, tg, L);
    ctx->launches++;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(ctx, e, "gs_task_kernel launch");
  return STENCIL_OK;
}

template <typename T, class Ar>
static int gs_tiles(stencil_ctx* ctx, T* u, const T* f, const Geom& g, Coef<T> c, int tx, int ty, int tz, int nt,
                    int nsweeps, bool direct, cudaStream_t st);

// Column march (gs_column.cu; nt 2..4: gs_column_ns.cuh) with the integer-pipe share of the additions.
template <typename T, class Ar>
static int gs_column_go(stencil_ctx* ctx, T* u, const T* f, const Geom& g, Coef<T> c, int nt, int tx, int ty, int tz,
                        int nsweeps, bool persistent, int int_adds, double h, cudaStream_t st, bool pre_f = false) {
  if (nt == 1) return gs_column_run<T, Ar>(ctx, u, f, g, c, tx, ty, tz, nsweeps, persistent, int_adds, h, st, pre_f);
  if (nt == 2) return gs_column_ns_run<T, Ar, 2>(ctx, u, f, g, c, tx, ty, tz, nsweeps, persistent, int_adds, h, st, pre_f);
  if (nt == 3) return gs_column_ns_run<T, Ar, 3>(ctx, u, f, g, c, tx, ty, tz, nsweeps, persistent, int_adds, h, st, pre_f);
  return gs_column_ns_run<T, Ar, 4>(ctx, u, f, g, c, tx, ty, tz, nsweeps, persistent, int_adds, h, st, pre_f);
}

template <typename T>
static int gs_column_dispatch(stencil_ctx* ctx, T* u, const T* f, const Geom& g, double h, int nsweeps, int nt,
                              const stencil_params* p, cudaStream_t st) {
  Coef<T> c;
  c.a = T(0);
  c.b = (T)((p && p->b != 0.0) ? p->b : 1.0 / 6.0);
  c.hh = (T)(h * h);
  int tx = p ? p->tile_x : 0, ty = p ? p->tile_y : 0, tz = p ? p->tile_z : 0;
  const bool persistent = p && p->variant == 5;
  const int int_adds = (p && p->int_adds >= 0) ? p->int_adds : kDefaultIntAddsColumn;
  if (int_adds < 0 || int_adds > kIntAddsAdaptive)
    return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "int_adds = %d (supported 0..6)", int_adds);
  if (nt > 1) {
    // several sweeps per task: tiles 8x8 (FP64) / 16x8 (FP32), chunks as the one-sweep march (at least nt planes)
    if (tx == 0) tx = sizeof(T) == 8 ? 8 : 16;
    if (ty == 0) ty = 8;
    if (tz <= 0) {
      // the shifted boxes span nz + nt - 1 planes: equal chunks of at most cap + nt - 1 of them, so that no
      // chunk holds only the last sweeps' shifted planes
      const int cap = (nsweeps < 8 ? 16 : 100) + nt - 1;
      const int span = g.nz + nt - 1;
      const int chunks = (span + cap - 1) / cap;
      tz = (span + chunks - 1) / chunks;
    }
    if (tz < nt) tz = nt;
    if (sizeof(T) == 8 && int_adds != 0 && int_adds != 2 && int_adds != kIntAddsAdaptive)
      return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "column march with %d sweeps per task: int_adds = %d (0, 2 or 6)",
                     nt, int_adds);
  }
  if constexpr (sizeof(T) == 8) {
    // f over several sweeps: hh*f once into workspace, the sweeps add it as it is (one FP64 multiplication
    // per site fewer; at int_adds 0, 2 and 6, and only when the workspace budget has room for it)
    if (f && nsweeps >= 2 && (int_adds == 0 || int_adds == 2 || int_adds == kIntAddsAdaptive)) {
      const size_t n = (size_t)g.sy * (size_t)(g.nz + 2);
      double* w = (double*)ws_try(ctx, SLOT_F_SCALED, n * sizeof(double));
      if (w) {
        cudaError_t e = prescale_f(f, w, n, (double)c.hh, ctx->sm_count, st);
        ctx->launches++;
        if (e != cudaSuccess) return cuda_err(ctx, e, "prescale_f launch");
        if (int_adds == kIntAddsAdaptive)
          return gs_column_go<T, AdaptColumnPre>(ctx, u, w, g, c, nt, tx, ty, tz, nsweeps, persistent, int_adds, h,
                                                 st, true);
        if (int_adds == 2)
          return gs_column_go<T, ArithPreF<ArithF64Mix<0x15u>>>(ctx, u, w, g, c, nt, tx, ty, tz, nsweeps, persistent,
                                                                int_adds, h, st, true);
        return gs_column_go<T, ArithPreF<ArithF64Fma>>(ctx, u, w, g, c, nt, tx, ty, tz, nsweeps, persistent,
                                                       int_adds, h, st, true);
      }
    }
    if (nt == 1) {
      if (int_adds == 1) return gs_column_run<T, ArithF64Mix<0x1Du>>(ctx, u, f, g, c, tx, ty, tz, nsweeps, persistent, int_adds, h, st);
      if (int_adds == 3) return gs_column_run<T, ArithF64Mix<0x12u>>(ctx, u, f, g, c, tx, ty, tz, nsweeps, persistent, int_adds, h, st);
      if (int_adds == 4) return gs_column_run<T, ArithF64Mix<0x10u>>(ctx, u, f, g, c, tx, ty, tz, nsweeps, persistent, int_adds, h, st);
      if (int_adds == 5) return gs_column_run<T, ArithF64Mix<0x00u>>(ctx, u, f, g, c, tx, ty, tz, nsweeps, persistent, int_adds, h, st);
    }
    if (int_adds == 2)
      return gs_column_go<T, ArithF64Mix<0x15u>>(ctx, u, f, g, c, nt, tx, ty, tz, nsweeps, persistent, int_adds, h, st);
    if (int_adds == kIntAddsAdaptive)
      return gs_column_go<T, AdaptColumn>(ctx, u, f, g, c, nt, tx, ty, tz, nsweeps, persistent, int_adds, h, st);
  }
  return gs_column_go<T, typename DefaultArith<T>::type>(ctx, u, f, g, c, nt, tx, ty, tz, nsweeps, persistent,
                                                         int_adds, h, st);
}

template <typename T>
int gs_run(stencil_ctx* ctx, T* u, const T* f, const Geom& g, double h, int nsweeps, const stencil_params* p,
           cudaStream_t st) {
  if (nsweeps == 0 || g.nx == 0 || g.ny == 0 || g.nz == 0) return STENCIL_OK;
  const int nt = (p && p->nt > 0) ? p->nt : 1;
  // variant: in place through L1 or the staged shared-memory box; 4: column march, one launch per
  // level; 5: column march, one persistent dataflow launch
  const int variant = p ? p->variant : 0;
  if (variant < 0 || variant > 5) return set_err(ctx, STENCIL_ERR_ARG, "variant = %d", variant);
  // one sweep per pass without an explicit tile: the column march is the default
  const bool tiled = p && (p->tile_x || p->tile_y || p->tile_z);
  if (variant == 4 || variant == 5 || (variant == 0 && nt <= 4 && !tiled)) {
    if (nt > 4) return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "column-march Gauss-Seidel runs nt = 1..4");
    return gs_column_dispatch<T>(ctx, u, f, g, h, nsweeps, nt, p, st);
  }
  const int tx = (p && p->tile_x) ? p->tile_x : 16;
  const int ty = (p && p->tile_y) ? p->tile_y : 16;
  const int tz = (p && p->tile_z) ? p->tile_z : 16;
  // the staged box of variant 1 holds (W+nt+1)(H+nt+1)(D+nt+1) values in shared memory: FP64 stops at nt = 8;
  // the tasks updated through L1 (variants 2, 3) take nt up to 16 with either dtype
  const int maxnt = (sizeof(T) == 8 && variant == 1) ? 8 : 16;
  const bool direct = variant != 1;
  if (variant == 3) {
    T* const a[1] = {u};
    const T* const fs[1] = {f};
    const int ns[1] = {nsweeps};
    const double hs[1] = {h};
    return dataflow_run<T>(ctx, STENCIL_GS, 1, a, nullptr, fs, &g, ns, hs, tx, ty, tz, nt, ctx->df_timeout_ns,
                           ctx->df_poison, st);
  }
  if (nt > maxnt) return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "Gauss-Seidel nt = %d > %d for this dtype", nt, maxnt);
  if (nt > tx || nt > ty || nt > tz)
    return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "nt = %d needs every tile extent >= nt (tile %dx%dx%d)", nt, tx, ty,
                   tz);
  Coef<T> c;
  c.a = T(0);
  c.b = (T)((p && p->b != 0.0) ? p->b : 1.0 / 6.0);
  c.hh = (T)(h * h);
  // the adaptive form is the column march's: these tiles take their own default for it
  const int int_adds = (p && p->int_adds >= 0 && p->int_adds != kIntAddsAdaptive) ? p->int_adds : kDefaultIntAdds;
  if (int_adds < 0 || int_adds > 5)
    return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "int_adds = %d (supported 0..6)", int_adds);
  if constexpr (sizeof(T) == 8) {
    if (int_adds == 1) return gs_tiles<T, ArithF64Mix<0x1Du>>(ctx, u, f, g, c, tx, ty, tz, nt, nsweeps, direct, st);
    if (int_adds == 2) return gs_tiles<T, ArithF64Mix<0x15u>>(ctx, u, f, g, c, tx, ty, tz, nt, nsweeps, direct, st);
    if (int_adds == 3) return gs_tiles<T, ArithF64Mix<0x12u>>(ctx, u, f, g, c, tx, ty, tz, nt, nsweeps, direct, st);
    if (int_adds == 4) return gs_tiles<T, ArithF64Mix<0x10u>>(ctx, u, f, g, c, tx, ty, tz, nt, nsweeps, direct, st);
    if (int_adds == 5) return gs_tiles<T, ArithF64Mix<0x00u>>(ctx, u, f, g, c, tx, ty, tz, nt, nsweeps, direct, st);
  }
  return gs_tiles<T, typename DefaultArith<T>::type>(ctx, u, f, g, c, tx, ty, tz, nt, nsweeps, direct, st);
}

template <typename T, class Ar>
static int gs_tiles(stencil_ctx* ctx, T* u, const T* f, const Geom& g, Coef<T> c, int tx, int ty, int tz, int nt,
                    int nsweeps, bool direct, cudaStream_t st) {
  TileGeom tg;
  int rc;
#define GS_TILE(WW, HH, DD)                                                              \
  if (tx == WW && ty == HH && tz == DD) {                                                \
    tg = make_tile_geom(g, WW, HH, DD, nt, nsweeps);                                     \
    if ((rc = ensure_slices(ctx, tg, st)) != STENCIL_OK) return rc;                      \
    if ((rc = ensure_sites(ctx, tg, st)) != STENCIL_OK) return rc;                       \
    return f ? gs_levels<T, Ar, true, WW, HH, DD>(ctx, u, f, g, c, tg, direct, st)       \
             : gs_levels<T, Ar, false, WW, HH, DD>(ctx, u, f, g, c, tg, direct, st);     \
  }
  GS_TILE(16, 16, 16)
  GS_TILE(8, 8, 8)
  GS_TILE(32, 8, 8)
  GS_TILE(32, 16, 16)
#undef GS_TILE
  return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "Gauss-Seidel tile %dx%dx%d (supported 16^3, 8^3, 32x8x8, 32x16x16)",
                 tx, ty, tz);
}

template int gs_run<double>(stencil_ctx*, double*, const double*, const Geom&, double, int, const stencil_params*,
                            cudaStream_t);
template int gs_run<float>(stencil_ctx*, float*, const float*, const Geom&, double, int, const stencil_params*,
                           cudaStream_t);

}  // namespace stn
