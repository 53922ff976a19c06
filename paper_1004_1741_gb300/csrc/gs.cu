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
#include <algorithm>
#include <vector>

#include "internal.h"
#include "tiles.h"

namespace stn {

constexpr int GS_THREADS = 256;

template <typename T, class Ar, bool HAS_F, int W, int H, int D>
__global__ void __launch_bounds__(GS_THREADS) gs_task_kernel(T* __restrict__ u, const T* __restrict__ f, Geom g,
                                                              Coef<T> c, const uint64_t* __restrict__ slices,
                                                              const int* __restrict__ slice_off,
                                                              const uint32_t* __restrict__ sites,
                                                              const int* __restrict__ site_off,
                                                              const int* __restrict__ site_base, TileGeom tg,
                                                              int level) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int tid = threadIdx.x;

  // ---- which task: blocks of this level enumerate the passes' slices in order
  int b = blockIdx.x;
  int p = level / tg.cstride;
  if (p > tg.npass - 1) p = tg.npass - 1;
  int sigma = level - tg.cstride * p;
  for (;;) {
    int cnt = (sigma <= tg.sigma_max) ? slice_off[sigma + 1] - slice_off[sigma] : 0;
    if (b < cnt) break;
    b -= cnt;
    --p;
    sigma += tg.cstride;
    if (p < 0) return;  // cannot happen for a correct launch size
  }
  int I, J, K;
  unpack_tile(slices[slice_off[sigma] + b], &I, &J, &K);
  const int ns = min(tg.nt, tg.nsweeps - p * tg.nt);
  const int X0 = I * W, Y0 = J * H, Z0 = K * D;

  // ---- stage the box [X0-ns, X0+W] x [Y0-ns, Y0+H] x [Z0-ns, Z0+D]
  const int bw = W + ns + 1, bh = H + ns + 1, bd = D + ns + 1;
  const int bx0 = X0 - ns, by0 = Y0 - ns, bz0 = Z0 - ns;
  const int nbox = bw * bh * bd;
  for (int e = tid; e < nbox; e += GS_THREADS) {
    const int lx = e % bw;
    const int r = e / bw;
    const int ly = r % bh;
    const int lz = r / bh;
    const int x = bx0 + lx, y = by0 + ly, z = bz0 + lz;
    if (x >= -1 && x <= g.nx && y >= -1 && y <= g.ny && z >= -1 && z <= g.nz) sm[e] = u[g.at(x, y, z)];
  }
  __syncthreads();

  // ---- tile-local levels ii+jj+kk-s, from -(ns-1) to W+H+D-3
  const int nlv = W + H + D - 2 + ns - 1;
  const int* so = site_off + site_base[ns];
  const int plane = bw * bh;
  for (int lv = 0; lv < nlv; ++lv) {
    const int beg = so[lv], end = so[lv + 1];
    for (int e = beg + tid; e < end; e += GS_THREADS) {
      const uint32_t s = sites[e];
      const int sw = (int)(s >> 24);
      const int x = X0 - sw + (int)(s & 0xFF);
      const int y = Y0 - sw + (int)((s >> 8) & 0xFF);
      const int z = Z0 - sw + (int)((s >> 16) & 0xFF);
      if (x >= 0 && x < g.nx && y >= 0 && y < g.ny && z >= 0 && z < g.nz) {
        const int li = ((z - bz0) * bh + (y - by0)) * bw + (x - bx0);
        T fv = T(0);
        if (HAS_F) fv = f[g.at(x, y, z)];
        sm[li] = site_update<T, Ar, HAS_F, false>(sm[li - 1], sm[li + 1], sm[li - bw], sm[li + bw], sm[li - plane],
                                                  sm[li + plane], fv, T(0), c);
      }
    }
    __syncthreads();
  }

  // ---- write back every site this task updated (its last value here)
  for (int e = tid; e < nbox; e += GS_THREADS) {
    const int lx = e % bw;
    const int r = e / bw;
    const int ly = r % bh;
    const int lz = r / bh;
    const int x = bx0 + lx, y = by0 + ly, z = bz0 + lz;
    if (x < 0 || x >= g.nx || y < 0 || y >= g.ny || z < 0 || z >= g.nz) continue;
    const int s_lo = max(max(X0 - x, Y0 - y), max(Z0 - z, 0));
    const int s_hi = min(min(X0 + W - x, Y0 + H - y), min(Z0 + D - z, ns));
    if (s_lo < s_hi) u[g.at(x, y, z)] = sm[e];
  }
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
int ensure_slices(stencil_ctx* ctx, const TileGeom& tg, cudaStream_t st) {
  if (ctx->gs_key[0] == tg.NI && ctx->gs_key[1] == tg.NJ && ctx->gs_key[2] == tg.NK && ctx->slots[SLOT_GS_SLICES].ptr)
    return STENCIL_OK;
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
  int status;
  unsigned char* d = (unsigned char*)ws_get(ctx, SLOT_GS_SLICES, bytes, &status);
  if (!d) return status;
  cudaError_t e = cudaMemcpyAsync(d, tiles.data(), tiles.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d + tiles.size() * sizeof(uint64_t), off.data(), off.size() * sizeof(int),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host vectors go out of scope
  if (e != cudaSuccess) return cuda_err(ctx, e, "upload of tile slices");
  ctx->gs_key[0] = tg.NI; ctx->gs_key[1] = tg.NJ; ctx->gs_key[2] = tg.NK;
  ctx->gs_slice_off = off;
  return STENCIL_OK;
}

static const uint64_t* slices_ptr(stencil_ctx* ctx) { return (const uint64_t*)ctx->slots[SLOT_GS_SLICES].ptr; }
static const int* slice_off_ptr(stencil_ctx* ctx) {
  size_t ntiles = (size_t)ctx->gs_slice_off.back();
  return (const int*)((const unsigned char*)ctx->slots[SLOT_GS_SLICES].ptr + ntiles * sizeof(uint64_t));
}

// Number of tasks of level L.
int tasks_at_level(const stencil_ctx* ctx, const TileGeom& tg, int L) {
  int n = 0;
  for (int p = std::min(tg.npass - 1, L / tg.cstride); p >= 0; --p) {
    int sigma = L - tg.cstride * p;
    if (sigma > tg.sigma_max) break;
    n += ctx->gs_slice_off[sigma + 1] - ctx->gs_slice_off[sigma];
  }
  return n;
}

// Site tables of the tile-local levels ii+jj+kk-s for ns = 1..nt, cached per (W, H, D, nt).
static int ensure_sites(stencil_ctx* ctx, const TileGeom& tg, cudaStream_t st) {
  if (ctx->gs_key[3] == tg.W && ctx->gs_key[4] == tg.H && ctx->gs_key[5] == tg.D && ctx->gs_key[6] == tg.nt &&
      ctx->slots[SLOT_GS_SITES].ptr)
    return STENCIL_OK;
  std::vector<uint32_t> sites;
  std::vector<int> off;
  std::vector<int> base(tg.nt + 1, 0);
  for (int ns = 1; ns <= tg.nt; ++ns) {
    base[ns] = (int)off.size();
    const int lo = -(ns - 1), hi = tg.W + tg.H + tg.D - 3;
    for (int lv = lo; lv <= hi; ++lv) {
      off.push_back((int)sites.size());
      for (int s = 0; s < ns; ++s)
        for (int kk = 0; kk < tg.D; ++kk)
          for (int jj = 0; jj < tg.H; ++jj) {
            int ii = lv + s - kk - jj;
            if (ii >= 0 && ii < tg.W) sites.push_back(pack_site(ii, jj, kk, s));
          }
    }
    off.push_back((int)sites.size());
  }
  const size_t b_sites = sites.size() * sizeof(uint32_t);
  const size_t b_off = off.size() * sizeof(int);
  const size_t b_base = base.size() * sizeof(int);
  int status;
  unsigned char* d = (unsigned char*)ws_get(ctx, SLOT_GS_SITES, b_sites + b_off + b_base + 64, &status);
  if (!d) return status;
  cudaError_t e = cudaMemcpyAsync(d, sites.data(), b_sites, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d + b_sites, off.data(), b_off, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d + b_sites + b_off, base.data(), b_base, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(ctx, e, "upload of site table");
  ctx->gs_key[3] = tg.W; ctx->gs_key[4] = tg.H; ctx->gs_key[5] = tg.D; ctx->gs_key[6] = tg.nt;
  ctx->gs_key[7] = (int64_t)sites.size();
  return STENCIL_OK;
}

template <typename T, class Ar, bool HAS_F, int W, int H, int D>
static int gs_levels(stencil_ctx* ctx, T* u, const T* f, const Geom& g, Coef<T> c, const TileGeom& tg,
                     cudaStream_t st) {
  const size_t smem = (size_t)(W + tg.nt + 1) * (H + tg.nt + 1) * (D + tg.nt + 1) * sizeof(T);
  auto kern = gs_task_kernel<T, Ar, HAS_F, W, H, D>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_err(ctx, e, "gs smem attribute");
  const unsigned char* sb = (const unsigned char*)ctx->slots[SLOT_GS_SITES].ptr;
  const size_t nsites = (size_t)ctx->gs_key[7];
  const uint32_t* sites = (const uint32_t*)sb;
  const int* site_off = (const int*)(sb + nsites * sizeof(uint32_t));
  // off has one entry per level per ns plus one terminator per ns
  size_t noff = 0;
  for (int ns = 1; ns <= tg.nt; ++ns) noff += (size_t)(W + H + D - 2 + ns - 1) + 1;
  const int* site_base = site_off + noff;
  const uint64_t* slices = slices_ptr(ctx);
  const int* soff = slice_off_ptr(ctx);
  for (int L = 0; L < tg.nlevels; ++L) {
    int n = tasks_at_level(ctx, tg, L);
    if (n == 0) continue;
    kern<<<n, GS_THREADS, smem, st>>>(u, f, g, c, slices, soff, sites, site_off, site_base, tg, L);
    ctx->launches++;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(ctx, e, "gs_task_kernel launch");
  return STENCIL_OK;
}

template <typename T>
int gs_run(stencil_ctx* ctx, T* u, const T* f, const Geom& g, double h, int nsweeps, const stencil_params* p,
           cudaStream_t st) {
  if (nsweeps == 0 || g.nx == 0 || g.ny == 0 || g.nz == 0) return STENCIL_OK;
  const int nt = (p && p->nt > 0) ? p->nt : 1;
  const int tx = (p && p->tile_x) ? p->tile_x : 16;
  const int ty = (p && p->tile_y) ? p->tile_y : 16;
  const int tz = (p && p->tile_z) ? p->tile_z : 16;
  const int maxnt = sizeof(T) == 8 ? 8 : 16;
  if (nt > maxnt) return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "Gauss-Seidel nt = %d > %d for this dtype", nt, maxnt);
  Coef<T> c;
  c.a = T(0);
  c.b = (T)((p && p->b != 0.0) ? p->b : 1.0 / 6.0);
  c.hh = (T)(h * h);
  TileGeom tg;
  using Ar = typename DefaultArith<T>::type;
  int rc;
#define GS_TILE(WW, HH, DD)                                                              \
  if (tx == WW && ty == HH && tz == DD) {                                                \
    tg = make_tile_geom(g, WW, HH, DD, nt, nsweeps);                                     \
    if ((rc = ensure_slices(ctx, tg, st)) != STENCIL_OK) return rc;                      \
    if ((rc = ensure_sites(ctx, tg, st)) != STENCIL_OK) return rc;                       \
    return f ? gs_levels<T, Ar, true, WW, HH, DD>(ctx, u, f, g, c, tg, st)               \
             : gs_levels<T, Ar, false, WW, HH, DD>(ctx, u, f, g, c, tg, st);             \
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
