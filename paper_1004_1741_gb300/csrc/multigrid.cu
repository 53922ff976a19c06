// Multigrid V-cycle solve of -Lap_h u = f with the library's smoothers.
//
// Sec. 1 and Sec. 3 name multigrid solvers as the place where Jacobi and
// Gauss-Seidel smoothers spend their time; the paper does not define the
// cycle, so the textbook one is used: level l+1 has extents (n-1)/2 and
// spacing 2h while every extent is odd and >= 3 (coarse site I on fine site
// 2I+1); nu1 smoothing sweeps, residual, full-weighting restriction, the
// coarse correction from zero with zero Dirichlet values, trilinear
// prolongation added to u, nu2 smoothing sweeps; ncoarse sweeps on the
// coarsest level.  Smoothers: weighted Jacobi with omega = 6/7 (a = b = 1/7),
// lexicographic Gauss-Seidel (b = 1/6) or red-black Gauss-Seidel (b = 1/6).  The transfers are written in one
// fixed order of IEEE operations (x, then y, then z; each weighted mean as
// ((w a + w' b) + w c), each interpolated mean as (a + b) * 0.5), so the
// whole cycle is deterministic and the same bits as the serial definition.
// The same cycle runs in binary32 (every operation in float, the FP32
// residual and smoothers) as the inner solver of the mixed-precision defect
// correction stencil_solve_mixed_mg, whose residual and update stay FP64.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "internal.h"

namespace stn {

// The transfers' arithmetic: one IEEE round-to-nearest operation per + and *,
// in binary64 or binary32 with the same order and weights.
template <typename T>
using MGArith = typename std::conditional<sizeof(T) == 8, ArithF64, ArithF32>::type;

// fc(I,J,K) = full weighting of r around fine site (2I+1, 2J+1, 2K+1).
template <typename T>
__global__ void __launch_bounds__(128) mg_restrict_kernel(const T* __restrict__ r, Geom gf, T* __restrict__ fc,
                                                          Geom gc) {
  using A = MGArith<T>;
  const T q = T(0.25), hf = T(0.5);
  const int I = blockIdx.x * 32 + threadIdx.x;
  const int J = blockIdx.y * 4 + threadIdx.y;
  const int K = blockIdx.z;
  if (I >= gc.nx || J >= gc.ny) return;
  T sy[3];
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz) {
    T sx[3];
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int64_t c = gf.at(2 * I + 1, 2 * J + 1 + dy, 2 * K + 1 + dz);
      sx[dy + 1] = A::add(A::add(A::mul(q, r[c - 1]), A::mul(hf, r[c])), A::mul(q, r[c + 1]));
    }
    sy[dz + 1] = A::add(A::add(A::mul(q, sx[0]), A::mul(hf, sx[1])), A::mul(q, sx[2]));
  }
  fc[gc.at(I, J, K)] = A::add(A::add(A::mul(q, sy[0]), A::mul(hf, sy[1])), A::mul(q, sy[2]));
}

// u(i,j,k) += trilinear interpolation of e (coarse, zero halo): per axis an odd
// fine index takes coarse site (i-1)/2, an even one the mean of coarse sites
// i/2-1 and i/2 (-1 and n_c being the zero halo); x, then y, then z.
template <typename T>
__global__ void __launch_bounds__(128) mg_prolong_add_kernel(T* __restrict__ u, Geom gf, const T* __restrict__ e,
                                                             Geom gc) {
  using A = MGArith<T>;
  const T hf = T(0.5);
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 4 + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= gf.nx || j >= gf.ny) return;
  const int xa = (i & 1) ? (i - 1) / 2 : i / 2 - 1, xb = (i & 1) ? xa : i / 2;
  const int ya = (j & 1) ? (j - 1) / 2 : j / 2 - 1, yb = (j & 1) ? ya : j / 2;
  const int za = (k & 1) ? (k - 1) / 2 : k / 2 - 1, zb = (k & 1) ? za : k / 2;
  T ey[2];
#pragma unroll
  for (int zz = 0; zz < 2; ++zz) {
    const int Z = zz ? zb : za;
    T ex[2];
#pragma unroll
    for (int yy = 0; yy < 2; ++yy) {
      const int Y = yy ? yb : ya;
      const T a = e[gc.at(xa, Y, Z)];
      ex[yy] = (i & 1) ? a : A::mul(A::add(a, e[gc.at(xb, Y, Z)]), hf);
    }
    ey[zz] = (j & 1) ? ex[0] : A::mul(A::add(ex[0], ex[1]), hf);
  }
  const T ez = (k & 1) ? ey[0] : A::mul(A::add(ey[0], ey[1]), hf);
  const int64_t c = gf.at(i, j, k);
  u[c] = A::add(u[c], ez);
}

namespace {

template <typename T>
struct MGLevel {
  Geom g;
  double h;
  T* u;
  const T* f;
  T* fw;  // writable right-hand side (coarse levels)
};

template <typename T>
struct MGRun {
  stencil_ctx* ctx;
  std::vector<MGLevel<T>> lv;
  T* r = nullptr;
  int smoother, nu1, nu2, ncoarse;
  cudaStream_t st;
};

// Smoothing sweeps on level l in the level's precision: weighted Jacobi
// (a = b = 1/7 rounded to T), lexicographic or red-black Gauss-Seidel (b = 1/6).
template <typename T>
int mg_smooth(MGRun<T>& m, int l, int nsweeps) {
  if (nsweeps <= 0) return STENCIL_OK;
  MGLevel<T>& L = m.lv[(size_t)l];
  stencil_params q{};
  q.int_adds = -1;
  if (m.smoother == STENCIL_JACOBI) {
    q.a = 1.0 / 7.0;
    q.b = 1.0 / 7.0;
    return jacobi_run<T>(m.ctx, L.u, L.f, L.g, L.h, nsweeps, &q, m.st);
  }
  if (m.smoother == STENCIL_GS_RB) return gs_rb_run<T>(m.ctx, L.u, L.f, L.g, L.h, nsweeps, &q, m.st);
  return gs_run<T>(m.ctx, L.u, L.f, L.g, L.h, nsweeps, &q, m.st);
}

// r = f - A u on level L into m.r (no norm).
int mg_residual(MGRun<double>& m, MGLevel<double>& L) {
  double* dres;
  return residual_launch(m.ctx, L.u, L.f, L.g, L.h, m.r, nullptr, &dres, m.st, false);
}
int mg_residual(MGRun<float>& m, MGLevel<float>& L) {
  return residual32_launch(m.ctx, L.u, L.f, L.g, L.h, m.r, m.st);
}

template <typename T>
int mg_vcycle(MGRun<T>& m, int l) {
  const int nlev = (int)m.lv.size();
  if (l == nlev - 1) return mg_smooth(m, l, m.ncoarse);
  MGLevel<T>& L = m.lv[(size_t)l];
  MGLevel<T>& C = m.lv[(size_t)l + 1];
  int rc = mg_smooth(m, l, m.nu1);
  if (rc) return rc;
  if ((rc = mg_residual(m, L))) return rc;
  mg_restrict_kernel<T><<<dim3((C.g.nx + 31) / 32, (C.g.ny + 3) / 4, C.g.nz), dim3(32, 4), 0, m.st>>>(m.r, L.g, C.fw,
                                                                                                      C.g);
  m.ctx->launches++;
  cudaError_t e = cudaMemsetAsync(C.u, 0, (size_t)C.g.sy * (size_t)(C.g.nz + 2) * sizeof(T), m.st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(m.ctx, e, "multigrid restriction");
  if ((rc = mg_vcycle(m, l + 1))) return rc;
  mg_prolong_add_kernel<T><<<dim3((L.g.nx + 31) / 32, (L.g.ny + 3) / 4, L.g.nz), dim3(32, 4), 0, m.st>>>(L.u, L.g,
                                                                                                         C.u, C.g);
  m.ctx->launches++;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(m.ctx, e, "multigrid prolongation");
  return mg_smooth(m, l, m.nu2);
}

// One V-cycle, replayed from a CUDA graph once the same cycle recurs.  A call's
// first cycle with given arguments runs its launches directly (it also sets up
// the workspace and tile tables); the next one is captured into a graph (one
// launch of some hundred kernels instead of as many launches, which is what
// bounds the cycles of small grids); later ones replay it.  The graph is kept
// in the context, keyed by the arguments, every level's buffers and the
// workspace generation (a reallocated slot or an evicted table makes a new
// key), for later calls on the same grids (the served solves call once per
// round).  A capture that fails falls back to direct launches.
template <typename T>
int mg_cycle(MGRun<T>& m) {
  stencil_ctx* ctx = m.ctx;
  std::vector<int64_t> key = {(int64_t)sizeof(T), m.smoother, m.nu1, m.nu2, m.ncoarse, (int64_t)m.lv.size(),
                              (int64_t)(intptr_t)m.r, (int64_t)ctx->ws_gen};
  for (const MGLevel<T>& L : m.lv) {
    int64_t hb;
    memcpy(&hb, &L.h, sizeof(hb));
    key.insert(key.end(), {L.g.nx, L.g.ny, L.g.nz, hb, (int64_t)(intptr_t)L.u, (int64_t)(intptr_t)L.f});
  }
  MGGraph* e = nullptr;
  for (MGGraph& c : ctx->mg_graphs)
    if (c.key == key) e = &c;
  if (!e) {
    if (ctx->mg_graphs.size() >= 32) {  // drop the least recently used
      auto it = std::min_element(ctx->mg_graphs.begin(), ctx->mg_graphs.end(),
                                 [](const MGGraph& a, const MGGraph& b) { return a.last_use < b.last_use; });
      if (it->exec) cudaGraphExecDestroy(it->exec);
      ctx->mg_graphs.erase(it);
    }
    ctx->mg_graphs.push_back(MGGraph{});
    e = &ctx->mg_graphs.back();
    e->key = key;
  }
  e->last_use = ++ctx->mg_clock;
  if (e->exec) {
    cudaError_t err = cudaGraphLaunch(e->exec, m.st);
    if (err != cudaSuccess) return cuda_err(ctx, err, "multigrid cycle graph");
    ctx->launches += e->nlaunch;
    return STENCIL_OK;
  }
  if (e->uses < 0) return mg_vcycle(m, 0);     // a capture of these arguments failed before
  if (e->uses++ == 0) return mg_vcycle(m, 0);  // first use: direct
  if (!ctx->cstream) {
    cudaError_t err = cudaStreamCreateWithFlags(&ctx->cstream, cudaStreamNonBlocking);
    if (err != cudaSuccess) return cuda_err(ctx, err, "cudaStreamCreate");
  }
  MGRun<T> mc = m;
  mc.st = ctx->cstream;
  const unsigned long long l0 = ctx->launches;
  const std::string saved = ctx->err;
  cudaError_t err = cudaStreamBeginCapture(mc.st, cudaStreamCaptureModeThreadLocal);
  int rc = err == cudaSuccess ? mg_vcycle(mc, 0) : STENCIL_ERR_CUDA;
  cudaGraph_t graph = nullptr;
  if (err == cudaSuccess) err = cudaStreamEndCapture(mc.st, &graph);
  const unsigned long long n = ctx->launches - l0;
  ctx->launches = l0;  // the capture launched nothing
  cudaGraphExec_t exec = nullptr;
  if (rc == STENCIL_OK && err == cudaSuccess && graph) err = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (rc != STENCIL_OK || err != cudaSuccess || !exec) {
    cudaGetLastError();
    ctx->err = saved;
    e->uses = -1;
    return mg_vcycle(m, 0);
  }
  e->exec = exec;
  e->nlaunch = n;
  err = cudaGraphLaunch(exec, m.st);
  if (err != cudaSuccess) return cuda_err(ctx, err, "multigrid cycle graph");
  ctx->launches += n;
  return STENCIL_OK;
}

// Builds the level hierarchy over (u, f) on g0 and takes its workspace: every
// coarse level's correction and right-hand side from slot `levels` (halos
// zeroed once), one residual grid of the finest size from slot `rslot`.
template <typename T>
int mg_setup(stencil_ctx* ctx, MGRun<T>& m, T* u, const T* f, const Geom& g0, double h, int max_levels,
             SlotId levels, SlotId rslot) {
  m.lv.clear();
  m.lv.push_back(MGLevel<T>{g0, h, u, f, nullptr});
  while ((int)m.lv.size() < max_levels) {
    const Geom& p = m.lv.back().g;
    if (p.nx < 3 || p.ny < 3 || p.nz < 3 || p.nx % 2 == 0 || p.ny % 2 == 0 || p.nz % 2 == 0) break;
    m.lv.push_back(MGLevel<T>{make_geom((p.nx - 1) / 2, (p.ny - 1) / 2, (p.nz - 1) / 2), 2.0 * m.lv.back().h,
                              nullptr, nullptr, nullptr});
  }
  size_t coarse = 0;
  for (size_t l = 1; l < m.lv.size(); ++l) coarse += 2 * (size_t)m.lv[l].g.sy * (size_t)(m.lv[l].g.nz + 2);
  if (coarse == 0) return STENCIL_OK;
  int status;
  T* base = (T*)ws_get(ctx, levels, coarse * sizeof(T), &status);
  if (!base) return status;
  m.r = (T*)ws_get(ctx, rslot, (size_t)g0.sy * (size_t)(g0.nz + 2) * sizeof(T), &status);
  if (!m.r) return status;
  cudaError_t e = cudaMemsetAsync(base, 0, coarse * sizeof(T), m.st);  // zero halos of every coarse grid
  if (e != cudaSuccess) return cuda_err(ctx, e, "multigrid workspace");
  for (size_t l = 1; l < m.lv.size(); ++l) {
    const size_t n = (size_t)m.lv[l].g.sy * (size_t)(m.lv[l].g.nz + 2);
    m.lv[l].u = base;
    m.lv[l].fw = base + n;
    m.lv[l].f = m.lv[l].fw;
    base += 2 * n;
  }
  return STENCIL_OK;
}

int mg_checks(stencil_ctx* ctx, const void* u, const int64_t dims[3], double h, int smoother, int nu1, int nu2,
              int ncoarse, int max_levels, double rtol, int max_cycles, Geom* g0) {
  if (!ctx) return STENCIL_ERR_ARG;
  ctx->err.clear();
  int rc = check_dims(ctx, dims, g0);
  if (rc) return rc;
  if (!u) return set_err(ctx, STENCIL_ERR_ARG, "u is NULL");
  if (!(h > 0.0) || !std::isfinite(h)) return set_err(ctx, STENCIL_ERR_ARG, "h must be finite and > 0");
  if (smoother != STENCIL_JACOBI && smoother != STENCIL_GS && smoother != STENCIL_GS_RB)
    return set_err(ctx, STENCIL_ERR_ARG, "bad smoother");
  if (nu1 < 0 || nu2 < 0 || ncoarse < 0 || max_cycles < 0 || !(rtol >= 0.0))
    return set_err(ctx, STENCIL_ERR_ARG, "bad sweep counts or limits");
  if (max_levels < 1 || max_levels > 32) return set_err(ctx, STENCIL_ERR_ARG, "max_levels must be in 1..32");
  if (g0->nz > 65535) return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "multigrid: nz = %d > 65535", g0->nz);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  return STENCIL_OK;
}

}  // namespace
}  // namespace stn

using namespace stn;

extern "C" int stencil_mg_solve(stencil_ctx* ctx, double* u, const double* f, const int64_t dims[3], double h,
                                int smoother, int nu1, int nu2, int ncoarse, int max_levels, double rtol,
                                int max_cycles, double* out_rel, int* out_cycles, void* stream) {
  Geom g0;
  int rc = mg_checks(ctx, u, dims, h, smoother, nu1, nu2, ncoarse, max_levels, rtol, max_cycles, &g0);
  if (rc) return rc;
  MGRun<double> m;
  m.ctx = ctx;
  m.smoother = smoother;
  m.nu1 = nu1;
  m.nu2 = nu2;
  m.ncoarse = ncoarse;
  m.st = (cudaStream_t)stream;
  if ((rc = mg_setup(ctx, m, u, f, g0, h, max_levels, SLOT_MG_LEVELS, SLOT_MG_R))) return rc;
  double* dres;
  double sums[2];
  if ((rc = residual_launch(ctx, u, f, g0, h, nullptr, nullptr, &dres, m.st))) return rc;
  if ((rc = read_sums(ctx, dres, sums, m.st))) return rc;
  const double fn = std::sqrt(sums[1]);
  double rn = std::sqrt(sums[0]);
  const double denom = fn > 0.0 ? fn : rn;
  double rel = denom > 0.0 ? rn / denom : 0.0;
  int it = 0;
  while (rel > rtol && it < max_cycles) {
    if ((rc = mg_cycle(m))) return rc;
    ++it;
    if ((rc = residual_launch(ctx, u, f, g0, h, nullptr, nullptr, &dres, m.st))) return rc;
    if ((rc = read_sums(ctx, dres, sums, m.st))) return rc;
    rn = std::sqrt(sums[0]);
    rel = denom > 0.0 ? rn / denom : 0.0;
  }
  if (out_rel) *out_rel = rel;
  if (out_cycles) *out_cycles = it;
  return rel <= rtol ? STENCIL_OK : STENCIL_ERR_NOT_CONVERGED;
}

// Defect correction with an FP32 multigrid inner solver: the FP64 residual
// (which also gives the stopping test) is rounded to FP32 in the same pass,
// inner_cycles FP32 V-cycles solve A e = r32 from e = 0 on the same level
// hierarchy, and u += (double) e in FP64.
extern "C" int stencil_solve_mixed_mg(stencil_ctx* ctx, double* u, const double* f, const int64_t dims[3], double h,
                                      int smoother, int nu1, int nu2, int ncoarse, int max_levels, double rtol,
                                      int max_outer, int inner_cycles, double* out_rel, int* out_iters,
                                      void* stream) {
  Geom g0;
  int rc = mg_checks(ctx, u, dims, h, smoother, nu1, nu2, ncoarse, max_levels, rtol, max_outer, &g0);
  if (rc) return rc;
  if (inner_cycles < 0) return set_err(ctx, STENCIL_ERR_ARG, "inner_cycles = %d < 0", inner_cycles);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = (size_t)g0.sy * (size_t)(g0.nz + 2);
  int status;
  float* r32 = (float*)ws_get(ctx, SLOT_MIX_R32, n * sizeof(float), &status);
  if (!r32) return status;
  float* e32 = (float*)ws_get(ctx, SLOT_MIX_E32, n * sizeof(float), &status);
  if (!e32) return status;
  cudaError_t e = cudaMemsetAsync(r32, 0, n * sizeof(float), st);  // r32's halo is never read: defined anyway
  if (e != cudaSuccess) return cuda_err(ctx, e, "memset r32");
  MGRun<float> m;
  m.ctx = ctx;
  m.smoother = smoother;
  m.nu1 = nu1;
  m.nu2 = nu2;
  m.ncoarse = ncoarse;
  m.st = st;
  if ((rc = mg_setup(ctx, m, e32, (const float*)r32, g0, h, max_levels, SLOT_MG32_LEVELS, SLOT_MG32_R))) return rc;
  double* dres;
  double sums[2];
  if ((rc = residual_launch(ctx, u, f, g0, h, nullptr, r32, &dres, st))) return rc;
  if ((rc = read_sums(ctx, dres, sums, st))) return rc;
  const double fn = std::sqrt(sums[1]);
  double rn = std::sqrt(sums[0]);
  const double denom = fn > 0.0 ? fn : rn;
  double rel = denom > 0.0 ? rn / denom : 0.0;
  int it = 0;
  while (rel > rtol && it < max_outer) {
    e = cudaMemsetAsync(e32, 0, n * sizeof(float), st);
    if (e != cudaSuccess) return cuda_err(ctx, e, "memset e32");
    for (int c = 0; c < inner_cycles; ++c)
      if ((rc = mg_cycle(m))) return rc;
    if ((rc = correct_launch(ctx, u, e32, g0, st))) return rc;
    ++it;
    if ((rc = residual_launch(ctx, u, f, g0, h, nullptr, r32, &dres, st))) return rc;
    if ((rc = read_sums(ctx, dres, sums, st))) return rc;
    rn = std::sqrt(sums[0]);
    rel = denom > 0.0 ? rn / denom : 0.0;
  }
  if (out_rel) *out_rel = rel;
  if (out_iters) *out_iters = it;
  if (rel > rtol)
    return set_err(ctx, STENCIL_ERR_NOT_CONVERGED, "relative residual %.3e > %.3e after %d outer", rel, rtol, it);
  return STENCIL_OK;
}
