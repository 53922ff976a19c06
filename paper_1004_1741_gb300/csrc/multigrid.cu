// Multigrid V-cycle solve of -Lap_h u = f with the library's smoothers.
//
// Sec. 1 and Sec. 3 name multigrid solvers as the place where Jacobi and
// Gauss-Seidel smoothers spend their time; the paper does not define the
// cycle, so the textbook one is used: level l+1 has extents (n-1)/2 and
// spacing 2h while every extent is odd and >= 3 (coarse site I on fine site
// 2I+1); nu1 smoothing sweeps, residual, full-weighting restriction, the
// coarse correction from zero with zero Dirichlet values, trilinear
// prolongation added to u, nu2 smoothing sweeps; ncoarse sweeps on the
// coarsest level.  Smoothers: weighted Jacobi with omega = 6/7 (a = b = 1/7)
// or lexicographic Gauss-Seidel (b = 1/6).  The transfers are written in one
// fixed order of IEEE operations (x, then y, then z; each weighted mean as
// ((w a + w' b) + w c), each interpolated mean as (a + b) * 0.5), so the
// whole cycle is deterministic and the same bits as the serial definition.
#include <cmath>
#include <vector>

#include "internal.h"

namespace stn {

// fc(I,J,K) = full weighting of r around fine site (2I+1, 2J+1, 2K+1).
__global__ void __launch_bounds__(128) mg_restrict_kernel(const double* __restrict__ r, Geom gf,
                                                          double* __restrict__ fc, Geom gc) {
  const int I = blockIdx.x * 32 + threadIdx.x;
  const int J = blockIdx.y * 4 + threadIdx.y;
  const int K = blockIdx.z;
  if (I >= gc.nx || J >= gc.ny) return;
  double sy[3];
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz) {
    double sx[3];
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int64_t c = gf.at(2 * I + 1, 2 * J + 1 + dy, 2 * K + 1 + dz);
      sx[dy + 1] = __dadd_rn(__dadd_rn(__dmul_rn(0.25, r[c - 1]), __dmul_rn(0.5, r[c])), __dmul_rn(0.25, r[c + 1]));
    }
    sy[dz + 1] = __dadd_rn(__dadd_rn(__dmul_rn(0.25, sx[0]), __dmul_rn(0.5, sx[1])), __dmul_rn(0.25, sx[2]));
  }
  fc[gc.at(I, J, K)] = __dadd_rn(__dadd_rn(__dmul_rn(0.25, sy[0]), __dmul_rn(0.5, sy[1])), __dmul_rn(0.25, sy[2]));
}

// u(i,j,k) += trilinear interpolation of e (coarse, zero halo): per axis an odd
// fine index takes coarse site (i-1)/2, an even one the mean of coarse sites
// i/2-1 and i/2 (-1 and n_c being the zero halo); x, then y, then z.
__global__ void __launch_bounds__(128) mg_prolong_add_kernel(double* __restrict__ u, Geom gf,
                                                             const double* __restrict__ e, Geom gc) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 4 + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= gf.nx || j >= gf.ny) return;
  const int xa = (i & 1) ? (i - 1) / 2 : i / 2 - 1, xb = (i & 1) ? xa : i / 2;
  const int ya = (j & 1) ? (j - 1) / 2 : j / 2 - 1, yb = (j & 1) ? ya : j / 2;
  const int za = (k & 1) ? (k - 1) / 2 : k / 2 - 1, zb = (k & 1) ? za : k / 2;
  double ey[2];
#pragma unroll
  for (int zz = 0; zz < 2; ++zz) {
    const int Z = zz ? zb : za;
    double ex[2];
#pragma unroll
    for (int yy = 0; yy < 2; ++yy) {
      const int Y = yy ? yb : ya;
      const double a = e[gc.at(xa, Y, Z)];
      ex[yy] = (i & 1) ? a : __dmul_rn(__dadd_rn(a, e[gc.at(xb, Y, Z)]), 0.5);
    }
    ey[zz] = (j & 1) ? ex[0] : __dmul_rn(__dadd_rn(ex[0], ex[1]), 0.5);
  }
  const double ez = (k & 1) ? ey[0] : __dmul_rn(__dadd_rn(ey[0], ey[1]), 0.5);
  const int64_t c = gf.at(i, j, k);
  u[c] = __dadd_rn(u[c], ez);
}

namespace {

struct MGLevel {
  Geom g;
  double h;
  double* u;
  const double* f;
  double* fw;  // writable right-hand side (coarse levels)
};

struct MGRun {
  stencil_ctx* ctx;
  std::vector<MGLevel> lv;
  double* r;
  int smoother, nu1, nu2, ncoarse;
  cudaStream_t st;
};

int mg_smooth(MGRun& m, int l, int nsweeps) {
  if (nsweeps <= 0) return STENCIL_OK;
  MGLevel& L = m.lv[(size_t)l];
  stencil_params q{};
  q.int_adds = -1;
  if (m.smoother == STENCIL_JACOBI) {
    q.a = 1.0 / 7.0;
    q.b = 1.0 / 7.0;
    return jacobi_run<double>(m.ctx, L.u, L.f, L.g, L.h, nsweeps, &q, m.st);
  }
  return gs_run<double>(m.ctx, L.u, L.f, L.g, L.h, nsweeps, &q, m.st);
}

int mg_vcycle(MGRun& m, int l) {
  const int nlev = (int)m.lv.size();
  if (l == nlev - 1) return mg_smooth(m, l, m.ncoarse);
  MGLevel& L = m.lv[(size_t)l];
  MGLevel& C = m.lv[(size_t)l + 1];
  int rc = mg_smooth(m, l, m.nu1);
  if (rc) return rc;
  double* dres;
  if ((rc = residual_launch(m.ctx, L.u, L.f, L.g, L.h, m.r, nullptr, &dres, m.st, false))) return rc;
  mg_restrict_kernel<<<dim3((C.g.nx + 31) / 32, (C.g.ny + 3) / 4, C.g.nz), dim3(32, 4), 0, m.st>>>(m.r, L.g, C.fw,
                                                                                                   C.g);
  m.ctx->launches++;
  cudaError_t e = cudaMemsetAsync(C.u, 0, (size_t)C.g.sy * (size_t)(C.g.nz + 2) * sizeof(double), m.st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(m.ctx, e, "multigrid restriction");
  if ((rc = mg_vcycle(m, l + 1))) return rc;
  mg_prolong_add_kernel<<<dim3((L.g.nx + 31) / 32, (L.g.ny + 3) / 4, L.g.nz), dim3(32, 4), 0, m.st>>>(L.u, L.g, C.u,
                                                                                                      C.g);
  m.ctx->launches++;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(m.ctx, e, "multigrid prolongation");
  return mg_smooth(m, l, m.nu2);
}

}  // namespace
}  // namespace stn

using namespace stn;

extern "C" int stencil_mg_solve(stencil_ctx* ctx, double* u, const double* f, const int64_t dims[3], double h,
                                int smoother, int nu1, int nu2, int ncoarse, int max_levels, double rtol,
                                int max_cycles, double* out_rel, int* out_cycles, void* stream) {
  if (!ctx) return STENCIL_ERR_ARG;
  ctx->err.clear();
  Geom g0;
  int rc = check_dims(ctx, dims, &g0);
  if (rc) return rc;
  if (!u) return set_err(ctx, STENCIL_ERR_ARG, "u is NULL");
  if (!(h > 0.0) || !std::isfinite(h)) return set_err(ctx, STENCIL_ERR_ARG, "h must be finite and > 0");
  if (smoother != STENCIL_JACOBI && smoother != STENCIL_GS) return set_err(ctx, STENCIL_ERR_ARG, "bad smoother");
  if (nu1 < 0 || nu2 < 0 || ncoarse < 0 || max_cycles < 0 || !(rtol >= 0.0))
    return set_err(ctx, STENCIL_ERR_ARG, "bad sweep counts or limits");
  if (max_levels < 1 || max_levels > 32) return set_err(ctx, STENCIL_ERR_ARG, "max_levels must be in 1..32");
  if (g0.nz > 65535) return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "multigrid: nz = %d > 65535", g0.nz);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  MGRun m;
  m.ctx = ctx;
  m.smoother = smoother;
  m.nu1 = nu1;
  m.nu2 = nu2;
  m.ncoarse = ncoarse;
  m.st = (cudaStream_t)stream;
  m.lv.push_back(MGLevel{g0, h, u, f, nullptr});
  while ((int)m.lv.size() < max_levels) {
    const Geom& p = m.lv.back().g;
    if (p.nx < 3 || p.ny < 3 || p.nz < 3 || p.nx % 2 == 0 || p.ny % 2 == 0 || p.nz % 2 == 0) break;
    m.lv.push_back(MGLevel{make_geom((p.nx - 1) / 2, (p.ny - 1) / 2, (p.nz - 1) / 2), 2.0 * m.lv.back().h, nullptr,
                           nullptr, nullptr});
  }
  // workspace: every coarse level's correction and right-hand side; one residual grid of the finest size
  size_t coarse = 0;
  for (size_t l = 1; l < m.lv.size(); ++l) coarse += 2 * (size_t)m.lv[l].g.sy * (size_t)(m.lv[l].g.nz + 2);
  int status;
  if (coarse > 0) {
    double* base = (double*)ws_get(ctx, SLOT_MG_LEVELS, coarse * sizeof(double), &status);
    if (!base) return status;
    m.r = (double*)ws_get(ctx, SLOT_MG_R, (size_t)g0.sy * (size_t)(g0.nz + 2) * sizeof(double), &status);
    if (!m.r) return status;
    e = cudaMemsetAsync(base, 0, coarse * sizeof(double), m.st);  // zero halos of every coarse grid
    if (e != cudaSuccess) return cuda_err(ctx, e, "multigrid workspace");
    for (size_t l = 1; l < m.lv.size(); ++l) {
      const size_t n = (size_t)m.lv[l].g.sy * (size_t)(m.lv[l].g.nz + 2);
      m.lv[l].u = base;
      m.lv[l].fw = base + n;
      m.lv[l].f = m.lv[l].fw;
      base += 2 * n;
    }
  }
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
    if ((rc = mg_vcycle(m, 0))) return rc;
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
