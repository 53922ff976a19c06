/*
 * Oracle for the 3D 7-point Jacobi and lexicographic Gauss-Seidel smoothers.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library and its Python binding) never calls it and shares no
 * code, header, table or constant with it.
 *
 * Everything here is the plain serial definition, written out loop by loop:
 *
 *  - Jacobi (Sec. 3, first listing): out of place, two arrays, every site
 *        dst = a*src + b*(W + E + S + N + B + T)
 *    with the neighbour sum taken left to right in the listing's order
 *    (i-1, i+1, j-1, j+1, k-1, k+1).  For a Poisson right-hand side
 *    (Sec. 3 names "the Jacobi method for a Poisson problem") the reading is
 *    -Lap_h u = f, so the bracket becomes (sum + h*h*f).  With a == 0 the
 *    a*src term is dropped.
 *  - Gauss-Seidel (Sec. 3, second listing): in place, k outermost, then j,
 *    then i, all ascending; at the moment of an update the i-1, j-1, k-1
 *    neighbours already hold this sweep's values.
 *  - Residual r = f - A u with A u = (6 u - sum) / h^2, and its 2-norm
 *    (not in the paper; compensated summation so the oracle's norm is
 *    correct to rounding).
 *  - Defect correction with single-precision inner sweeps (not in the
 *    paper): r in double, e solves A e = r by FP32 sweeps from e = 0,
 *    u += e in double.
 *
 * Storage: (nz+2)(ny+2)(nx+2) elements, C order u[k][j][i], i fastest, with a
 * one-cell Dirichlet halo that is read, never written.  Halo edges and
 * corners are never read.
 *
 * Build with -O2 -ffp-contract=off -fno-fast-math: every + and * below is
 * one IEEE-754 operation rounded to nearest, never fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_OOM (-2)
#define ORC_NOT_CONVERGED (-5)

typedef struct {
  int64_t nx, ny, nz; /* interior extents */
  int64_t sx, sy;     /* strides of j and k in elements: sx = nx+2, sy = (nx+2)(ny+2) */
} orc_grid;

static int orc_grid_make(orc_grid* g, int64_t nx, int64_t ny, int64_t nz) {
  if (nx < 0 || ny < 0 || nz < 0) return ORC_ERR_ARG;
  g->nx = nx; g->ny = ny; g->nz = nz;
  g->sx = nx + 2;
  g->sy = (nx + 2) * (ny + 2);
  return ORC_OK;
}

static size_t orc_total(const orc_grid* g) { return (size_t)g->sy * (size_t)(g->nz + 2); }

/* index of interior site (i,j,k), 0-based interior coordinates */
static size_t orc_at(const orc_grid* g, int64_t i, int64_t j, int64_t k) {
  return (size_t)((k + 1) * g->sy + (j + 1) * g->sx + (i + 1));
}

/* ---------------------------------------------------------------------------
 * Double precision
 * ------------------------------------------------------------------------- */

/* Neighbour sum in the listing's order, left to right. */
static double orc_sum_d(const double* u, size_t c, int64_t sx, int64_t sy) {
  double s = u[c - 1] + u[c + 1];
  s = s + u[c - sx];
  s = s + u[c + sx];
  s = s + u[c - sy];
  s = s + u[c + sy];
  return s;
}

/* One site of the smoother: a*u + b*(sum + hh*f). */
static double orc_site_d(const double* src, const double* f, size_t c, int64_t sx, int64_t sy,
                         double a, double b, double hh) {
  double t = orc_sum_d(src, c, sx, sy);
  if (f) t = t + hh * f[c];
  double v = b * t;
  if (a != 0.0) v = a * src[c] + v;
  return v;
}

/* Jacobi, Sec. 3 first listing: nsweeps out-of-place sweeps, result in u. */
int oracle_jacobi_f64(double* u, const double* f, int64_t nx, int64_t ny, int64_t nz, double h,
                      double a, double b, int nsweeps) {
  orc_grid g;
  if (!u || nsweeps < 0 || orc_grid_make(&g, nx, ny, nz) != ORC_OK) return ORC_ERR_ARG;
  if (nsweeps == 0 || nx == 0 || ny == 0 || nz == 0) return ORC_OK;
  size_t n = orc_total(&g);
  double* tmp = (double*)malloc(n * sizeof(double));
  if (!tmp) return ORC_ERR_OOM;
  memcpy(tmp, u, n * sizeof(double)); /* the second array carries the same halo */
  const double hh = h * h;
  double* src = u;
  double* dst = tmp;
  for (int it = 0; it < nsweeps; ++it) {
    for (int64_t k = 0; k < nz; ++k)
      for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
          size_t c = orc_at(&g, i, j, k);
          dst[c] = orc_site_d(src, f, c, g.sx, g.sy, a, b, hh);
        }
    double* sw = src; src = dst; dst = sw;
  }
  if (src != u) memcpy(u, src, n * sizeof(double));
  free(tmp);
  return ORC_OK;
}

/* Gauss-Seidel, Sec. 3 second listing: in place, lexicographic. */
int oracle_gs_lex_f64(double* u, const double* f, int64_t nx, int64_t ny, int64_t nz, double h,
                      double b, int nsweeps) {
  orc_grid g;
  if (!u || nsweeps < 0 || orc_grid_make(&g, nx, ny, nz) != ORC_OK) return ORC_ERR_ARG;
  const double hh = h * h;
  for (int it = 0; it < nsweeps; ++it)
    for (int64_t k = 0; k < nz; ++k)
      for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
          size_t c = orc_at(&g, i, j, k);
          u[c] = orc_site_d(u, f, c, g.sx, g.sy, 0.0, b, hh);
        }
  return ORC_OK;
}

/* Red-black Gauss-Seidel (Sec. 3 names it as the usual parallel
 * alternative): all sites with (i+j+k) even, then all with (i+j+k) odd, each
 * colour in lexicographic order, in place.  Interior coordinates 0-based. */
int oracle_gs_rb_f64(double* u, const double* f, int64_t nx, int64_t ny, int64_t nz, double h,
                     double b, int nsweeps) {
  orc_grid g;
  if (!u || nsweeps < 0 || orc_grid_make(&g, nx, ny, nz) != ORC_OK) return ORC_ERR_ARG;
  const double hh = h * h;
  for (int it = 0; it < nsweeps; ++it)
    for (int colour = 0; colour < 2; ++colour)
      for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
          for (int64_t i = 0; i < nx; ++i) {
            if (((i + j + k) & 1) != colour) continue;
            size_t c = orc_at(&g, i, j, k);
            u[c] = orc_site_d(u, f, c, g.sx, g.sy, 0.0, b, hh);
          }
  return ORC_OK;
}

/* Neumaier-compensated accumulation of x into (s, c). */
static void orc_acc(double* s, double* c, double x) {
  double t = *s + x;
  if (fabs(*s) >= fabs(x))
    *c += (*s - t) + x;
  else
    *c += (x - t) + *s;
  *s = t;
}

/* Residual r = f - A u, A u = (6 u - sum) * (1/h^2), f == NULL meaning f = 0.
 * r (optional) receives the residual on the interior (halo untouched).
 * out_norm receives ||r||_2 over the interior; out_fnorm (optional) ||f||_2. */
int oracle_residual_f64(const double* u, const double* f, int64_t nx, int64_t ny, int64_t nz,
                        double h, double* r, double* out_norm, double* out_fnorm) {
  orc_grid g;
  if (!u || !out_norm || orc_grid_make(&g, nx, ny, nz) != ORC_OK || !(h > 0.0)) return ORC_ERR_ARG;
  const double ih2 = 1.0 / (h * h);
  double s = 0.0, cs = 0.0, fs = 0.0, fc = 0.0;
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        size_t c = orc_at(&g, i, j, k);
        double au = (6.0 * u[c] - orc_sum_d(u, c, g.sx, g.sy)) * ih2;
        double fv = f ? f[c] : 0.0;
        double rv = fv - au;
        if (r) r[c] = rv;
        orc_acc(&s, &cs, rv * rv);
        orc_acc(&fs, &fc, fv * fv);
      }
  *out_norm = sqrt(s + cs);
  if (out_fnorm) *out_fnorm = sqrt(fs + fc);
  return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Single precision: the same definitions with every operation in float.
 * hh = (float)(h*h), b given as the float constant.
 * ------------------------------------------------------------------------- */

static float orc_sum_s(const float* u, size_t c, int64_t sx, int64_t sy) {
  float s = u[c - 1] + u[c + 1];
  s = s + u[c - sx];
  s = s + u[c + sx];
  s = s + u[c - sy];
  s = s + u[c + sy];
  return s;
}

static float orc_site_s(const float* src, const float* f, size_t c, int64_t sx, int64_t sy,
                        float a, float b, float hh) {
  float t = orc_sum_s(src, c, sx, sy);
  if (f) t = t + hh * f[c];
  float v = b * t;
  if (a != 0.0f) v = a * src[c] + v;
  return v;
}

int oracle_jacobi_f32(float* u, const float* f, int64_t nx, int64_t ny, int64_t nz, double h,
                      float a, float b, int nsweeps) {
  orc_grid g;
  if (!u || nsweeps < 0 || orc_grid_make(&g, nx, ny, nz) != ORC_OK) return ORC_ERR_ARG;
  if (nsweeps == 0 || nx == 0 || ny == 0 || nz == 0) return ORC_OK;
  size_t n = orc_total(&g);
  float* tmp = (float*)malloc(n * sizeof(float));
  if (!tmp) return ORC_ERR_OOM;
  memcpy(tmp, u, n * sizeof(float));
  const float hh = (float)(h * h);
  float* src = u;
  float* dst = tmp;
  for (int it = 0; it < nsweeps; ++it) {
    for (int64_t k = 0; k < nz; ++k)
      for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
          size_t c = orc_at(&g, i, j, k);
          dst[c] = orc_site_s(src, f, c, g.sx, g.sy, a, b, hh);
        }
    float* sw = src; src = dst; dst = sw;
  }
  if (src != u) memcpy(u, src, n * sizeof(float));
  free(tmp);
  return ORC_OK;
}

int oracle_gs_lex_f32(float* u, const float* f, int64_t nx, int64_t ny, int64_t nz, double h,
                      float b, int nsweeps) {
  orc_grid g;
  if (!u || nsweeps < 0 || orc_grid_make(&g, nx, ny, nz) != ORC_OK) return ORC_ERR_ARG;
  const float hh = (float)(h * h);
  for (int it = 0; it < nsweeps; ++it)
    for (int64_t k = 0; k < nz; ++k)
      for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
          size_t c = orc_at(&g, i, j, k);
          u[c] = orc_site_s(u, f, c, g.sx, g.sy, 0.0f, b, hh);
        }
  return ORC_OK;
}

/* Red-black Gauss-Seidel in single precision (same order as the FP64 one). */
int oracle_gs_rb_f32(float* u, const float* f, int64_t nx, int64_t ny, int64_t nz, double h, float b,
                     int nsweeps) {
  orc_grid g;
  if (!u || nsweeps < 0 || orc_grid_make(&g, nx, ny, nz) != ORC_OK) return ORC_ERR_ARG;
  const float hh = (float)(h * h);
  for (int it = 0; it < nsweeps; ++it)
    for (int colour = 0; colour < 2; ++colour)
      for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
          for (int64_t i = 0; i < nx; ++i) {
            if (((i + j + k) & 1) != colour) continue;
            size_t c = orc_at(&g, i, j, k);
            u[c] = orc_site_s(u, f, c, g.sx, g.sy, 0.0f, b, hh);
          }
  return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Defect correction with FP32 inner sweeps.
 *
 *   r  = f - A u                         (double, oracle_residual_f64)
 *   rel = ||r|| / ||f||  (||r0|| if f == 0)
 *   while rel > rtol and outer < max_outer:
 *       r32 = (float) r                  (interior; halo of e and r32 zero)
 *       e32 = 0
 *       inner_sweeps FP32 sweeps of the chosen smoother on A e = r32
 *       u  += (double) e32               (interior)
 *       r = f - A u ; rel = ...
 *
 * smoother: 0 = Jacobi (a = 0), 1 = lexicographic Gauss-Seidel.
 * Returns ORC_OK when rel <= rtol, ORC_NOT_CONVERGED otherwise; out_rel and
 * out_iters are filled either way.
 * ------------------------------------------------------------------------- */
int oracle_solve_mixed(double* u, const double* f, int64_t nx, int64_t ny, int64_t nz, double h,
                       int smoother, double rtol, int max_outer, int inner_sweeps,
                       double* out_rel, int* out_iters) {
  orc_grid g;
  if (!u || orc_grid_make(&g, nx, ny, nz) != ORC_OK || !(h > 0.0) || max_outer < 0 ||
      inner_sweeps < 0 || (smoother != 0 && smoother != 1))
    return ORC_ERR_ARG;
  size_t n = orc_total(&g);
  double* r = (double*)calloc(n, sizeof(double));
  float* r32 = (float*)calloc(n, sizeof(float));
  float* e32 = (float*)calloc(n, sizeof(float));
  if (!r || !r32 || !e32) { free(r); free(r32); free(e32); return ORC_ERR_OOM; }
  const float b32 = (float)(1.0 / 6.0);
  double rn = 0.0, fn = 0.0;
  oracle_residual_f64(u, f, nx, ny, nz, h, r, &rn, &fn);
  const double denom = fn > 0.0 ? fn : rn;
  double rel = denom > 0.0 ? rn / denom : 0.0;
  int it = 0;
  while (rel > rtol && it < max_outer) {
    for (int64_t k = 0; k < nz; ++k)
      for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
          size_t c = orc_at(&g, i, j, k);
          r32[c] = (float)r[c];
          e32[c] = 0.0f;
        }
    if (smoother == 0)
      oracle_jacobi_f32(e32, r32, nx, ny, nz, h, 0.0f, b32, inner_sweeps);
    else
      oracle_gs_lex_f32(e32, r32, nx, ny, nz, h, b32, inner_sweeps);
    for (int64_t k = 0; k < nz; ++k)
      for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
          size_t c = orc_at(&g, i, j, k);
          u[c] = u[c] + (double)e32[c];
        }
    ++it;
    oracle_residual_f64(u, f, nx, ny, nz, h, r, &rn, NULL);
    rel = denom > 0.0 ? rn / denom : 0.0;
  }
  free(r); free(r32); free(e32);
  if (out_rel) *out_rel = rel;
  if (out_iters) *out_iters = it;
  return rel <= rtol ? ORC_OK : ORC_NOT_CONVERGED;
}

/* Double-precision-only solve for comparison: plain FP64 sweeps of the
 * chosen smoother, the residual checked every check_every sweeps, until
 * rel <= rtol or max_sweeps.  out_sweeps receives the sweeps done. */
int oracle_solve_f64(double* u, const double* f, int64_t nx, int64_t ny, int64_t nz, double h,
                     int smoother, double rtol, int max_sweeps, int check_every,
                     double* out_rel, int* out_sweeps) {
  orc_grid g;
  if (!u || orc_grid_make(&g, nx, ny, nz) != ORC_OK || !(h > 0.0) || max_sweeps < 0 ||
      check_every <= 0 || (smoother != 0 && smoother != 1))
    return ORC_ERR_ARG;
  const double b = 1.0 / 6.0;
  double rn = 0.0, fn = 0.0;
  oracle_residual_f64(u, f, nx, ny, nz, h, NULL, &rn, &fn);
  const double denom = fn > 0.0 ? fn : rn;
  double rel = denom > 0.0 ? rn / denom : 0.0;
  int done = 0;
  while (rel > rtol && done < max_sweeps) {
    int step = check_every < max_sweeps - done ? check_every : max_sweeps - done;
    if (smoother == 0)
      oracle_jacobi_f64(u, f, nx, ny, nz, h, 0.0, b, step);
    else
      oracle_gs_lex_f64(u, f, nx, ny, nz, h, b, step);
    done += step;
    oracle_residual_f64(u, f, nx, ny, nz, h, NULL, &rn, NULL);
    rel = denom > 0.0 ? rn / denom : 0.0;
  }
  if (out_rel) *out_rel = rel;
  if (out_sweeps) *out_sweeps = done;
  return rel <= rtol ? ORC_OK : ORC_NOT_CONVERGED;
}

/* ---------------------------------------------------------------------------
 * Multigrid V-cycle with these smoothers (Sec. 1 and Sec. 3 name multigrid
 * solvers as the place where the smoothers spend their time; the grid
 * transfers below are the textbook ones, written out in a fixed order).
 *
 * Levels: level 0 is the given grid; while fewer than max_levels levels exist
 * and every extent of the last one is odd and >= 3, the next level has
 * extents (n-1)/2 and spacing 2h.  Coarse site I sits on fine site 2I+1
 * (0-based interior coordinates), so every fine neighbour of a coarse site is
 * interior.
 *
 * Smoothers: 0 = weighted Jacobi with omega = 6/7 (a = 1 - omega = 1/7,
 * b = omega/6 = 1/7), 1 = lexicographic Gauss-Seidel (b = 1/6), 2 = red-black
 * Gauss-Seidel (b = 1/6; red = (i+j+k) even first).
 *
 * Restriction (full weighting, weights 1/4, 1/2, 1/4 per axis), in this order:
 *   along x:  sx = (0.25*r[i-1] + 0.5*r[i]) + 0.25*r[i+1]
 *   along y:  sy = (0.25*sx[j-1] + 0.5*sx[j]) + 0.25*sx[j+1]
 *   along z:  fc = (0.25*sy[k-1] + 0.5*sy[k]) + 0.25*sy[k+1]
 * Prolongation (trilinear, zero on the coarse boundary), added to u:
 *   per axis, an odd fine index takes its coarse site, an even one the mean
 *   (a + b) * 0.5 of the two coarse sites around it; x first, then y, then z.
 *
 * V-cycle at level l < L-1: nu1 smoothing sweeps; r = f - A u (the residual
 * above); f_{l+1} = restriction of r; u_{l+1} = 0 (halo included: the error
 * has zero Dirichlet values); V-cycle at l+1; u_l += prolongation of u_{l+1};
 * nu2 smoothing sweeps.  At the coarsest level: ncoarse sweeps.
 *
 * Solve: rel = ||r||/||f|| (||r0|| if f == 0) before and after each cycle;
 * cycles while rel > rtol and fewer than max_cycles cycles ran.
 * ------------------------------------------------------------------------- */
typedef struct {
  orc_grid g;
  double h;
  double* u; /* level > 0: the correction */
  double* f; /* level > 0: the restricted residual */
  double* r;
} orc_level;

static void orc_mg_smooth(orc_level* L, int smoother, int nsweeps) {
  if (nsweeps <= 0) return;
  if (smoother == 0)
    oracle_jacobi_f64(L->u, L->f, L->g.nx, L->g.ny, L->g.nz, L->h, 1.0 / 7.0, 1.0 / 7.0, nsweeps);
  else if (smoother == 1)
    oracle_gs_lex_f64(L->u, L->f, L->g.nx, L->g.ny, L->g.nz, L->h, 1.0 / 6.0, nsweeps);
  else
    oracle_gs_rb_f64(L->u, L->f, L->g.nx, L->g.ny, L->g.nz, L->h, 1.0 / 6.0, nsweeps);
}

/* fc (coarse interior) = full weighting of r (fine interior). */
int oracle_mg_restrict_f64(const double* r, int64_t nx, int64_t ny, int64_t nz, double* fc) {
  orc_grid gf, gc;
  if (!r || !fc || orc_grid_make(&gf, nx, ny, nz) != ORC_OK) return ORC_ERR_ARG;
  if (nx % 2 == 0 || ny % 2 == 0 || nz % 2 == 0) return ORC_ERR_ARG;
  orc_grid_make(&gc, (nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2);
  for (int64_t K = 0; K < gc.nz; ++K)
    for (int64_t J = 0; J < gc.ny; ++J)
      for (int64_t I = 0; I < gc.nx; ++I) {
        double sy[3];
        for (int dz = -1; dz <= 1; ++dz) {
          double sx[3];
          for (int dy = -1; dy <= 1; ++dy) {
            size_t c = orc_at(&gf, 2 * I + 1, 2 * J + 1 + dy, 2 * K + 1 + dz);
            sx[dy + 1] = (0.25 * r[c - 1] + 0.5 * r[c]) + 0.25 * r[c + 1];
          }
          sy[dz + 1] = (0.25 * sx[0] + 0.5 * sx[1]) + 0.25 * sx[2];
        }
        fc[orc_at(&gc, I, J, K)] = (0.25 * sy[0] + 0.5 * sy[1]) + 0.25 * sy[2];
      }
  return ORC_OK;
}

/* u (fine interior) += trilinear prolongation of e (coarse, zero halo). */
int oracle_mg_prolong_add_f64(double* u, int64_t nx, int64_t ny, int64_t nz, const double* e) {
  orc_grid gf, gc;
  if (!u || !e || orc_grid_make(&gf, nx, ny, nz) != ORC_OK) return ORC_ERR_ARG;
  if (nx % 2 == 0 || ny % 2 == 0 || nz % 2 == 0) return ORC_ERR_ARG;
  orc_grid_make(&gc, (nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2);
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        /* coarse interior coordinates around (i, j, k); -1 and n_c are the zero halo */
        const int64_t xa = (i % 2) ? (i - 1) / 2 : i / 2 - 1, xb = (i % 2) ? xa : i / 2;
        const int64_t ya = (j % 2) ? (j - 1) / 2 : j / 2 - 1, yb = (j % 2) ? ya : j / 2;
        const int64_t za = (k % 2) ? (k - 1) / 2 : k / 2 - 1, zb = (k % 2) ? za : k / 2;
        double ey[2];
        for (int zz = 0; zz < 2; ++zz) {
          const int64_t Z = zz ? zb : za;
          double ex[2];
          for (int yy = 0; yy < 2; ++yy) {
            const int64_t Y = yy ? yb : ya;
            const double a = e[orc_at(&gc, xa, Y, Z)];
            ex[yy] = (i % 2) ? a : (a + e[orc_at(&gc, xb, Y, Z)]) * 0.5;
          }
          ey[zz] = (j % 2) ? ex[0] : (ex[0] + ex[1]) * 0.5;
        }
        const double ez = (k % 2) ? ey[0] : (ey[0] + ey[1]) * 0.5;
        const size_t c = orc_at(&gf, i, j, k);
        u[c] = u[c] + ez;
      }
  return ORC_OK;
}

static void orc_vcycle(orc_level* lv, int l, int nlev, int smoother, int nu1, int nu2, int ncoarse) {
  orc_level* L = &lv[l];
  if (l == nlev - 1) {
    orc_mg_smooth(L, smoother, ncoarse);
    return;
  }
  orc_level* C = &lv[l + 1];
  orc_mg_smooth(L, smoother, nu1);
  double rn;
  oracle_residual_f64(L->u, L->f, L->g.nx, L->g.ny, L->g.nz, L->h, L->r, &rn, NULL);
  oracle_mg_restrict_f64(L->r, L->g.nx, L->g.ny, L->g.nz, C->f);
  memset(C->u, 0, orc_total(&C->g) * sizeof(double));
  orc_vcycle(lv, l + 1, nlev, smoother, nu1, nu2, ncoarse);
  oracle_mg_prolong_add_f64(L->u, L->g.nx, L->g.ny, L->g.nz, C->u);
  orc_mg_smooth(L, smoother, nu2);
}

int oracle_mg_solve_f64(double* u, const double* f, int64_t nx, int64_t ny, int64_t nz, double h, int smoother,
                        int nu1, int nu2, int ncoarse, int max_levels, double rtol, int max_cycles, double* out_rel,
                        int* out_cycles) {
  orc_grid g0;
  if (!u || orc_grid_make(&g0, nx, ny, nz) != ORC_OK || !(h > 0.0) || (smoother < 0 || smoother > 2) ||
      nu1 < 0 || nu2 < 0 || ncoarse < 0 || max_levels < 1 || max_levels > 32 || max_cycles < 0)
    return ORC_ERR_ARG;
  orc_level lv[32];
  memset(lv, 0, sizeof(lv));
  int nlev = 1;
  lv[0].g = g0;
  lv[0].h = h;
  lv[0].u = u;
  lv[0].f = (double*)f;
  while (nlev < max_levels) {
    const orc_grid* p = &lv[nlev - 1].g;
    if (p->nx < 3 || p->ny < 3 || p->nz < 3 || p->nx % 2 == 0 || p->ny % 2 == 0 || p->nz % 2 == 0) break;
    orc_grid_make(&lv[nlev].g, (p->nx - 1) / 2, (p->ny - 1) / 2, (p->nz - 1) / 2);
    lv[nlev].h = 2.0 * lv[nlev - 1].h;
    ++nlev;
  }
  int rc = ORC_OK;
  for (int l = 0; l < nlev; ++l) {
    const size_t n = orc_total(&lv[l].g);
    lv[l].r = (double*)calloc(n, sizeof(double));
    if (l > 0) {
      lv[l].u = (double*)calloc(n, sizeof(double));
      lv[l].f = (double*)calloc(n, sizeof(double));
    }
    if (!lv[l].r || (l > 0 && (!lv[l].u || !lv[l].f))) rc = ORC_ERR_OOM;
  }
  double rel = 0.0;
  int it = 0;
  if (rc == ORC_OK) {
    double rn = 0.0, fn = 0.0;
    oracle_residual_f64(u, f, nx, ny, nz, h, NULL, &rn, &fn);
    const double denom = fn > 0.0 ? fn : rn;
    rel = denom > 0.0 ? rn / denom : 0.0;
    while (rel > rtol && it < max_cycles) {
      orc_vcycle(lv, 0, nlev, smoother, nu1, nu2, ncoarse);
      ++it;
      oracle_residual_f64(u, f, nx, ny, nz, h, NULL, &rn, NULL);
      rel = denom > 0.0 ? rn / denom : 0.0;
    }
  }
  for (int l = 0; l < nlev; ++l) {
    free(lv[l].r);
    if (l > 0) {
      free(lv[l].u);
      free(lv[l].f);
    }
  }
  if (rc != ORC_OK) return rc;
  if (out_rel) *out_rel = rel;
  if (out_cycles) *out_cycles = it;
  return rel <= rtol ? ORC_OK : ORC_NOT_CONVERGED;
}

/* ---------------------------------------------------------------------------
 * Single-precision multigrid and the mixed-precision multigrid solve (not in
 * the paper; the paper's smoothers inside the multigrid solver that Sec. 1
 * and Sec. 3 name as their setting, run on binary32 storage inside an FP64
 * defect correction).
 *
 * The FP32 cycle is the FP64 cycle above with every operation in float:
 *  - residual r = f - (6u - sum) * ih2, ih2 = (float)(1/(h*h)) with 1/(h*h)
 *    formed in double; 6u is the float product 6.0f*u;
 *  - smoothers: weighted Jacobi a = b = (float)(1/7), Gauss-Seidel
 *    b = (float)(1/6), hh = (float)(h*h) (the FP32 sweeps above);
 *  - restriction and prolongation with the float weights 0.25f, 0.5f in the
 *    same order as the FP64 transfers.
 *
 * Mixed solve (defect correction with an FP32 multigrid inner solver):
 *   r = f - A u (double); rel = ||r||/||f|| (||r0|| if f == 0)
 *   while rel > rtol and outer < max_outer:
 *       r32 = (float) r on the interior; e32 = 0
 *       inner_cycles FP32 V-cycles on A e = r32 (levels, nu1, nu2, ncoarse
 *       as the FP64 cycle)
 *       u += (double) e32 on the interior
 *       r = f - A u; rel = ...
 * ------------------------------------------------------------------------- */

/* FP32 residual r = f - (6u - sum) * ih2 on the interior (halo of r untouched). */
int oracle_residual_f32(const float* u, const float* f, int64_t nx, int64_t ny, int64_t nz, double h, float* r) {
  orc_grid g;
  if (!u || !r || orc_grid_make(&g, nx, ny, nz) != ORC_OK || !(h > 0.0)) return ORC_ERR_ARG;
  const float ih2 = (float)(1.0 / (h * h));
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        size_t c = orc_at(&g, i, j, k);
        float au = (6.0f * u[c] - orc_sum_s(u, c, g.sx, g.sy)) * ih2;
        float fv = f ? f[c] : 0.0f;
        r[c] = fv - au;
      }
  return ORC_OK;
}

/* FP32 full weighting, the same order as oracle_mg_restrict_f64. */
int oracle_mg_restrict_f32(const float* r, int64_t nx, int64_t ny, int64_t nz, float* fc) {
  orc_grid gf, gc;
  if (!r || !fc || orc_grid_make(&gf, nx, ny, nz) != ORC_OK) return ORC_ERR_ARG;
  if (nx % 2 == 0 || ny % 2 == 0 || nz % 2 == 0) return ORC_ERR_ARG;
  orc_grid_make(&gc, (nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2);
  for (int64_t K = 0; K < gc.nz; ++K)
    for (int64_t J = 0; J < gc.ny; ++J)
      for (int64_t I = 0; I < gc.nx; ++I) {
        float sy[3];
        for (int dz = -1; dz <= 1; ++dz) {
          float sx[3];
          for (int dy = -1; dy <= 1; ++dy) {
            size_t c = orc_at(&gf, 2 * I + 1, 2 * J + 1 + dy, 2 * K + 1 + dz);
            sx[dy + 1] = (0.25f * r[c - 1] + 0.5f * r[c]) + 0.25f * r[c + 1];
          }
          sy[dz + 1] = (0.25f * sx[0] + 0.5f * sx[1]) + 0.25f * sx[2];
        }
        fc[orc_at(&gc, I, J, K)] = (0.25f * sy[0] + 0.5f * sy[1]) + 0.25f * sy[2];
      }
  return ORC_OK;
}

/* FP32 trilinear prolongation added to u, the same order as the FP64 one. */
int oracle_mg_prolong_add_f32(float* u, int64_t nx, int64_t ny, int64_t nz, const float* e) {
  orc_grid gf, gc;
  if (!u || !e || orc_grid_make(&gf, nx, ny, nz) != ORC_OK) return ORC_ERR_ARG;
  if (nx % 2 == 0 || ny % 2 == 0 || nz % 2 == 0) return ORC_ERR_ARG;
  orc_grid_make(&gc, (nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2);
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        const int64_t xa = (i % 2) ? (i - 1) / 2 : i / 2 - 1, xb = (i % 2) ? xa : i / 2;
        const int64_t ya = (j % 2) ? (j - 1) / 2 : j / 2 - 1, yb = (j % 2) ? ya : j / 2;
        const int64_t za = (k % 2) ? (k - 1) / 2 : k / 2 - 1, zb = (k % 2) ? za : k / 2;
        float ey[2];
        for (int zz = 0; zz < 2; ++zz) {
          const int64_t Z = zz ? zb : za;
          float ex[2];
          for (int yy = 0; yy < 2; ++yy) {
            const int64_t Y = yy ? yb : ya;
            const float a = e[orc_at(&gc, xa, Y, Z)];
            ex[yy] = (i % 2) ? a : (a + e[orc_at(&gc, xb, Y, Z)]) * 0.5f;
          }
          ey[zz] = (j % 2) ? ex[0] : (ex[0] + ex[1]) * 0.5f;
        }
        const float ez = (k % 2) ? ey[0] : (ey[0] + ey[1]) * 0.5f;
        const size_t c = orc_at(&gf, i, j, k);
        u[c] = u[c] + ez;
      }
  return ORC_OK;
}

typedef struct {
  orc_grid g;
  double h;
  float* u;
  float* f;
  float* r;
} orc_level32;

static void orc_mg_smooth32(orc_level32* L, int smoother, int nsweeps) {
  if (nsweeps <= 0) return;
  if (smoother == 0)
    oracle_jacobi_f32(L->u, L->f, L->g.nx, L->g.ny, L->g.nz, L->h, (float)(1.0 / 7.0), (float)(1.0 / 7.0), nsweeps);
  else if (smoother == 1)
    oracle_gs_lex_f32(L->u, L->f, L->g.nx, L->g.ny, L->g.nz, L->h, (float)(1.0 / 6.0), nsweeps);
  else
    oracle_gs_rb_f32(L->u, L->f, L->g.nx, L->g.ny, L->g.nz, L->h, (float)(1.0 / 6.0), nsweeps);
}

static void orc_vcycle32(orc_level32* lv, int l, int nlev, int smoother, int nu1, int nu2, int ncoarse) {
  orc_level32* L = &lv[l];
  if (l == nlev - 1) {
    orc_mg_smooth32(L, smoother, ncoarse);
    return;
  }
  orc_level32* C = &lv[l + 1];
  orc_mg_smooth32(L, smoother, nu1);
  oracle_residual_f32(L->u, L->f, L->g.nx, L->g.ny, L->g.nz, L->h, L->r);
  oracle_mg_restrict_f32(L->r, L->g.nx, L->g.ny, L->g.nz, C->f);
  memset(C->u, 0, orc_total(&C->g) * sizeof(float));
  orc_vcycle32(lv, l + 1, nlev, smoother, nu1, nu2, ncoarse);
  oracle_mg_prolong_add_f32(L->u, L->g.nx, L->g.ny, L->g.nz, C->u);
  orc_mg_smooth32(L, smoother, nu2);
}

/* ncycles FP32 V-cycles on A u = f (u, f float, in place on u); levels as
 * oracle_mg_solve_f64.  No stopping test: exactly ncycles cycles. */
int oracle_mg_cycles_f32(float* u, const float* f, int64_t nx, int64_t ny, int64_t nz, double h, int smoother,
                         int nu1, int nu2, int ncoarse, int max_levels, int ncycles) {
  orc_grid g0;
  if (!u || !f || orc_grid_make(&g0, nx, ny, nz) != ORC_OK || !(h > 0.0) || (smoother < 0 || smoother > 2) ||
      nu1 < 0 || nu2 < 0 || ncoarse < 0 || max_levels < 1 || max_levels > 32 || ncycles < 0)
    return ORC_ERR_ARG;
  orc_level32 lv[32];
  memset(lv, 0, sizeof(lv));
  int nlev = 1;
  lv[0].g = g0;
  lv[0].h = h;
  lv[0].u = u;
  lv[0].f = (float*)f;
  while (nlev < max_levels) {
    const orc_grid* p = &lv[nlev - 1].g;
    if (p->nx < 3 || p->ny < 3 || p->nz < 3 || p->nx % 2 == 0 || p->ny % 2 == 0 || p->nz % 2 == 0) break;
    orc_grid_make(&lv[nlev].g, (p->nx - 1) / 2, (p->ny - 1) / 2, (p->nz - 1) / 2);
    lv[nlev].h = 2.0 * lv[nlev - 1].h;
    ++nlev;
  }
  int rc = ORC_OK;
  for (int l = 0; l < nlev; ++l) {
    const size_t n = orc_total(&lv[l].g);
    lv[l].r = (float*)calloc(n, sizeof(float));
    if (l > 0) {
      lv[l].u = (float*)calloc(n, sizeof(float));
      lv[l].f = (float*)calloc(n, sizeof(float));
    }
    if (!lv[l].r || (l > 0 && (!lv[l].u || !lv[l].f))) rc = ORC_ERR_OOM;
  }
  if (rc == ORC_OK)
    for (int c = 0; c < ncycles; ++c) orc_vcycle32(lv, 0, nlev, smoother, nu1, nu2, ncoarse);
  for (int l = 0; l < nlev; ++l) {
    free(lv[l].r);
    if (l > 0) {
      free(lv[l].u);
      free(lv[l].f);
    }
  }
  return rc;
}

int oracle_solve_mixed_mg(double* u, const double* f, int64_t nx, int64_t ny, int64_t nz, double h, int smoother,
                          int nu1, int nu2, int ncoarse, int max_levels, double rtol, int max_outer, int inner_cycles,
                          double* out_rel, int* out_iters) {
  orc_grid g;
  if (!u || orc_grid_make(&g, nx, ny, nz) != ORC_OK || !(h > 0.0) || max_outer < 0 || inner_cycles < 0 ||
      (smoother < 0 || smoother > 2))
    return ORC_ERR_ARG;
  size_t n = orc_total(&g);
  double* r = (double*)calloc(n, sizeof(double));
  float* r32 = (float*)calloc(n, sizeof(float));
  float* e32 = (float*)calloc(n, sizeof(float));
  if (!r || !r32 || !e32) { free(r); free(r32); free(e32); return ORC_ERR_OOM; }
  double rn = 0.0, fn = 0.0;
  oracle_residual_f64(u, f, nx, ny, nz, h, r, &rn, &fn);
  const double denom = fn > 0.0 ? fn : rn;
  double rel = denom > 0.0 ? rn / denom : 0.0;
  int it = 0, rc = ORC_OK;
  while (rel > rtol && it < max_outer) {
    for (int64_t k = 0; k < nz; ++k)
      for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
          size_t c = orc_at(&g, i, j, k);
          r32[c] = (float)r[c];
          e32[c] = 0.0f;
        }
    rc = oracle_mg_cycles_f32(e32, r32, nx, ny, nz, h, smoother, nu1, nu2, ncoarse, max_levels, inner_cycles);
    if (rc != ORC_OK) break;
    for (int64_t k = 0; k < nz; ++k)
      for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
          size_t c = orc_at(&g, i, j, k);
          u[c] = u[c] + (double)e32[c];
        }
    ++it;
    oracle_residual_f64(u, f, nx, ny, nz, h, r, &rn, NULL);
    rel = denom > 0.0 ? rn / denom : 0.0;
  }
  free(r); free(r32); free(e32);
  if (rc != ORC_OK) return rc;
  if (out_rel) *out_rel = rel;
  if (out_iters) *out_iters = it;
  return rel <= rtol ? ORC_OK : ORC_NOT_CONVERGED;
}
