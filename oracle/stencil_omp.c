/*
 * All-core CPU baseline for the 7-point Jacobi and lexicographic Gauss-Seidel
 * smoothers: the oracle's per-site arithmetic, run on every host core.
 *
 * TEST INFRASTRUCTURE ONLY (like stencil_oracle.c): loaded by the test-suite
 * and by the CPU-baseline leg of the benchmark, never by the product path.
 *
 *  - Jacobi (Sec. 3, first listing), threaded as in the paper's domain
 *    decomposition: every sweep's planes k are split among the threads; each
 *    site is the oracle's expression, so the result is bit-identical.
 *  - Gauss-Seidel (Sec. 3, second listing), pipeline-parallel as Sec. 3
 *    describes it (Fig. pipeline_gs(a)): the rows j of every plane are split
 *    into one block per thread; thread t updates plane k of its block once
 *    thread t-1 has finished plane k of its own (so the j-1 neighbours across
 *    the block boundary are this sweep's values) and once thread t+1 has
 *    finished plane k of the previous sweep (so the j+1 neighbours are the
 *    previous sweep's values, and not yet this sweep's).  Each thread visits
 *    its rows and sites in lexicographic order, so every site sees exactly
 *    the neighbours of the serial loop: the same result bit for bit.
 *    Progress counters use C11 acquire/release atomics.
 *
 * Build with -O2 -ffp-contract=off -fno-fast-math -fopenmp.
 */
#include <omp.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OMP_OK 0
#define OMP_ERR_ARG (-1)
#define OMP_ERR_OOM (-2)

static size_t at(int64_t sx, int64_t sy, int64_t i, int64_t j, int64_t k) {
  return (size_t)((k + 1) * sy + (j + 1) * sx + (i + 1));
}

/* the oracle's site update, a*src + b*(sum + hh*f), the neighbours in the listing's order */
static double site(const double* src, const double* f, size_t c, int64_t sx, int64_t sy, double a, double b,
                   double hh) {
  double s = src[c - 1] + src[c + 1];
  s = s + src[c - sx];
  s = s + src[c + sx];
  s = s + src[c - sy];
  s = s + src[c + sy];
  if (f) s = s + hh * f[c];
  double v = b * s;
  if (a != 0.0) v = a * src[c] + v;
  return v;
}

int omp_jacobi_f64(double* u, const double* f, int64_t nx, int64_t ny, int64_t nz, double h, double a, double b,
                   int nsweeps, int nthreads) {
  if (!u || nx < 0 || ny < 0 || nz < 0 || nsweeps < 0) return OMP_ERR_ARG;
  if (nsweeps == 0 || nx == 0 || ny == 0 || nz == 0) return OMP_OK;
  const int64_t sx = nx + 2, sy = (nx + 2) * (ny + 2);
  const size_t n = (size_t)sy * (size_t)(nz + 2);
  double* tmp = (double*)malloc(n * sizeof(double));
  if (!tmp) return OMP_ERR_OOM;
  memcpy(tmp, u, n * sizeof(double));
  const double hh = h * h;
  double* src = u;
  double* dst = tmp;
  if (nthreads > 0) omp_set_num_threads(nthreads);
  for (int it = 0; it < nsweeps; ++it) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nz; ++k)
      for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
          const size_t c = at(sx, sy, i, j, k);
          dst[c] = site(src, f, c, sx, sy, a, b, hh);
        }
    double* sw = src;
    src = dst;
    dst = sw;
  }
  if (src != u) memcpy(u, src, n * sizeof(double));
  free(tmp);
  return OMP_OK;
}

int omp_gs_lex_f64(double* u, const double* f, int64_t nx, int64_t ny, int64_t nz, double h, double b, int nsweeps,
                   int nthreads) {
  if (!u || nx < 0 || ny < 0 || nz < 0 || nsweeps < 0) return OMP_ERR_ARG;
  if (nsweeps == 0 || nx == 0 || ny == 0 || nz == 0) return OMP_OK;
  const int64_t sx = nx + 2, sy = (nx + 2) * (ny + 2);
  const double hh = h * h;
  int T = nthreads > 0 ? nthreads : omp_get_max_threads();
  if (T > ny) T = (int)ny;
  if (T < 1) T = 1;
  /* done[t] = planes (over all sweeps, in order) thread t has finished */
  atomic_llong* done = (atomic_llong*)malloc((size_t)T * sizeof(atomic_llong));
  if (!done) return OMP_ERR_OOM;
  for (int t = 0; t < T; ++t) atomic_init(&done[t], 0);
  const long long total = (long long)nsweeps * nz;
#pragma omp parallel num_threads(T)
  {
    const int t = omp_get_thread_num();
    const int64_t j0 = ny * t / T, j1 = ny * (t + 1) / T;
    for (long long p = 0; p < total; ++p) {
      const int64_t k = p % nz;
      /* the block above has finished this plane; the block below has finished it in the previous sweep */
      if (t > 0)
        while (atomic_load_explicit(&done[t - 1], memory_order_acquire) < p + 1) {
        }
      if (t + 1 < T)
        while (atomic_load_explicit(&done[t + 1], memory_order_acquire) < p + 1 - nz) {
        }
      for (int64_t j = j0; j < j1; ++j)
        for (int64_t i = 0; i < nx; ++i) {
          const size_t c = at(sx, sy, i, j, k);
          u[c] = site(u, f, c, sx, sy, 0.0, b, hh);
        }
      atomic_store_explicit(&done[t], p + 1, memory_order_release);
    }
  }
  free(done);
  return OMP_OK;
}

int omp_max_threads(void) { return omp_get_max_threads(); }
