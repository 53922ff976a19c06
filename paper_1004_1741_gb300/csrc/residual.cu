// Residual r = f - A u of the Poisson problem -Lap_h u = f, its FP64 2-norm,
// the FP64 correction u += e, and the defect-correction solves built on them
// (not in the paper; they make the smoothers usable as a solver with FP32
// inner sweeps).
//
// The norm is reduced in a fixed order (per-thread running sums over a fixed
// set of sites, a fixed tree per CTA, then one CTA over the per-CTA partials
// in index order), so a given grid shape always gives the same bits.
#include <cmath>

#include "internal.h"
#include "residual_kernels.cuh"

namespace stn {

int residual_launch(stencil_ctx* ctx, const double* u, const double* f, const Geom& g, double h, double* r_out,
                    float* r32_out, double** result, cudaStream_t st, bool norm) {
  const dim3 block(RES_BX, RES_BY);
  const dim3 grid = residual_grid(g);
  const int64_t nblk = (int64_t)grid.x * grid.y * grid.z;
  int status;
  double* part = (double*)ws_get(ctx, SLOT_RED_PARTIALS, (size_t)(nblk > 0 ? nblk : 1) * 2 * sizeof(double), &status);
  if (!part) return status;
  double* res = (double*)ws_get(ctx, SLOT_RED_RESULT, 4 * sizeof(double), &status);
  if (!res) return status;
  *result = res;
  const double ih2 = 1.0 / (h * h);
  if (!norm) {  // r only (the multigrid cycle): no sums, no reduction
    if (nblk > 0) {
      if (!r_out || r32_out) return set_err(ctx, STENCIL_ERR_ARG, "residual without norm writes FP64 r only");
      if (f)
        residual_kernel<true, true, false, false><<<grid, block, 0, st>>>(u, f, r_out, nullptr, g, ih2, part);
      else
        residual_kernel<false, true, false, false><<<grid, block, 0, st>>>(u, f, r_out, nullptr, g, ih2, part);
      ctx->launches++;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(ctx, e, "residual kernel");
    return STENCIL_OK;
  }
  if (nblk > 0) {
#define RES_GO(HF, WR, W32) residual_kernel<HF, WR, W32, true><<<grid, block, 0, st>>>(u, f, r_out, r32_out, g, ih2, part)
    const bool hf = f != nullptr, wr = r_out != nullptr, w32 = r32_out != nullptr;
    if (hf && wr && w32) RES_GO(true, true, true);
    else if (hf && wr) RES_GO(true, true, false);
    else if (hf && w32) RES_GO(true, false, true);
    else if (hf) RES_GO(true, false, false);
    else if (wr && w32) RES_GO(false, true, true);
    else if (wr) RES_GO(false, true, false);
    else if (w32) RES_GO(false, false, true);
    else RES_GO(false, false, false);
#undef RES_GO
  }
  reduce_pairs_kernel<1024><<<1, 1024, 0, st>>>(part, nblk, res);
  ctx->launches += nblk > 0 ? 2 : 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(ctx, e, "residual kernels");
  return STENCIL_OK;
}

int residual32_launch(stencil_ctx* ctx, const float* u, const float* f, const Geom& g, double h, float* r_out,
                      cudaStream_t st) {
  const dim3 grid = residual_grid(g);
  if ((int64_t)grid.x * grid.y * grid.z == 0) return STENCIL_OK;
  const float ih2 = (float)(1.0 / (h * h));
  if (f)
    residual_f32_kernel<true><<<grid, dim3(RES_BX, RES_BY), 0, st>>>(u, f, r_out, g, ih2);
  else
    residual_f32_kernel<false><<<grid, dim3(RES_BX, RES_BY), 0, st>>>(u, f, r_out, g, ih2);
  ctx->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(ctx, e, "residual_f32_kernel");
  return STENCIL_OK;
}

__global__ void correct_kernel(double* __restrict__ u, const float* __restrict__ e, Geom g) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 8 + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int z0 = blockIdx.z * 32, z1 = min(g.nz, z0 + 32);
  for (int z = z0; z < z1; ++z) {
    const int64_t c = g.at(x, y, z);
    u[c] = __dadd_rn(u[c], (double)e[c]);
  }
}

int correct_launch(stencil_ctx* ctx, double* u, const float* e, const Geom& g, cudaStream_t st) {
  dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, (g.nz + 31) / 32);
  correct_kernel<<<grid, dim3(32, 8), 0, st>>>(u, e, g);
  ctx->launches++;
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return cuda_err(ctx, err, "correct_kernel");
  return STENCIL_OK;
}

// Reads the two sums (||r||^2, ||f||^2) to the host.
int read_sums(stencil_ctx* ctx, const double* dres, double* sums, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(sums, dres, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(ctx, e, "reading residual sums");
  return STENCIL_OK;
}

}  // namespace stn

using namespace stn;

static int solve_checks(stencil_ctx* ctx, const void* u, const int64_t dims[3], double h, Geom* g) {
  if (!ctx) return STENCIL_ERR_ARG;
  ctx->err.clear();
  int rc = check_dims(ctx, dims, g);
  if (rc) return rc;
  if (!u) return set_err(ctx, STENCIL_ERR_ARG, "u is NULL");
  if (!(h > 0.0) || !std::isfinite(h)) return set_err(ctx, STENCIL_ERR_ARG, "h must be finite and > 0");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  return STENCIL_OK;
}

extern "C" {

int residual_norm(stencil_ctx* ctx, const double* u, const double* f, const int64_t dims[3], double h,
                  double* r_out, double* out_abs, double* out_rel, void* stream) {
  Geom g;
  int rc = solve_checks(ctx, u, dims, h, &g);
  if (rc) return rc;
  if (!out_abs) return set_err(ctx, STENCIL_ERR_ARG, "out_abs is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  double* dres = nullptr;
  rc = residual_launch(ctx, u, f, g, h, r_out, nullptr, &dres, st);
  if (rc) return rc;
  double sums[2];
  rc = read_sums(ctx, dres, sums, st);
  if (rc) return rc;
  const double rn = std::sqrt(sums[0]), fn = std::sqrt(sums[1]);
  *out_abs = rn;
  if (out_rel) *out_rel = fn > 0.0 ? rn / fn : rn;
  return STENCIL_OK;
}

int stencil_solve_mixed(stencil_ctx* ctx, double* u, const double* f, const int64_t dims[3], double h, int smoother,
                        double rtol, int max_outer, int inner_sweeps, double* out_rel, int* out_iters,
                        void* stream) {
  Geom g;
  int rc = solve_checks(ctx, u, dims, h, &g);
  if (rc) return rc;
  if (!f) return set_err(ctx, STENCIL_ERR_ARG, "f is NULL");
  if (smoother != STENCIL_JACOBI && smoother != STENCIL_GS) return set_err(ctx, STENCIL_ERR_ARG, "bad smoother");
  if (max_outer < 0 || inner_sweeps < 0 || !(rtol >= 0.0)) return set_err(ctx, STENCIL_ERR_ARG, "bad limits");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = (size_t)g.sy * (size_t)(g.nz + 2);
  int status;
  float* r32 = (float*)ws_get(ctx, SLOT_MIX_R32, n * sizeof(float), &status);
  if (!r32) return status;
  float* e32 = (float*)ws_get(ctx, SLOT_MIX_E32, n * sizeof(float), &status);
  if (!e32) return status;
  // the halo of r32 is never read; zero it once so the buffer is defined
  cudaError_t e = cudaMemsetAsync(r32, 0, n * sizeof(float), st);
  if (e != cudaSuccess) return cuda_err(ctx, e, "memset r32");
  double* dres;
  double sums[2];
  if ((rc = residual_launch(ctx, u, f, g, h, nullptr, r32, &dres, st))) return rc;
  if ((rc = read_sums(ctx, dres, sums, st))) return rc;
  const double fn = std::sqrt(sums[1]);
  double rn = std::sqrt(sums[0]);
  const double denom = fn > 0.0 ? fn : rn;
  double rel = denom > 0.0 ? rn / denom : 0.0;
  int it = 0;
  while (rel > rtol && it < max_outer) {
    e = cudaMemsetAsync(e32, 0, n * sizeof(float), st);
    if (e != cudaSuccess) return cuda_err(ctx, e, "memset e32");
    // FP32 inner sweeps: Jacobi with on-chip temporal blocking (3 sweeps per
    // pass), Gauss-Seidel as the persistent column march (one sweep per task)
    stencil_params q{};
    q.int_adds = -1;
    if (smoother == STENCIL_JACOBI) {
      q.variant = 4;
      q.nt = 3;
      q.tile_y = 32;
      q.tile_z = 64;
      rc = jacobi_run<float>(ctx, e32, r32, g, h, inner_sweeps, &q, st);
    } else {
      q.nt = 1;
      q.variant = 5;
      rc = gs_run<float>(ctx, e32, r32, g, h, inner_sweeps, &q, st);
    }
    if (rc) return rc;
    if ((rc = correct_launch(ctx, u, e32, g, st))) return rc;
    ++it;
    if ((rc = residual_launch(ctx, u, f, g, h, nullptr, r32, &dres, st))) return rc;
    if ((rc = read_sums(ctx, dres, sums, st))) return rc;
    rn = std::sqrt(sums[0]);
    rel = denom > 0.0 ? rn / denom : 0.0;
  }
  if (out_rel) *out_rel = rel;
  if (out_iters) *out_iters = it;
  if (rel > rtol) return set_err(ctx, STENCIL_ERR_NOT_CONVERGED, "relative residual %.3e > %.3e after %d outer", rel,
                                 rtol, it);
  return STENCIL_OK;
}

int stencil_solve_f64(stencil_ctx* ctx, double* u, const double* f, const int64_t dims[3], double h, int smoother,
                      double rtol, int max_sweeps, int check_every, const stencil_params* params, double* out_rel,
                      int* out_sweeps, void* stream) {
  Geom g;
  int rc = solve_checks(ctx, u, dims, h, &g);
  if (rc) return rc;
  if (smoother != STENCIL_JACOBI && smoother != STENCIL_GS) return set_err(ctx, STENCIL_ERR_ARG, "bad smoother");
  if (max_sweeps < 0 || check_every <= 0 || !(rtol >= 0.0)) return set_err(ctx, STENCIL_ERR_ARG, "bad limits");
  cudaStream_t st = (cudaStream_t)stream;
  double* dres;
  double sums[2];
  if ((rc = residual_launch(ctx, u, f, g, h, nullptr, nullptr, &dres, st))) return rc;
  if ((rc = read_sums(ctx, dres, sums, st))) return rc;
  const double fn = std::sqrt(sums[1]);
  double rn = std::sqrt(sums[0]);
  const double denom = fn > 0.0 ? fn : rn;
  double rel = denom > 0.0 ? rn / denom : 0.0;
  int done = 0;
  while (rel > rtol && done < max_sweeps) {
    const int step = check_every < max_sweeps - done ? check_every : max_sweeps - done;
    if (smoother == STENCIL_JACOBI)
      rc = jacobi_run<double>(ctx, u, f, g, h, step, params, st);
    else
      rc = gs_run<double>(ctx, u, f, g, h, step, params, st);
    if (rc) return rc;
    done += step;
    if ((rc = residual_launch(ctx, u, f, g, h, nullptr, nullptr, &dres, st))) return rc;
    if ((rc = read_sums(ctx, dres, sums, st))) return rc;
    rn = std::sqrt(sums[0]);
    rel = denom > 0.0 ? rn / denom : 0.0;
  }
  if (out_rel) *out_rel = rel;
  if (out_sweeps) *out_sweeps = done;
  if (rel > rtol) return set_err(ctx, STENCIL_ERR_NOT_CONVERGED, "relative residual %.3e > %.3e after %d sweeps",
                                 rel, rtol, done);
  return STENCIL_OK;
}

}  // extern "C"
