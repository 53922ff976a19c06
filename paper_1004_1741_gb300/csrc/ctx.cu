// Context, workspace and the C-ABI entry points of the stencil library.
#include <stdarg.h>
#include <stdio.h>

#include <cmath>
#include <new>

#include "internal.h"

namespace stn {

static thread_local std::string g_create_err;

int set_err(stencil_ctx* ctx, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx)
    ctx->err = buf;
  else
    g_create_err = buf;
  return code;
}

int cuda_err(stencil_ctx* ctx, cudaError_t e, const char* where) {
  return set_err(ctx, STENCIL_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorString(e), cudaGetErrorName(e));
}

void* ws_try(stencil_ctx* ctx, SlotId id, size_t bytes) {
  const Slot& s = ctx->slots[id];
  if (s.bytes >= bytes && s.ptr) return s.ptr;
  if (ctx->budget && ctx->held - s.bytes + bytes > ctx->budget) return nullptr;
  const std::string saved = ctx->err;
  int status;
  void* p = ws_get(ctx, id, bytes, &status);
  if (!p) ctx->err = saved;
  return p;
}

void* ws_get(stencil_ctx* ctx, SlotId id, size_t bytes, int* status) {
  Slot& s = ctx->slots[id];
  *status = STENCIL_OK;
  if (bytes == 0) bytes = 16;
  if (s.bytes >= bytes) return s.ptr;
  size_t grown = bytes;
  size_t after = ctx->held - s.bytes + grown;
  if (ctx->budget && after > ctx->budget) {
    *status = set_err(ctx, STENCIL_ERR_OOM, "workspace slot %d needs %zu bytes; %zu held, budget %zu", (int)id,
                      grown, ctx->held, ctx->budget);
    return nullptr;
  }
  if (s.ptr) {
    cudaError_t e = cudaFree(s.ptr);
    ctx->held -= s.bytes;
    s.ptr = nullptr;
    s.bytes = 0;
    if (e != cudaSuccess) {
      *status = cuda_err(ctx, e, "cudaFree(workspace)");
      return nullptr;
    }
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, grown);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *status = set_err(ctx, STENCIL_ERR_OOM, "cudaMalloc(%zu) for workspace slot %d: %s", grown, (int)id,
                      cudaGetErrorString(e));
    return nullptr;
  }
  s.ptr = p;
  s.bytes = grown;
  ctx->ws_gen++;
  ctx->held += grown;
  return p;
}

int check_dims(stencil_ctx* ctx, const int64_t dims[3], Geom* g) {
  if (!dims) return set_err(ctx, STENCIL_ERR_ARG, "dims is NULL");
  for (int d = 0; d < 3; ++d) {
    if (dims[d] < 0 || dims[d] > (1 << 20))
      return set_err(ctx, STENCIL_ERR_ARG, "dims[%d] = %lld out of range [0, 2^20]", d, (long long)dims[d]);
  }
  double total = (double)(dims[0] + 2) * (double)(dims[1] + 2) * (double)(dims[2] + 2);
  if (total >= 1099511627776.0) return set_err(ctx, STENCIL_ERR_ARG, "padded grid too large");
  *g = make_geom((int)dims[0], (int)dims[1], (int)dims[2]);
  return STENCIL_OK;
}

static int check_params(stencil_ctx* ctx, const stencil_params* p, bool allow_a) {
  if (!p) return STENCIL_OK;
  if (p->nt < 0 || p->nt > 16) return set_err(ctx, STENCIL_ERR_ARG, "nt = %d out of range [0, 16]", p->nt);
  if (p->tile_x < 0 || p->tile_y < 0 || p->tile_z < 0) return set_err(ctx, STENCIL_ERR_ARG, "negative tile");
  if (!std::isfinite(p->a) || !std::isfinite(p->b)) return set_err(ctx, STENCIL_ERR_ARG, "a, b must be finite");
  if (!allow_a && p->a != 0.0) return set_err(ctx, STENCIL_ERR_ARG, "a != 0 is only accepted by Jacobi");
  return STENCIL_OK;
}

static int common_checks(stencil_ctx* ctx, const void* u, const int64_t dims[3], double h, int nsweeps,
                         const stencil_params* p, bool allow_a, Geom* g) {
  if (!ctx) return STENCIL_ERR_ARG;
  ctx->err.clear();
  int rc = check_dims(ctx, dims, g);
  if (rc) return rc;
  if (!u) return set_err(ctx, STENCIL_ERR_ARG, "u is NULL");
  if (nsweeps < 0) return set_err(ctx, STENCIL_ERR_ARG, "nsweeps = %d < 0", nsweeps);
  if (!(h > 0.0) || !std::isfinite(h)) return set_err(ctx, STENCIL_ERR_ARG, "h = %g must be finite and > 0", h);
  rc = check_params(ctx, p, allow_a);
  if (rc) return rc;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  return STENCIL_OK;
}

}  // namespace stn

using namespace stn;

extern "C" {

int stencil_create(stencil_ctx** out, int device, size_t hbm_budget_bytes) {
  if (!out) return set_err(nullptr, STENCIL_ERR_ARG, "out is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(nullptr, STENCIL_ERR_CUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
  }
  if (device < 0 || device >= n) return set_err(nullptr, STENCIL_ERR_ARG, "device %d not in [0, %d)", device, n);
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return set_err(nullptr, STENCIL_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  stencil_ctx* c = new (std::nothrow) stencil_ctx();
  if (!c) return set_err(nullptr, STENCIL_ERR_OOM, "host allocation failed");
  c->device = device;
  c->budget = hbm_budget_bytes;
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  *out = c;
  return STENCIL_OK;
}

void stencil_destroy(stencil_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  dataflow_release(ctx);
  for (auto& s : ctx->slots)
    if (s.ptr) cudaFree(s.ptr);
  for (auto& en : ctx->slices)
    if (en.dev) cudaFree(en.dev);
  for (auto& mg : ctx->mg_graphs)
    if (mg.exec) cudaGraphExecDestroy(mg.exec);
  if (ctx->cstream) cudaStreamDestroy(ctx->cstream);
  if (ctx->ev) cudaEventDestroy(ctx->ev);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  delete ctx;
}

const char* stencil_last_error(const stencil_ctx* ctx) {
  if (!ctx) return g_create_err.c_str();
  return ctx->err.c_str();
}

size_t stencil_workspace_bytes(const stencil_ctx* ctx) { return ctx ? ctx->held : 0; }

unsigned long long stencil_kernel_launches(const stencil_ctx* ctx) { return ctx ? ctx->launches : 0; }

int stencil_jacobi_ex(stencil_ctx* ctx, double* u, const double* f, const int64_t dims[3], double h, int nsweeps,
                      const stencil_params* p, void* stream) {
  Geom g;
  int rc = common_checks(ctx, u, dims, h, nsweeps, p, true, &g);
  if (rc) return rc;
  return jacobi_run<double>(ctx, u, f, g, h, nsweeps, p, (cudaStream_t)stream);
}

int stencil_jacobi(stencil_ctx* ctx, double* u, const double* f, const int64_t dims[3], double h, int nsweeps,
                   void* stream) {
  return stencil_jacobi_ex(ctx, u, f, dims, h, nsweeps, nullptr, stream);
}

int stencil_jacobi_f32(stencil_ctx* ctx, float* u, const float* f, const int64_t dims[3], double h, int nsweeps,
                       const stencil_params* p, void* stream) {
  Geom g;
  int rc = common_checks(ctx, u, dims, h, nsweeps, p, true, &g);
  if (rc) return rc;
  return jacobi_run<float>(ctx, u, f, g, h, nsweeps, p, (cudaStream_t)stream);
}

int stencil_gs_lex_ex(stencil_ctx* ctx, double* u, const double* f, const int64_t dims[3], double h, int nsweeps,
                      const stencil_params* p, void* stream) {
  Geom g;
  int rc = common_checks(ctx, u, dims, h, nsweeps, p, false, &g);
  if (rc) return rc;
  return gs_run<double>(ctx, u, f, g, h, nsweeps, p, (cudaStream_t)stream);
}

int stencil_gs_lex(stencil_ctx* ctx, double* u, const double* f, const int64_t dims[3], double h, int nsweeps,
                   void* stream) {
  return stencil_gs_lex_ex(ctx, u, f, dims, h, nsweeps, nullptr, stream);
}

int stencil_gs_lex_f32(stencil_ctx* ctx, float* u, const float* f, const int64_t dims[3], double h, int nsweeps,
                       const stencil_params* p, void* stream) {
  Geom g;
  int rc = common_checks(ctx, u, dims, h, nsweeps, p, false, &g);
  if (rc) return rc;
  return gs_run<float>(ctx, u, f, g, h, nsweeps, p, (cudaStream_t)stream);
}

}  // extern "C"
