// Temporally blocked Jacobi (Sec. 4) on the skewed-tile task schedule.
#include "internal.h"
#include "tiles.h"

namespace stn {

template <typename T>
int tb_jacobi_run(stencil_ctx* ctx, T* u, T* tmp, const T* f, const Geom& g, double h, int nsweeps,
                  const stencil_params* p, cudaStream_t st) {
  (void)u; (void)tmp; (void)f; (void)g; (void)h; (void)nsweeps; (void)st;
  return set_err(ctx, STENCIL_ERR_UNSUPPORTED, "Jacobi nt = %d not built yet", p ? p->nt : 0);
}

template int tb_jacobi_run<double>(stencil_ctx*, double*, double*, const double*, const Geom&, double, int,
                                   const stencil_params*, cudaStream_t);
template int tb_jacobi_run<float>(stencil_ctx*, float*, float*, const float*, const Geom&, double, int,
                                  const stencil_params*, cudaStream_t);

}  // namespace stn
