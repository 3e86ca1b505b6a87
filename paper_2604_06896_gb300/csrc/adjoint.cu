// Equilibrium gradients: implicit adjoint by conjugate gradients on a
// Hessian-vector product, and equilibrium propagation.
#include "tissue.h"
#include "vx_internal.h"

namespace vx {
vx_status equilibrium_grad(vx_tissue_s* t, const double* Xstar, const ParamsD& prm,
                           const double* dCdX, const vx_grad_opts* o, double* g_lambda, double* g_A0,
                           double* g_P0, vx_grad_result* r, cudaStream_t s) {
  set_error("not built yet");
  return VX_ERR_INVALID_ARG;
}
}  // namespace vx
