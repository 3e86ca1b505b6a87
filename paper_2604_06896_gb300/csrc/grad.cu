// Drivers of the equilibrium gradients (Methods, "Gradient computation
// methods"):
//   adjoint implicit differentiation (Methods, "Implicit differentiation",
//   adjoint form): the persistent preconditioned CG on the Hessian-vector
//   product, or the plain path's one launch per sub-step;
//   equilibrium propagation (Methods, "Equilibrium propagation"): two
//   nudged persistent minimisations from X*, then the difference of
//   d_theta E over beta.
// Both run without allocating (every buffer is in the tissue's workspace).
// The synchronous form returns the result to the host; the asynchronous
// form launches everything on the stream and has the GPU write the result
// into device or pinned memory, so that it can be captured in a CUDA graph.
#include <cuda_runtime.h>

#include <string>

#include "persistent.cuh"
#include "tissue.h"
#include "vx_internal.h"

namespace vx {

// defined in adjoint.cu
View<PolF64> topo_view(vx_tissue_s* t, const double* X);
__global__ void k_ep_grad(View<PolF64> vp, View<PolF64> vm, ParamsD prm, double beta,
                          double* g_lam, double* g_A0, double* g_P0);
__global__ void k_v2v_cost(View<PolF64> v, const double* Xt, double* out);
__global__ void k_aniso_cells(View<PolF64> v, double2* cent, int* kk, double* part);
__global__ void k_aniso_final(const double* part, int nb, int n, const double* qt, double* g);
__global__ void k_aniso_grad(View<PolF64> v, const double2* cent, const int* kk, const double* g,
                             double2* out);
vx_status adjoint_plain(vx_tissue_s* t, const double* Xstar, const ParamsD& prm, const AdjParams& ap,
                        int check_every, AdjOut* out, cudaStream_t s);
vx_status adjoint_minres(vx_tissue_s* t, const double* Xstar, const ParamsD& prm,
                         const AdjParams& ap, int check_every, AdjOut* out, cudaStream_t s);
// defined in persistent.cu
vx_status adjoint_solve(vx_tissue_s* t, const double* Xstar, const ParamsD& prm, const AdjParams& ap,
                        int path, AdjOut* out_host, AdjOut* out_dev, cudaStream_t s);
vx_status minimize_launch(vx_tissue_s* t, double* X, const ParamsD& prm, const MinParams& mp,
                          int path, MinOut* out_dev, int* path_used, cudaStream_t s);
bool resident_fits(vx_tissue_s* t, bool adjoint);
bool cluster_fits(vx_tissue_s* t);

namespace {

// What one gradient call leaves on the device (at the end of the EP region).
struct GradDev {
  AdjOut adj;
  MinOut plus, minus;
  double cost;
};

// Layout of the anisotropy region: grad_X C [V][2] | centroids [n] (double2)
// | corner counts [n] (int, in n doubles) | block partials [3 nb] | (C, dC/dQ).
struct AnisoWs {
  double* gradX;
  double2* cent;
  int* kk;
  double* part;
  double* g;
};
AnisoWs aniso_ws(vx_tissue_s* t) {
  AnisoWs a;
  double* w = work_aniso(t);
  const int nb = (t->n + 255) / 256;
  a.gradX = w;
  a.cent = (double2*)(w + 2 * (size_t)t->V);
  a.kk = (int*)(w + 2 * (size_t)t->V + 2 * (size_t)t->n);
  a.part = w + 2 * (size_t)t->V + 3 * (size_t)t->n;
  a.g = a.part + 3 * (size_t)nb;
  return a;
}

GradDev* grad_dev(vx_tissue_s* t) {
  return (GradDev*)(work_ep(t) + 4 * (size_t)t->V + 8);
}

// C (and, with gradX, grad_X C) of the anisotropy cost at X, into a.g[0]
// (and a.gradX).
void aniso_cost_launch(vx_tissue_s* t, const double* X, const double* q_target, bool grad,
                       cudaStream_t s) {
  const AnisoWs a = aniso_ws(t);
  const int nb = (t->n + 255) / 256;
  View<PolF64> v = topo_view(t, X);
  v.ccor = nullptr;
  k_aniso_cells<<<nb, 256, 0, s>>>(v, a.cent, a.kk, a.part);
  k_aniso_final<<<1, 32, 0, s>>>(a.part, nb, t->n, q_target, a.g);
  if (grad) k_aniso_grad<<<(t->V + 255) / 256, 256, 0, s>>>(v, a.cent, a.kk, a.g, (double2*)a.gradX);
}

__global__ void k_copy_scalar(const double* src, double* dst) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *dst = *src;
}

// The result of an adjoint call (mode 0) or an EP call (modes 1, 2) from
// the device-side records into r (device or pinned host memory).
__global__ void k_grad_result(const GradDev* g, int mode, int centered, int cost_from_adj,
                              vx_grad_result* r) {
  if (threadIdx.x || blockIdx.x) return;
  vx_grad_result o;
  if (mode == VX_ADJOINT_CG || mode == VX_ADJOINT_MINRES) {
    o.status = g->adj.status;
    o.cg_iters = g->adj.iters;
    o.cg_rel_residual = g->adj.rel_residual;
    o.cost = cost_from_adj ? g->adj.cost : g->cost;
    o.nudged_iters[0] = o.nudged_iters[1] = 0;
  } else {
    o.status = (g->plus.status == VX_OK && (!centered || g->minus.status == VX_OK)) ? VX_OK
                                                                                     : VX_NOT_CONVERGED;
    o.cg_iters = 0;
    o.cg_rel_residual = 0.0;
    o.cost = g->cost;
    o.nudged_iters[0] = g->plus.iters;
    o.nudged_iters[1] = centered ? g->minus.iters : 0;
  }
  *r = o;
}

// Runs the nudged phases of an FP32 tissue in FP64 arithmetic: a tissue's
// buffers hold either precision (positions 16 bytes per vertex, cell
// coefficients 16 bytes per cell), so only the kernel template changes.
struct PrecisionScope {
  vx_tissue_s* t;
  int saved;
  PrecisionScope(vx_tissue_s* t_, bool f64) : t(t_), saved(t_->dtype) {
    if (f64) t->dtype = VX_F64;
  }
  ~PrecisionScope() { t->dtype = saved; }
};

MinParams nudged_params(const vx_grad_opts* o, vx_tissue_s* t) {
  MinParams mp = {};
  const vx_min_opts& in = o->inner;
  mp.method = in.method;
  mp.tol = in.tol;
  mp.patience = in.patience;
  mp.max_iter = in.max_iter;
  mp.gd_lr = in.gd_lr;
  mp.dt0 = in.dt0;
  mp.dt_max = in.dt_max;
  mp.n_min = in.n_min;
  mp.f_inc = in.f_inc;
  mp.f_dec = in.f_dec;
  mp.alpha0 = in.alpha0;
  mp.f_alpha = in.f_alpha;
  mp.l_min = 0.0;   // fixed topology in the nudged phases
  mp.wrap = 0;      // X+ and X- are differenced on one set of offsets
  mp.cost = o->cost;
  mp.cost_data = o->cost_data;
  mp.aniso_ws = o->cost == VX_COST_ANISO ? (double*)aniso_ws(t).cent : nullptr;
  mp.aniso_nudge = o->cost == VX_COST_ANISO ? aniso_ws(t).gradX : nullptr;  // free in EP
  return mp;
}

}  // namespace

// One gradient call.  r_host != NULL: synchronous, the result goes to the
// host; r_dev != NULL: asynchronous (resident and cluster paths only), the
// GPU writes the result to r_dev.
vx_status equilibrium_grad_impl(vx_tissue_s* t, const double* Xstar, const ParamsD& prm,
                                const double* dCdX, const vx_grad_opts* o, double* g_lambda,
                                double* g_A0, double* g_P0, vx_grad_result* r_host,
                                vx_grad_result* r_dev, cudaStream_t s) {
  const bool async = r_dev != nullptr;
  GradDev* gd = grad_dev(t);
  if (o->mode == VX_ADJOINT_CG || o->mode == VX_ADJOINT_MINRES) {
    const bool minres = o->mode == VX_ADJOINT_MINRES;
    const double* rhs = dCdX;
    const bool aniso = !dCdX && o->cost == VX_COST_ANISO;
    if (aniso) {
      aniso_cost_launch(t, Xstar, o->cost_data, true, s);
      rhs = aniso_ws(t).gradX;
      k_copy_scalar<<<1, 1, 0, s>>>(aniso_ws(t).g, &gd->cost);
    }
    AdjParams ap = {};
    ap.dCdX = rhs;
    ap.cost = o->cost;
    ap.cost_data = o->cost_data;
    ap.rtol = o->cg_rtol;
    ap.max_iter = o->cg_max_iter;
    ap.g_lam = g_lambda;
    ap.g_A0 = g_A0;
    ap.g_P0 = g_P0;
    AdjOut out = {};
    vx_status st;
    if (o->inner.path == VX_PATH_PLAIN || minres) {
      // one launch per sub-step, status polled by the host
      if (async) {
        set_error("the plain adjoint path and MINRES poll the host and cannot run asynchronously");
        return VX_ERR_INVALID_ARG;
      }
      st = minres ? adjoint_minres(t, Xstar, prm, ap, o->inner.check_every, &out, s)
                  : adjoint_plain(t, Xstar, prm, ap, o->inner.check_every, &out, s);
    } else {
      st = adjoint_solve(t, Xstar, prm, ap, o->inner.path, async ? nullptr : &out, &gd->adj, s);
    }
    if (st != VX_OK) return st;
    if (async) {
      k_grad_result<<<1, 1, 0, s>>>(gd, o->mode, 0, aniso ? 0 : 1, r_dev);
      return cudaGetLastError() == cudaSuccess ? VX_OK : VX_ERR_CUDA;
    }
    double c = 0.0;
    if (aniso && (cudaMemcpyAsync(&c, &gd->cost, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                  cudaStreamSynchronize(s) != cudaSuccess)) {
      set_error(std::string("anisotropy cost: ") + cudaGetErrorString(cudaGetLastError()));
      return VX_ERR_CUDA;
    }
    r_host->status = out.status;
    r_host->cg_iters = out.iters;
    r_host->cg_rel_residual = out.rel_residual;
    r_host->cost = dCdX ? 0.0 : (aniso ? c : out.cost);
    r_host->nudged_iters[0] = r_host->nudged_iters[1] = 0;
    if (out.status == VX_ERR_INDEFINITE) {
      set_error("CG met a direction of non-positive curvature (the Hessian is not positive definite)");
      return VX_ERR_INDEFINITE;
    }
    return VX_OK;
  }
  // Equilibrium propagation.
  if (!resident_fits(t, false) && !cluster_fits(t)) {
    set_error("equilibrium propagation needs the resident or cluster minimiser");
    return VX_ERR_INVALID_ARG;
  }
  const size_t V2 = 2 * (size_t)t->V;
  double* Xp = work_ep(t);
  double* Xm = Xp + V2;
  const bool centered = o->mode == VX_EP_CENTERED;
  const int path = o->inner.path == VX_PATH_PLAIN ? VX_PATH_AUTO : o->inner.path;
  // C at X* first (the anisotropy phases reuse the centroid scratch)
  View<PolF64> vs = topo_view(t, Xstar);
  if (o->cost == VX_COST_V2V) {
    k_v2v_cost<<<1, 256, 0, s>>>(vs, o->cost_data, &gd->cost);
  } else {
    aniso_cost_launch(t, Xstar, o->cost_data, false, s);
    k_copy_scalar<<<1, 1, 0, s>>>(aniso_ws(t).g, &gd->cost);
  }
  if (cudaMemcpyAsync(Xp, Xstar, 8 * V2, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(Xm, Xstar, 8 * V2, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
    set_error("vx_equilibrium_grad: copy failed");
    return VX_ERR_CUDA;
  }
  MinParams mp = nudged_params(o, t);
  MinOut op = {}, om = {};
  {
    PrecisionScope scope(t, o->ep_f64 != 0);
    int used = 0;
    mp.nudge_s = centered ? 0.5 * o->beta : o->beta;
    vx_status st = async ? minimize_launch(t, Xp, prm, mp, path, &gd->plus, &used, s)
                         : minimize(t, Xp, prm, mp, path, o->inner.check_every, &op, &used, s);
    if (st != VX_OK) return st;
    if (centered) {
      mp.nudge_s = -0.5 * o->beta;
      st = async ? minimize_launch(t, Xm, prm, mp, path, &gd->minus, &used, s)
                 : minimize(t, Xm, prm, mp, path, o->inner.check_every, &om, &used, s);
      if (st != VX_OK) return st;
    }
  }
  // one-sided: the difference with the free equilibrium X* itself
  View<PolF64> vp = topo_view(t, Xp), vm = topo_view(t, centered ? Xm : Xstar);
  const int nb = (t->E + 255) / 256;
  k_ep_grad<<<nb, 256, 0, s>>>(vp, vm, prm, o->beta, g_lambda, g_A0, g_P0);
  if (async) {
    k_grad_result<<<1, 1, 0, s>>>(gd, o->mode, centered ? 1 : 0, 0, r_dev);
    return cudaGetLastError() == cudaSuccess ? VX_OK : VX_ERR_CUDA;
  }
  double c = 0;
  if (cudaMemcpyAsync(&c, &gd->cost, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    set_error(std::string("equilibrium propagation: ") + cudaGetErrorString(cudaGetLastError()));
    return VX_ERR_CUDA;
  }
  r_host->status = (op.status == VX_OK && (!centered || om.status == VX_OK)) ? VX_OK : VX_NOT_CONVERGED;
  r_host->cg_iters = 0;
  r_host->cg_rel_residual = 0;
  r_host->cost = c;
  r_host->nudged_iters[0] = op.iters;
  r_host->nudged_iters[1] = centered ? om.iters : 0;
  return VX_OK;
}

vx_status equilibrium_grad(vx_tissue_s* t, const double* Xstar, const ParamsD& prm,
                           const double* dCdX, const vx_grad_opts* o, double* g_lambda, double* g_A0,
                           double* g_P0, vx_grad_result* r, cudaStream_t s) {
  return equilibrium_grad_impl(t, Xstar, prm, dCdX, o, g_lambda, g_A0, g_P0, r, nullptr, s);
}

}  // namespace vx
