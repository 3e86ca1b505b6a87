// Equilibrium gradients (Methods, "Gradient computation methods"):
//   adjoint implicit differentiation through the persistent CG kernels, and
//   equilibrium propagation through two nudged persistent minimisations
//   followed by the difference of d_theta E; plus the Hessian-vector product
//   entry point.
#include <cuda_runtime.h>

#include "persistent.cuh"
#include "tissue.h"
#include "vx_internal.h"

namespace vx {

vx_status adjoint_solve(vx_tissue_s* t, const double* Xstar, const ParamsD& prm, const AdjParams& ap,
                        int path, AdjOut* out, cudaStream_t s);
bool resident_fits(vx_tissue_s* t, bool adjoint);
bool cluster_fits(vx_tissue_s* t);

static View<PolF64> topo_view(vx_tissue_s* t, const double* X) {
  View<PolF64> v;
  v.X = (double2*)X;
  v.tgt = t->tgt;
  v.nxt = t->nxt;
  v.face = t->face;
  v.vout = t->vout;
  v.ffirst = t->ffirst;
  v.n = t->n;
  v.V = t->V;
  v.E = t->E;
  v.box = PolF64::make_box(t->Lx, t->Ly);
  v.Lx = t->Lx;
  v.Ly = t->Ly;
  v.vnb = t->vnb;
  v.vfc = t->vfc;
  v.ccnt = t->ccnt;
  v.ccor = t->ccor;
  v.cedge = t->cedge;
  return v;
}

// (1/beta) [d_theta E(X+) - d_theta E(X-)] with d E / d Lambda_e = l_e,
// d E / d A0 = -2 K_A (A - A0), d E / d P0 = -2 K_P (P - P0).
__global__ void k_ep_grad(View<PolF64> vp, View<PolF64> vm, ParamsD prm, double beta,
                          double* g_lam, double* g_A0, double* g_P0) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
  if (g_lam)
    for (int e = tid; e < vp.E; e += st)
      g_lam[e] = (edge_len_d(vp, 2 * e) - edge_len_d(vm, 2 * e)) / beta;
  for (int c = tid; c < vp.n; c += st) {
    double Ap, Pp, Am, Pm;
    cell_geometry(vp, c, Ap, Pp, 0.0, nullptr);
    cell_geometry(vm, c, Am, Pm, 0.0, nullptr);
    if (g_A0) g_A0[c] = -2.0 * prm.ka(c) * (Ap - Am) / beta;
    if (g_P0) g_P0[c] = -2.0 * prm.kp(c) * (Pp - Pm) / beta;
  }
}

__global__ void k_v2v_cost(View<PolF64> v, const double* Xt, double* out) {
  __shared__ double red[32];
  double s = 0;
  for (int i = threadIdx.x; i < v.V; i += blockDim.x) {
    double gx, gy;
    v2v_grad(v, i, Xt, gx, gy);
    s += 0.5 * v.V * (gx * gx + gy * gy);
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double c = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) c += red[q];
    *out = c;
  }
}

static bool ensure_work(vx_tissue_s* t, size_t doubles) {
  if (t->work_doubles >= doubles) return true;
  if (t->work) cudaFree(t->work);
  t->work = nullptr;
  t->work_doubles = 0;
  if (cudaMalloc(&t->work, 8 * doubles) != cudaSuccess) return false;
  t->work_doubles = doubles;
  return true;
}

vx_status equilibrium_grad(vx_tissue_s* t, const double* Xstar, const ParamsD& prm,
                           const double* dCdX, const vx_grad_opts* o, double* g_lambda, double* g_A0,
                           double* g_P0, vx_grad_result* r, cudaStream_t s) {
  if (o->cost == VX_COST_ANISO) {
    set_error("the anisotropy cost is not available in this build");
    return VX_ERR_INVALID_ARG;
  }
  if (o->mode == VX_ADJOINT_CG) {
    AdjParams ap = {};
    ap.dCdX = dCdX;
    ap.cost = o->cost;
    ap.cost_data = o->cost_data;
    ap.rtol = o->cg_rtol;
    ap.max_iter = o->cg_max_iter;
    ap.g_lam = g_lambda;
    ap.g_A0 = g_A0;
    ap.g_P0 = g_P0;
    AdjOut out = {};
    const vx_status st = adjoint_solve(t, Xstar, prm, ap, o->inner.path, &out, s);
    if (st != VX_OK) return st;
    r->status = out.status;
    r->cg_iters = out.iters;
    r->cg_rel_residual = out.rel_residual;
    r->cost = dCdX ? 0.0 : out.cost;
    r->nudged_iters[0] = r->nudged_iters[1] = 0;
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
  if (!ensure_work(t, 2 * V2 + 8)) {
    set_error("out of device memory for the equilibrium-propagation workspace");
    return VX_ERR_OOM;
  }
  double* Xp = t->work;
  double* Xm = t->work + V2;
  double* cst = t->work + 2 * V2;
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
  mp.l_min = 0.0;  // fixed topology in the nudged phases
  mp.cost = 1;
  mp.cost_data = o->cost_data;
  const bool centered = o->mode == VX_EP_CENTERED;
  const int path = in.path == VX_PATH_PLAIN ? VX_PATH_AUTO : in.path;
  if (cudaMemcpyAsync(Xp, Xstar, 8 * V2, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(Xm, Xstar, 8 * V2, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
    set_error("vx_equilibrium_grad: copy failed");
    return VX_ERR_CUDA;
  }
  MinOut op = {}, om = {};
  int used = 0;
  mp.nudge_s = centered ? 0.5 * o->beta : o->beta;
  vx_status st = minimize(t, Xp, prm, mp, path, in.check_every, &op, &used, s);
  if (st != VX_OK) return st;
  if (centered) {
    mp.nudge_s = -0.5 * o->beta;
    st = minimize(t, Xm, prm, mp, path, in.check_every, &om, &used, s);
    if (st != VX_OK) return st;
  }
  View<PolF64> vp = topo_view(t, Xp), vm = topo_view(t, Xm), vs = topo_view(t, Xstar);
  const int nb = (t->E + 255) / 256;
  k_ep_grad<<<nb, 256, 0, s>>>(vp, vm, prm, o->beta, g_lambda, g_A0, g_P0);
  k_v2v_cost<<<1, 256, 0, s>>>(vs, o->cost_data, cst);
  double c = 0;
  if (cudaMemcpyAsync(&c, cst, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    set_error(std::string("equilibrium propagation: ") + cudaGetErrorString(cudaGetLastError()));
    return VX_ERR_CUDA;
  }
  r->status = (op.status == VX_OK && (!centered || om.status == VX_OK)) ? VX_OK : VX_NOT_CONVERGED;
  r->cg_iters = 0;
  r->cg_rel_residual = 0;
  r->cost = c;
  r->nudged_iters[0] = op.iters;
  r->nudged_iters[1] = centered ? om.iters : 0;
  return VX_OK;
}

// ------------------------------------------------------ Hessian x vector

template <class P>
__global__ void k_hvp_cells(View<P> v, ParamsD prm, const double2* vec,
                            typename Vec2Of<typename P::R>::T4* cell4) {
  using R = typename P::R;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < v.n; c += gridDim.x * blockDim.x) {
    R A, Pp, sA, sP;
    cell_geometry(v, c, A, Pp, (R)0, nullptr);
    cell_dir(v, c, vec, sA, sP);
    typename Vec2Of<R>::T4 q;
    q.x = (R)(2.0 * prm.ka(c) * ((double)A - prm.a0(c)));
    q.y = (R)(2.0 * prm.kp(c) * ((double)Pp - prm.p0(c)));
    q.z = (R)(2.0 * prm.ka(c)) * sA;
    q.w = (R)(2.0 * prm.kp(c)) * sP;
    cell4[c] = q;
  }
}

template <class P>
__global__ void k_hvp_vertices(View<P> v, const typename Vec2Of<typename P::R>::T4* cell4,
                               ParamsD prm, const double2* vec, double2* out) {
  using R = typename P::R;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < v.V; i += gridDim.x * blockDim.x) {
    R hx, hy;
    vertex_hvp(v, i, cell4, prm.lam, prm.lam_s, vec, hx, hy);
    out[i] = make_double2((double)hx, (double)hy);
  }
}

template <class P>
__global__ void k_load_pos(const double* X, typename P::Pos* out, int V) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x)
    out[i] = P::from_d(X[2 * i], X[2 * i + 1]);
}

template <class P>
static vx_status hvp_impl(vx_tissue_s* t, const double* X, const ParamsD& prm, const double* vec,
                          double* Hv, cudaStream_t s) {
  if (!ensure_work(t, 4 * (size_t)t->n + 8)) return VX_ERR_OOM;
  View<P> v;
  v.X = (typename P::Pos*)t->Xw;
  v.tgt = t->tgt;
  v.nxt = t->nxt;
  v.face = t->face;
  v.vout = t->vout;
  v.ffirst = t->ffirst;
  v.n = t->n;
  v.V = t->V;
  v.E = t->E;
  v.box = P::make_box(t->Lx, t->Ly);
  v.Lx = t->Lx;
  v.Ly = t->Ly;
  v.vnb = t->vnb;
  v.vfc = t->vfc;
  v.ccnt = t->ccnt;
  v.ccor = t->ccor;
  v.cedge = t->cedge;
  using C4 = typename Vec2Of<typename P::R>::T4;
  C4* cell4 = (C4*)t->work;
  const int th = 256;
  k_load_pos<P><<<(t->V + th - 1) / th, th, 0, s>>>(X, v.X, t->V);
  k_hvp_cells<P><<<(t->n + th - 1) / th, th, 0, s>>>(v, prm, (const double2*)vec, cell4);
  k_hvp_vertices<P><<<(t->V + th - 1) / th, th, 0, s>>>(v, cell4, prm, (const double2*)vec,
                                                          (double2*)Hv);
  return cudaGetLastError() == cudaSuccess ? VX_OK : VX_ERR_CUDA;
}

vx_status hessian_vector(vx_tissue_s* t, const double* X, const ParamsD& prm, const double* vec,
                         double* Hv, cudaStream_t s) {
  return t->dtype == VX_F64 ? hvp_impl<PolF64>(t, X, prm, vec, Hv, s)
                            : hvp_impl<PolF32>(t, X, prm, vec, Hv, s);
}

}  // namespace vx
