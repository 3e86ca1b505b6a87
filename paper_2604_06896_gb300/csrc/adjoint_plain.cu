// The plain GPU path of the implicit adjoint (Methods, "Implicit
// differentiation"): the block-Jacobi preconditioned CG of the persistent
// kernels for H lambda = Pi grad_X C, written as one grid-wide launch per
// sub-step (HVP cell pass, HVP vertex pass with p.Hp, update with r.z and
// r.r, new direction).  The scalars of the iteration stay on the device: the
// last block to finish each reduction sums the per-block partials in block
// order (deterministic) and takes the step's decision; the host polls the
// status every check_every iterations.  This is the baseline the persistent
// adjoint is measured against.  CG vectors are FP64 on this path.
#include <cuda_runtime.h>

#include <string>

#include "persistent.cuh"
#include "tissue.h"
#include "vx_internal.h"

namespace vx {

bool ensure_work(vx_tissue_s* t, size_t doubles);

namespace {

constexpr int kT = 256;

struct CgCtrl {
  unsigned counter;
  int status;  // VX_NOT_CONVERGED while running
  int it;      // completed iterations
  int done;
  double rz, pHp, alpha, beta, bnorm, rnorm, cost, mx, my;
};

template <class P>
View<P> plain_view(vx_tissue_s* t) {
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
  return v;
}

// Block sum of NV doubles into part[NV * blockIdx.x + k]; returns true in
// thread 0 of the last block to finish, after a fence, so that it may read
// every block's partials.
template <int NV>
__device__ __forceinline__ bool block_partials(double (&v)[NV], double* part, unsigned* counter) {
  __shared__ double red[kT / 32][NV];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const double x = warp_sum(v[k]);
    if (lane == 0) red[w][k] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0;
      for (int q = 0; q < kT / 32; ++q) s += red[q][k];
      part[NV * blockIdx.x + k] = s;
    }
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return false;
  __threadfence();
  *counter = 0;
  return true;
}

template <int NV>
__device__ __forceinline__ void sum_partials(const double* part, int nb, double (&s)[NV]) {
#pragma unroll
  for (int k = 0; k < NV; ++k) s[k] = 0;
  for (int b = 0; b < nb; ++b)
#pragma unroll
    for (int k = 0; k < NV; ++k) s[k] += __ldcg(&part[NV * b + k]);
}

template <class P>
__global__ void k_pl_load(const double* X, typename P::Pos* out, int V) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x)
    out[i] = P::from_d(X[2 * i], X[2 * i + 1]);
}

// (cA, cP, 2 K_A, 2 K_P) per cell at X*.
template <class P>
__global__ void k_pl_cells0(View<P> v, ParamsD prm, typename Vec2Of<typename P::R>::T4* cell4) {
  using R = typename P::R;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < v.n; c += gridDim.x * blockDim.x) {
    R A, Pp;
    cell_geometry(v, c, A, Pp, (R)0, nullptr);
    typename Vec2Of<R>::T4 q;
    q.x = (R)(2.0 * prm.ka(c) * ((double)A - prm.a0(c)));
    q.y = (R)(2.0 * prm.kp(c) * ((double)Pp - prm.p0(c)));
    q.z = (R)(2.0 * prm.ka(c));
    q.w = (R)(2.0 * prm.kp(c));
    cell4[c] = q;
  }
}

// Preconditioner (inverse 2 x 2 diagonal blocks of H, as the persistent
// kernels build it) and the right side grad_X C; partial sums of the right
// side (for its mean) and of the built-in cost.
template <class P, class LamT>
__global__ void k_pl_setup(View<P> v, const typename Vec2Of<typename P::R>::T4* cell4,
                           const LamT* lam, double lam_s, const double* dCdX, const double* Xt,
                           double4* pre, double2* r, double* part, CgCtrl* ctrl) {
  double acc[3] = {0, 0, 0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < v.V; i += gridDim.x * blockDim.x) {
    double dxx, dxy, dyy;
    vertex_diag(v, i, cell4, lam, lam_s, dxx, dxy, dyy);
    const double det = dxx * dyy - dxy * dxy;
    double4 q;
    if (dxx > 0 && det > 1e-300 * dxx * dxx) {
      q.x = dyy / det;
      q.y = -dxy / det;
      q.z = dxx / det;
    } else {
      const double tr = fabs(dxx) + fabs(dyy);
      q.x = q.z = tr > 0 ? 2.0 / tr : 1.0;
      q.y = 0;
    }
    q.w = 0;
    pre[i] = q;
    double gx, gy;
    if (dCdX) {
      gx = dCdX[2 * i];
      gy = dCdX[2 * i + 1];
    } else {
      v2v_grad(v, i, Xt, gx, gy);
      acc[2] += 0.5 * v.V * (gx * gx + gy * gy);
    }
    r[i] = make_double2(gx, gy);
    acc[0] += gx;
    acc[1] += gy;
  }
  if (!block_partials<3>(acc, part, &ctrl->counter)) return;
  double s[3];
  sum_partials<3>(part, gridDim.x, s);
  ctrl->mx = s[0] / v.V;
  ctrl->my = s[1] / v.V;
  ctrl->cost = s[2];
}

// r = Pi g (mean removed), x = 0, p = z = M r; r.z and |r|.
__global__ void k_pl_start(int V, const double4* pre, double2* r, double2* p, double2* x,
                           double* part, CgCtrl* ctrl) {
  const double mx = ctrl->mx, my = ctrl->my;
  double acc[2] = {0, 0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    double2 ri = r[i];
    ri.x -= mx;
    ri.y -= my;
    r[i] = ri;
    const double4 q = pre[i];
    const double zx = q.x * ri.x + q.y * ri.y, zy = q.y * ri.x + q.z * ri.y;
    p[i] = make_double2(zx, zy);
    x[i] = make_double2(0.0, 0.0);
    acc[0] += ri.x * zx + ri.y * zy;
    acc[1] += ri.x * ri.x + ri.y * ri.y;
  }
  if (!block_partials<2>(acc, part, &ctrl->counter)) return;
  double s[2];
  sum_partials<2>(part, gridDim.x, s);
  ctrl->rz = s[0];
  ctrl->bnorm = ctrl->rnorm = sqrt(s[1]);
  ctrl->it = 0;
  ctrl->status = s[1] == 0.0 ? VX_OK : VX_NOT_CONVERGED;
  ctrl->done = s[1] == 0.0;
}

// HVP cell pass: (2 K_A sA, 2 K_P sP) along p.
template <class P>
__global__ void k_pl_cg_cells(View<P> v, ParamsD prm, const double2* p,
                              typename Vec2Of<typename P::R>::T4* cell4, const CgCtrl* ctrl) {
  using R = typename P::R;
  if (ctrl->done) return;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < v.n; c += gridDim.x * blockDim.x) {
    R sA, sP;
    cell_dir(v, c, p, sA, sP);
    typename Vec2Of<R>::T4 q = cell4[c];
    q.z = (R)(2.0 * prm.ka(c)) * sA;
    q.w = (R)(2.0 * prm.kp(c)) * sP;
    cell4[c] = q;
  }
}

// HVP vertex pass h = H p and p.Hp; the last block sets alpha or flags a
// direction of non-positive curvature.
template <class P, class LamT>
__global__ void k_pl_cg_hvp(View<P> v, const typename Vec2Of<typename P::R>::T4* cell4,
                            const LamT* lam, double lam_s, const double2* p, double2* h,
                            double* part, CgCtrl* ctrl) {
  using R = typename P::R;
  if (ctrl->done) return;
  double acc[1] = {0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < v.V; i += gridDim.x * blockDim.x) {
    R hx, hy;
    vertex_hvp(v, i, cell4, lam, lam_s, p, hx, hy);
    h[i] = make_double2((double)hx, (double)hy);
    const double2 pi = p[i];
    acc[0] += pi.x * (double)hx + pi.y * (double)hy;
  }
  if (!block_partials<1>(acc, part, &ctrl->counter)) return;
  double s[1];
  sum_partials<1>(part, gridDim.x, s);
  ctrl->pHp = s[0];
  if (!(s[0] > 0)) {
    ctrl->status = VX_ERR_INDEFINITE;
    ctrl->done = 1;
  } else {
    ctrl->alpha = ctrl->rz / s[0];
  }
}

// x += alpha p, r -= alpha h, z = M r (into h); r.z and |r|; the last block
// tests convergence and sets beta.
__global__ void k_pl_cg_update(int V, const double4* pre, const double2* p, double2* h, double2* x,
                               double2* r, double* part, CgCtrl* ctrl, double rtol, int max_iter) {
  if (ctrl->done) return;
  const double al = ctrl->alpha;
  double acc[2] = {0, 0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    const double2 pi = p[i], hi = h[i];
    double2 xi = x[i], ri = r[i];
    xi.x += al * pi.x;
    xi.y += al * pi.y;
    ri.x -= al * hi.x;
    ri.y -= al * hi.y;
    x[i] = xi;
    r[i] = ri;
    const double4 q = pre[i];
    const double zx = q.x * ri.x + q.y * ri.y, zy = q.y * ri.x + q.z * ri.y;
    h[i] = make_double2(zx, zy);
    acc[0] += ri.x * zx + ri.y * zy;
    acc[1] += ri.x * ri.x + ri.y * ri.y;
  }
  if (!block_partials<2>(acc, part, &ctrl->counter)) return;
  double s[2];
  sum_partials<2>(part, gridDim.x, s);
  ctrl->it += 1;
  ctrl->rnorm = sqrt(s[1]);
  if (!(ctrl->rnorm == ctrl->rnorm)) {
    ctrl->status = VX_ERR_NONFINITE;
    ctrl->done = 1;
    return;
  }
  if (ctrl->rnorm <= rtol * ctrl->bnorm) {
    ctrl->status = VX_OK;
    ctrl->done = 1;
  } else if (ctrl->it >= max_iter) {
    ctrl->done = 1;
  }
  ctrl->beta = s[0] / ctrl->rz;
  ctrl->rz = s[0];
}

// p = z + beta p.
__global__ void k_pl_cg_dir(int V, const double2* z, double2* p, const CgCtrl* ctrl) {
  if (ctrl->done) return;
  const double be = ctrl->beta;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    const double2 zi = z[i];
    double2 pi = p[i];
    pi.x = zi.x + be * pi.x;
    pi.y = zi.y + be * pi.y;
    p[i] = pi;
  }
}

// g = -(d^2E / dX dtheta)^T lambda: per edge -u_e . (lambda_t - lambda_s),
// per cell 2 K_A (grad A . lambda), 2 K_P (grad P . lambda).
template <class P>
__global__ void k_pl_vjp(View<P> v, ParamsD prm, const double2* lam_x, double* g_lam,
                         double* g_A0, double* g_P0) {
  using R = typename P::R;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
  if (g_lam)
    for (int e = tid; e < v.E; e += st) {
      const int h = 2 * e;
      const uint32_t tg = v.tgt[h];
      const int s = src_of(v, h), t = tgt_v(tg);
      R dx, dy;
      P::diff(v.X[t], v.X[s], tgt_ox(tg), tgt_oy(tg), v.box, dx, dy);
      const double il = 1.0 / sqrt((double)(dx * dx + dy * dy));
      const double2 lt = lam_x[t], ls = lam_x[s];
      g_lam[e] = -((double)dx * (lt.x - ls.x) + (double)dy * (lt.y - ls.y)) * il;
    }
  if (g_A0 || g_P0)
    for (int c = tid; c < v.n; c += st) {
      R sA, sP;
      cell_dir(v, c, lam_x, sA, sP);
      if (g_A0) g_A0[c] = 2.0 * prm.ka(c) * (double)sA;
      if (g_P0) g_P0[c] = 2.0 * prm.kp(c) * (double)sP;
    }
}

}  // namespace

template <class P>
static vx_status adjoint_plain_t(vx_tissue_s* t, const double* Xstar, const ParamsD& prm,
                                 const AdjParams& ap, int check_every, AdjOut* out, cudaStream_t s) {
  using C4 = typename Vec2Of<typename P::R>::T4;
  const int V = t->V, n = t->n;
  const int nbv = (V + kT - 1) / kT, nbc = (n + kT - 1) / kT;
  // x, r, p, h [V][2]; pre [V][4]; cell4 [n][4]; partials [nbv][3]; control
  const size_t need = 12 * (size_t)V + 4 * (size_t)n + 3 * (size_t)nbv + sizeof(CgCtrl) / 8 + 8;
  if (!ensure_work(t, need)) {
    set_error("out of device memory for the adjoint workspace");
    return VX_ERR_OOM;
  }
  double* w = t->work;
  double2* x = (double2*)w;
  double2* r = (double2*)(w + 2 * (size_t)V);
  double2* p = (double2*)(w + 4 * (size_t)V);
  double2* h = (double2*)(w + 6 * (size_t)V);
  double4* pre = (double4*)(w + 8 * (size_t)V);
  C4* cell4 = (C4*)(w + 12 * (size_t)V);
  double* part = w + 12 * (size_t)V + 4 * (size_t)n;
  CgCtrl* ctrl = (CgCtrl*)(part + 3 * (size_t)nbv);
  View<P> v = plain_view<P>(t);
  cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(CgCtrl), s);
  k_pl_load<P><<<nbv, kT, 0, s>>>(Xstar, v.X, V);
  k_pl_cells0<P><<<nbc, kT, 0, s>>>(v, prm, cell4);
  k_pl_setup<P><<<nbv, kT, 0, s>>>(v, cell4, prm.lam, prm.lam_s, ap.dCdX, ap.cost_data, pre, r,
                                   part, ctrl);
  k_pl_start<<<nbv, kT, 0, s>>>(V, pre, r, p, x, part, ctrl);
  CgCtrl hc = {};
  const int ce = check_every > 0 ? check_every : 1;
  for (int it = 0; e == cudaSuccess && it < ap.max_iter;) {
    const int k = ap.max_iter - it < ce ? ap.max_iter - it : ce;
    for (int j = 0; j < k; ++j) {
      k_pl_cg_cells<P><<<nbc, kT, 0, s>>>(v, prm, p, cell4, ctrl);
      k_pl_cg_hvp<P><<<nbv, kT, 0, s>>>(v, cell4, prm.lam, prm.lam_s, p, h, part, ctrl);
      k_pl_cg_update<<<nbv, kT, 0, s>>>(V, pre, p, h, x, r, part, ctrl, ap.rtol, ap.max_iter);
      k_pl_cg_dir<<<nbv, kT, 0, s>>>(V, h, p, ctrl);
    }
    it += k;
    e = cudaMemcpyAsync(&hc, ctrl, sizeof(CgCtrl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && hc.done) break;
  }
  if (e == cudaSuccess)
    k_pl_vjp<P><<<nbv, kT, 0, s>>>(v, prm, x, ap.g_lam, ap.g_A0, ap.g_P0);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, ctrl, sizeof(CgCtrl), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error(std::string("plain adjoint: ") + cudaGetErrorString(e));
    return VX_ERR_CUDA;
  }
  out->status = hc.status;
  out->iters = hc.it;
  out->rel_residual = hc.bnorm > 0 ? hc.rnorm / hc.bnorm : 0.0;
  out->cost = hc.cost;
  return VX_OK;
}

vx_status adjoint_plain(vx_tissue_s* t, const double* Xstar, const ParamsD& prm, const AdjParams& ap,
                        int check_every, AdjOut* out, cudaStream_t s) {
  return t->dtype == VX_F64 ? adjoint_plain_t<PolF64>(t, Xstar, prm, ap, check_every, out, s)
                            : adjoint_plain_t<PolF32>(t, Xstar, prm, ap, check_every, out, s);
}

}  // namespace vx
