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

#include <cstddef>
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

// ------------------------------------------------------------ MINRES
//
// MINRES (Paige and Saunders, SIAM J. Numer. Anal. 12, 617, 1975) for
// H x = b when H is symmetric but indefinite (Methods, "Implicit
// differentiation": Krylov solves for Hessians that are not positive
// definite).  Lanczos: beta_1 v_1 = b; p = H v_k - beta_k v_{k-1},
// alpha_k = v_k.p, p -= alpha_k v_k, beta_{k+1} = |p|, v_{k+1} = p / beta_{k+1}.
// The tridiagonal T_k is reduced by Givens rotations G_j = [c s; -s c] on
// rows (j, j+1): column k becomes (eps_k, delta_k, gamma_k) with
// eps_k = s_{k-2} beta_k, dbar = c_{k-2} beta_k, delta_k = c_{k-1} dbar +
// s_{k-1} alpha_k, gbar = c_{k-1} alpha_k - s_{k-1} dbar,
// gamma_k = |(gbar, beta_{k+1})|, c_k = gbar / gamma_k, s_k = beta_{k+1} /
// gamma_k; the right side gives phi_k = c_k phibar_{k-1}, phibar_k =
// -s_k phibar_{k-1} (phibar_0 = beta_1, |r_k| = |phibar_k|); then
// w_k = (v_k - delta_k w_{k-1} - eps_k w_{k-2}) / gamma_k and
// x_k = x_{k-1} + phi_k w_k.  Vectors FP64, one launch per sub-step.

struct MrCtrl {
  unsigned counter;
  int status, it, done, stop;
  double beta, beta_next, alpha, beta1, c1, s1, c2, s2, phibar, eps, delta, gamma, phi;
  double mx, my, cost;
};

// v_1 = Pi b / |Pi b|, v_0 = w = w_prev = x = 0 (b in r, its mean in ctrl).
__global__ void k_mr_start(int V, double2* r, double2* v0, double2* v1, double2* w, double2* wp,
                           double2* x, double* part, CgCtrl* cg, MrCtrl* ctrl) {
  const double mx = cg->mx, my = cg->my;
  double acc[1] = {0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    double2 ri = r[i];
    ri.x -= mx;
    ri.y -= my;
    r[i] = ri;
    acc[0] += ri.x * ri.x + ri.y * ri.y;
  }
  if (!block_partials<1>(acc, part, &ctrl->counter)) return;
  double s[1];
  sum_partials<1>(part, gridDim.x, s);
  const double b1 = sqrt(s[0]);
  ctrl->beta1 = b1;
  ctrl->beta = 0.0;
  ctrl->phibar = b1;
  ctrl->c1 = ctrl->c2 = 1.0;
  ctrl->s1 = ctrl->s2 = 0.0;
  ctrl->it = 0;
  ctrl->cost = cg->cost;
  ctrl->status = b1 == 0.0 ? VX_OK : VX_NOT_CONVERGED;
  ctrl->done = b1 == 0.0;
  ctrl->stop = 0;
}

// v_1 = r / beta_1 and zeroed vectors (after k_mr_start's reduction).
__global__ void k_mr_init(int V, const double2* r, double2* v0, double2* v1, double2* w,
                          double2* wp, double2* x, const MrCtrl* ctrl) {
  const double ib = ctrl->beta1 > 0 ? 1.0 / ctrl->beta1 : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    const double2 ri = r[i];
    v1[i] = make_double2(ri.x * ib, ri.y * ib);
    const double2 z = make_double2(0.0, 0.0);
    v0[i] = z;
    w[i] = z;
    wp[i] = z;
    x[i] = z;
  }
}

// p = H v_k - beta_k v_{k-1} and alpha_k = v_k.p.
template <class P, class LamT>
__global__ void k_mr_hvp(View<P> v, const typename Vec2Of<typename P::R>::T4* cell4,
                         const LamT* lam, double lam_s, const double2* v1, const double2* v0,
                         double2* p, double* part, MrCtrl* ctrl) {
  using R = typename P::R;
  if (ctrl->done) return;
  const double be = ctrl->beta;
  double acc[1] = {0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < v.V; i += gridDim.x * blockDim.x) {
    R hx, hy;
    vertex_hvp(v, i, cell4, lam, lam_s, v1, hx, hy);
    const double2 a = v1[i], b = v0[i];
    const double px = (double)hx - be * b.x, py = (double)hy - be * b.y;
    p[i] = make_double2(px, py);
    acc[0] += a.x * px + a.y * py;
  }
  if (!block_partials<1>(acc, part, &ctrl->counter)) return;
  double s[1];
  sum_partials<1>(part, gridDim.x, s);
  ctrl->alpha = s[0];
}

// p -= alpha_k v_k, beta_{k+1} = |p|; the rotations and the step's phi.
__global__ void k_mr_lanczos(int V, const double2* v1, double2* p, double* part, MrCtrl* ctrl,
                             double rtol, int max_iter) {
  if (ctrl->done) return;
  const double al = ctrl->alpha;
  double acc[1] = {0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    const double2 a = v1[i];
    double2 q = p[i];
    q.x -= al * a.x;
    q.y -= al * a.y;
    p[i] = q;
    acc[0] += q.x * q.x + q.y * q.y;
  }
  if (!block_partials<1>(acc, part, &ctrl->counter)) return;
  double s[1];
  sum_partials<1>(part, gridDim.x, s);
  const double bn = sqrt(s[0]), bk = ctrl->beta;
  // rotation k-2 (c2, s2) and k-1 (c1, s1) applied to column k
  const double eps = ctrl->s2 * bk;
  const double dbar = ctrl->c2 * bk;
  const double delta = ctrl->c1 * dbar + ctrl->s1 * al;
  const double gbar = ctrl->c1 * al - ctrl->s1 * dbar;
  double gamma = sqrt(gbar * gbar + bn * bn);
  if (!(gamma > 0)) gamma = 1e-300;
  const double c = gbar / gamma, sn = bn / gamma;
  ctrl->eps = eps;
  ctrl->delta = delta;
  ctrl->gamma = gamma;
  ctrl->phi = c * ctrl->phibar;
  ctrl->phibar = -sn * ctrl->phibar;
  ctrl->c2 = ctrl->c1;
  ctrl->s2 = ctrl->s1;
  ctrl->c1 = c;
  ctrl->s1 = sn;
  ctrl->beta_next = bn;
  ctrl->it += 1;
  if (!(bn == bn) || !(ctrl->phibar == ctrl->phibar)) {
    ctrl->status = VX_ERR_NONFINITE;
    ctrl->done = 1;
  } else if (fabs(ctrl->phibar) <= rtol * ctrl->beta1 || bn == 0.0) {
    ctrl->status = VX_OK;   // the update below is still applied
    ctrl->stop = 1;
  } else if (ctrl->it >= max_iter) {
    ctrl->stop = 1;         // VX_NOT_CONVERGED, after this update
  }
}

// w_k = (v_k - delta w_{k-1} - eps w_{k-2}) / gamma, x += phi w_k; then
// v_{k-1} = v_k, v_k = p / beta_{k+1}.
__global__ void k_mr_update(int V, double2* v0, double2* v1, const double2* p, double2* w,
                            double2* wp, double2* x, MrCtrl* ctrl) {
  if (ctrl->done) return;
  const double de = ctrl->delta, ep = ctrl->eps, ig = 1.0 / ctrl->gamma, ph = ctrl->phi;
  const double bn = ctrl->beta_next, ib = bn > 0 ? 1.0 / bn : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    const double2 a = v1[i], wc = w[i], wo = wp[i], q = p[i];
    const double2 wn = make_double2((a.x - de * wc.x - ep * wo.x) * ig,
                                    (a.y - de * wc.y - ep * wo.y) * ig);
    wp[i] = wc;
    w[i] = wn;
    double2 xi = x[i];
    xi.x += ph * wn.x;
    xi.y += ph * wn.y;
    x[i] = xi;
    v0[i] = a;
    v1[i] = make_double2(q.x * ib, q.y * ib);
  }
}

// The last update's control: move to the next iteration (run alone, after
// k_mr_update, so that every block has read this iteration's scalars).
__global__ void k_mr_advance(MrCtrl* ctrl) {
  if (threadIdx.x || blockIdx.x || ctrl->done) return;
  ctrl->beta = ctrl->beta_next;
  if (ctrl->stop) ctrl->done = 1;
}

// Sen-ID right sides: m = d(grad_X E)/d theta for one parameter (kind 0:
// Lambda_e -> -u_e at the source, +u_e at the target; kind 1: A0_c ->
// -2 K_A grad A_c; kind 2: P0_c -> -2 K_P grad P_c), written into the
// zeroed r by one thread.
template <class P>
__global__ void k_sen_rhs(View<P> v, ParamsD prm, int kind, int idx, double2* r) {
  if (threadIdx.x || blockIdx.x) return;
  if (kind == 0) {
    const int h = 2 * idx;
    double dx, dy;
    edge_vec_d(v, h, dx, dy);
    const double l = sqrt(dx * dx + dy * dy);
    const int s = src_of(v, h), t = tgt_v(v.tgt[h]);
    r[t].x += dx / l;
    r[t].y += dy / l;
    r[s].x -= dx / l;
    r[s].y -= dy / l;
    return;
  }
  // corners of cell idx: dA/dx_k = (y_{k+1} - y_{k-1}) / 2, dA/dy_k =
  // (x_{k-1} - x_{k+1}) / 2; dP/dx_k = u_{k-1} - u_k (edge k from corner k)
  const int h0 = v.ffirst[idx];
  const double2 X0 = P::to_d(v.X[src_of(v, h0)]);
  int vid[kMaxCorners];
  double qx[kMaxCorners], qy[kMaxCorners];
  int m = 0, cx = 0, cy = 0, h = h0;
  vid[0] = src_of(v, h0);
  qx[0] = qy[0] = 0;
  do {
    const uint32_t tg = v.tgt[h];
    cx += tgt_ox(tg);
    cy += tgt_oy(tg);
    h = v.nxt[h];
    ++m;
    if (h != h0 && m < kMaxCorners) {
      vid[m] = tgt_v(tg);
      const double2 Xt = P::to_d(v.X[tgt_v(tg)]);
      qx[m] = (Xt.x + cx * v.Lx) - X0.x;
      qy[m] = (Xt.y + cy * v.Ly) - X0.y;
    }
  } while (h != h0 && m < kMaxCorners);
  const double f = kind == 1 ? -2.0 * prm.ka(idx) : -2.0 * prm.kp(idx);
  for (int k = 0; k < m; ++k) {
    const int kp = (k + 1) % m, km = (k + m - 1) % m;
    double gx, gy;
    if (kind == 1) {
      gx = 0.5 * (qy[kp] - qy[km]);
      gy = 0.5 * (qx[km] - qx[kp]);
    } else {
      const double ax = qx[k] - qx[km], ay = qy[k] - qy[km];
      const double bx = qx[kp] - qx[k], by = qy[kp] - qy[k];
      const double la = sqrt(ax * ax + ay * ay), lb = sqrt(bx * bx + by * by);
      gx = ax / la - bx / lb;
      gy = ay / la - by / lb;
    }
    r[vid[k]].x += f * gx;
    r[vid[k]].y += f * gy;
  }
}

// out = -a.(Pi b) = -(sum a.b - (sum a).(sum b) / V): the solution b of a
// singular solve carries an arbitrary rigid translation (the preconditioned
// CG iterates leave the range of H), which the projection removes (FP64,
// one block, fixed order).
__global__ void k_neg_dot(int V, const double2* a, const double2* b, double* out) {
  __shared__ double red[5][kT / 32];
  double s[5] = {0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < V; i += blockDim.x) {
    const double2 x = a[i], y = b[i];
    s[0] += x.x * y.x + x.y * y.y;
    s[1] += x.x;
    s[2] += x.y;
    s[3] += y.x;
    s[4] += y.y;
  }
  for (int q = 0; q < 5; ++q) {
    const double w = warp_sum(s[q]);
    if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = w;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[5] = {0, 0, 0, 0, 0};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
      for (int q = 0; q < 5; ++q) t[q] += red[q][w];
    *out = -(t[0] - (t[1] * t[3] + t[2] * t[4]) / V);
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

namespace {

// k_pl_cg_cells tests `done` through a CgCtrl pointer; MINRES passes its own
// control block, whose leading words have the same layout.
static_assert(offsetof(MrCtrl, done) == offsetof(CgCtrl, done), "control layouts");

// The solver region of the workspace on this path: x, r, p, h [V][2]
// (MINRES: x, r, v_{k-1}, v_k, p, w, w_{k-1} use the same twelve V doubles
// and the four of pre), pre [V][4], cell4 [n][4], partials [nbv][3],
// control words.
struct PlainWs {
  double2 *x, *r, *p, *h, *m0, *m1, *m2;
  double4* pre;
  void* cell4;
  double* part;
  CgCtrl* ctrl;
  MrCtrl* mctrl;
};

PlainWs plain_ws(vx_tissue_s* t) {
  const int V = t->V, n = t->n, nbv = (V + kT - 1) / kT;
  double* w = t->work;
  PlainWs a;
  a.x = (double2*)w;
  a.r = (double2*)(w + 2 * (size_t)V);
  a.p = (double2*)(w + 4 * (size_t)V);
  a.h = (double2*)(w + 6 * (size_t)V);
  a.pre = (double4*)(w + 8 * (size_t)V);
  a.m0 = (double2*)(w + 8 * (size_t)V);     // MINRES only (no preconditioner)
  a.m1 = (double2*)(w + 10 * (size_t)V);
  a.m2 = a.p;                               // unused name for clarity of layout
  a.cell4 = w + 12 * (size_t)V;
  a.part = w + 12 * (size_t)V + 4 * (size_t)n;
  a.ctrl = (CgCtrl*)(a.part + 3 * (size_t)nbv);
  a.mctrl = (MrCtrl*)(a.ctrl + 1);
  return a;
}

// Solve H x = Pi rhs at X* on the plain path: block-Jacobi preconditioned CG
// (minres = false) or MINRES.  rhs is dCdX (device [V][2]) or, when NULL,
// the v2v cost gradient for the target Xt.  The solution stays in the
// workspace (plain_ws(t).x); out receives status, iterations, residual and
// the v2v cost.
template <class P>
vx_status plain_solve(vx_tissue_s* t, const double* Xstar, const ParamsD& prm, const double* rhs,
                      const double* Xt, bool minres, double rtol, int max_iter, int check_every,
                      AdjOut* out, cudaStream_t s) {
  using C4 = typename Vec2Of<typename P::R>::T4;
  const int V = t->V, n = t->n;
  const int nbv = (V + kT - 1) / kT, nbc = (n + kT - 1) / kT;
  const size_t need = 12 * (size_t)V + 4 * (size_t)n + 3 * (size_t)nbv +
                      (sizeof(CgCtrl) + sizeof(MrCtrl)) / 8 + 8;
  if (!ensure_work(t, need)) {
    set_error("the adjoint workspace is too small");
    return VX_ERR_INVALID_ARG;
  }
  const PlainWs a = plain_ws(t);
  C4* cell4 = (C4*)a.cell4;
  View<P> v = plain_view<P>(t);
  cudaError_t e = cudaMemsetAsync(a.ctrl, 0, sizeof(CgCtrl) + sizeof(MrCtrl), s);
  k_pl_load<P><<<nbv, kT, 0, s>>>(Xstar, v.X, V);
  k_pl_cells0<P><<<nbc, kT, 0, s>>>(v, prm, cell4);
  k_pl_setup<P><<<nbv, kT, 0, s>>>(v, cell4, prm.lam, prm.lam_s, rhs, Xt, a.pre, a.r, a.part,
                                   a.ctrl);
  const int ce = check_every > 0 ? check_every : 1;
  if (!minres) {
    k_pl_start<<<nbv, kT, 0, s>>>(V, a.pre, a.r, a.p, a.x, a.part, a.ctrl);
    CgCtrl hc = {};
    for (int it = 0; e == cudaSuccess && it < max_iter;) {
      const int k = max_iter - it < ce ? max_iter - it : ce;
      for (int j = 0; j < k; ++j) {
        k_pl_cg_cells<P><<<nbc, kT, 0, s>>>(v, prm, a.p, cell4, a.ctrl);
        k_pl_cg_hvp<P><<<nbv, kT, 0, s>>>(v, cell4, prm.lam, prm.lam_s, a.p, a.h, a.part, a.ctrl);
        k_pl_cg_update<<<nbv, kT, 0, s>>>(V, a.pre, a.p, a.h, a.x, a.r, a.part, a.ctrl, rtol,
                                          max_iter);
        k_pl_cg_dir<<<nbv, kT, 0, s>>>(V, a.h, a.p, a.ctrl);
      }
      it += k;
      e = cudaMemcpyAsync(&hc, a.ctrl, sizeof(CgCtrl), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e == cudaSuccess && hc.done) break;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, a.ctrl, sizeof(CgCtrl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_error(std::string("plain CG: ") + cudaGetErrorString(e));
      return VX_ERR_CUDA;
    }
    out->status = hc.status;
    out->iters = hc.it;
    out->rel_residual = hc.bnorm > 0 ? hc.rnorm / hc.bnorm : 0.0;
    out->cost = hc.cost;
    return VX_OK;
  }
  // MINRES: vectors x, r (right side), v_{k-1} = m0, v_k = m1, p, w = h,
  // w_{k-1} = p's neighbour: p holds the Lanczos residual, h the current w
  // and the pre area the two Lanczos vectors.
  double2 *v0 = a.m0, *v1 = a.m1, *pv = a.p, *w = a.h, *wp = a.r;
  k_mr_start<<<nbv, kT, 0, s>>>(V, a.r, v0, v1, w, wp, a.x, a.part, a.ctrl, a.mctrl);
  k_mr_init<<<nbv, kT, 0, s>>>(V, a.r, v0, v1, w, wp, a.x, a.mctrl);
  MrCtrl hm = {};
  for (int it = 0; e == cudaSuccess && it < max_iter;) {
    const int k = max_iter - it < ce ? max_iter - it : ce;
    for (int j = 0; j < k; ++j) {
      k_pl_cg_cells<P><<<nbc, kT, 0, s>>>(v, prm, v1, cell4, (const CgCtrl*)a.mctrl);
      k_mr_hvp<P><<<nbv, kT, 0, s>>>(v, cell4, prm.lam, prm.lam_s, v1, v0, pv, a.part, a.mctrl);
      k_mr_lanczos<<<nbv, kT, 0, s>>>(V, v1, pv, a.part, a.mctrl, rtol, max_iter);
      k_mr_update<<<nbv, kT, 0, s>>>(V, v0, v1, pv, w, wp, a.x, a.mctrl);
      k_mr_advance<<<1, 1, 0, s>>>(a.mctrl);
    }
    it += k;
    e = cudaMemcpyAsync(&hm, a.mctrl, sizeof(MrCtrl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && hm.done) break;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hm, a.mctrl, sizeof(MrCtrl), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error(std::string("plain MINRES: ") + cudaGetErrorString(e));
    return VX_ERR_CUDA;
  }
  out->status = hm.status;
  out->iters = hm.it;
  out->rel_residual = hm.beta1 > 0 ? fabs(hm.phibar) / hm.beta1 : 0.0;
  out->cost = hm.cost;
  return VX_OK;
}

}  // namespace

template <class P>
static vx_status adjoint_plain_t(vx_tissue_s* t, const double* Xstar, const ParamsD& prm,
                                 const AdjParams& ap, bool minres, int check_every, AdjOut* out,
                                 cudaStream_t s) {
  const vx_status st = plain_solve<P>(t, Xstar, prm, ap.dCdX, ap.cost_data, minres, ap.rtol,
                                      ap.max_iter, check_every, out, s);
  if (st != VX_OK) return st;
  const int nbv = (t->V + kT - 1) / kT;
  k_pl_vjp<P><<<nbv, kT, 0, s>>>(plain_view<P>(t), prm, plain_ws(t).x, ap.g_lam, ap.g_A0, ap.g_P0);
  const cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error(std::string("plain adjoint: ") + cudaGetErrorString(e));
    return VX_ERR_CUDA;
  }
  return VX_OK;
}

// Forward sensitivity (Sen-ID): for each parameter theta_k, solve
// H s_k = m_k with m_k = d(grad_X E)/d theta_k, then dC/d theta_k =
// -grad_X C . Pi s_k (Pi removes the rigid translation, along which H is
// singular and X* undetermined).  One solve per parameter.
template <class P>
static vx_status sensitivity_t(vx_tissue_s* t, const double* Xstar, const ParamsD& prm,
                               const double* dCdX, int count, const int32_t* kind,
                               const int32_t* index, bool minres, double rtol, int max_iter,
                               int check_every, double* out, int32_t* status, cudaStream_t s) {
  double* rhs = work_ep(t);      // [V][2] right side (the EP region is free here)
  double* dev_out = rhs + 2 * (size_t)t->V;
  View<P> v = plain_view<P>(t);
  const int nbv = (t->V + kT - 1) / kT;
  k_pl_load<P><<<nbv, kT, 0, s>>>(Xstar, v.X, t->V);
  for (int k = 0; k < count; ++k) {
    cudaError_t e = cudaMemsetAsync(rhs, 0, 16 * (size_t)t->V, s);
    if (e != cudaSuccess) return VX_ERR_CUDA;
    k_sen_rhs<P><<<1, 1, 0, s>>>(v, prm, kind[k], index[k], (double2*)rhs);
    AdjOut o = {};
    const vx_status st = plain_solve<P>(t, Xstar, prm, rhs, nullptr, minres, rtol, max_iter,
                                        check_every, &o, s);
    if (st != VX_OK) return st;
    k_neg_dot<<<1, kT, 0, s>>>(t->V, (const double2*)dCdX, plain_ws(t).x, dev_out);
    e = cudaMemcpyAsync(out + k, dev_out, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_error(std::string("sensitivity: ") + cudaGetErrorString(e));
      return VX_ERR_CUDA;
    }
    if (status) status[k] = o.status;
  }
  return VX_OK;
}

namespace {

__global__ void k_nt_step(int V, double* X, const double2* d, double* backup) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    const double2 x = make_double2(X[2 * i], X[2 * i + 1]);
    backup[2 * i] = x.x;
    backup[2 * i + 1] = x.y;
    X[2 * i] = x.x + d[i].x;
    X[2 * i + 1] = x.y + d[i].y;
  }
}

__global__ void k_nt_fmax(int V, const double2* F, double* out) {
  __shared__ double red[kT / 32];
  double m = 0;
  for (int i = threadIdx.x; i < V; i += blockDim.x) {
    const double2 f = F[i];
    m = fmax(m, f.x * f.x + f.y * f.y);
  }
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
    *out = sqrt(r);
  }
}

}  // namespace

vx_status newton_refine(vx_tissue_s* t, double* X, const ParamsD& prm, double tol, int max_steps,
                        int* steps, double* fmax, cudaStream_t s) {
  const int V = t->V, nb = (V + kT - 1) / kT;
  double* F = work_ep(t);                 // [V][2]; the EP region is free here
  double* backup = F + 2 * (size_t)V;     // [V][2]
  double* dev_f = backup + 2 * (size_t)V; // one double
  const int saved = t->dtype;
  auto residual = [&](double* fm) -> vx_status {
    t->dtype = VX_F64;
    vx_status st = energy_forces(t, X, prm, F, nullptr, s);
    t->dtype = saved;
    if (st != VX_OK) return st;
    k_nt_fmax<<<1, kT, 0, s>>>(V, (const double2*)F, dev_f);
    cudaError_t e = cudaMemcpyAsync(fm, dev_f, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? VX_OK : VX_ERR_CUDA;
  };
  *steps = 0;
  double f0 = 0;
  vx_status st = residual(&f0);
  if (st != VX_OK) return st;
  for (int k = 0; k < max_steps && f0 >= tol && f0 == f0; ++k) {
    AdjOut o = {};
    st = saved == VX_F64 ? plain_solve<PolF64>(t, X, prm, F, nullptr, false, 1e-4, 5000, 20, &o, s)
                         : plain_solve<PolF32>(t, X, prm, F, nullptr, false, 1e-4, 5000, 20, &o, s);
    if (st != VX_OK) return st;
    if (o.status != VX_OK) break;          // negative curvature or no convergence
    k_nt_step<<<nb, kT, 0, s>>>(V, X, plain_ws(t).x, backup);
    double f1 = 0;
    st = residual(&f1);
    if (st != VX_OK) return st;
    if (!(f1 < f0)) {                      // not an improvement: undo
      cudaError_t e = cudaMemcpyAsync(X, backup, 16 * (size_t)V, cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return VX_ERR_CUDA;
      break;
    }
    f0 = f1;
    ++*steps;
  }
  *fmax = f0;
  return VX_OK;
}

vx_status adjoint_plain(vx_tissue_s* t, const double* Xstar, const ParamsD& prm, const AdjParams& ap,
                        int check_every, AdjOut* out, cudaStream_t s) {
  return t->dtype == VX_F64
             ? adjoint_plain_t<PolF64>(t, Xstar, prm, ap, false, check_every, out, s)
             : adjoint_plain_t<PolF32>(t, Xstar, prm, ap, false, check_every, out, s);
}

vx_status adjoint_minres(vx_tissue_s* t, const double* Xstar, const ParamsD& prm,
                         const AdjParams& ap, int check_every, AdjOut* out, cudaStream_t s) {
  return t->dtype == VX_F64
             ? adjoint_plain_t<PolF64>(t, Xstar, prm, ap, true, check_every, out, s)
             : adjoint_plain_t<PolF32>(t, Xstar, prm, ap, true, check_every, out, s);
}

vx_status sensitivity(vx_tissue_s* t, const double* Xstar, const ParamsD& prm, const double* dCdX,
                      int count, const int32_t* kind, const int32_t* index, bool minres,
                      double rtol, int max_iter, int check_every, double* out, int32_t* status,
                      cudaStream_t s) {
  return t->dtype == VX_F64
             ? sensitivity_t<PolF64>(t, Xstar, prm, dCdX, count, kind, index, minres, rtol,
                                     max_iter, check_every, out, status, s)
             : sensitivity_t<PolF32>(t, Xstar, prm, dCdX, count, kind, index, minres, rtol,
                                     max_iter, check_every, out, status, s);
}

}  // namespace vx
