// Kernels of the equilibrium gradients (Methods, "Gradient computation
// methods"; the drivers are in grad.cu): the equilibrium-propagation
// difference of d_theta E, the v2v cost, the anisotropy cost and its
// gradient; plus the Hessian-vector product entry point.
#include <cuda_runtime.h>

#include "persistent.cuh"
#include "tissue.h"
#include "vx_internal.h"

namespace vx {

View<PolF64> topo_view(vx_tissue_s* t, const double* X) {
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

// ------------------------------------------------ anisotropy outer cost

// Per cell: corner count k, centroid (absolute, unwrapped from corner 0) and
// the shape tensor S = (1/k) sum (q - c)(q - c)^T; per-block sums of S.
__global__ void k_aniso_cells(View<PolF64> v, double2* cent, int* kk, double* part) {
  __shared__ double red[3][32];
  double s[3] = {0, 0, 0};
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < v.n; c += gridDim.x * blockDim.x) {
    const int h0 = v.ffirst[c];
    const int v0 = src_of(v, h0);
    const double2 X0 = v.X[v0];
    double qx[kMaxCorners * 2], qy[kMaxCorners * 2];
    qx[0] = 0;
    qy[0] = 0;
    int m = 1, cx = 0, cy = 0, h = h0;
    double mx = 0, my = 0;
    do {
      const uint32_t tg = v.tgt[h];
      cx += tgt_ox(tg);
      cy += tgt_oy(tg);
      h = v.nxt[h];
      if (h != h0) {
        const double2 Xt = v.X[tgt_v(tg)];
        qx[m] = (Xt.x + cx * v.Lx) - X0.x;
        qy[m] = (Xt.y + cy * v.Ly) - X0.y;
        ++m;
      }
    } while (h != h0 && m < 2 * kMaxCorners);
    for (int k = 0; k < m; ++k) {
      mx += qx[k];
      my += qy[k];
    }
    mx /= m;
    my /= m;
    double sxx = 0, syy = 0, sxy = 0;
    for (int k = 0; k < m; ++k) {
      const double wx = qx[k] - mx, wy = qy[k] - my;
      sxx += wx * wx;
      syy += wy * wy;
      sxy += wx * wy;
    }
    cent[c] = make_double2(X0.x + mx, X0.y + my);
    kk[c] = m;
    s[0] += sxx / m;
    s[1] += syy / m;
    s[2] += sxy / m;
  }
  for (int q = 0; q < 3; ++q) {
    double x = warp_sum(s[q]);
    if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double x = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x += red[threadIdx.x][w];
    part[3 * blockIdx.x + threadIdx.x] = x;
  }
}

// Q = mean S, q = ((Qxx - Qyy)/tr Q, 2 Qxy / tr Q), C = |q - q_target|^2 and
// G = dC/dQ into g[0..3] = (C, Gxx, Gyy, Gxy).
__global__ void k_aniso_final(const double* part, int nb, int n, const double* qt, double* g) {
  if (threadIdx.x || blockIdx.x) return;
  double Q[3] = {0, 0, 0};
  for (int b = 0; b < nb; ++b)
    for (int q = 0; q < 3; ++q) Q[q] += part[3 * b + q];
  const double Qxx = Q[0] / n, Qyy = Q[1] / n, Qxy = Q[2] / n, T = Qxx + Qyy;
  const double q1 = (Qxx - Qyy) / T, q2 = 2.0 * Qxy / T;
  const double r1 = 2.0 * (q1 - qt[0]), r2 = 2.0 * (q2 - qt[1]);
  g[0] = (q1 - qt[0]) * (q1 - qt[0]) + (q2 - qt[1]) * (q2 - qt[1]);
  g[1] = r1 * 2.0 * Qyy / (T * T) - r2 * 2.0 * Qxy / (T * T);
  g[2] = -r1 * 2.0 * Qxx / (T * T) - r2 * 2.0 * Qxy / (T * T);
  g[3] = r2 * 2.0 / T;
}

// dC/dx_i = sum over the cells of i of (1 / (n k)) (2 Gxx wx + Gxy wy,
// 2 Gyy wy + Gxy wx), w = x_i - centroid (minimum image).
__global__ void k_aniso_grad(View<PolF64> v, const double2* cent, const int* kk, const double* g,
                             double2* out) {
  const double Gxx = g[1], Gyy = g[2], Gxy = g[3];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < v.V; i += gridDim.x * blockDim.x) {
    const double2 x = v.X[i];
    double gx = 0, gy = 0;
    for (int a = 0; a < 3; ++a) {
      const int c = v.face[v.vout[a * v.V + i]];
      double wx = x.x - cent[c].x, wy = x.y - cent[c].y;
      wx -= v.Lx * rint(wx / v.Lx);
      wy -= v.Ly * rint(wy / v.Ly);
      const double s = 1.0 / ((double)v.n * kk[c]);
      gx += s * (2.0 * Gxx * wx + Gxy * wy);
      gy += s * (2.0 * Gyy * wy + Gxy * wx);
    }
    out[i] = make_double2(gx, gy);
  }
}

vx_status adjoint_plain(vx_tissue_s* t, const double* Xstar, const ParamsD& prm, const AdjParams& ap,
                        int check_every, AdjOut* out, cudaStream_t s);

size_t aniso_scratch_doubles(int n) { return 3 * (size_t)n + 3 * (size_t)((n + 255) / 256) + 8; }

// The anisotropy cost of one tissue given as an FP64 view (X = positions):
// C to the host, grad_X C to gradX [V][2] (device).  `scratch` holds
// aniso_scratch_doubles(n) doubles.  Synchronises s.
vx_status aniso_cost_view(const View<PolF64>& v, const double* q_target, double* gradX,
                          double* scratch, double* C, cudaStream_t s) {
  const int nb = (v.n + 255) / 256;
  double2* cent = (double2*)scratch;
  int* kk = (int*)(scratch + 2 * (size_t)v.n);
  double* part = scratch + 3 * (size_t)v.n;
  double* g = part + 3 * (size_t)nb;
  k_aniso_cells<<<nb, 256, 0, s>>>(v, cent, kk, part);
  k_aniso_final<<<1, 32, 0, s>>>(part, nb, v.n, q_target, g);
  k_aniso_grad<<<(v.V + 255) / 256, 256, 0, s>>>(v, cent, kk, g, (double2*)gradX);
  if (cudaMemcpyAsync(C, g, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    set_error(std::string("anisotropy cost: ") + cudaGetErrorString(cudaGetLastError()));
    return VX_ERR_CUDA;
  }
  return VX_OK;
}

// The solver region of the workspace (allocated by vx_tissue_create) holds
// `doubles`; nothing is allocated here.
bool ensure_work(vx_tissue_s* t, size_t doubles) {
  return t->work && doubles <= work_solver_doubles(t->n, t->V);
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
