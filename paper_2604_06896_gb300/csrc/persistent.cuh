// Persistent per-tissue bodies, written once for any Team (team.cuh):
//   min_body  - the whole FIRE / GD loop with T1 checks (Methods,
//               "Simulation engine", "T1 transitions"), optionally nudged by
//               -s Pi grad_X C (a phase of equilibrium propagation);
//   adj_body  - the implicit adjoint (Methods, "Implicit differentiation"):
//               preconditioned CG for H lam = Pi grad_X C on a Hessian-vector
//               product, then g = -(d^2E / dX dtheta)^T lam.
// Per-item state (velocities, forces, CG vectors) lives in registers of the
// thread that owns the item; positions, topology, cell coefficients and the
// CG direction live wherever the View points (shared memory for a resident
// CTA, L2-resident global memory for a cluster).
#pragma once
#include <type_traits>
#include "device_math.cuh"
#include "t1.cuh"
#include "kernels.cuh"
#include "team.cuh"

namespace vx {

template <class R>
struct Vec2Of;
template <>
struct Vec2Of<float> {
  using T = float2;
  using T4 = float4;
};
template <>
struct Vec2Of<double> {
  using T = double2;
  using T4 = double4;
};

// Slots for team reductions: three independent banks (each used at most once
// between two team barriers).
struct Slots {
  double* a;
  double* b;
  double* c;
  // cells the T1 pass changed (rank 0's shared memory); without it, a T1
  // pass is followed by a full cell pass
  int* dirty = nullptr;
  int dirty_cap = 0;
};

// Minimum-image v2v cost gradient at vertex i: (x_i - x_target,i) / N.
template <class P>
__device__ __forceinline__ void v2v_grad(const View<P>& v, int i, const double* Xt, double& gx,
                                         double& gy) {
  const double2 x = P::to_d(v.X[i]);
  double dx = x.x - Xt[2 * i], dy = x.y - Xt[2 * i + 1];
  dx -= v.Lx * rint(dx / v.Lx);
  dy -= v.Ly * rint(dy / v.Ly);
  gx = dx / v.V;
  gy = dy / v.V;
}

// Mean cell-shape-tensor anisotropy (the inverse-design outer cost):
// S_c = (1/k) sum (r_i - c)(r_i - c)^T over the k corners of cell c (c their
// mean), Q = mean_c S_c, q = ((Qxx - Qyy)/tr Q, 2 Qxy/tr Q),
// C = |q - q_target|^2.  Per cell, the centroid (absolute, FP64) and k go to
// `cent` / `kk`; the cell's S is returned (FP64 whatever the tissue's
// precision: the cost is a small nudge on top of the forces).
template <class P>
__device__ __forceinline__ void cell_shape(const View<P>& v, int c, double2* cent, int* kk,
                                           double& sxx, double& syy, double& sxy) {
  const int h0 = v.ffirst[c];
  const double2 X0 = P::to_d(v.X[src_of(v, h0)]);
  double qx[kMaxCorners], qy[kMaxCorners];
  int m = 0, cx = 0, cy = 0, h = h0;
  qx[0] = 0;
  qy[0] = 0;
  do {
    const uint32_t tg = v.tgt[h];
    cx += tgt_ox(tg);
    cy += tgt_oy(tg);
    h = v.nxt[h];
    ++m;
    if (h != h0 && m < kMaxCorners) {
      const double2 Xt = P::to_d(v.X[tgt_v(tg)]);
      qx[m] = (Xt.x + cx * v.Lx) - X0.x;
      qy[m] = (Xt.y + cy * v.Ly) - X0.y;
    }
  } while (h != h0 && m < kMaxCorners);
  double mx = 0, my = 0;
  for (int k = 0; k < m; ++k) {
    mx += qx[k];
    my += qy[k];
  }
  mx /= m;
  my /= m;
  sxx = syy = sxy = 0;
  for (int k = 0; k < m; ++k) {
    const double wx = qx[k] - mx, wy = qy[k] - my;
    sxx += wx * wx;
    syy += wy * wy;
    sxy += wx * wy;
  }
  sxx /= m;
  syy /= m;
  sxy /= m;
  cent[c] = make_double2(X0.x + mx, X0.y + my);
  kk[c] = m;
}

// dC/dQ = (Gxx, Gyy, Gxy) from Q = (Qxx, Qyy, Qxy) and q_target.
__device__ __forceinline__ void aniso_dC_dQ(const double (&Q)[3], const double* qt,
                                            double (&G)[3]) {
  const double T = Q[0] + Q[1];
  const double q1 = (Q[0] - Q[1]) / T, q2 = 2.0 * Q[2] / T;
  const double r1 = 2.0 * (q1 - qt[0]), r2 = 2.0 * (q2 - qt[1]);
  G[0] = r1 * 2.0 * Q[1] / (T * T) - r2 * 2.0 * Q[2] / (T * T);
  G[1] = -r1 * 2.0 * Q[0] / (T * T) - r2 * 2.0 * Q[2] / (T * T);
  G[2] = r2 * 2.0 / T;
}

// dC/dx_i = sum over the three cells c of i of (1/(n k_c)) (2 Gxx wx + Gxy wy,
// 2 Gyy wy + Gxy wx), w = x_i - centroid_c (minimum image).
template <class P>
__device__ __forceinline__ void aniso_grad_vertex(const View<P>& v, int i, const double2* cent,
                                                  const int* kk, const double (&G)[3], double& gx,
                                                  double& gy) {
  const double2 x = P::to_d(v.X[i]);
  gx = gy = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int c = v.vfc ? v.vfc[a * v.V + i] : v.face[v.vout[a * v.V + i]];
    double wx = x.x - cent[c].x, wy = x.y - cent[c].y;
    wx -= v.Lx * rint(wx / v.Lx);
    wy -= v.Ly * rint(wy / v.Ly);
    const double s = 1.0 / ((double)v.n * kk[c]);
    gx += s * (2.0 * G[0] * wx + G[2] * wy);
    gy += s * (2.0 * G[1] * wy + G[2] * wx);
  }
}

// The anisotropy nudge of a nudged phase, out of line so that the solver
// loops carry none of its registers: the shape tensors of the cells
// c = first + k stride (partial Q into Q), then, after a team barrier has
// published the centroids, grad_X C of the vertices i = first + k stride
// into nudge[i].
template <class P>
__device__ __noinline__ void aniso_q_pass(View<P> v, int first, int stride, double* ws,
                                          double* Q) {
  double2* cent = (double2*)ws;
  int* kk = (int*)(ws + 2 * (size_t)v.n);
  Q[0] = Q[1] = Q[2] = 0;
  for (int c = first; c < v.n; c += stride) {
    double sxx, syy, sxy;
    cell_shape(v, c, cent, kk, sxx, syy, sxy);
    Q[0] += sxx;
    Q[1] += syy;
    Q[2] += sxy;
  }
}
template <class P>
__device__ __noinline__ void aniso_nudge_pass(View<P> v, int first, int stride, const double* ws,
                                              double G0, double G1, double G2, double2* nudge) {
  const double G[3] = {G0, G1, G2};
  const double2* cent = (const double2*)ws;
  const int* kk = (const int*)(ws + 2 * (size_t)v.n);
  for (int i = first; i < v.V; i += stride) {
    double gx, gy;
    aniso_grad_vertex(v, i, cent, kk, G, gx, gy);
    nudge[i] = make_double2(gx, gy);
  }
}

// --------------------------------------------------------------- minimiser

// Coefficients (cA, cP) of the listed cells, by the 32 lanes of one warp,
// with the same arithmetic as the cell pass of min_body: after a T1 pass
// only the cells around a moved edge change.  Kept out of line so that the
// solver loop does not carry its registers.
template <class P, class R2>
__device__ __noinline__ void refresh_cells(View<P> vw, R2* cell, const ParamsD& prm,
                                           const int* list, int count) {
  using R = typename P::R;
  for (int q = (int)(threadIdx.x & 31); q < count; q += 32) {
    const int c = list[q];
    R A, Pp;
    cell_geometry(vw, c, A, Pp, (R)0, (uint32_t*)nullptr);
    R2 cc;
    cc.x = (R)2 * (R)prm.ka(c) * (A - (R)prm.a0(c));
    cc.y = (R)2 * (R)prm.kp(c) * (Pp - (R)prm.p0(c));
    cell[c] = cc;
  }
}

// The same for the whole CTA (out of line: the array-state loop keeps its
// registers).
template <class P, class R2>
__device__ __noinline__ void refresh_cells_cta(View<P> vw, R2* cell, const ParamsD& prm,
                                               const int* list, int count) {
  using R = typename P::R;
  for (int q = (int)threadIdx.x; q < count; q += (int)blockDim.x) {
    const int c = list[q];
    R A, Pp;
    cell_geometry(vw, c, A, Pp, (R)0, (uint32_t*)nullptr);
    R2 cc;
    cc.x = (R)2 * (R)prm.ka(c) * (A - (R)prm.a0(c));
    cc.y = (R)2 * (R)prm.kp(c) * (Pp - (R)prm.p0(c));
    cell[c] = cc;
  }
}

template <class P, class Team, int MAXC, class LamT>
__device__ void min_body(const Team& tm, View<P> vw, typename Vec2Of<typename P::R>::T* cell,
                         const LamT* lam, uint32_t* shortbits, uint32_t* touched, Slots sl,
                         const ParamsD& prm, const MinParams& mp, const double* Xin,
                         double* Xout, MinOut* out) {
  using R = typename P::R;
  using R2 = typename Vec2Of<R>::T;
  constexpr int MAXV = 2 * MAXC;
  const int n = vw.n, V = vw.V, E = vw.E;
  const int f0 = tm.first(), st = tm.stride();

  // Positions in (the owner converts), registers for per-item state.
  if (Xin)
#pragma unroll
    for (int k = 0; k < MAXV; ++k) {
      const int i = f0 + k * st;
      if (i < V) vw.X[i] = P::from_d(Xin[2 * i], Xin[2 * i + 1]);
    }
  R vx[MAXV], vy[MAXV], fx[MAXV], fy[MAXV];
#pragma unroll
  for (int k = 0; k < MAXV; ++k) vx[k] = vy[k] = fx[k] = fy[k] = 0;
  tm.sync();

  // Nudged phase: -s Pi grad C, with the mean of grad C taken once (the
  // centroid is conserved because every force term sums to zero).
  double nmx = 0, nmy = 0;
  const bool nudged = mp.cost == 1 && mp.nudge_s != 0.0;
  const bool nudged_aniso = mp.cost == 2 && mp.nudge_s != 0.0 && mp.aniso_ws != nullptr &&
                            mp.aniso_nudge != nullptr;
  if (nudged) {
    double s2[2] = {0, 0};
#pragma unroll
    for (int k = 0; k < MAXV; ++k) {
      const int i = f0 + k * st;
      if (i < V) {
        double gx, gy;
        v2v_grad(vw, i, mp.cost_data, gx, gy);
        s2[0] += gx;
        s2[1] += gy;
      }
    }
    tm.template reduce<2>(s2, sl.c, 0);
    nmx = s2[0] / V;
    nmy = s2[1] / V;
  }

  const R lminR = (R)mp.l_min;
  double dt = mp.dt0, alpha = mp.alpha0, fmx = 0;
  int npos = 0, below = 0, it = 0, status = VX_NOT_CONVERGED, n_t1 = 0, n_st = 0;

  auto cell_pass = [&](R lm) -> bool {
    bool fl = false;
#pragma unroll
    for (int k = 0; k < MAXC; ++k) {
      const int c = f0 + k * st;
      if (c < n) {
        R A, Pp;
        fl |= cell_geometry(vw, c, A, Pp, lm, shortbits);
        R2 cc;
        // per-cell parameters are read where used (no registers held)
        cc.x = (R)2 * (R)prm.ka(c) * (A - (R)prm.a0(c));
        cc.y = (R)2 * (R)prm.kp(c) * (Pp - (R)prm.p0(c));
        cell[c] = cc;
      }
    }
    return fl;
  };

  for (it = 0;; ++it) {
    const bool fl = cell_pass(lminR);
    if (mp.l_min > 0) {
      if (tm.sync_or(fl, sl.b)) {
        bool ovf = false;
        if (tm.rank() == 0) {
          T1Stats s1 = {0, 0, 0};
          int nd = 0;
          t1_pass_block(vw, prm, mp.l_min, shortbits, touched, &s1, sl.dirty, sl.dirty_cap,
                        sl.dirty ? &nd : nullptr, mp.edge_events);
          n_t1 += s1.n_t1;
          n_st += s1.n_stretch;
          if (threadIdx.x < 32) {
            nd = __shfl_sync(0xffffffffu, nd, 0);
            ovf = !sl.dirty || nd > sl.dirty_cap;
            if (!ovf) refresh_cells(vw, cell, prm, sl.dirty, nd);
          }
        }
        const bool full = tm.sync_or(ovf, sl.c);
        // The moved vertices restart from rest.  The 32 vertices of a mask
        // word belong to the 32 lanes of one warp, which clears the word.
#pragma unroll
        for (int k = 0; k < MAXV; ++k) {
          const int i = f0 + k * st;
          const uint32_t word = i < V ? touched[i >> 5] : 0u;
          if ((word >> (i & 31)) & 1u) vx[k] = vy[k] = 0;
          __syncwarp();
          if ((threadIdx.x & 31) == 0 && word) touched[i >> 5] = 0;
        }
        if (full) {
          cell_pass((R)0);
          tm.sync();
        }
      }
    } else {
      tm.sync();
    }
    // Anisotropy nudging: the cells' centroids and shape tensors, then
    // dC/dQ from the team-wide mean Q (the reduction's barrier publishes the
    // centroids to the whole team; the nudged phases run without T1, so
    // bank c is free here).
    if (nudged_aniso) {
      double Q[3];
      aniso_q_pass(vw, f0, st, mp.aniso_ws, Q);
      tm.template reduce<3>(Q, sl.c, 0);
      Q[0] /= n;
      Q[1] /= n;
      Q[2] /= n;
      double G[3];
      aniso_dC_dQ(Q, mp.cost_data, G);
      // each thread reads back only its own vertices' nudges
      aniso_nudge_pass(vw, f0, st, mp.aniso_ws, G[0], G[1], G[2], (double2*)mp.aniso_nudge);
    }
    // F.F, F.v, v.v, max |F_i|^2: FP32 tissues sum their per-thread and
    // per-warp parts in FP32 and combine warps in FP64
    constexpr bool kF32 = std::is_same<R, float>::value;
    double red[4] = {0, 0, 0, 0};
    float redf[4] = {0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < MAXV; ++k) {
      const int i = f0 + k * st;
      if (i < V) vertex_force(vw, i, cell, lam, prm.lam_s, fx[k], fy[k]);
    }
#pragma unroll
    for (int k = 0; k < MAXV; ++k) {
      const int i = f0 + k * st;
      if (i < V) {
        if (nudged) {
          double gx, gy;
          v2v_grad(vw, i, mp.cost_data, gx, gy);
          fx[k] -= (R)(mp.nudge_s * (gx - nmx));
          fy[k] -= (R)(mp.nudge_s * (gy - nmy));
        }
        if (nudged_aniso) {
          // sum_i dC/dx_i = 0 (each cell's w sum to zero): no projection
          const double2 g = ((const double2*)mp.aniso_nudge)[i];
          fx[k] -= (R)(mp.nudge_s * g.x);
          fy[k] -= (R)(mp.nudge_s * g.y);
        }
        if constexpr (kF32) {
          const float f2 = fx[k] * fx[k] + fy[k] * fy[k];
          redf[0] += f2;
          redf[1] += fx[k] * vx[k] + fy[k] * vy[k];
          redf[2] += vx[k] * vx[k] + vy[k] * vy[k];
          redf[3] = fmaxf(redf[3], f2);
        } else {
          const double f2 = (double)(fx[k] * fx[k] + fy[k] * fy[k]);
          red[0] += f2;
          red[1] += (double)(fx[k] * vx[k] + fy[k] * vy[k]);
          red[2] += (double)(vx[k] * vx[k] + vy[k] * vy[k]);
          red[3] = fmax(red[3], f2);
        }
      }
    }
    if constexpr (kF32)
      tm.template reduce_f<4>(redf, red, sl.a, 1);
    else
      tm.template reduce<4>(red, sl.a, 1);
    if (tm.failed()) {
      status = VX_ERR_TIMEOUT;
      break;
    }
    fmx = kF32 ? (double)sqrtf((float)red[3]) : sqrt(red[3]);
    if (!(fmx == fmx) || isinf(fmx) || !(red[0] == red[0])) {
      status = VX_ERR_NONFINITE;
      break;
    }
    below = (fmx < mp.tol) ? below + 1 : 0;
    if (below >= mp.patience) {
      status = VX_OK;
      break;
    }
    if (it >= mp.max_iter) {
      status = VX_NOT_CONVERGED;
      break;
    }
    if (mp.method == 1) {
      const R s = (R)mp.gd_lr;
#pragma unroll
      for (int k = 0; k < MAXV; ++k) {
        const int i = f0 + k * st;
        if (i < V) P::add(vw.X[i], s * fx[k], s * fy[k]);
      }
    } else {
      R mA = 0, mB = 0;
      bool zero;
      if (red[1] > 0) {
        mA = (R)(1.0 - alpha);
        mB = (R)alpha * sqrt((R)red[2]) / sqrt((R)red[0]);
        zero = false;
        if (npos > mp.n_min) {
          dt = fmin(dt * mp.f_inc, mp.dt_max);
          alpha *= mp.f_alpha;
        }
        ++npos;
      } else {
        zero = true;
        dt *= mp.f_dec;
        alpha = mp.alpha0;
        npos = 0;
      }
      const R dtR = (R)dt;
      typename P::Pos xs[MAXV];
#pragma unroll
      for (int k = 0; k < MAXV; ++k) {
        const int i = f0 + k * st;
        if (i < V) xs[k] = vw.X[i];
      }
#pragma unroll
      for (int k = 0; k < MAXV; ++k) {
        const int i = f0 + k * st;
        if (i < V) {
          R ux = zero ? (R)0 : mA * vx[k] + mB * fx[k];
          R uy = zero ? (R)0 : mA * vy[k] + mB * fy[k];
          ux += dtR * fx[k];
          uy += dtR * fy[k];
          vx[k] = ux;
          vy[k] = uy;
          P::add(xs[k], dtR * ux, dtR * uy);
          vw.X[i] = xs[k];
        }
      }
    }
    tm.sync();
  }
  tm.sync();

  // Energy, inverted cells and short edges at the returned X.
  double fin[3] = {0, 0, 0};
#pragma unroll
  for (int k = 0; k < MAXC; ++k) {
    const int c = f0 + k * st;
    if (c < n) {
      R A, Pp;
      double el = 0;
      cell_geometry(vw, c, A, Pp, (R)0, shortbits, &el, &prm);
      const double dA = (double)A - prm.a0(c), dP = (double)Pp - prm.p0(c);
      fin[0] += prm.ka(c) * dA * dA + prm.kp(c) * dP * dP + el;
      fin[1] += (A <= 0) ? 1.0 : 0.0;
    }
  }
  if (mp.l_min > 0)
    for (int e = f0; e < E; e += st) fin[2] += edge_len_d(vw, 2 * e) < mp.l_min ? 1.0 : 0.0;
  tm.template reduce<3>(fin, sl.c, 0);
  if (tm.leader() && out) {
    MinOut o;
    o.status = status;
    o.iters = it;
    o.n_t1 = n_t1;
    o.n_stretch = n_st;
    o.n_short = (int)fin[2];
    o.n_inverted = (int)fin[1];
    o.force_evals = it + 1;
    o.wrap_err = 0;
    o.fmax = fmx;
    o.energy = fin[0];
    *out = o;
  }
  if (Xout)
    for (int i = f0; i < V; i += st) {
      const double2 d = P::to_d(vw.X[i]);
      Xout[2 * i] = d.x;
      Xout[2 * i + 1] = d.y;
    }
}

// ----------------------------------------------------------------- adjoint

struct AdjParams {
  const double* dCdX;   // [V][2] or null (then the built-in cost)
  int cost;             // 1 v2v
  const double* cost_data;
  double rtol;
  int max_iter;
  double* g_lam;        // [E] or null
  double* g_A0;         // [n] or null
  double* g_P0;         // [n] or null
};

struct AdjOut {
  int status, iters;
  double rel_residual, cost;
};

// Directional derivatives of one cell's area and perimeter along `vec`:
// sA = grad A . vec = 1/2 sum [cross(q_k, w_{k+1}) + cross(w_k, q_{k+1})],
// sP = grad P . vec = sum u_k . (w_{k+1} - w_k).
template <class P, class VT>
__device__ __forceinline__ void cell_dir(const View<P>& v, int c, const VT* vec,
                                         typename P::R& sA, typename P::R& sP) {
  using R = typename P::R;
  if (v.ccor) {
    const int m = v.ccnt[c];
    const uint32_t* cor = v.ccor + (size_t)c * kMaxCorners;
    const int v0 = tgt_v(cor[0]);
    const typename P::Pos X0 = v.X[v0];
    const VT w0 = vec[v0];
    VT w = w0;
    R qx = 0, qy = 0, a = 0, pp = 0;
    for (int k = 1; k <= m; ++k) {
      R nx = 0, ny = 0;
      VT wn = w0;
      if (k < m) {
        const uint32_t t = cor[k];
        P::diff(v.X[tgt_v(t)], X0, tgt_ox(t), tgt_oy(t), v.box, nx, ny);
        wn = vec[tgt_v(t)];
      }
      a += qx * (R)wn.y - qy * (R)wn.x + (R)w.x * ny - (R)w.y * nx;
      const R ex = nx - qx, ey = ny - qy;
      const R rl = P::rsqrt(ex * ex + ey * ey);
      pp += (ex * ((R)wn.x - (R)w.x) + ey * ((R)wn.y - (R)w.y)) * rl;
      qx = nx;
      qy = ny;
      w = wn;
    }
    sA = (R)0.5 * a;
    sP = pp;
    return;
  }
  const int h0 = v.ffirst[c];
  const int v0 = src_of(v, h0);
  const typename P::Pos X0 = v.X[v0];
  VT w = vec[v0];
  R qx = 0, qy = 0, a = 0, pp = 0;
  int cx = 0, cy = 0, h = h0, guard = 0;
  do {
    const uint32_t tg = v.tgt[h];
    cx += tgt_ox(tg);
    cy += tgt_oy(tg);
    R nx, ny;
    const int j = tgt_v(tg);
    P::diff(v.X[j], X0, cx, cy, v.box, nx, ny);
    const VT wn = vec[j];
    a += qx * (R)wn.y - qy * (R)wn.x + (R)w.x * ny - (R)w.y * nx;
    const R ex = nx - qx, ey = ny - qy;
    const R rl = P::rsqrt(ex * ex + ey * ey);
    pp += (ex * ((R)wn.x - (R)w.x) + ey * ((R)wn.y - (R)w.y)) * rl;
    qx = nx;
    qy = ny;
    w = wn;
    h = v.nxt[h];
  } while (h != h0 && ++guard < 4096);
  sA = (R)0.5 * a;
  sP = pp;
}

// (H vec)_i, with per cell (cA, cP, 2 K_A sA, 2 K_P sP) in cell4.
template <class P, class C4, class LamT, class VT>
__device__ __forceinline__ void vertex_hvp(const View<P>& v, int i, const C4* cell4,
                                           const LamT* lam, double lam_s, const VT* vec,
                                           typename P::R& hx, typename P::R& hy) {
  using R = typename P::R;
  const typename P::Pos Xi = v.X[i];
  const VT vi = vec[i];
  R dx[3], dy[3], ux[3], uy[3], il[3], cA[3], cP[3], zA[3], zP[3], la[3], wx[3], wy[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int h = v.vout[a * v.V + i];
    const uint32_t tg = v.vnb ? v.vnb[a * v.V + i] : v.tgt[h];
    const int j = tgt_v(tg);
    P::diff(v.X[j], Xi, tgt_ox(tg), tgt_oy(tg), v.box, dx[a], dy[a]);
    il[a] = P::rsqrt(dx[a] * dx[a] + dy[a] * dy[a]);
    ux[a] = dx[a] * il[a];
    uy[a] = dy[a] * il[a];
    const C4 cc = cell4[v.vfc ? v.vfc[a * v.V + i] : v.face[h]];
    cA[a] = (R)cc.x;
    cP[a] = (R)cc.y;
    zA[a] = (R)cc.z;
    zP[a] = (R)cc.w;
    la[a] = lam ? (R)lam[h >> 1] : (R)lam_s;
    const VT wj = vec[j];
    wx[a] = (R)wj.x;
    wy[a] = (R)wj.y;
  }
  R gx = 0, gy = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int am = (a + 2) % 3, ap = (a + 1) % 3;
    const R T = la[a] + cP[a] + cP[am];
    // T M_a (v_i - w_a), M = (I - u u^T) / l
    const R ex = (R)vi.x - wx[a], ey = (R)vi.y - wy[a];
    const R ue = ux[a] * ex + uy[a] * ey;
    gx += T * il[a] * (ex - ue * ux[a]);
    gy += T * il[a] * (ey - ue * uy[a]);
    // 2 K_A sA grad_i A = zA * 1/2 rot(d_a - d_{a+1})
    gx += (R)0.5 * zA[a] * (dy[a] - dy[ap]);
    gy -= (R)0.5 * zA[a] * (dx[a] - dx[ap]);
    // 2 K_A (A - A0) (grad^2 A vec)_i = cA * 1/2 rot(w_a - w_{a+1})
    gx += (R)0.5 * cA[a] * (wy[a] - wy[ap]);
    gy -= (R)0.5 * cA[a] * (wx[a] - wx[ap]);
    // 2 K_P sP grad_i P = zP * (-u_a - u_{a+1})
    gx -= zP[a] * (ux[a] + ux[ap]);
    gy -= zP[a] * (uy[a] + uy[ap]);
  }
  hx = gx;
  hy = gy;
}

// 2 x 2 diagonal block of H at vertex i (K2A, K2P = 2 K_A, 2 K_P per cell in
// cell4.z / .w): sum_a T_a M_a + 2 K_A gA gA^T + 2 K_P gP gP^T.
template <class P, class C4, class LamT>
__device__ __forceinline__ void vertex_diag(const View<P>& v, int i, const C4* cell4,
                                            const LamT* lam, double lam_s, double& dxx,
                                            double& dxy, double& dyy) {
  using R = typename P::R;
  const typename P::Pos Xi = v.X[i];
  double dx[3], dy[3], ux[3], uy[3], il[3], cP[3], kA[3], kP[3], la[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int h = v.vout[a * v.V + i];
    const uint32_t tg = v.tgt[h];
    R ddx, ddy;
    P::diff(v.X[tgt_v(tg)], Xi, tgt_ox(tg), tgt_oy(tg), v.box, ddx, ddy);
    dx[a] = ddx;
    dy[a] = ddy;
    il[a] = 1.0 / sqrt(dx[a] * dx[a] + dy[a] * dy[a]);
    ux[a] = dx[a] * il[a];
    uy[a] = dy[a] * il[a];
    const C4 cc = cell4[v.face[h]];
    cP[a] = (double)cc.y;
    kA[a] = (double)cc.z;
    kP[a] = (double)cc.w;
    la[a] = lam ? (double)lam[h >> 1] : lam_s;
  }
  dxx = dxy = dyy = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int am = (a + 2) % 3, ap = (a + 1) % 3;
    const double T = la[a] + cP[a] + cP[am];
    dxx += T * il[a] * (1.0 - ux[a] * ux[a]);
    dxy += T * il[a] * (-ux[a] * uy[a]);
    dyy += T * il[a] * (1.0 - uy[a] * uy[a]);
    const double gAx = 0.5 * (dy[a] - dy[ap]), gAy = -0.5 * (dx[a] - dx[ap]);
    const double gPx = -(ux[a] + ux[ap]), gPy = -(uy[a] + uy[ap]);
    dxx += kA[a] * gAx * gAx + kP[a] * gPx * gPx;
    dxy += kA[a] * gAx * gAy + kP[a] * gPx * gPy;
    dyy += kA[a] * gAy * gAy + kP[a] * gPy * gPy;
  }
}

template <class P, class Team, int MAXC, class LamT>
__device__ void adj_body(const Team& tm, View<P> vw, typename Vec2Of<typename P::R>::T4* cell4,
                         const LamT* lam, typename Vec2Of<typename P::R>::T* pvec, Slots sl,
                         const ParamsD& prm, const AdjParams& ap, const double* Xin,
                         AdjOut* out) {
  using R = typename P::R;
  using R2 = typename Vec2Of<R>::T;
  using R4 = typename Vec2Of<R>::T4;
  constexpr int MAXV = 2 * MAXC;
  const int n = vw.n, V = vw.V, E = vw.E;
  const int f0 = tm.first(), st = tm.stride();

  if (Xin)
    for (int i = f0; i < V; i += st) vw.X[i] = P::from_d(Xin[2 * i], Xin[2 * i + 1]);
  R k2a[MAXC], k2p[MAXC];
#pragma unroll
  for (int k = 0; k < MAXC; ++k) {
    const int c = f0 + k * st;
    const int cc = c < n ? c : 0;
    k2a[k] = (R)(2.0 * prm.ka(cc));
    k2p[k] = (R)(2.0 * prm.kp(cc));
  }
  tm.sync();
  // Forward geometry at X*: (cA, cP, 2 K_A, 2 K_P) per cell.
#pragma unroll
  for (int k = 0; k < MAXC; ++k) {
    const int c = f0 + k * st;
    if (c < n) {
      R A, Pp;
      cell_geometry(vw, c, A, Pp, (R)0, nullptr);
      R4 q;
      q.x = (R)(2.0 * prm.ka(c) * ((double)A - prm.a0(c)));
      q.y = (R)(2.0 * prm.kp(c) * ((double)Pp - prm.p0(c)));
      q.z = k2a[k];
      q.w = k2p[k];
      cell4[c] = q;
    }
  }
  tm.sync();
  // Preconditioner (inverse of the 2 x 2 diagonal blocks) and right side.
  R ia[MAXV], ib[MAXV], ic[MAXV], rx[MAXV], ry[MAXV], lx[MAXV], ly[MAXV];
  double s3[3] = {0, 0, 0};
#pragma unroll
  for (int k = 0; k < MAXV; ++k) {
    const int i = f0 + k * st;
    rx[k] = ry[k] = lx[k] = ly[k] = 0;
    ia[k] = ic[k] = 1;
    ib[k] = 0;
    if (i < V) {
      double dxx, dxy, dyy;
      vertex_diag(vw, i, cell4, lam, prm.lam_s, dxx, dxy, dyy);
      const double det = dxx * dyy - dxy * dxy;
      if (dxx > 0 && det > 1e-300 * dxx * dxx) {
        ia[k] = (R)(dyy / det);
        ib[k] = (R)(-dxy / det);
        ic[k] = (R)(dxx / det);
      } else {
        const double tr = fabs(dxx) + fabs(dyy);
        ia[k] = ic[k] = (R)(tr > 0 ? 2.0 / tr : 1.0);
      }
      double gx, gy;
      if (ap.dCdX) {
        gx = ap.dCdX[2 * i];
        gy = ap.dCdX[2 * i + 1];
      } else {
        v2v_grad(vw, i, ap.cost_data, gx, gy);
        s3[2] += 0.5 * V * (gx * gx + gy * gy);  // C = (1/2N) sum |D|^2, g = D/N
      }
      rx[k] = (R)gx;
      ry[k] = (R)gy;
      s3[0] += gx;
      s3[1] += gy;
    }
  }
  tm.template reduce<3>(s3, sl.a, 0);
  const R mx = (R)(s3[0] / V), my = (R)(s3[1] / V);
  const double cost = s3[2];
  double s2[2] = {0, 0};  // r.z, r.r
#pragma unroll
  for (int k = 0; k < MAXV; ++k) {
    const int i = f0 + k * st;
    if (i < V) {
      rx[k] -= mx;
      ry[k] -= my;
      const R zx = ia[k] * rx[k] + ib[k] * ry[k], zy = ib[k] * rx[k] + ic[k] * ry[k];
      R2 pz;
      pz.x = zx;
      pz.y = zy;
      pvec[i] = pz;
      s2[0] += (double)(rx[k] * zx + ry[k] * zy);
      s2[1] += (double)(rx[k] * rx[k] + ry[k] * ry[k]);
    }
  }
  tm.template reduce<2>(s2, sl.b, 0);
  double rz = s2[0];
  const double bnorm = sqrt(s2[1]);
  double rnorm = bnorm;
  int status = VX_NOT_CONVERGED, it = 0;
  if (bnorm == 0.0) status = VX_OK;
  tm.sync();
  for (it = 0; status == VX_NOT_CONVERGED && it < ap.max_iter; ++it) {
    // HVP, cell pass: (2 K_A sA, 2 K_P sP) along p.
#pragma unroll
    for (int k = 0; k < MAXC; ++k) {
      const int c = f0 + k * st;
      if (c < n) {
        R sA, sP;
        cell_dir(vw, c, pvec, sA, sP);
        R4 q = cell4[c];
        q.z = k2a[k] * sA;
        q.w = k2p[k] * sP;
        cell4[c] = q;
      }
    }
    tm.sync();
    R hx[MAXV], hy[MAXV], px[MAXV], py[MAXV];
    double s1[1] = {0};
#pragma unroll
    for (int k = 0; k < MAXV; ++k) {
      const int i = f0 + k * st;
      hx[k] = hy[k] = px[k] = py[k] = 0;
      if (i < V) {
        vertex_hvp(vw, i, cell4, lam, prm.lam_s, pvec, hx[k], hy[k]);
        const R2 pp = pvec[i];
        px[k] = pp.x;
        py[k] = pp.y;
        s1[0] += (double)(px[k] * hx[k] + py[k] * hy[k]);
      }
    }
    tm.template reduce<1>(s1, sl.a, 0);
    if (!(s1[0] > 0)) {
      status = VX_ERR_INDEFINITE;
      break;
    }
    const R al = (R)(rz / s1[0]);
    double s2b[2] = {0, 0};
    R zx[MAXV], zy[MAXV];
#pragma unroll
    for (int k = 0; k < MAXV; ++k) {
      const int i = f0 + k * st;
      zx[k] = zy[k] = 0;
      if (i < V) {
        lx[k] += al * px[k];
        ly[k] += al * py[k];
        rx[k] -= al * hx[k];
        ry[k] -= al * hy[k];
        zx[k] = ia[k] * rx[k] + ib[k] * ry[k];
        zy[k] = ib[k] * rx[k] + ic[k] * ry[k];
        s2b[0] += (double)(rx[k] * zx[k] + ry[k] * zy[k]);
        s2b[1] += (double)(rx[k] * rx[k] + ry[k] * ry[k]);
      }
    }
    tm.template reduce<2>(s2b, sl.b, 0);
    rnorm = sqrt(s2b[1]);
    if (!(rnorm == rnorm)) {
      status = VX_ERR_NONFINITE;
      break;
    }
    if (rnorm <= ap.rtol * bnorm) status = VX_OK;
    const R be = (R)(s2b[0] / rz);
    rz = s2b[0];
#pragma unroll
    for (int k = 0; k < MAXV; ++k) {
      const int i = f0 + k * st;
      if (i < V && status == VX_NOT_CONVERGED) {
        R2 pp;
        pp.x = zx[k] + be * px[k];
        pp.y = zy[k] + be * py[k];
        pvec[i] = pp;
      }
    }
    tm.sync();
  }
  tm.sync();
  // lambda into pvec, then g = -(d^2E/dX dtheta)^T lambda.
#pragma unroll
  for (int k = 0; k < MAXV; ++k) {
    const int i = f0 + k * st;
    if (i < V) {
      R2 l;
      l.x = lx[k];
      l.y = ly[k];
      pvec[i] = l;
    }
  }
  tm.sync();
  if (ap.g_lam)
    for (int e = f0; e < E; e += st) {
      const int h = 2 * e;
      const uint32_t tg = vw.tgt[h];
      const int s = src_of(vw, h), t = tgt_v(tg);
      R dx, dy;
      P::diff(vw.X[t], vw.X[s], tgt_ox(tg), tgt_oy(tg), vw.box, dx, dy);
      const R il = P::rsqrt(dx * dx + dy * dy);
      const R2 lt = pvec[t], ls = pvec[s];
      ap.g_lam[e] = -(double)((dx * (lt.x - ls.x) + dy * (lt.y - ls.y)) * il);
    }
  if (ap.g_A0 || ap.g_P0)
    for (int c = f0; c < n; c += st) {
      R sA, sP;
      cell_dir(vw, c, pvec, sA, sP);
      if (ap.g_A0) ap.g_A0[c] = 2.0 * prm.ka(c) * (double)sA;
      if (ap.g_P0) ap.g_P0[c] = 2.0 * prm.kp(c) * (double)sP;
    }
  if (tm.leader() && out) {
    AdjOut o;
    o.status = status;
    o.iters = it;
    o.rel_residual = bnorm > 0 ? rnorm / bnorm : 0.0;
    o.cost = cost;
    *out = o;
  }
}

}  // namespace vx

namespace vx {

// ------------------------------------------------- minimiser, memory state

// The same iteration as min_body for one CTA, with the per-vertex state
// (velocities, forces) in arrays instead of registers and the per-cell
// parameters read where they are needed, so that one kernel serves tissues
// of any size (the batched path).  `vel` and `frc` may live in shared or
// global memory.
template <class P, int T, class LamT>
__device__ void min_body_mem(View<P> vw, typename Vec2Of<typename P::R>::T* cell,
                             typename Vec2Of<typename P::R>::T* vel,
                             typename Vec2Of<typename P::R>::T* frc, const LamT* lam,
                             uint32_t* shortbits, uint32_t* touched, Slots sl,
                             const ParamsD& prm, const MinParams& mp, const double* Xin,
                             double* Xout, MinOut* out) {
  using R = typename P::R;
  using R2 = typename Vec2Of<R>::T;
  BlockTeam<T> tm;
  const int n = vw.n, V = vw.V, E = vw.E, tid = threadIdx.x;
  for (int i = tid; i < V; i += T) {
    if (Xin) vw.X[i] = P::from_d(Xin[2 * i], Xin[2 * i + 1]);
    R2 z;
    z.x = 0;
    z.y = 0;
    vel[i] = z;
  }
  for (int w = tid; w < (E + 31) / 32; w += T) shortbits[w] = 0;
  for (int w = tid; w < (V + 31) / 32; w += T) touched[w] = 0;
  tm.sync();
  // Nudged phase of equilibrium propagation: -s Pi grad_X C (v2v: the mean
  // of grad C taken once, the centroid being conserved; anisotropy: the
  // gradient sums to zero by itself).
  const bool nudged_v2v = mp.cost == 1 && mp.nudge_s != 0.0;
  const bool nudged_aniso = mp.cost == 2 && mp.nudge_s != 0.0 && mp.aniso_ws != nullptr &&
                            mp.aniso_nudge != nullptr;
  double nmx = 0, nmy = 0;
  if (nudged_v2v) {
    double s2[2] = {0, 0};
    for (int i = tid; i < V; i += T) {
      double gx, gy;
      v2v_grad(vw, i, mp.cost_data, gx, gy);
      s2[0] += gx;
      s2[1] += gy;
    }
    tm.template reduce<2>(s2, sl.c, 0);
    nmx = s2[0] / V;
    nmy = s2[1] / V;
    tm.sync();
  }
  const R lminR = (R)mp.l_min;
  double dt = mp.dt0, alpha = mp.alpha0, fmx = 0;
  int npos = 0, below = 0, it = 0, status = VX_NOT_CONVERGED, n_t1 = 0, n_st = 0;
  // uniform parameters converted once (FP64 operations, conversions
  // included, are slow on this GPU); the values are those of the per-cell
  // expressions
  const R ka2_s = (R)(2.0 * prm.KA_s), kp2_s = (R)(2.0 * prm.KP_s);
  const R a0_s = (R)prm.A0_s, p0_s = (R)prm.P0_s;
  auto cell_coef = [&](int c, R A, R Pp) {
    R2 cc;
    cc.x = (prm.KA ? (R)(2.0 * prm.KA[c]) : ka2_s) * (A - (prm.A0 ? (R)prm.A0[c] : a0_s));
    cc.y = (prm.KP ? (R)(2.0 * prm.KP[c]) : kp2_s) * (Pp - (prm.P0 ? (R)prm.P0[c] : p0_s));
    cell[c] = cc;
  };
  auto cell_pass = [&](R lm) -> bool {
    bool fl = false;
    if (vw.ccor) {
      // two cells per thread with both gathers in flight (flat tables)
      for (int c0 = tid; c0 < n; c0 += 2 * T) {
        const int c1 = c0 + T;
        CGather<P> g0, g1;
        cell_gather(vw, c0, g0);
        if (c1 < n) cell_gather(vw, c1, g1);
        R A, Pp;
        fl |= cell_geometry_g(vw, c0, g0, A, Pp, lm, shortbits);
        cell_coef(c0, A, Pp);
        if (c1 < n) {
          fl |= cell_geometry_g(vw, c1, g1, A, Pp, lm, shortbits);
          cell_coef(c1, A, Pp);
        }
      }
      return fl;
    }
    for (int c = tid; c < n; c += T) {
      R A, Pp;
      fl |= cell_geometry(vw, c, A, Pp, lm, shortbits);
      cell_coef(c, A, Pp);
    }
    return fl;
  };
  for (it = 0;; ++it) {
    const bool fl = cell_pass(lminR);
    if (mp.l_min > 0) {
      if (__syncthreads_or(fl)) {
        // cells the pass changed (shared memory); their coefficients are
        // recomputed by the whole CTA, or every cell's if the list overflows
        constexpr int kMemDirty = 512;
        __shared__ int mdirty[kMemDirty];
        __shared__ int mnd;
        {
          T1Stats s1 = {0, 0, 0};
          int nd = 0;
          t1_pass_block(vw, prm, mp.l_min, shortbits, touched, &s1, mdirty, kMemDirty, &nd,
                        mp.edge_events);
          n_t1 += s1.n_t1;
          n_st += s1.n_stretch;
          if (tid == 0) mnd = nd;
        }
        __syncthreads();
        const int nd = mnd;
        for (int w = tid; w < (V + 31) / 32; w += T) {
          uint32_t b = touched[w];
          touched[w] = 0;
          while (b) {
            const int i = (w << 5) + __ffs(b) - 1;
            b &= b - 1;
            R2 z;
            z.x = 0;
            z.y = 0;
            vel[i] = z;
          }
        }
        if (nd > kMemDirty) {
          cell_pass((R)0);
        } else {
          refresh_cells_cta(vw, cell, prm, mdirty, nd);
        }
        __syncthreads();
      }
    } else {
      __syncthreads();
    }
    // Nudged phases (no T1, so bank c is free): anisotropy dC/dQ from the
    // cells' shapes; the reduction's barrier publishes the centroids.
    if (nudged_aniso) {
      double Q[3];
      aniso_q_pass(vw, tid, T, mp.aniso_ws, Q);
      tm.template reduce<3>(Q, sl.c, 0);
      Q[0] /= n;
      Q[1] /= n;
      Q[2] /= n;
      double G[3];
      aniso_dC_dQ(Q, mp.cost_data, G);
      aniso_nudge_pass(vw, tid, T, mp.aniso_ws, G[0], G[1], G[2], (double2*)mp.aniso_nudge);
    }
    // F.F, F.v, v.v, max |F|^2: FP32 tissues sum their per-thread parts in
    // FP32 and combine warps in FP64 (FP64 issues slowly on this GPU)
    constexpr bool kF32 = std::is_same<R, float>::value;
    double red[4] = {0, 0, 0, 0};
    float redf[4] = {0, 0, 0, 0};
    auto vertex_tail = [&](int i, R fx, R fy) {
      if (nudged_v2v) {
        double gx, gy;
        v2v_grad(vw, i, mp.cost_data, gx, gy);
        fx -= (R)(mp.nudge_s * (gx - nmx));
        fy -= (R)(mp.nudge_s * (gy - nmy));
      }
      if (nudged_aniso) {
        const double2 g = ((const double2*)mp.aniso_nudge)[i];
        fx -= (R)(mp.nudge_s * g.x);
        fy -= (R)(mp.nudge_s * g.y);
      }
      R2 f;
      f.x = fx;
      f.y = fy;
      frc[i] = f;
      const R2 u = vel[i];
      if constexpr (kF32) {
        const float f2 = fx * fx + fy * fy;
        redf[0] += f2;
        redf[1] += fx * u.x + fy * u.y;
        redf[2] += u.x * u.x + u.y * u.y;
        redf[3] = fmaxf(redf[3], f2);
      } else {
        const double f2 = (double)(fx * fx + fy * fy);
        red[0] += f2;
        red[1] += (double)(fx * u.x + fy * u.y);
        red[2] += (double)(u.x * u.x + u.y * u.y);
        red[3] = fmax(red[3], f2);
      }
    };
    // two vertices per thread with both gathers in flight
    for (int i0 = tid; i0 < V; i0 += 2 * T) {
      const int i1 = i0 + T;
      VGather<P> g0, g1;
      vertex_gather(vw, i0, cell, lam, prm.lam_s, g0);
      if (i1 < V) vertex_gather(vw, i1, cell, lam, prm.lam_s, g1);
      R fx, fy;
      vertex_compute(vw, g0, fx, fy);
      vertex_tail(i0, fx, fy);
      if (i1 < V) {
        vertex_compute(vw, g1, fx, fy);
        vertex_tail(i1, fx, fy);
      }
    }
    if constexpr (kF32)
      tm.template reduce_f<4>(redf, red, sl.a, 1);
    else
      tm.template reduce<4>(red, sl.a, 1);
    fmx = kF32 ? (double)sqrtf((float)red[3]) : sqrt(red[3]);
    if (!(fmx == fmx) || isinf(fmx)) {
      status = VX_ERR_NONFINITE;
      break;
    }
    below = (fmx < mp.tol) ? below + 1 : 0;
    if (below >= mp.patience) {
      status = VX_OK;
      break;
    }
    if (it >= mp.max_iter) {
      status = VX_NOT_CONVERGED;
      break;
    }
    R mA = 0, mB = 0;
    bool zero = true;
    R dtR;
    if (mp.method == 1) {
      dtR = (R)mp.gd_lr;
    } else {
      if (red[1] > 0) {
        mA = (R)(1.0 - alpha);
        mB = (R)(alpha * sqrt(red[2]) / sqrt(red[0]));
        zero = false;
        if (npos > mp.n_min) {
          dt = fmin(dt * mp.f_inc, mp.dt_max);
          alpha *= mp.f_alpha;
        }
        ++npos;
      } else {
        dt *= mp.f_dec;
        alpha = mp.alpha0;
        npos = 0;
      }
      dtR = (R)dt;
    }
    for (int i = tid; i < V; i += T) {
      const R2 f = frc[i];
      if (mp.method == 1) {
        P::add(vw.X[i], dtR * f.x, dtR * f.y);
        continue;
      }
      R2 u = vel[i];
      R ux = zero ? (R)0 : mA * u.x + mB * f.x;
      R uy = zero ? (R)0 : mA * u.y + mB * f.y;
      ux += dtR * f.x;
      uy += dtR * f.y;
      u.x = ux;
      u.y = uy;
      vel[i] = u;
      P::add(vw.X[i], dtR * ux, dtR * uy);
    }
    __syncthreads();
  }
  __syncthreads();
  double fin[3] = {0, 0, 0};
  for (int c = tid; c < n; c += T) {
    R A, Pp;
    double el = 0;
    cell_geometry(vw, c, A, Pp, (R)0, shortbits, &el, &prm);
    const double dA = (double)A - prm.a0(c), dP = (double)Pp - prm.p0(c);
    fin[0] += prm.ka(c) * dA * dA + prm.kp(c) * dP * dP + el;
    fin[1] += (A <= 0) ? 1.0 : 0.0;
  }
  if (mp.l_min > 0)
    for (int e = tid; e < E; e += T) fin[2] += edge_len_d(vw, 2 * e) < mp.l_min ? 1.0 : 0.0;
  tm.template reduce<3>(fin, sl.c, 0);
  if (tid == 0 && out) {
    MinOut o;
    o.status = status;
    o.iters = it;
    o.n_t1 = n_t1;
    o.n_stretch = n_st;
    o.n_short = (int)fin[2];
    o.n_inverted = (int)fin[1];
    o.force_evals = it + 1;
    o.wrap_err = 0;
    o.fmax = fmx;
    o.energy = fin[0];
    *out = o;
  }
  if (Xout)
    for (int i = tid; i < V; i += T) {
      const double2 d = P::to_d(vw.X[i]);
      Xout[2 * i] = d.x;
      Xout[2 * i + 1] = d.y;
    }
}

// ------------------------------------------------- adjoint, memory state

// The implicit adjoint of adj_body for one CTA, with the CG vectors (x, r,
// p, z) and the inverse diagonal blocks in arrays instead of registers, so
// that one kernel serves tissues of any size (the batched path).  The right
// side grad_X C comes in dCdX; the same preconditioned CG, stop rule and
// parameter VJP as adj_body.
template <class P, int T, class LamT>
__device__ void adj_body_mem(View<P> vw, typename Vec2Of<typename P::R>::T4* cell4,
                             typename Vec2Of<typename P::R>::T* x,
                             typename Vec2Of<typename P::R>::T* r,
                             typename Vec2Of<typename P::R>::T* p,
                             typename Vec2Of<typename P::R>::T* z,
                             typename Vec2Of<typename P::R>::T4* pre, const LamT* lam, Slots sl,
                             const ParamsD& prm, const double* dCdX, double rtol, int max_iter,
                             const double* Xin, double* g_lam, double* g_A0, double* g_P0,
                             AdjOut* out) {
  using R = typename P::R;
  using R2 = typename Vec2Of<R>::T;
  using R4 = typename Vec2Of<R>::T4;
  BlockTeam<T> tm;
  const int n = vw.n, V = vw.V, E = vw.E, tid = threadIdx.x;
  if (Xin)
    for (int i = tid; i < V; i += T) vw.X[i] = P::from_d(Xin[2 * i], Xin[2 * i + 1]);
  tm.sync();
  for (int c = tid; c < n; c += T) {
    R A, Pp;
    cell_geometry(vw, c, A, Pp, (R)0, nullptr);
    R4 q;
    q.x = (R)(2.0 * prm.ka(c) * ((double)A - prm.a0(c)));
    q.y = (R)(2.0 * prm.kp(c) * ((double)Pp - prm.p0(c)));
    q.z = (R)(2.0 * prm.ka(c));
    q.w = (R)(2.0 * prm.kp(c));
    cell4[c] = q;
  }
  tm.sync();
  double s2[2] = {0, 0};
  for (int i = tid; i < V; i += T) {
    double dxx, dxy, dyy;
    vertex_diag(vw, i, cell4, lam, prm.lam_s, dxx, dxy, dyy);
    const double det = dxx * dyy - dxy * dxy;
    R4 q;
    if (dxx > 0 && det > 1e-300 * dxx * dxx) {
      q.x = (R)(dyy / det);
      q.y = (R)(-dxy / det);
      q.z = (R)(dxx / det);
    } else {
      const double tr = fabs(dxx) + fabs(dyy);
      q.x = q.z = (R)(tr > 0 ? 2.0 / tr : 1.0);
      q.y = 0;
    }
    q.w = 0;
    pre[i] = q;
    const double gx = dCdX[2 * i], gy = dCdX[2 * i + 1];
    R2 g;
    g.x = (R)gx;
    g.y = (R)gy;
    r[i] = g;
    s2[0] += gx;
    s2[1] += gy;
  }
  tm.template reduce<2>(s2, sl.a, 0);
  const R mx = (R)(s2[0] / V), my = (R)(s2[1] / V);
  double s2a[2] = {0, 0};  // r.z, r.r
  for (int i = tid; i < V; i += T) {
    R2 ri = r[i];
    ri.x -= mx;
    ri.y -= my;
    r[i] = ri;
    const R4 q = pre[i];
    R2 zi;
    zi.x = q.x * ri.x + q.y * ri.y;
    zi.y = q.y * ri.x + q.z * ri.y;
    p[i] = zi;
    R2 zero;
    zero.x = 0;
    zero.y = 0;
    x[i] = zero;
    s2a[0] += (double)(ri.x * zi.x + ri.y * zi.y);
    s2a[1] += (double)(ri.x * ri.x + ri.y * ri.y);
  }
  tm.template reduce<2>(s2a, sl.b, 0);
  double rz = s2a[0];
  const double bnorm = sqrt(s2a[1]);
  double rnorm = bnorm;
  int status = VX_NOT_CONVERGED, it = 0;
  if (bnorm == 0.0) status = VX_OK;
  tm.sync();
  for (it = 0; status == VX_NOT_CONVERGED && it < max_iter; ++it) {
    for (int c = tid; c < n; c += T) {
      R sA, sP;
      cell_dir(vw, c, p, sA, sP);
      R4 q = cell4[c];
      q.z = (R)(2.0 * prm.ka(c)) * sA;
      q.w = (R)(2.0 * prm.kp(c)) * sP;
      cell4[c] = q;
    }
    tm.sync();
    double s1[1] = {0};
    for (int i = tid; i < V; i += T) {
      R hx, hy;
      vertex_hvp(vw, i, cell4, lam, prm.lam_s, p, hx, hy);
      R2 h;
      h.x = hx;
      h.y = hy;
      z[i] = h;  // H p, until the update below replaces it by M r
      const R2 pi = p[i];
      s1[0] += (double)(pi.x * hx + pi.y * hy);
    }
    tm.template reduce<1>(s1, sl.a, 0);
    if (!(s1[0] > 0)) {
      status = VX_ERR_INDEFINITE;
      break;
    }
    const R al = (R)(rz / s1[0]);
    double s2b[2] = {0, 0};
    for (int i = tid; i < V; i += T) {
      const R2 pi = p[i], hi = z[i];
      R2 xi = x[i], ri = r[i];
      xi.x += al * pi.x;
      xi.y += al * pi.y;
      ri.x -= al * hi.x;
      ri.y -= al * hi.y;
      x[i] = xi;
      r[i] = ri;
      const R4 q = pre[i];
      R2 zi;
      zi.x = q.x * ri.x + q.y * ri.y;
      zi.y = q.y * ri.x + q.z * ri.y;
      z[i] = zi;
      s2b[0] += (double)(ri.x * zi.x + ri.y * zi.y);
      s2b[1] += (double)(ri.x * ri.x + ri.y * ri.y);
    }
    tm.template reduce<2>(s2b, sl.b, 0);
    rnorm = sqrt(s2b[1]);
    if (!(rnorm == rnorm)) {
      status = VX_ERR_NONFINITE;
      break;
    }
    if (rnorm <= rtol * bnorm) status = VX_OK;
    const R be = (R)(s2b[0] / rz);
    rz = s2b[0];
    if (status == VX_NOT_CONVERGED)
      for (int i = tid; i < V; i += T) {
        const R2 zi = z[i];
        R2 pi = p[i];
        pi.x = zi.x + be * pi.x;
        pi.y = zi.y + be * pi.y;
        p[i] = pi;
      }
    tm.sync();
  }
  tm.sync();
  // g = -(d^2E / dX dtheta)^T lambda with lambda = x.
  if (g_lam)
    for (int e = tid; e < E; e += T) {
      const int h = 2 * e;
      const uint32_t tg = vw.tgt[h];
      const int s = src_of(vw, h), t = tgt_v(tg);
      R dx, dy;
      P::diff(vw.X[t], vw.X[s], tgt_ox(tg), tgt_oy(tg), vw.box, dx, dy);
      const R il = P::rsqrt(dx * dx + dy * dy);
      const R2 lt = x[t], ls = x[s];
      g_lam[e] = -(double)((dx * (lt.x - ls.x) + dy * (lt.y - ls.y)) * il);
    }
  if (g_A0 || g_P0)
    for (int c = tid; c < n; c += T) {
      R sA, sP;
      cell_dir(vw, c, x, sA, sP);
      if (g_A0) g_A0[c] = 2.0 * prm.ka(c) * (double)sA;
      if (g_P0) g_P0[c] = 2.0 * prm.kp(c) * (double)sP;
    }
  if (tid == 0 && out) {
    AdjOut o;
    o.status = status;
    o.iters = it;
    o.rel_residual = bnorm > 0 ? rnorm / bnorm : 0.0;
    o.cost = 0.0;
    *out = o;
  }
}

}  // namespace vx
