// Energy, forces and the inner minimiser: global-memory kernels (one kernel
// per sub-step; the reference "plain" path) and the shared-memory-resident
// persistent minimiser (one CTA holds a whole tissue for the whole FIRE / GD
// loop; HBM is touched only at entry and exit).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <type_traits>

#include "device_math.cuh"
#include "t1.cuh"
#include "kernels.cuh"
#include "tissue.h"

namespace vx {

template <class R>
using R2T = typename std::conditional<std::is_same<R, double>::value, double2, float2>::type;

template <class R>
__device__ __forceinline__ R2T<R> mk2(R a, R b) {
  R2T<R> r;
  r.x = a;
  r.y = b;
  return r;
}

// ---------------------------------------------------------------- helpers

template <class P>
__global__ void k_load_X(const double* __restrict__ X, typename P::Pos* __restrict__ out, int V) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x)
    out[i] = P::from_d(X[2 * i], X[2 * i + 1]);
}

template <class P>
__global__ void k_store_X(const typename P::Pos* __restrict__ in, double* __restrict__ X, int V) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    const double2 d = P::to_d(in[i]);
    X[2 * i] = d.x;
    X[2 * i + 1] = d.y;
  }
}

// Block-wide deterministic sum of NV doubles (fixed tree for a given block
// size); the result is valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* smem) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) smem[w * NV + k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < NV; ++k) {
      double s = 0;
      for (int q = 0; q < nw; ++q) s += smem[q * NV + k];
      v[k] = s;
    }
  }
}

// ------------------------------------------------------- plain: cell pass

// Per cell: cA = 2 K_A (A - A0), cP = 2 K_P (P - P0); optional per-block
// energy partials (cell terms + 1/2 Lambda l per half-edge) and short-edge
// flags.
template <class P>
__global__ void k_cells(View<P> v, ParamsD prm, R2T<typename P::R>* __restrict__ cellc,
                        uint32_t* shortbits, double lmin, FireCtrl* ctrl, double* partE) {
  using R = typename P::R;
  __shared__ double red[32 * 3];
  if (ctrl && ctrl->done) return;
  double acc[3] = {0, 0, 0};  // energy, short half-edges, inverted cells
  bool flagged = false;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < v.n; c += gridDim.x * blockDim.x) {
    R A, Pp;
    double el = 0;
    flagged |= cell_geometry(v, c, A, Pp, (R)lmin, shortbits, partE ? &el : nullptr, &prm);
    const double dA = (double)A - prm.a0(c), dP = (double)Pp - prm.p0(c);
    cellc[c] = mk2<R>((R)(2.0 * prm.ka(c) * dA), (R)(2.0 * prm.kp(c) * dP));
    if (partE) {
      acc[0] += prm.ka(c) * dA * dA + prm.kp(c) * dP * dP + el;
      acc[2] += (A <= 0) ? 1.0 : 0.0;
    }
  }
  if (ctrl && lmin > 0) {
    if (__syncthreads_or(flagged) && threadIdx.x == 0) atomicOr(&ctrl->any_short, 1);
  }
  if (partE) {
    block_sum<3>(acc, red);
    if (threadIdx.x == 0) {
      partE[3 * blockIdx.x] = acc[0];
      partE[3 * blockIdx.x + 1] = acc[1];
      partE[3 * blockIdx.x + 2] = acc[2];
    }
  }
}

// Fixed-order sum of per-block energy partials.
__global__ void k_sum_energy(const double* partE, int nb, double* E, MinOut* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0, inv = 0;
  for (int b = 0; b < nb; ++b) {
    s += partE[3 * b];
    inv += partE[3 * b + 2];
  }
  if (E) *E = s;
  if (out) {
    out->energy = s;
    out->n_inverted = (int)inv;
  }
}

// ------------------------------------------------------- plain: T1 pass

template <class P>
__global__ void k_t1(View<P> v, ParamsD prm, double lmin, uint32_t* shortbits, uint32_t* touched,
                     R2T<typename P::R>* vel, R2T<typename P::R>* cellc, FireCtrl* ctrl,
                     int* events) {
  using R = typename P::R;
  constexpr int CAP = 512;
  __shared__ int dirty[CAP];
  __shared__ int n_dirty;
  if (ctrl->done || !ctrl->any_short) return;
  if (threadIdx.x == 0) n_dirty = 0;
  __syncthreads();
  {
    T1Stats st = {0, 0, 0};
    t1_pass_block(v, prm, lmin, shortbits, touched, &st, dirty, CAP, &n_dirty, events);
    if (threadIdx.x == 0) {
      ctrl->n_t1 += st.n_t1;
      ctrl->n_stretch += st.n_stretch;
      ctrl->any_short = 0;
    }
  }
  __syncthreads();
  const int nw = (v.V + 31) >> 5;
  for (int w = threadIdx.x; w < nw; w += blockDim.x) {
    uint32_t b = touched[w];
    touched[w] = 0;
    while (b) {
      const int i = (w << 5) + __ffs(b) - 1;
      b &= b - 1;
      if (vel) vel[i] = mk2<R>(0, 0);
    }
  }
  const bool all = n_dirty > CAP;
  const int m = all ? v.n : n_dirty;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const int c = all ? k : dirty[k];
    R A, Pp;
    cell_geometry(v, c, A, Pp, (R)0, shortbits);
    const double dA = (double)A - prm.a0(c), dP = (double)Pp - prm.p0(c);
    cellc[c] = mk2<R>((R)(2.0 * prm.ka(c) * dA), (R)(2.0 * prm.kp(c) * dP));
  }
}

// ---------------------------------------------------- plain: vertex pass

// Forces; with `ctrl`, also the FIRE reductions (F.F, F.v, v.v, max |F|^2)
// per block, and the last block to finish reduces them in block order and
// takes the FIRE / GD control decision for the step.
template <class P, class OutT>
__global__ void k_vertices(View<P> v, const R2T<typename P::R>* __restrict__ cellc,
                           const double* __restrict__ lam, double lam_s, OutT* __restrict__ F,
                           const R2T<typename P::R>* __restrict__ vel, FireCtrl* ctrl,
                           double* part, MinParams mp) {
  using R = typename P::R;
  __shared__ double red[32 * 4];
  __shared__ bool last;
  if (ctrl && ctrl->done) return;
  double acc[4] = {0, 0, 0, 0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < v.V; i += gridDim.x * blockDim.x) {
    R fx, fy;
    vertex_force(v, i, cellc, lam, lam_s, fx, fy);
    OutT o;
    o.x = fx;
    o.y = fy;
    F[i] = o;
    if (ctrl) {
      const R2T<R> vv = vel[i];
      acc[0] += (double)(fx * fx + fy * fy);
      acc[1] += (double)(fx * vv.x + fy * vv.y);
      acc[2] += (double)(vv.x * vv.x + vv.y * vv.y);
      acc[3] = fmax(acc[3], (double)(fx * fx + fy * fy));
    }
  }
  if (!ctrl) return;
  // max via a separate warp/block pass
  double mx = acc[3];
  acc[3] = 0;
  double s3[3] = {acc[0], acc[1], acc[2]};
  mx = warp_max(mx);
  {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[96 + w] = mx;
  }
  block_sum<3>(s3, red);
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    double m = 0;
    for (int q = 0; q < nw; ++q) m = fmax(m, red[96 + q]);
    part[4 * blockIdx.x] = s3[0];
    part[4 * blockIdx.x + 1] = s3[1];
    part[4 * blockIdx.x + 2] = s3[2];
    part[4 * blockIdx.x + 3] = m;
    __threadfence();
    const unsigned t = atomicAdd(&ctrl->counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  double FF = 0, Pw = 0, VV = 0, M = 0;
  for (unsigned b = 0; b < gridDim.x; ++b) {
    FF += part[4 * b];
    Pw += part[4 * b + 1];
    VV += part[4 * b + 2];
    M = fmax(M, part[4 * b + 3]);
  }
  ctrl->counter = 0;
  ctrl->FF = FF;
  ctrl->P = Pw;
  ctrl->VV = VV;
  ctrl->fmax2 = M;
  const double fmax = sqrt(M);
  if (!(fmax == fmax) || isinf(fmax)) {
    ctrl->done = 1;
    ctrl->status = VX_ERR_NONFINITE;
    return;
  }
  ctrl->below = (fmax < mp.tol) ? ctrl->below + 1 : 0;
  if (ctrl->below >= mp.patience) {
    ctrl->done = 1;
    ctrl->status = VX_OK;
    return;
  }
  if (ctrl->it >= mp.max_iter) {
    ctrl->done = 1;
    ctrl->status = VX_NOT_CONVERGED;
    return;
  }
  if (mp.method == 1) {  // gradient descent
    ctrl->mixA = 0;
    ctrl->mixB = 0;
    ctrl->zero_v = 1;
    ctrl->dt_step = mp.gd_lr;
  } else if (Pw > 0) {
    ctrl->mixA = 1.0 - ctrl->alpha;
    ctrl->mixB = ctrl->alpha * sqrt(VV) / sqrt(FF);
    ctrl->zero_v = 0;
    if (ctrl->npos > mp.n_min) {
      ctrl->dt = fmin(ctrl->dt * mp.f_inc, mp.dt_max);
      ctrl->alpha *= mp.f_alpha;
    }
    ctrl->npos++;
    ctrl->dt_step = ctrl->dt;
  } else {
    ctrl->mixA = 0;
    ctrl->mixB = 0;
    ctrl->zero_v = 1;
    ctrl->dt *= mp.f_dec;
    ctrl->alpha = mp.alpha0;
    ctrl->npos = 0;
    ctrl->dt_step = ctrl->dt;
  }
  ctrl->it++;
}

template <class P>
__global__ void k_update(View<P> v, R2T<typename P::R>* __restrict__ vel,
                         const R2T<typename P::R>* __restrict__ F, FireCtrl* ctrl, int method) {
  using R = typename P::R;
  if (ctrl->done) return;
  const R mA = (R)ctrl->mixA, mB = (R)ctrl->mixB, dt = (R)ctrl->dt_step;
  const bool zero = ctrl->zero_v;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < v.V; i += gridDim.x * blockDim.x) {
    const R2T<R> f = F[i];
    if (method == 1) {
      P::add(v.X[i], dt * f.x, dt * f.y);
      continue;
    }
    R2T<R> u = vel[i];
    if (zero) {
      u.x = 0;
      u.y = 0;
    } else {
      u.x = mA * u.x + mB * f.x;
      u.y = mA * u.y + mB * f.y;
    }
    u.x += dt * f.x;
    u.y += dt * f.y;
    vel[i] = u;
    P::add(v.X[i], dt * u.x, dt * u.y);
  }
}

template <class P>
__global__ void k_final_short(View<P> v, double lmin, int* out) {
  if (threadIdx.x || blockIdx.x) return;
  int c = 0;
  if (lmin > 0)
    for (int e = 0; e < v.E; ++e) c += edge_len_d(v, 2 * e) < lmin;
  *out = c;
}

// ------------------------------------------------------------- host side

static int grid_for(int items, int threads) {
  int b = (items + threads - 1) / threads;
  return b < 1 ? 1 : b;
}

template <class P>
static View<P> make_view(vx_tissue_s* t) {
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

template <class P>
__global__ void k_rebuild_flat(View<P> v) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
  for (int w = tid; w < v.V; w += st) rebuild_vertex(v, w);
  for (int c = tid; c < v.n; c += st) rebuild_cell(v, c);
}

cudaError_t rebuild_flat(vx_tissue_s* t, cudaStream_t s) {
  View<PolF64> v = make_view<PolF64>(t);
  const int th = 256, nb = (t->V + th - 1) / th;
  k_rebuild_flat<PolF64><<<nb, th, 0, s>>>(v);
  return cudaGetLastError();
}

// --------------------------------------------------- bulk evaluation

// Per cell: (cA, cP) and the cell part of the energy (block partials in
// partE[2b], inverted cells in partE[2b + 1]); two cells per thread with
// both gathers in flight.
template <class P>
__global__ void __launch_bounds__(256) k_ef_cells(View<P> v, ParamsD prm,
                                                  R2T<typename P::R>* __restrict__ cellc,
                                                  double* partE) {
  using R = typename P::R;
  __shared__ double red[32 * 2];
  // Arithmetic in R: A and P are R values, so their differences from the
  // targets lose nothing in R; uniform parameters are converted once (on
  // FP32 tissues every FP64 operation, conversions included, runs on this
  // GPU's narrow FP64 pipe).  Per-thread energy sums of a few positive
  // terms in R, the block and grid stages in FP64.
  const R ka_s = (R)prm.KA_s, kp_s = (R)prm.KP_s, a0_s = (R)prm.A0_s, p0_s = (R)prm.P0_s;
  R er = 0;
  int inv = 0;
  auto finish = [&](int c, R A, R Pp) {
    const R ka = prm.KA ? (R)prm.KA[c] : ka_s, kp = prm.KP ? (R)prm.KP[c] : kp_s;
    const R dA = A - (prm.A0 ? (R)prm.A0[c] : a0_s), dP = Pp - (prm.P0 ? (R)prm.P0[c] : p0_s);
    cellc[c] = mk2<R>((R)2 * ka * dA, (R)2 * kp * dP);
    er += ka * dA * dA + kp * dP * dP;
    inv += (A <= 0) ? 1 : 0;
  };
  const int st = gridDim.x * blockDim.x;
  for (int c0 = blockIdx.x * blockDim.x + threadIdx.x; c0 < v.n; c0 += 2 * st) {
    const int c1 = c0 + st;
    R A, Pp;
    if (v.ccor) {
      CGather<P> g0, g1;
      cell_gather(v, c0, g0);
      if (c1 < v.n) cell_gather(v, c1, g1);
      cell_geometry_g(v, c0, g0, A, Pp, (R)0, (uint32_t*)nullptr);
      finish(c0, A, Pp);
      if (c1 < v.n) {
        cell_geometry_g(v, c1, g1, A, Pp, (R)0, (uint32_t*)nullptr);
        finish(c1, A, Pp);
      }
    } else {
      cell_geometry(v, c0, A, Pp, (R)0, (uint32_t*)nullptr);
      finish(c0, A, Pp);
      if (c1 < v.n) {
        cell_geometry(v, c1, A, Pp, (R)0, (uint32_t*)nullptr);
        finish(c1, A, Pp);
      }
    }
  }
  if (partE) {
    double acc[2] = {(double)er, (double)inv};
    block_sum<2>(acc, red);
    if (threadIdx.x == 0) {
      partE[2 * blockIdx.x] = acc[0];
      partE[2 * blockIdx.x + 1] = acc[1];
    }
  }
}

// Per vertex: F, and the line energy of its out-half-edges, 1/2 Lambda_e l_e
// each (every edge has one out-half-edge at each end), as block partials in
// partL[b]; two vertices per thread with both gathers in flight.
template <class P, class LamT>
__global__ void __launch_bounds__(256) k_ef_vertices(View<P> v,
                                                     const R2T<typename P::R>* __restrict__ cellc,
                                                     const LamT* __restrict__ lam, double lam_s,
                                                     double2* __restrict__ F, double* partL) {
  using R = typename P::R;
  __shared__ double red[32];
  // per-thread sums of positive terms in R (a handful per thread), the
  // block and grid stages in FP64
  R elr = 0;
  auto one = [&](int i, const VGather<P>& g) {
    R fx, fy;
    vertex_compute(v, g, fx, fy);
    if (F) F[i] = make_double2((double)fx, (double)fy);
    if (partL) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        R dx, dy;
        P::diff(g.Xj[a], g.Xi, tgt_ox(g.tg[a]), tgt_oy(g.tg[a]), v.box, dx, dy);
        elr += (R)0.5 * g.la[a] * sqrt(dx * dx + dy * dy);
      }
    }
  };
  const int st = gridDim.x * blockDim.x;
  for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < v.V; i0 += 2 * st) {
    const int i1 = i0 + st;
    VGather<P> g0, g1;
    vertex_gather(v, i0, cellc, lam, lam_s, g0);
    if (i1 < v.V) vertex_gather(v, i1, cellc, lam, lam_s, g1);
    one(i0, g0);
    if (i1 < v.V) one(i1, g1);
  }
  if (partL) {
    double el[1] = {(double)elr};
    block_sum<1>(el, red);
    if (threadIdx.x == 0) partL[blockIdx.x] = el[0];
  }
}

// E = cell partials + line partials: one block of 256 threads, each summing
// a fixed strided subset, then a fixed tree (deterministic).
__global__ void k_ef_sum(const double* partE, int nbc, const double* partL, int nbv, double* E) {
  __shared__ double red[32];
  double s[1] = {0};
  for (int b = threadIdx.x; b < nbc; b += blockDim.x) s[0] += partE[2 * b];
  for (int b = threadIdx.x; b < nbv; b += blockDim.x) s[0] += partL[b];
  block_sum<1>(s, red);
  if (threadIdx.x == 0) *E = s[0];
}

// Energy and forces of one tissue: the positions converted once into the
// tissue's precision (hi/lo pairs on FP32 tissues: FP64 arithmetic, slow on
// this GPU, is then needed per vertex only, not per edge), then one
// gathered pass per cell and one per vertex.
template <class P>
static vx_status energy_forces_impl(vx_tissue_s* t, const double* X, const ParamsD& prm,
                                    double* F, double* E, cudaStream_t s) {
  using R = typename P::R;
  const int th = 256;
  View<P> v = make_view<P>(t);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int gc = std::min(grid_for(t->n, 2 * th), 8 * sms);
  const int gv = std::min(grid_for(t->V, 2 * th), 8 * sms);
  double* partL = t->partE + 2 * (size_t)gc;   // fits: 2 gc + gv <= 3 ((n + 255) / 256 + 1)
  k_load_X<P><<<std::min(grid_for(t->V, th), 8 * sms), th, 0, s>>>(X, v.X, t->V);
  k_ef_cells<P><<<gc, th, 0, s>>>(v, prm, (R2T<R>*)t->cellc, E ? t->partE : nullptr);
  k_ef_vertices<P, double><<<gv, th, 0, s>>>(v, (const R2T<R>*)t->cellc, prm.lam, prm.lam_s,
                                             (double2*)F, E ? partL : nullptr);
  if (E) k_ef_sum<<<1, 256, 0, s>>>(t->partE, gc, partL, gv, E);
  return cudaGetLastError() == cudaSuccess ? VX_OK : VX_ERR_CUDA;
}

vx_status energy_forces(vx_tissue_s* t, const double* X, const ParamsD& prm, double* F, double* E,
                        cudaStream_t s) {
  return t->dtype == VX_F64 ? energy_forces_impl<PolF64>(t, X, prm, F, E, s)
                            : energy_forces_impl<PolF32>(t, X, prm, F, E, s);
}

// Plain path: one kernel per sub-step, convergence polled every k steps.
template <class P>
static vx_status minimize_plain(vx_tissue_s* t, double* X, const ParamsD& prm, const MinParams& mp,
                                int check_every, MinOut* out_h, cudaStream_t s) {
  using R = typename P::R;
  View<P> v = make_view<P>(t);
  const int th = 256;
  k_load_X<P><<<grid_for(t->V, th), th, 0, s>>>(X, v.X, t->V);
  cudaMemsetAsync(t->vel, 0, 2 * sizeof(R) * t->V, s);
  cudaMemsetAsync(t->shortbits, 0, sizeof(uint32_t) * ((t->E + 31) / 32), s);
  cudaMemsetAsync(t->touched, 0, sizeof(uint32_t) * ((t->V + 31) / 32), s);
  FireCtrl c0 = {};
  c0.dt = mp.dt0;
  c0.alpha = mp.alpha0;
  c0.status = VX_NOT_CONVERGED;
  cudaMemcpyAsync(t->ctrl, &c0, sizeof(FireCtrl), cudaMemcpyHostToDevice, s);
  const int nbc = grid_for(t->n, th), nbv = grid_for(t->V, th);
  R2T<R>* cellc = (R2T<R>*)t->cellc;
  R2T<R>* vel = (R2T<R>*)t->vel;
  R2T<R>* F = (R2T<R>*)t->F;
  FireCtrl ch;
  const int k = check_every > 0 ? check_every : 50;
  for (int it = 0; it <= mp.max_iter; ++it) {
    k_cells<P><<<nbc, th, 0, s>>>(v, prm, cellc, t->shortbits, mp.l_min, t->ctrl, nullptr);
    if (mp.l_min > 0)
      k_t1<P><<<1, 256, 0, s>>>(v, prm, mp.l_min, t->shortbits, t->touched, vel, cellc, t->ctrl,
                                mp.edge_events);
    k_vertices<P, R2T<R>><<<nbv, th, 0, s>>>(v, cellc, prm.lam, prm.lam_s, F, vel, t->ctrl,
                                             t->partF, mp);
    k_update<P><<<nbv, th, 0, s>>>(v, vel, F, t->ctrl, mp.method);
    if ((it + 1) % k == 0 || it == mp.max_iter) {
      cudaMemcpyAsync(&ch, t->ctrl, sizeof(FireCtrl), cudaMemcpyDeviceToHost, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) return VX_ERR_CUDA;
      if (ch.done) break;
    }
  }
  cudaMemcpyAsync(&ch, t->ctrl, sizeof(FireCtrl), cudaMemcpyDeviceToHost, s);
  // final energy and counts
  k_cells<P><<<nbc, th, 0, s>>>(v, prm, cellc, t->shortbits, 0.0, nullptr, t->partE);
  k_sum_energy<<<1, 32, 0, s>>>(t->partE, nbc, nullptr, t->dout);
  k_final_short<P><<<1, 32, 0, s>>>(v, mp.l_min, &t->dout->n_short);
  k_store_X<P><<<grid_for(t->V, th), th, 0, s>>>(v.X, X, t->V);
  if (mp.wrap && wrap_tissue(t, X, &t->dout->wrap_err, s) != VX_OK) return VX_ERR_CUDA;
  MinOut o;
  cudaMemcpyAsync(&o, t->dout, sizeof(MinOut), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return VX_ERR_CUDA;
  o.status = ch.status;
  o.iters = ch.it;
  o.n_t1 = ch.n_t1;
  o.n_stretch = ch.n_stretch;
  o.fmax = sqrt(ch.fmax2);
  o.force_evals = ch.it + 1;
  if (!mp.wrap) o.wrap_err = 0;
  *out_h = o;
  return VX_OK;
}

template <class P>
vx_status minimize_plain_t(vx_tissue_s* t, double* X, const ParamsD& prm, const MinParams& mp,
                           int check_every, MinOut* out_h, cudaStream_t s) {
  return minimize_plain<P>(t, X, prm, mp, check_every, out_h, s);
}
template vx_status minimize_plain_t<PolF64>(vx_tissue_s*, double*, const ParamsD&,
                                            const MinParams&, int, MinOut*, cudaStream_t);
template vx_status minimize_plain_t<PolF32>(vx_tissue_s*, double*, const ParamsD&,
                                            const MinParams&, int, MinOut*, cudaStream_t);

}  // namespace vx
