// Energy, forces and the inner minimiser: global-memory kernels (one kernel
// per sub-step; the reference "plain" path) and the shared-memory-resident
// persistent minimiser (one CTA holds a whole tissue for the whole FIRE / GD
// loop; HBM is touched only at entry and exit).
#include <cuda_runtime.h>

#include <cstdio>
#include <type_traits>

#include "device_math.cuh"
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
                     R2T<typename P::R>* vel, R2T<typename P::R>* cellc, FireCtrl* ctrl) {
  using R = typename P::R;
  constexpr int CAP = 512;
  __shared__ int dirty[CAP];
  __shared__ int n_dirty;
  if (ctrl->done || !ctrl->any_short) return;
  if (threadIdx.x == 0) {
    n_dirty = 0;
    T1Stats st = {0, 0, 0};
    t1_pass(v, prm, lmin, shortbits, touched, &st, dirty, CAP, &n_dirty);
    ctrl->n_t1 += st.n_t1;
    ctrl->n_stretch += st.n_stretch;
    ctrl->any_short = 0;
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

// --------------------------------------------------- resident minimiser

struct ResidentArgs {
  const double* Xin;
  double* Xout;
  int n, V, E, HE;
  double Lx, Ly;
  // global topology (read at entry, written back at exit)
  uint32_t* tgt;
  int32_t *nxt, *face, *vout, *ffirst;
  ParamsD prm;
  MinParams mp;
  MinOut* out;
};

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

template <class P>
__host__ __device__ inline size_t resident_bytes(int n, int V, int E, int HE, int nthreads) {
  using R = typename P::R;
  size_t b = 0;
  b += align16(sizeof(typename P::Pos) * V);
  b += align16(sizeof(uint32_t) * HE);
  b += align16(sizeof(int32_t) * HE);
  b += align16(sizeof(int32_t) * HE);
  b += align16(sizeof(int32_t) * 3 * V);
  b += align16(sizeof(int32_t) * n);
  b += align16(2 * sizeof(R) * n);
  b += align16(sizeof(R) * E);
  b += align16(sizeof(uint32_t) * ((E + 31) / 32));
  b += align16(sizeof(uint32_t) * ((V + 31) / 32));
  b += align16(sizeof(double) * 8 * ((nthreads + 31) / 32));
  return b;
}

template <class P, int T, int MAXC>
__global__ void __launch_bounds__(T) k_min_resident(ResidentArgs g) {
  using R = typename P::R;
  using Pos = typename P::Pos;
  using R2 = R2T<R>;
  constexpr int MAXV = 2 * MAXC;
  constexpr int NW = T / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = g.n, V = g.V, E = g.E, HE = g.HE;
  unsigned char* p = smem;
  Pos* sX = (Pos*)p;            p += align16(sizeof(Pos) * V);
  uint32_t* sTgt = (uint32_t*)p; p += align16(sizeof(uint32_t) * HE);
  int32_t* sNxt = (int32_t*)p;   p += align16(sizeof(int32_t) * HE);
  int32_t* sFace = (int32_t*)p;  p += align16(sizeof(int32_t) * HE);
  int32_t* sVout = (int32_t*)p;  p += align16(sizeof(int32_t) * 3 * V);
  int32_t* sFf = (int32_t*)p;    p += align16(sizeof(int32_t) * n);
  R2* sCell = (R2*)p;            p += align16(2 * sizeof(R) * n);
  R* sLam = (R*)p;               p += align16(sizeof(R) * E);
  uint32_t* sShort = (uint32_t*)p; p += align16(sizeof(uint32_t) * ((E + 31) / 32));
  uint32_t* sTouch = (uint32_t*)p; p += align16(sizeof(uint32_t) * ((V + 31) / 32));
  double* sRed = (double*)p;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

  for (int i = tid; i < V; i += T) sX[i] = P::from_d(g.Xin[2 * i], g.Xin[2 * i + 1]);
  for (int h = tid; h < HE; h += T) {
    sTgt[h] = g.tgt[h];
    sNxt[h] = g.nxt[h];
    sFace[h] = g.face[h];
  }
  for (int k = tid; k < 3 * V; k += T) sVout[k] = g.vout[k];
  for (int c = tid; c < n; c += T) sFf[c] = g.ffirst[c];
  for (int e = tid; e < E; e += T) sLam[e] = (R)g.prm.la(e);
  for (int w = tid; w < (E + 31) / 32; w += T) sShort[w] = 0;
  for (int w = tid; w < (V + 31) / 32; w += T) sTouch[w] = 0;

  View<P> vw;
  vw.X = sX;
  vw.tgt = sTgt;
  vw.nxt = sNxt;
  vw.face = sFace;
  vw.vout = sVout;
  vw.ffirst = sFf;
  vw.n = n;
  vw.V = V;
  vw.E = E;
  vw.box = P::make_box(g.Lx, g.Ly);
  vw.Lx = g.Lx;
  vw.Ly = g.Ly;

  R ka[MAXC], kp[MAXC], a0[MAXC], p0[MAXC];
#pragma unroll
  for (int k = 0; k < MAXC; ++k) {
    const int c = tid + k * T;
    const int cc = c < n ? c : 0;
    ka[k] = (R)g.prm.ka(cc);
    kp[k] = (R)g.prm.kp(cc);
    a0[k] = (R)g.prm.a0(cc);
    p0[k] = (R)g.prm.p0(cc);
  }
  R vx[MAXV], vy[MAXV], fx[MAXV], fy[MAXV];
#pragma unroll
  for (int k = 0; k < MAXV; ++k) vx[k] = vy[k] = fx[k] = fy[k] = 0;

  const MinParams& mp = g.mp;
  const R lminR = (R)mp.l_min;
  double dt = mp.dt0, alpha = mp.alpha0;
  int npos = 0, below = 0, it = 0, status = VX_NOT_CONVERGED, n_t1 = 0, n_st = 0;
  double fmx = 0;
  __syncthreads();

  auto cell_pass = [&](R lm) -> bool {
    bool fl = false;
#pragma unroll
    for (int k = 0; k < MAXC; ++k) {
      const int c = tid + k * T;
      if (c < n) {
        R A, Pp;
        fl |= cell_geometry(vw, c, A, Pp, lm, sShort);
        sCell[c] = mk2<R>((R)2 * ka[k] * (A - a0[k]), (R)2 * kp[k] * (Pp - p0[k]));
      }
    }
    return fl;
  };

  for (it = 0;; ++it) {
    const bool fl = cell_pass(lminR);
    if (mp.l_min > 0) {
      if (__syncthreads_or(fl)) {
        if (tid == 0) {
          T1Stats st = {0, 0, 0};
          int nd = 0;
          t1_pass(vw, g.prm, mp.l_min, sShort, sTouch, &st, nullptr, 0, &nd);
          n_t1 += st.n_t1;
          n_st += st.n_stretch;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < MAXV; ++k) {
          const int i = tid + k * T;
          if (i < V && (sTouch[i >> 5] >> (i & 31)) & 1u) vx[k] = vy[k] = 0;
        }
        __syncthreads();
        for (int w = tid; w < (V + 31) / 32; w += T) sTouch[w] = 0;
        cell_pass((R)0);
        __syncthreads();
      }
    } else {
      __syncthreads();
    }
    // Vertex pass and FIRE reductions.
    double ff = 0, pv = 0, vv = 0, m2 = 0;
#pragma unroll
    for (int k = 0; k < MAXV; ++k) {
      const int i = tid + k * T;
      if (i < V) {
        vertex_force(vw, i, sCell, sLam, 0.0, fx[k], fy[k]);
        ff += (double)(fx[k] * fx[k] + fy[k] * fy[k]);
        pv += (double)(fx[k] * vx[k] + fy[k] * vy[k]);
        vv += (double)(vx[k] * vx[k] + vy[k] * vy[k]);
        m2 = fmax(m2, (double)(fx[k] * fx[k] + fy[k] * fy[k]));
      }
    }
    ff = warp_sum(ff);
    pv = warp_sum(pv);
    vv = warp_sum(vv);
    m2 = warp_max(m2);
    if (lane == 0) {
      sRed[4 * wid] = ff;
      sRed[4 * wid + 1] = pv;
      sRed[4 * wid + 2] = vv;
      sRed[4 * wid + 3] = m2;
    }
    __syncthreads();
    double FF = 0, PW = 0, VVs = 0, M = 0;
#pragma unroll 4
    for (int q = 0; q < NW; ++q) {
      FF += sRed[4 * q];
      PW += sRed[4 * q + 1];
      VVs += sRed[4 * q + 2];
      M = fmax(M, sRed[4 * q + 3]);
    }
    fmx = sqrt(M);
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
    if (mp.method == 1) {
      const R s = (R)mp.gd_lr;
#pragma unroll
      for (int k = 0; k < MAXV; ++k) {
        const int i = tid + k * T;
        if (i < V) P::add(sX[i], s * fx[k], s * fy[k]);
      }
    } else {
      R mA = 0, mB = 0;
      bool zero;
      if (PW > 0) {
        mA = (R)(1.0 - alpha);
        mB = (R)(alpha * sqrt(VVs) / sqrt(FF));
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
#pragma unroll
      for (int k = 0; k < MAXV; ++k) {
        const int i = tid + k * T;
        if (i < V) {
          R ux = zero ? (R)0 : mA * vx[k] + mB * fx[k];
          R uy = zero ? (R)0 : mA * vy[k] + mB * fy[k];
          ux += dtR * fx[k];
          uy += dtR * fy[k];
          vx[k] = ux;
          vy[k] = uy;
          P::add(sX[i], dtR * ux, dtR * uy);
        }
      }
    }
    __syncthreads();
  }
  __syncthreads();

  // Final energy, inverted cells and short edges at the returned X.
  double en = 0, inv = 0;
#pragma unroll
  for (int k = 0; k < MAXC; ++k) {
    const int c = tid + k * T;
    if (c < n) {
      R A, Pp;
      double el = 0;
      cell_geometry(vw, c, A, Pp, (R)0, sShort, &el, &g.prm);
      const double dA = (double)A - g.prm.a0(c), dP = (double)Pp - g.prm.p0(c);
      en += g.prm.ka(c) * dA * dA + g.prm.kp(c) * dP * dP + el;
      inv += (A <= 0) ? 1.0 : 0.0;
    }
  }
  double nsh = 0;
  if (mp.l_min > 0)
    for (int e = tid; e < E; e += T) nsh += edge_len_d(vw, 2 * e) < mp.l_min ? 1.0 : 0.0;
  en = warp_sum(en);
  inv = warp_sum(inv);
  nsh = warp_sum(nsh);
  if (lane == 0) {
    sRed[4 * wid] = en;
    sRed[4 * wid + 1] = inv;
    sRed[4 * wid + 2] = nsh;
  }
  __syncthreads();
  if (tid == 0) {
    double E0 = 0, I0 = 0, S0 = 0;
    for (int q = 0; q < NW; ++q) {
      E0 += sRed[4 * q];
      I0 += sRed[4 * q + 1];
      S0 += sRed[4 * q + 2];
    }
    MinOut o;
    o.status = status;
    o.iters = it;
    o.n_t1 = n_t1;
    o.n_stretch = n_st;
    o.n_short = (int)S0;
    o.n_inverted = (int)I0;
    o.force_evals = it + 1;
    o.pad = 0;
    o.fmax = fmx;
    o.energy = E0;
    *g.out = o;
  }
  for (int i = tid; i < V; i += T) {
    const double2 d = P::to_d(sX[i]);
    g.Xout[2 * i] = d.x;
    g.Xout[2 * i + 1] = d.y;
  }
  for (int h = tid; h < HE; h += T) {
    g.tgt[h] = sTgt[h];
    g.nxt[h] = sNxt[h];
    g.face[h] = sFace[h];
  }
  for (int k = tid; k < 3 * V; k += T) g.vout[k] = sVout[k];
  for (int c = tid; c < n; c += T) g.ffirst[c] = sFf[c];
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
  return v;
}

template <class P>
static vx_status energy_forces_impl(vx_tissue_s* t, const double* X, const ParamsD& prm,
                                    double* F, double* E, cudaStream_t s) {
  using R = typename P::R;
  View<P> v = make_view<P>(t);
  const int th = 256;
  k_load_X<P><<<grid_for(t->V, th), th, 0, s>>>(X, v.X, t->V);
  const int nbc = grid_for(t->n, th);
  k_cells<P><<<nbc, th, 0, s>>>(v, prm, (R2T<R>*)t->cellc, t->shortbits, 0.0, nullptr,
                                E ? t->partE : nullptr);
  if (F) {
    MinParams mp = {};
    k_vertices<P, double2><<<grid_for(t->V, th), th, 0, s>>>(
        v, (const R2T<R>*)t->cellc, prm.lam, prm.lam_s, (double2*)F, nullptr, nullptr, nullptr, mp);
  }
  if (E) k_sum_energy<<<1, 32, 0, s>>>(t->partE, nbc, E, nullptr);
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
      k_t1<P><<<1, 256, 0, s>>>(v, prm, mp.l_min, t->shortbits, t->touched, vel, cellc, t->ctrl);
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
  MinOut o;
  cudaMemcpyAsync(&o, t->dout, sizeof(MinOut), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return VX_ERR_CUDA;
  o.status = ch.status;
  o.iters = ch.it;
  o.n_t1 = ch.n_t1;
  o.n_stretch = ch.n_stretch;
  o.fmax = sqrt(ch.fmax2);
  o.force_evals = ch.it + 1;
  *out_h = o;
  return VX_OK;
}

template <class P, int T, int MAXC>
static vx_status launch_resident(vx_tissue_s* t, double* X, const ParamsD& prm, const MinParams& mp,
                                 MinOut* out_h, cudaStream_t s) {
  const size_t smem = resident_bytes<P>(t->n, t->V, t->E, t->HE, T);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_min_resident<P, T, MAXC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024);
    attr_set = true;
  }
  ResidentArgs a;
  a.Xin = X;
  a.Xout = X;
  a.n = t->n;
  a.V = t->V;
  a.E = t->E;
  a.HE = t->HE;
  a.Lx = t->Lx;
  a.Ly = t->Ly;
  a.tgt = t->tgt;
  a.nxt = t->nxt;
  a.face = t->face;
  a.vout = t->vout;
  a.ffirst = t->ffirst;
  a.prm = prm;
  a.mp = mp;
  a.out = t->dout;
  k_min_resident<P, T, MAXC><<<1, T, smem, s>>>(a);
  if (cudaGetLastError() != cudaSuccess) return VX_ERR_CUDA;
  if (cudaMemcpyAsync(out_h, t->dout, sizeof(MinOut), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return VX_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return VX_ERR_CUDA;
  return VX_OK;
}

template <class P>
static bool resident_fits(vx_tissue_s* t, int T) {
  return resident_bytes<P>(t->n, t->V, t->E, t->HE, T) <= 227 * 1024;
}

template <class P>
static vx_status minimize_resident(vx_tissue_s* t, double* X, const ParamsD& prm,
                                   const MinParams& mp, MinOut* out, cudaStream_t s) {
  // threads per CTA: enough for one cell per thread up to 1024, then 2 / 4
  const int n = t->n;
  if (n <= 128) return launch_resident<P, 128, 1>(t, X, prm, mp, out, s);
  if (n <= 256) return launch_resident<P, 256, 1>(t, X, prm, mp, out, s);
  if (n <= 512) return launch_resident<P, 512, 1>(t, X, prm, mp, out, s);
  if (n <= 1024) return launch_resident<P, 1024, 1>(t, X, prm, mp, out, s);
  if (n <= 2048) return launch_resident<P, 1024, 2>(t, X, prm, mp, out, s);
  return launch_resident<P, 1024, 4>(t, X, prm, mp, out, s);
}

vx_status minimize(vx_tissue_s* t, double* X, const ParamsD& prm, const MinParams& mp, int path,
                   int check_every, MinOut* out, int* path_used, cudaStream_t s) {
  const bool f64 = t->dtype == VX_F64;
  const bool fits = f64 ? resident_fits<PolF64>(t, 1024) : resident_fits<PolF32>(t, 1024);
  if (path == VX_PATH_RESIDENT && !fits) return VX_ERR_INVALID_ARG;
  const bool use_res = (path == VX_PATH_RESIDENT) || (path == VX_PATH_AUTO && fits);
  *path_used = use_res ? VX_PATH_RESIDENT : VX_PATH_PLAIN;
  if (use_res)
    return f64 ? minimize_resident<PolF64>(t, X, prm, mp, out, s)
               : minimize_resident<PolF32>(t, X, prm, mp, out, s);
  return f64 ? minimize_plain<PolF64>(t, X, prm, mp, check_every, out, s)
             : minimize_plain<PolF32>(t, X, prm, mp, check_every, out, s);
}

size_t resident_smem_bytes(vx_tissue_s* t) {
  return t->dtype == VX_F64 ? resident_bytes<PolF64>(t->n, t->V, t->E, t->HE, 1024)
                            : resident_bytes<PolF32>(t->n, t->V, t->E, t->HE, 1024);
}

}  // namespace vx
