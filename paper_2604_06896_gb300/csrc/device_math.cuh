// Device-side arithmetic of the periodic vertex model, shared by the
// shared-memory-resident persistent kernels and the global-memory kernels.
//
// Geometry (Methods, "Vertex model formulation", "Periodic mode"):
//   a half-edge h runs from X[src] to X[tgt] + (offx Lx, offy Ly);
//   A_c = 1/2 sum cross(q_k, q_{k+1}) over the corners of cell c in a frame
//   local to the cell's first corner, P_c = sum |q_{k+1} - q_k|;
//   E = sum_c K_A (A - A0)^2 + K_P (P - P0)^2 + sum_e Lambda_e l_e.
// Forces on a 3-valent vertex i with outgoing half-edges h_0, h_1, h_2
// (counter-clockwise; cell c_a lies between h_a and h_{a+1}; edge a is shared
// by c_a and c_{a-1}), d_a the edge vector and u_a = d_a / l_a:
//   F_i = sum_a (Lambda_a + cP_{c_a} + cP_{c_{a-1}}) u_a
//         - 1/2 sum_a cA_{c_a} rot(d_a - d_{a+1}),   rot(x, y) = (y, -x),
// with cA = 2 K_A (A - A0) and cP = 2 K_P (P - P0) per cell.
//
// Internal half-edge numbering: edge e owns half-edges 2e and 2e + 1 (twin =
// h ^ 1), 2e being the one with the smaller index in the caller's table.
#pragma once
#include <type_traits>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace vx {

constexpr uint32_t kTgtMask = (1u << 28) - 1;

__host__ __device__ inline uint32_t pack_tgt(int v, int ox, int oy) {
  return (uint32_t)v | ((uint32_t)(ox + 1) << 28) | ((uint32_t)(oy + 1) << 30);
}
__host__ __device__ inline int tgt_v(uint32_t t) { return (int)(t & kTgtMask); }
__host__ __device__ inline int tgt_ox(uint32_t t) { return (int)((t >> 28) & 3u) - 1; }
__host__ __device__ inline int tgt_oy(uint32_t t) { return (int)((t >> 30) & 3u) - 1; }

// ------------------------------------------------------------ precisions

// Error of s = fl(a + b) (Knuth's TwoSum; exact in round-to-nearest).
__device__ __forceinline__ float two_sum_err(float a, float b, float s) {
  const float bb = __fsub_rn(s, a);
  return __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

struct PolF64 {
  using R = double;
  using Pos = double2;
  struct Box { double Lx, Ly; };
  static __host__ __device__ Box make_box(double Lx, double Ly) { return Box{Lx, Ly}; }
  static __device__ __forceinline__ void diff(const Pos& t, const Pos& s, int ox, int oy,
                                              const Box& b, R& dx, R& dy) {
    dx = (t.x + ox * b.Lx) - s.x;
    dy = (t.y + oy * b.Ly) - s.y;
  }
  static __device__ __forceinline__ void add(Pos& p, R dx, R dy) {
    p.x += dx;
    p.y += dy;
  }
  static __device__ __forceinline__ double2 to_d(const Pos& p) { return p; }
  static __device__ __forceinline__ Pos from_d(double x, double y) { return make_double2(x, y); }
  static __device__ __forceinline__ R rsqrt(R x) { return 1.0 / sqrt(x); }
};

// FP32 arithmetic on positions held as unevaluated hi + lo float pairs, so
// that differences of nearby vertices keep ~48 bits and the force tolerance is
// not limited by the absolute-coordinate quantum of one float.
struct PolF32 {
  using R = float;
  using Pos = float4;  // (hi.x, hi.y, lo.x, lo.y)
  struct Box { float Lxh, Lxl, Lyh, Lyl; };
  static __host__ __device__ Box make_box(double Lx, double Ly) {
    Box b;
    b.Lxh = (float)Lx;
    b.Lxl = (float)(Lx - (double)b.Lxh);
    b.Lyh = (float)Ly;
    b.Lyl = (float)(Ly - (double)b.Lyh);
    return b;
  }
  // A small integer as a float without a conversion instruction (those run
  // on the narrow FP64 pipe of this GPU): 1.5 * 2^23 + o is exact in a float
  // for |o| < 2^22 and its bit pattern is 0x4B400000 + o; subtracting
  // 1.5 * 2^23 leaves o exactly.
  static __device__ __forceinline__ float small_int(int o) {
    return __fsub_rn(__int_as_float(0x4B400000 + o), 12582912.0f);
  }
  // a_hi + a_lo - b_hi - b_lo + o (Lh + Ll), rounded once at the end.
  static __device__ __forceinline__ float dd(float ah, float al, float bh, float bl, int o,
                                             float Lh, float Ll) {
    const float s = __fsub_rn(ah, bh);
    const float e = two_sum_err(ah, -bh, s);
    const float of = small_int(o);
    const float oL = of * Lh;                  // exact: o in {-2..2}
    const float t = __fadd_rn(s, oL);
    const float e2 = two_sum_err(s, oL, t);
    return __fadd_rn(t, __fadd_rn(__fadd_rn(e, e2), __fadd_rn(__fsub_rn(al, bl), of * Ll)));
  }
  static __device__ __forceinline__ void diff(const Pos& t, const Pos& s, int ox, int oy,
                                              const Box& b, R& dx, R& dy) {
    dx = dd(t.x, t.z, s.x, s.z, ox, b.Lxh, b.Lxl);
    dy = dd(t.y, t.w, s.y, s.w, oy, b.Lyh, b.Lyl);
  }
  static __device__ __forceinline__ void add1(float& hi, float& lo, float d) {
    const float s = __fadd_rn(hi, d);
    const float e = two_sum_err(hi, d, s);
    const float l = __fadd_rn(lo, e);
    const float h2 = __fadd_rn(s, l);
    lo = __fsub_rn(l, __fsub_rn(h2, s));
    hi = h2;
  }
  static __device__ __forceinline__ void add(Pos& p, R dx, R dy) {
    add1(p.x, p.z, dx);
    add1(p.y, p.w, dy);
  }
  static __device__ __forceinline__ double2 to_d(const Pos& p) {
    return make_double2((double)p.x + (double)p.z, (double)p.y + (double)p.w);
  }
  static __device__ __forceinline__ Pos from_d(double x, double y) {
    const float hx = (float)x, hy = (float)y;
    return make_float4(hx, hy, (float)(x - (double)hx), (float)(y - (double)hy));
  }
  static __device__ __forceinline__ R rsqrt(R x) { return rsqrtf(x); }
};

// ------------------------------------------------------------ views

// Pointers to one tissue's topology and state.  The pointers may address
// shared or global memory: the same code runs in both residencies.
template <class P>
struct View {
  using R = typename P::R;
  using Pos = typename P::Pos;
  Pos* X;
  uint32_t* tgt;    // [HE]
  int32_t* nxt;     // [HE]
  int32_t* face;    // [HE]
  int32_t* vout;    // [3][V] (SoA)
  int32_t* ffirst;  // [n]
  int n, V, E;
  typename P::Box box;
  double Lx, Ly;
  // Optional flat tables (global-memory residencies): per vertex the packed
  // targets and faces of its three out-half-edges, per cell its corners
  // (vertex + image relative to corner 0) and half-edges.  They replace the
  // pointer chase through nxt / vout by one level of independent loads; T1
  // transitions rebuild the entries they invalidate.
  uint32_t* vnb;    // [3][V]
  int32_t* vfc;     // [3][V]
  int32_t* ccnt;    // [n]
  uint32_t* ccor;   // [n][kMaxCorners]
  int32_t* cedge;   // [n][kMaxCorners]
};

constexpr int kMaxCorners = 16;

// Parameters as the caller gave them (float64, per cell / per edge or
// uniform).
struct ParamsD {
  const double *KA, *KP, *A0, *P0, *lam;
  double KA_s, KP_s, A0_s, P0_s, lam_s;
  __device__ __forceinline__ double ka(int c) const { return KA ? KA[c] : KA_s; }
  __device__ __forceinline__ double kp(int c) const { return KP ? KP[c] : KP_s; }
  __device__ __forceinline__ double a0(int c) const { return A0 ? A0[c] : A0_s; }
  __device__ __forceinline__ double p0(int c) const { return P0 ? P0[c] : P0_s; }
  __device__ __forceinline__ double la(int e) const { return lam ? lam[e] : lam_s; }
};

template <class P>
__device__ __forceinline__ int src_of(const View<P>& v, int h) {
  return tgt_v(v.tgt[h ^ 1]);
}

// Area and perimeter of cell c; lengths below lmin flag their edge in
// `shortbits` (lmin <= 0 disables the check).  Returns whether any edge of
// the cell was flagged.
template <class P>
__device__ __forceinline__ bool cell_geometry(const View<P>& v, int c, typename P::R& A,
                                              typename P::R& Per, typename P::R lmin,
                                              uint32_t* shortbits, double* eline = nullptr,
                                              const ParamsD* prm = nullptr) {
  using R = typename P::R;
  if (v.ccor) {
    // The count and the first eight corner words (two 16-byte loads) are
    // loaded together; each chunk of four corners issues its four position
    // loads and the next chunk's first before any is used: three load
    // latencies for a cell of up to eight corners.
    using Pos = typename P::Pos;
    const uint32_t* cor = v.ccor + (size_t)c * kMaxCorners;
    const int32_t* ced = v.cedge + (size_t)c * kMaxCorners;
    const uint4 wa = reinterpret_cast<const uint4*>(cor)[0];
    const uint4 wb = reinterpret_cast<const uint4*>(cor)[1];
    const int m = v.ccnt[c];
    R qx = 0, qy = 0, A2 = 0, pp = 0;
    bool flagged = false;
    double el = 0.0;
    Pos X0;
    for (int base = 0; base < m; base += 4) {
      uint32_t cw[5];
      if (base == 0) {
        cw[0] = wa.x; cw[1] = wa.y; cw[2] = wa.z; cw[3] = wa.w; cw[4] = wb.x;
      } else if (base == 4) {
        cw[0] = wb.x; cw[1] = wb.y; cw[2] = wb.z; cw[3] = wb.w;
        cw[4] = m > 8 ? cor[8] : 0u;
      } else {
        const uint4 w = reinterpret_cast<const uint4*>(cor + base)[0];
        cw[0] = w.x; cw[1] = w.y; cw[2] = w.z; cw[3] = w.w;
        cw[4] = base + 4 < m ? cor[base + 4] : 0u;
      }
      Pos Xc[5];
#pragma unroll
      for (int k = 0; k < 5; ++k)
        if (base + k < m) Xc[k] = v.X[tgt_v(cw[k])];
      if (base == 0) X0 = Xc[0];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int kk = base + k;  // edge from corner kk to corner kk + 1
        if (kk < m) {
          R nx = 0, ny = 0;
          if (kk + 1 < m)
            P::diff(Xc[k + 1], X0, tgt_ox(cw[k + 1]), tgt_oy(cw[k + 1]), v.box, nx, ny);
          // q_kk -> q_{kk+1}; q_0 = 0
          A2 += qx * ny - nx * qy;
          const R ex = nx - qx, ey = ny - qy;
          const R l = sqrt(ex * ex + ey * ey);
          pp += l;
          if (l < lmin) {
            const int h = ced[kk];
            atomicOr(&shortbits[h >> 6], 1u << ((h >> 1) & 31));
            flagged = true;
          }
          if (eline) el += 0.5 * prm->la(ced[kk] >> 1) * (double)l;
          qx = nx;
          qy = ny;
        }
      }
    }
    A = (R)0.5 * A2;
    Per = pp;
    if (eline) *eline = el;
    return flagged;
  }
  const int h0 = v.ffirst[c];
  const int v0 = src_of(v, h0);
  const typename P::Pos X0 = v.X[v0];
  R qx = 0, qy = 0, A2 = 0, pp = 0;
  int cx = 0, cy = 0;
  int h = h0;
  bool flagged = false;
  double el = 0.0;
  int guard = 0;
  do {
    const uint32_t tg = v.tgt[h];
    cx += tgt_ox(tg);
    cy += tgt_oy(tg);
    R nx, ny;
    P::diff(v.X[tgt_v(tg)], X0, cx, cy, v.box, nx, ny);
    A2 += qx * ny - nx * qy;
    const R ex = nx - qx, ey = ny - qy;
    const R l = sqrt(ex * ex + ey * ey);
    pp += l;
    if (l < lmin) {
      atomicOr(&shortbits[h >> 6], 1u << ((h >> 1) & 31));
      flagged = true;
    }
    if (eline) el += 0.5 * prm->la(h >> 1) * (double)l;
    qx = nx;
    qy = ny;
    h = v.nxt[h];
  } while (h != h0 && ++guard < 4096);
  A = (R)0.5 * A2;
  Per = pp;
  if (eline) *eline = el;
  return flagged;
}

// What the geometry of one cell reads from the flat tables, loaded in one go
// (gather) and used afterwards (compute), so that a thread owning several
// cells has all their loads in flight together: the corner count, the first
// kGather corner words (two 16-byte loads) and their positions.  Corner
// words past the count are clamped into [0, V) before use as indices; their
// positions are loaded but never used.
constexpr int kGather = 8;
template <class P>
struct CGather {
  int m;
  uint32_t w[kGather];
  typename P::Pos X[kGather];
};

template <class P>
__device__ __forceinline__ void cell_gather(const View<P>& v, int c, CGather<P>& g) {
  g.m = v.ccnt[c];
  const uint4* row = reinterpret_cast<const uint4*>(v.ccor + (size_t)c * kMaxCorners);
  const uint4 a = row[0], b = row[1];
  g.w[0] = a.x; g.w[1] = a.y; g.w[2] = a.z; g.w[3] = a.w;
  g.w[4] = b.x; g.w[5] = b.y; g.w[6] = b.z; g.w[7] = b.w;
#pragma unroll
  for (int k = 0; k < kGather; ++k) g.X[k] = v.X[min(tgt_v(g.w[k]), v.V - 1)];
}

// cell_geometry's flat-table arithmetic, in the same order, from a gather
// (corners past kGather are loaded here).
template <class P>
__device__ __forceinline__ bool cell_geometry_g(const View<P>& v, int c, const CGather<P>& g,
                                                typename P::R& A, typename P::R& Per,
                                                typename P::R lmin, uint32_t* shortbits,
                                                double* eline = nullptr,
                                                const ParamsD* prm = nullptr) {
  using R = typename P::R;
  const int m = g.m;
  const int32_t* ced = v.cedge + (size_t)c * kMaxCorners;
  R qx = 0, qy = 0, A2 = 0, pp = 0;
  bool flagged = false;
  double el = 0.0;
  auto edge = [&](int kk, R nx, R ny) {
    A2 += qx * ny - nx * qy;
    const R ex = nx - qx, ey = ny - qy;
    const R l = sqrt(ex * ex + ey * ey);
    pp += l;
    if (l < lmin) {
      const int h = ced[kk];
      atomicOr(&shortbits[h >> 6], 1u << ((h >> 1) & 31));
      flagged = true;
    }
    if (eline) el += 0.5 * prm->la(ced[kk] >> 1) * (double)l;
    qx = nx;
    qy = ny;
  };
#pragma unroll
  for (int kk = 0; kk < kGather; ++kk) {
    if (kk < m) {
      R nx = 0, ny = 0;
      if (kk + 1 < m) {
        if (kk + 1 < kGather) {
          P::diff(g.X[kk + 1], g.X[0], tgt_ox(g.w[kk + 1]), tgt_oy(g.w[kk + 1]), v.box, nx, ny);
        } else {
          const uint32_t t = v.ccor[(size_t)c * kMaxCorners + kk + 1];
          P::diff(v.X[tgt_v(t)], g.X[0], tgt_ox(t), tgt_oy(t), v.box, nx, ny);
        }
      }
      edge(kk, nx, ny);
    }
  }
  for (int kk = kGather; kk < m; ++kk) {
    R nx = 0, ny = 0;
    if (kk + 1 < m) {
      const uint32_t t = v.ccor[(size_t)c * kMaxCorners + kk + 1];
      P::diff(v.X[tgt_v(t)], g.X[0], tgt_ox(t), tgt_oy(t), v.box, nx, ny);
    }
    edge(kk, nx, ny);
  }
  A = (R)0.5 * A2;
  Per = pp;
  if (eline) *eline = el;
  return flagged;
}

// Everything the force on one vertex reads, loaded in one go (gather) and
// used afterwards (compute), so that a thread owning several vertices has
// all their loads in flight together.
template <class P>
struct VGather {
  typename P::Pos Xi, Xj[3];
  uint32_t tg[3];
  typename P::R cA[3], cP[3], la[3];
};

template <class P, class CellC, class LamT>
__device__ __forceinline__ void vertex_gather(const View<P>& v, int i, const CellC* cellc,
                                              const LamT* lam, double lam_s, VGather<P>& g) {
  using R = typename P::R;
  int h[3], f[3];
  g.Xi = v.X[i];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    h[a] = v.vout[a * v.V + i];
    g.tg[a] = v.vnb ? v.vnb[a * v.V + i] : v.tgt[h[a]];
    f[a] = v.vfc ? v.vfc[a * v.V + i] : v.face[h[a]];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    g.Xj[a] = v.X[tgt_v(g.tg[a])];
    const CellC cc = cellc[f[a]];
    g.cA[a] = (R)cc.x;
    g.cP[a] = (R)cc.y;
    g.la[a] = lam ? (R)lam[h[a] >> 1] : (R)lam_s;
  }
}

template <class P>
__device__ __forceinline__ void vertex_compute(const View<P>& v, const VGather<P>& g,
                                               typename P::R& fx, typename P::R& fy) {
  using R = typename P::R;
  R dx[3], dy[3], ux[3], uy[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    P::diff(g.Xj[a], g.Xi, tgt_ox(g.tg[a]), tgt_oy(g.tg[a]), v.box, dx[a], dy[a]);
    const R r = P::rsqrt(dx[a] * dx[a] + dy[a] * dy[a]);
    ux[a] = dx[a] * r;
    uy[a] = dy[a] * r;
  }
  R gx = 0, gy = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int am = (a + 2) % 3, ap = (a + 1) % 3;
    const R T = g.la[a] + g.cP[a] + g.cP[am];
    gx += T * ux[a];
    gy += T * uy[a];
    // -1/2 cA rot(d_a - d_{a+1}),  rot(x, y) = (y, -x)
    const R wx = dx[a] - dx[ap], wy = dy[a] - dy[ap];
    gx -= (R)0.5 * g.cA[a] * wy;
    gy += (R)0.5 * g.cA[a] * wx;
  }
  fx = gx;
  fy = gy;
}

// Force on vertex i from the cell coefficients (cA, cP) and edge tensions.
template <class P, class CellC, class LamT>
__device__ __forceinline__ void vertex_force(const View<P>& v, int i, const CellC* cellc,
                                             const LamT* lam, double lam_s, typename P::R& fx,
                                             typename P::R& fy) {
  VGather<P> g;
  vertex_gather(v, i, cellc, lam, lam_s, g);
  vertex_compute(v, g, fx, fy);
}

// ------------------------------------------------------------ T1 (serial)

// Slot of half-edge h in the out-list of its source vertex s.
template <class P>
__device__ __forceinline__ int out_slot(const View<P>& v, int s, int h) {
  return (v.vout[s] == h) ? 0 : (v.vout[v.V + s] == h ? 1 : 2);
}
// prev(h): the twin of the out-half-edge after h (counter-clockwise).
template <class P>
__device__ __forceinline__ int prev_of(const View<P>& v, int h) {
  const int s = src_of(v, h);
  const int k = out_slot(v, s, h);
  return v.vout[((k + 1) % 3) * v.V + s] ^ 1;
}

template <class P>
__device__ __forceinline__ void edge_vec_d(const View<P>& v, int h, double& dx, double& dy) {
  const uint32_t tg = v.tgt[h];
  const double2 a = P::to_d(v.X[src_of(v, h)]);
  const double2 b = P::to_d(v.X[tgt_v(tg)]);
  dx = (b.x + tgt_ox(tg) * v.Lx) - a.x;
  dy = (b.y + tgt_oy(tg) * v.Ly) - a.y;
}

template <class P>
__device__ __forceinline__ double edge_len_d(const View<P>& v, int h) {
  double dx, dy;
  edge_vec_d(v, h, dx, dy);
  return sqrt(dx * dx + dy * dy);
}

template <class P>
__device__ __forceinline__ int face_size(const View<P>& v, int h0) {
  int k = 0, h = h0;
  do {
    ++k;
    h = v.nxt[h];
  } while (h != h0 && k < 4096);
  return k;
}

// Edge length in the tissue's precision (the T1 length checks): FP64
// tissues in FP64, FP32 tissues in FP32 from the TwoSum-exact local
// difference (as the cell and force passes do).
template <class P>
__device__ __forceinline__ double edge_len_p(const View<P>& v, int h) {
  if constexpr (std::is_same<typename P::R, double>::value) {
    return edge_len_d(v, h);
  } else {
    const uint32_t tg = v.tgt[h];
    float dx, dy;
    P::diff(v.X[tgt_v(tg)], v.X[src_of(v, h)], tgt_ox(tg), tgt_oy(tg), v.box, dx, dy);
    return (double)sqrtf(dx * dx + dy * dy);
  }
}

// Rebuild the flat-table entries of vertex w and of cell c from the
// half-edge tables (after a T1 rewired them).
template <class P>
__device__ void rebuild_vertex(const View<P>& v, int w) {
  for (int a = 0; a < 3; ++a) {
    const int h = v.vout[a * v.V + w];
    v.vnb[a * v.V + w] = v.tgt[h];
    v.vfc[a * v.V + w] = v.face[h];
  }
}
template <class P>
__device__ void rebuild_cell(const View<P>& v, int c) {
  const int h0 = v.ffirst[c];
  uint32_t* cor = v.ccor + (size_t)c * kMaxCorners;
  int32_t* ced = v.cedge + (size_t)c * kMaxCorners;
  int h = h0, k = 0, cx = 0, cy = 0;
  cor[0] = pack_tgt(src_of(v, h0), 0, 0);
  do {
    const uint32_t tg = v.tgt[h];
    ced[k] = h;
    cx += tgt_ox(tg);
    cy += tgt_oy(tg);
    ++k;
    if (k < kMaxCorners) cor[k] = pack_tgt(tgt_v(tg), cx, cy);
    h = v.nxt[h];
  } while (h != h0 && k < kMaxCorners);
  v.ccnt[c] = k;
}

struct T1Stats {
  int n_t1, n_stretch, err;
};

constexpr double kT1Stretch = 1.5;  // both candidates: length 1.5 l_min

// ------------------------------------------------------------ wrap

// One coordinate of the exit-time wrap (Methods, "Periodic mode"):
// x' = x - k L in [0, L) with k = floor(x / L), corrected by one period when
// rounding left x' outside [0, L); a result that rounds to L is taken as 0.
// Explicitly rounded operations: no fused multiply-add changes a result.
__device__ __forceinline__ double wrap_coord(double x, double L, int& k) {
  const double q = floor(__ddiv_rn(x, L));
  double w = __dsub_rn(x, __dmul_rn(q, L));
  int kk = (int)q;
  if (w >= L) {
    w = __dsub_rn(w, L);
    ++kk;
  }
  if (w < 0.0) {
    w = __dadd_rn(w, L);
    --kk;
  }
  if (w >= L) w = 0.0;
  k = kk;
  return w;
}

// ------------------------------------------------------------ reductions

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
__device__ __forceinline__ double warp_max(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

}  // namespace vx
