// T1 transitions (Methods, "T1 transitions"): when an edge is shorter than
// l_min, two candidates are compared by energy and the lower one is kept:
// (1) the edge stretched along its direction, (2) the edge removed and a new
// edge orthogonal to it created (a neighbour exchange).  Both candidates give
// the edge length 1.5 l_min about its old midpoint; a T1 is not a candidate
// when a cell losing the edge is a triangle, when the four cells around the
// edge are not distinct, when an offset would leave {-1, 0, 1} or when a cell
// would outgrow the flat tables.  Edges are taken in increasing id, each
// against the positions the previous ones left; edges with a larger id that a
// change makes short join the same pass.
//
// Naming, for the edge's half-edge h = a -> b and its twin h^1 = b -> a:
// C1 = face(h), C2 = face(h^1); p -> a = prev(h) (in C1), b -> y = next(h),
// z -> b = prev(h^1) (in C2), a -> x = next(h^1); C3 = face(a -> p),
// C4 = face(b -> z).  After the T1, a sits on C1's side joined to p and y,
// b on C2's side joined to x and z, and the edge a - b separates C3 from C4:
// C1 loses b, C2 loses a, C3 = (.. x, b, a, p ..), C4 = (.. y, a, b, z ..).
//
// The candidates are evaluated without changing the tissue: only the four
// cells and the five edges at a and b differ between them, and each cell is
// walked once, accumulating its area and perimeter for both candidates (the
// T1 cycles are the current ones with one corner dropped or inserted, and a,
// b at their new positions in the frames the current offsets give them).
#pragma once
#include <type_traits>

#include "device_math.cuh"

namespace vx {

// Both candidates of the short edge e as one warp sees them (every lane).
template <class P>
struct T1Cand {
  using Pos = typename P::Pos;
  int h, a, b, C[4];
  int hp1, hn1, hp2, hn2, p, x, y, z;
  int kbx, kby, kpx, kpy, kxx, kxy, kyx, kyy, kzx, kzy;
  bool allow;
  Pos Xas, Xbs;   // stretch: a, b in their own frames
  Pos Xat, Xbt;   // T1: a and b, both in a's frame
  double Es, Et;  // local energies (four cells, five edges)
};

// Area and perimeter of a closed polygon whose corners (positions relative
// to any fixed origin) arrive one at a time.
template <class R>
struct PolyAcc {
  R fx, fy, px, py, a2, pp;
  int m;
  __device__ __forceinline__ void init() {
    a2 = pp = 0;
    m = 0;
  }
  __device__ __forceinline__ void add(R x, R y) {
    if (m == 0) {
      fx = x;
      fy = y;
    } else {
      a2 += px * y - x * py;
      const R ex = x - px, ey = y - py;
      pp += sqrt(ex * ex + ey * ey);
    }
    px = x;
    py = y;
    ++m;
  }
  __device__ __forceinline__ void close(R& A, R& Per) {
    a2 += px * fy - fx * py;
    const R ex = fx - px, ey = fy - py;
    pp += sqrt(ex * ex + ey * ey);
    A = (R)0.5 * a2;
    Per = pp;
  }
};

// Energy K_A (A - A0)^2 + K_P (P - P0)^2 of cell c under both candidates.
// role 0 (C1): the T1 drops b; role 1 (C2): drops a; role 2 (C3): inserts
// b before a; role 3 (C4): inserts a before b.
template <class P>
__device__ __noinline__ void t1_cell_pair(const View<P>& v, const ParamsD& prm, int c, int role,
                                          const T1Cand<P>& k, double& es, double& et) {
  using R = typename P::R;
  using Pos = typename P::Pos;
  PolyAcc<R> s, t;
  s.init();
  t.init();
  const int h0 = v.ffirst[c];
  const Pos X0 = v.X[src_of(v, h0)];
  // b's T1 position in b's current frame, a's T1 position in b's frame
  const double2 at = P::to_d(k.Xat), bt = P::to_d(k.Xbt);
  const Pos Xbt_b = P::from_d(bt.x - k.kbx * v.Lx, bt.y - k.kby * v.Ly);
  const Pos Xat_b = P::from_d(at.x - k.kbx * v.Lx, at.y - k.kby * v.Ly);
  int cx = 0, cy = 0, h = h0, guard = 0, vv = src_of(v, h0);
  do {
    const bool is_a = vv == k.a, is_b = vv == k.b;
    R dx, dy;
    P::diff(is_a ? k.Xas : (is_b ? k.Xbs : v.X[vv]), X0, cx, cy, v.box, dx, dy);
    s.add(dx, dy);
    if (role == 2 && is_a) {
      R ix, iy;
      P::diff(k.Xbt, X0, cx, cy, v.box, ix, iy);
      t.add(ix, iy);
    }
    if (role == 3 && is_b) {
      R ix, iy;
      P::diff(Xat_b, X0, cx, cy, v.box, ix, iy);
      t.add(ix, iy);
    }
    const bool drop = (role == 0 && is_b) || (role == 1 && is_a);
    if (!drop) {
      if (is_a || is_b) P::diff(is_a ? k.Xat : Xbt_b, X0, cx, cy, v.box, dx, dy);
      t.add(dx, dy);
    }
    const uint32_t tg = v.tgt[h];
    cx += tgt_ox(tg);
    cy += tgt_oy(tg);
    vv = tgt_v(tg);
    h = v.nxt[h];
  } while (h != h0 && ++guard < 4096);
  R As, Ps, At, Pt;
  s.close(As, Ps);
  t.close(At, Pt);
  const double a0 = prm.a0(c), p0 = prm.p0(c), ka = prm.ka(c), kp = prm.kp(c);
  const double dAs = (double)As - a0, dPs = (double)Ps - p0;
  const double dAt = (double)At - a0, dPt = (double)Pt - p0;
  es = ka * dAs * dAs + kp * dPs * dPs;
  et = ka * dAt * dAt + kp * dPt * dPt;
}

// Length of the segment from s to t + o L (positions as stored).
template <class P>
__device__ __forceinline__ double seg_len(const View<P>& v, const typename P::Pos& t,
                                          const typename P::Pos& s, int ox, int oy) {
  typename P::R dx, dy;
  P::diff(t, s, ox, oy, v.box, dx, dy);
  return (double)sqrt(dx * dx + dy * dy);
}

// Everything about the short edge e, evaluated by the 32 lanes of one warp
// (every lane must call; every lane gets the result).  Returns false when
// the edge is no longer shorter than lmin.
template <class P>
__device__ __noinline__ bool t1_evaluate(const View<P>& v, const ParamsD& prm, double lmin, int e,
                                         T1Cand<P>& k) {
  using Pos = typename P::Pos;
  const int lane = threadIdx.x & 31;
  const int h = 2 * e, hq = h ^ 1;
  if (edge_len_p(v, h) >= lmin) return false;
  k.h = h;
  k.a = src_of(v, h);
  k.b = tgt_v(v.tgt[h]);
  k.C[0] = v.face[h];
  k.C[1] = v.face[hq];
  k.hp1 = prev_of(v, h);
  k.hn1 = v.nxt[h];
  k.hp2 = prev_of(v, hq);
  k.hn2 = v.nxt[hq];
  const int ta_p = k.hp1 ^ 1, tb_z = k.hp2 ^ 1;
  k.C[2] = v.face[ta_p];
  k.C[3] = v.face[tb_z];
  const uint32_t tg_h = v.tgt[h], tg_ap = v.tgt[ta_p], tg_n2 = v.tgt[k.hn2];
  const uint32_t tg_n1 = v.tgt[k.hn1], tg_bz = v.tgt[tb_z];
  k.p = tgt_v(tg_ap);
  k.y = tgt_v(tg_n1);
  k.x = tgt_v(tg_n2);
  k.z = tgt_v(tg_bz);
  k.kbx = tgt_ox(tg_h);
  k.kby = tgt_oy(tg_h);
  k.kpx = tgt_ox(tg_ap);
  k.kpy = tgt_oy(tg_ap);
  k.kxx = tgt_ox(tg_n2);
  k.kxy = tgt_oy(tg_n2);
  k.kyx = k.kbx + tgt_ox(tg_n1);
  k.kyy = k.kby + tgt_oy(tg_n1);
  k.kzx = k.kbx + tgt_ox(tg_bz);
  k.kzy = k.kby + tgt_oy(tg_bz);
  // face sizes of C1..C4 in parallel
  const int fh[4] = {h, hq, ta_p, tb_z};
  const int fs = lane < 4 ? face_size(v, fh[lane]) : 0;
  const int s1 = __shfl_sync(0xffffffffu, fs, 0), s2 = __shfl_sync(0xffffffffu, fs, 1);
  const int s3 = __shfl_sync(0xffffffffu, fs, 2), s4 = __shfl_sync(0xffffffffu, fs, 3);
  const int* C = k.C;
  k.allow = s1 > 3 && s2 > 3 && s3 < kMaxCorners && s4 < kMaxCorners &&
            C[0] != C[1] && C[0] != C[2] &&
            C[0] != C[3] && C[1] != C[2] && C[1] != C[3] && C[2] != C[3] && k.kyx >= -1 &&
            k.kyx <= 1 && k.kyy >= -1 && k.kyy <= 1 && k.kzx >= -1 && k.kzx <= 1 && k.kzy >= -1 &&
            k.kzy <= 1;
  // new positions (FP64 geometry of the edge in a's frame)
  double dx, dy;
  edge_vec_d(v, h, dx, dy);
  const double ell = sqrt(dx * dx + dy * dy);
  const double ux = dx / ell, uy = dy / ell;
  const double2 Xa = P::to_d(v.X[k.a]);
  const double mx = Xa.x + 0.5 * dx, my = Xa.y + 0.5 * dy;
  const double lnew = kT1Stretch * lmin;
  k.Xas = P::from_d(mx - 0.5 * lnew * ux, my - 0.5 * lnew * uy);
  k.Xbs = P::from_d(mx + 0.5 * lnew * ux - k.kbx * v.Lx, my + 0.5 * lnew * uy - k.kby * v.Ly);
  const double px = -uy, py = ux;  // into C1
  k.Xat = P::from_d(mx + 0.5 * lnew * px, my + 0.5 * lnew * py);
  k.Xbt = P::from_d(mx - 0.5 * lnew * px, my - 0.5 * lnew * py);
  // lanes 0..3: the four cells under both candidates; lanes 4..8: the five
  // edges h, p - a, (b|a) - y, z - b, (a|b) - x
  double es = 0.0, et = 0.0;
  if (lane < 4) {
    t1_cell_pair(v, prm, C[lane], lane, k, es, et);
  } else if (lane < 9) {
    const int q = lane - 4;
    const int he[5] = {h, k.hp1, k.hn1, k.hp2, k.hn2};
    const double la = prm.la(he[q] >> 1);
    const Pos Xp = v.X[k.p], Xx = v.X[k.x], Xy = v.X[k.y], Xz = v.X[k.z];
    double ls = 0.0, lt = 0.0;
    switch (q) {
      case 0:   // a - b
        ls = seg_len(v, k.Xbs, k.Xas, k.kbx, k.kby);
        lt = seg_len(v, k.Xbt, k.Xat, 0, 0);
        break;
      case 1:   // p - a
        ls = seg_len(v, k.Xas, Xp, -k.kpx, -k.kpy);
        lt = seg_len(v, k.Xat, Xp, -k.kpx, -k.kpy);
        break;
      case 2:   // b - y, then a - y
        ls = seg_len(v, Xy, k.Xbs, k.kyx - k.kbx, k.kyy - k.kby);
        lt = seg_len(v, Xy, k.Xat, k.kyx, k.kyy);
        break;
      case 3:   // z - b
        ls = seg_len(v, k.Xbs, Xz, k.kbx - k.kzx, k.kby - k.kzy);
        lt = seg_len(v, k.Xbt, Xz, -k.kzx, -k.kzy);
        break;
      default:  // a - x, then b - x
        ls = seg_len(v, Xx, k.Xas, k.kxx, k.kxy);
        lt = seg_len(v, Xx, k.Xbt, k.kxx, k.kxy);
        break;
    }
    es = la * ls;
    et = la * lt;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    es += __shfl_xor_sync(0xffffffffu, es, o);
    et += __shfl_xor_sync(0xffffffffu, et, o);
  }
  k.Es = es;
  k.Et = et;
  return true;
}

// Applies the chosen candidate (lane 0 writes, the flat-table rebuild is
// spread over lanes) and flags the vertices whose velocities restart.
template <class P>
__device__ __forceinline__ void t1_commit(const View<P>& v, const T1Cand<P>& k, bool take_t1,
                                          uint32_t* touched) {
  const int lane = threadIdx.x & 31;
  const int h = k.h, hq = h ^ 1;
  const int ta_p = k.hp1 ^ 1, tb_y = k.hn1 ^ 1, tb_z = k.hp2 ^ 1, tx_a = k.hn2 ^ 1;
  if (lane == 0) {
    touched[k.a >> 5] |= 1u << (k.a & 31);
    touched[k.b >> 5] |= 1u << (k.b & 31);
    if (take_t1) {
      v.X[k.a] = k.Xat;
      v.X[k.b] = k.Xbt;
      v.nxt[k.hp1] = k.hn1;
      v.nxt[k.hp2] = k.hn2;
      v.nxt[tx_a] = hq;
      v.nxt[hq] = ta_p;
      v.nxt[tb_y] = h;
      v.nxt[h] = tb_z;
      v.face[hq] = k.C[2];
      v.face[h] = k.C[3];
      v.tgt[ta_p] = pack_tgt(k.p, k.kpx, k.kpy);
      v.tgt[k.hp1] = pack_tgt(k.a, -k.kpx, -k.kpy);
      v.tgt[k.hn1] = pack_tgt(k.y, k.kyx, k.kyy);
      v.tgt[tb_y] = pack_tgt(k.a, -k.kyx, -k.kyy);
      v.tgt[k.hn2] = pack_tgt(k.x, k.kxx, k.kxy);
      v.tgt[tx_a] = pack_tgt(k.b, -k.kxx, -k.kxy);
      v.tgt[tb_z] = pack_tgt(k.z, k.kzx, k.kzy);
      v.tgt[k.hp2] = pack_tgt(k.b, -k.kzx, -k.kzy);
      v.tgt[h] = pack_tgt(k.b, 0, 0);
      v.tgt[hq] = pack_tgt(k.a, 0, 0);
      v.vout[k.a] = h;
      v.vout[v.V + k.a] = k.hn1;
      v.vout[2 * v.V + k.a] = ta_p;
      v.vout[k.b] = hq;
      v.vout[v.V + k.b] = k.hn2;
      v.vout[2 * v.V + k.b] = tb_z;
      if (v.ffirst[k.C[0]] == h) v.ffirst[k.C[0]] = k.hn1;
      if (v.ffirst[k.C[1]] == hq) v.ffirst[k.C[1]] = k.hn2;
    } else {
      v.X[k.a] = k.Xas;
      v.X[k.b] = k.Xbs;
    }
  }
  __syncwarp();
  if (take_t1 && v.ccor) {
    const int ws[6] = {k.a, k.b, k.p, k.x, k.y, k.z};
    if (lane < 6) rebuild_vertex(v, ws[lane]);
    else if (lane < 10) rebuild_cell(v, k.C[lane - 6]);
  }
  __syncwarp();
}

// The T1 pass over the edges flagged in `shortbits`, by all warps of one
// CTA, with the result of taking the flagged edges one at a time in
// increasing id (edges with a larger id that a commit makes short join the
// pass; `shortbits` ends cleared; cells whose geometry changed are appended
// to `dirty`, up to `dirty_cap`, while `*n_dirty` counts them all; `events`,
// optional [E][2], counts each edge's stretches and T1s).  Each round, the
// next (up to) eight flagged edges in id order are evaluated at once, one
// warp each, against the current tissue; warp 0 then commits them in id
// order.  A candidate's evaluation reads
// only the four cells around its edge (their corners, half-edges and
// parameters), and a commit changes only the four cells around its own
// edge, so the evaluation of a later candidate whose cells are disjoint
// from every cell committed before it in the round is the one the
// sequential pass would make.  The round stops at the first candidate that
// fails this test, at a candidate that a join (an edge made short by a
// commit, with a larger id than the committed edge) precedes, and at a
// candidate found no longer short after an earlier commit of the round
// (its cells are not known); the next round starts there.  Every thread of
// the CTA must call it.
template <class P>
__device__ __noinline__ void t1_pass_block(View<P> v, const ParamsD& prm, double lmin,
                                           uint32_t* shortbits, uint32_t* touched, T1Stats* st,
                                           int* dirty = nullptr, int dirty_cap = 0,
                                           int* n_dirty = nullptr, int* events = nullptr) {
  constexpr int kNW = 8;
  __shared__ T1Cand<P> slot[kNW];
  __shared__ int cand[kNW], okv[kNW], rcells[4 * kNW];
  __shared__ int ncand, s_cursor;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (int)(blockDim.x >> 5) < kNW ? (int)(blockDim.x >> 5) : kNW;
  const int nwords = (v.E + 31) >> 5;
  if (threadIdx.x == 0) s_cursor = 0;
  __syncthreads();
  for (;;) {
    // the next flagged edges at or after the cursor, in id order
    if (warp == 0) {
      const int cursor = s_cursor;
      int count = 0;
      for (int w0 = cursor >> 5; w0 < nwords && count < nw; w0 += 32) {
        const int w = w0 + lane;
        uint32_t bits = w < nwords ? ((volatile const uint32_t*)shortbits)[w] : 0u;
        if (w == (cursor >> 5)) bits &= ~((1u << (cursor & 31)) - 1u);
        unsigned nz = __ballot_sync(0xffffffffu, bits != 0);
        while (nz && count < nw) {
          const int src = __ffs(nz) - 1;
          nz &= nz - 1;
          uint32_t b = __shfl_sync(0xffffffffu, bits, src);
          while (b && count < nw) {
            const int bit = __ffs(b) - 1;
            b &= b - 1;
            if (lane == 0) cand[count] = ((w0 + src) << 5) + bit;
            ++count;
          }
        }
      }
      if (lane == 0) ncand = count;
    }
    __syncthreads();
    const int k = ncand;
    if (k == 0) break;
    if (warp < k) {
      T1Cand<P> c;
      const bool r = t1_evaluate(v, prm, lmin, cand[warp], c);
      if (lane == 0) {
        slot[warp] = c;
        okv[warp] = r ? 1 : 0;
      }
    }
    __syncthreads();
    if (warp == 0) {
      int nr = 0, minjoin = 0x7fffffff, next = s_cursor;
      for (int j = 0; j < k; ++j) {
        const int e = cand[j];
        if (j > 0) {
          if (minjoin < e) break;
          if (!okv[j] && nr > 0) break;
          bool conflict = false;
          if (okv[j])
            for (int q = 0; q < 4 && !conflict; ++q)
              for (int r = 0; r < nr; ++r)
                if (slot[j].C[q] == rcells[r]) {
                  conflict = true;
                  break;
                }
          if (conflict) break;
        }
        if (lane == 0) atomicAnd(&shortbits[e >> 5], ~(1u << (e & 31)));
        next = e + 1;
        __syncwarp();
        if (!okv[j]) continue;
        const T1Cand<P> c = slot[j];
        const bool take_t1 = c.allow && c.Et < c.Es;
        if (lane == 0 && events) events[2 * e + (take_t1 ? 1 : 0)] += 1;
        t1_commit(v, c, take_t1, touched);
        if (lane == 0) {
          if (take_t1) st->n_t1++;
          else st->n_stretch++;
          if (n_dirty) {
            for (int q = 0; q < 4; ++q) {
              if (*n_dirty < dirty_cap) dirty[*n_dirty] = c.C[q];
              ++*n_dirty;
            }
          }
          for (int q = 0; q < 4; ++q) rcells[nr + q] = c.C[q];
        }
        nr += 4;
        __syncwarp();
        // edges at a or b with a larger id that are now short join the pass
        int join = 0x7fffffff;
        if (lane < 6) {
          const int vv = lane < 3 ? c.a : c.b;
          const int hh = v.vout[(lane % 3) * v.V + vv];
          const int f = hh >> 1;
          if (f > e && edge_len_p(v, hh) < lmin) {
            atomicOr(&shortbits[f >> 5], 1u << (f & 31));
            join = f;
          }
        }
        join = __reduce_min_sync(0xffffffffu, join);
        if (join < minjoin) minjoin = join;
        __syncwarp();
      }
      if (lane == 0) s_cursor = next;
    }
    __syncthreads();
  }
}

}  // namespace vx
