// Host builder of the periodic Voronoi tessellation (vx_build_mesh).
//
// Methods, "Mesh initialization" / "Periodic mode": the Voronoi cell of every
// seed on the torus, with periodic offsets on the half-edges that cross the
// box.  The cell of seed i is found by clipping a square around it with the
// perpendicular bisectors of nearby seed images, nearest first, until no
// remaining image can cut it (the security radius: twice the distance to the
// cell's farthest corner).  Each corner of the clipped polygon is the meeting
// point of the bisectors of two images, so it names its Delaunay triangle
// (i, j + s_j, k + s_k) combinatorially; keys, vertex order, half-edge order
// and edge ids then follow the canonical indexing documented in vx.h.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "vx_internal.h"

namespace vx {
namespace {

struct Img {          // a seed image: seed index and integer box shift
  int32_t seed, sx, sy;
  double x, y;        // position
  double d2;          // squared distance to the clipped cell's seed
};

struct Corner {       // a polygon corner; edge (k -> k+1) is generated by gen[k]
  double x, y;
};

// Key of a Delaunay triangle of the torus: (a, b, sbx, sby, c, scx, scy).
using Key = std::array<int32_t, 7>;

struct Tri {          // three CCW corners (seed, sx, sy)
  int32_t s[3], sx[3], sy[3];
};

// Smallest normalised rotation; t = shift subtracted to reach the key frame.
void canonical_key(const Tri& tr, Key* key, int32_t* tx, int32_t* ty) {
  bool have = false;
  for (int r = 0; r < 3; ++r) {
    int a = r, b = (r + 1) % 3, c = (r + 2) % 3;
    Key k = {tr.s[a], tr.s[b], tr.sx[b] - tr.sx[a], tr.sy[b] - tr.sy[a],
             tr.s[c], tr.sx[c] - tr.sx[a], tr.sy[c] - tr.sy[a]};
    if (!have || k < *key) {
      *key = k;
      *tx = tr.sx[a];
      *ty = tr.sy[a];
      have = true;
    }
  }
}

void circumcentre(double px, double py, double qx, double qy, double rx, double ry,
                  double* cx, double* cy) {
  const double bx = qx - px, by = qy - py, ex = rx - px, ey = ry - py;
  const double d = 2.0 * (bx * ey - by * ex);
  const double b2 = bx * bx + by * by, e2 = ex * ex + ey * ey;
  *cx = px + (ey * b2 - by * e2) / d;
  *cy = py + (bx * e2 - ex * b2) / d;
}

struct Grid {
  int gx, gy;
  double Lx, Ly, wx, wy;
  std::vector<int32_t> start, items;
  Grid(const double* seeds, int n, double Lx_, double Ly_) : Lx(Lx_), Ly(Ly_) {
    const double cell = std::sqrt(Lx * Ly / n);
    gx = std::max(1, (int)std::floor(Lx / cell));
    gy = std::max(1, (int)std::floor(Ly / cell));
    wx = Lx / gx;
    wy = Ly / gy;
    std::vector<int32_t> cnt(gx * gy + 1, 0);
    std::vector<int32_t> b(n);
    for (int i = 0; i < n; ++i) {
      int bx = std::min(gx - 1, std::max(0, (int)(seeds[2 * i] / wx)));
      int by = std::min(gy - 1, std::max(0, (int)(seeds[2 * i + 1] / wy)));
      b[i] = by * gx + bx;
      cnt[b[i] + 1]++;
    }
    for (int k = 0; k < gx * gy; ++k) cnt[k + 1] += cnt[k];
    start = cnt;
    items.resize(n);
    std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
    for (int i = 0; i < n; ++i) items[fill[b[i]]++] = i;
  }
};

inline int floordiv(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }

struct CellOut {
  std::vector<Key> keys;          // per corner, in CCW order
  std::vector<int32_t> tx, ty;    // key translation per corner
  int status = 0;                 // 0 ok, else a vx_status
};

// Voronoi cell of seed i by half-plane clipping.
void clip_cell(const double* seeds, int n, const Grid& g, int i, CellOut* out) {
  const double sx0 = seeds[2 * i], sy0 = seeds[2 * i + 1];
  const double B = 1.5 * std::max(g.Lx, g.Ly);
  const int bx0 = std::min(g.gx - 1, std::max(0, (int)(sx0 / g.wx)));
  const int by0 = std::min(g.gy - 1, std::max(0, (int)(sy0 / g.wy)));
  const double wmin = std::min(g.wx, g.wy);
  int rings = 3;
  for (int attempt = 0; attempt < 12; ++attempt, rings *= 2) {
    // Gather every image in the (2 rings + 1)^2 buckets around the seed.
    std::vector<Img> cand;
    for (int dy = -rings; dy <= rings; ++dy)
      for (int dx = -rings; dx <= rings; ++dx) {
        const int bx = bx0 + dx, by = by0 + dy;
        const int shx = floordiv(bx, g.gx), shy = floordiv(by, g.gy);
        const int pb = (by - shy * g.gy) * g.gx + (bx - shx * g.gx);
        for (int q = g.start[pb]; q < g.start[pb + 1]; ++q) {
          const int j = g.items[q];
          if (j == i && shx == 0 && shy == 0) continue;
          Img m;
          m.seed = j;
          m.sx = shx;
          m.sy = shy;
          m.x = seeds[2 * j] + shx * g.Lx;
          m.y = seeds[2 * j + 1] + shy * g.Ly;
          const double ddx = m.x - sx0, ddy = m.y - sy0;
          m.d2 = ddx * ddx + ddy * ddy;
          cand.push_back(m);
        }
      }
    std::sort(cand.begin(), cand.end(), [](const Img& a, const Img& b) {
      if (a.d2 != b.d2) return a.d2 < b.d2;
      if (a.seed != b.seed) return a.seed < b.seed;
      if (a.sx != b.sx) return a.sx < b.sx;
      return a.sy < b.sy;
    });
    // Covered radius: every image closer than this is in `cand`.
    const double covered = rings * wmin;
    // Initial square; generators -1 .. -4 mark its sides.
    std::vector<Corner> poly = {{sx0 - B, sy0 - B}, {sx0 + B, sy0 - B},
                                {sx0 + B, sy0 + B}, {sx0 - B, sy0 + B}};
    std::vector<int32_t> gen = {-1, -2, -3, -4};
    double r2max = 2 * B * B;
    size_t used = 0;
    for (; used < cand.size(); ++used) {
      const Img& m = cand[used];
      if (m.d2 > 4.0 * r2max) break;  // no remaining image can cut the cell
      const double nx = m.x - sx0, ny = m.y - sy0;
      const double mx = 0.5 * (m.x + sx0), my = 0.5 * (m.y + sy0);
      const size_t K = poly.size();
      std::vector<double> f(K);
      bool any_out = false;
      for (size_t k = 0; k < K; ++k) {
        f[k] = (poly[k].x - mx) * nx + (poly[k].y - my) * ny;
        any_out |= f[k] > 0;
      }
      if (!any_out) continue;
      std::vector<Corner> np;
      std::vector<int32_t> ng;
      np.reserve(K + 1);
      ng.reserve(K + 1);
      for (size_t k = 0; k < K; ++k) {
        const size_t k1 = (k + 1) % K;
        const bool in0 = f[k] <= 0, in1 = f[k1] <= 0;
        if (in0) {
          np.push_back(poly[k]);
          ng.push_back(gen[k]);
        }
        if (in0 != in1) {
          const double s = f[k] / (f[k] - f[k1]);
          Corner c = {poly[k].x + s * (poly[k1].x - poly[k].x),
                      poly[k].y + s * (poly[k1].y - poly[k].y)};
          np.push_back(c);
          // Entering the kept side starts the bisector edge (generator = m);
          // leaving it continues the old edge k.
          ng.push_back(in0 ? (int32_t)used : gen[k]);
        }
      }
      poly.swap(np);
      gen.swap(ng);
      if (poly.size() < 3) {
        out->status = VX_ERR_DEGENERATE_SEEDS;
        return;
      }
      r2max = 0;
      for (const Corner& c : poly) {
        const double ddx = c.x - sx0, ddy = c.y - sy0;
        r2max = std::max(r2max, ddx * ddx + ddy * ddy);
      }
    }
    const double rmax = std::sqrt(r2max);
    bool square_left = false;
    for (int32_t v : gen) square_left |= v < 0;
    if (square_left || 2.0 * rmax > covered) continue;  // widen the search
    // Corner k sits between edges k-1 and k: triangle (i, gen[k-1], gen[k]).
    const size_t K = poly.size();
    out->keys.resize(K);
    out->tx.resize(K);
    out->ty.resize(K);
    for (size_t k = 0; k < K; ++k) {
      const Img& a = cand[gen[(k + K - 1) % K]];
      const Img& b = cand[gen[k]];
      Tri tr;
      tr.s[0] = i; tr.sx[0] = 0; tr.sy[0] = 0;
      tr.s[1] = a.seed; tr.sx[1] = a.sx; tr.sy[1] = a.sy;
      tr.s[2] = b.seed; tr.sx[2] = b.sx; tr.sy[2] = b.sy;
      const double o = (a.x - sx0) * (b.y - sy0) - (a.y - sy0) * (b.x - sx0);
      if (o < 0) {  // keep the corners counter-clockwise
        std::swap(tr.s[1], tr.s[2]);
        std::swap(tr.sx[1], tr.sx[2]);
        std::swap(tr.sy[1], tr.sy[2]);
      }
      canonical_key(tr, &out->keys[k], &out->tx[k], &out->ty[k]);
    }
    out->status = 0;
    return;
  }
  out->status = VX_ERR_DEGENERATE_SEEDS;
}

}  // namespace

vx_status build_mesh(const double* seeds, int n, double Lx, double Ly, double* vert,
                     int32_t* he, int32_t* face_he, int32_t* edge_id, std::string* err) {
  Grid g(seeds, n, Lx, Ly);
  std::vector<CellOut> cells(n);
  {
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (n < 2000) nt = 1;
    std::vector<std::thread> pool;
    for (unsigned w = 0; w < nt; ++w)
      pool.emplace_back([&, w]() {
        for (int i = (int)w; i < n; i += (int)nt) clip_cell(seeds, n, g, i, &cells[i]);
      });
    for (auto& th : pool) th.join();
  }
  for (int i = 0; i < n; ++i)
    if (cells[i].status) {
      *err = "Voronoi cell of seed " + std::to_string(i) + " could not be built";
      return VX_ERR_DEGENERATE_SEEDS;
    }
  // Vertices: the sorted unique keys.  The order is lexicographic and a
  // key's first entry is a seed, so a counting sort by that seed followed
  // by a sort of each (small) bucket gives the sorted order; bstart[a] ..
  // bstart[a + 1] are then the vertices whose key starts with seed a.
  size_t HE = 0;
  for (int i = 0; i < n; ++i) HE += cells[i].keys.size();
  std::vector<int32_t> bstart(n + 1, 0);
  for (int i = 0; i < n; ++i)
    for (const Key& k : cells[i].keys) bstart[k[0] + 1]++;
  for (int a = 0; a < n; ++a) bstart[a + 1] += bstart[a];
  std::vector<Key> keys(HE);
  {
    std::vector<int32_t> fill(bstart.begin(), bstart.end() - 1);
    for (int i = 0; i < n; ++i)
      for (const Key& k : cells[i].keys) keys[fill[k[0]]++] = k;
  }
  {
    size_t w = 0;
    for (int a = 0; a < n; ++a) {
      const size_t b0 = bstart[a], b1 = bstart[a + 1];
      std::sort(keys.begin() + b0, keys.begin() + b1);
      bstart[a] = (int32_t)w;
      for (size_t q = b0; q < b1; ++q)
        if (q == b0 || keys[q] != keys[q - 1]) keys[w++] = keys[q];
    }
    bstart[n] = (int32_t)w;
    keys.resize(w);
  }
  const int V = (int)keys.size();
  if (V != 2 * n || HE != (size_t)6 * n) {
    *err = "not a 3-valent torus tessellation (V=" + std::to_string(V) +
           ", HE=" + std::to_string(HE) + ", n=" + std::to_string(n) + ")";
    return VX_ERR_DEGENERATE_SEEDS;
  }
  auto vertex_of = [&](const Key& k) -> int32_t {
    for (int32_t v = bstart[k[0]]; v < bstart[k[0] + 1]; ++v)
      if (keys[v] == k) return v;
    return -1;
  };
  std::vector<int32_t> wrapx(V), wrapy(V);
  for (int v = 0; v < V; ++v) {
    const Key& k = keys[v];
    double cx, cy;
    circumcentre(seeds[2 * k[0]], seeds[2 * k[0] + 1],
                 seeds[2 * k[1]] + k[2] * Lx, seeds[2 * k[1] + 1] + k[3] * Ly,
                 seeds[2 * k[4]] + k[5] * Lx, seeds[2 * k[4] + 1] + k[6] * Ly, &cx, &cy);
    const double wx = std::floor(cx / Lx), wy = std::floor(cy / Ly);
    vert[2 * v] = cx - wx * Lx;
    vert[2 * v + 1] = cy - wy * Ly;
    wrapx[v] = (int32_t)wx;
    wrapy[v] = (int32_t)wy;
  }
  // Faces: CCW corners from the smallest vertex index; corner image
  // k = wrap + t (the corner's triangle is the key triangle shifted by t).
  int32_t h = 0;
  std::vector<int32_t> cv, ckx, cky;
  for (int a = 0; a < n; ++a) {
    const CellOut& c = cells[a];
    const int m = (int)c.keys.size();
    cv.resize(m);
    ckx.resize(m);
    cky.resize(m);
    for (int q = 0; q < m; ++q) {
      cv[q] = vertex_of(c.keys[q]);
      if (cv[q] < 0) {
        *err = "inconsistent tessellation";
        return VX_ERR_DEGENERATE_SEEDS;
      }
      ckx[q] = wrapx[cv[q]] + c.tx[q];
      cky[q] = wrapy[cv[q]] + c.ty[q];
    }
    int start = 0;
    for (int q = 1; q < m; ++q)
      if (cv[q] < cv[start]) start = q;
    for (int q = 0; q < m; ++q)
      for (int r = q + 1; r < m; ++r)
        if (cv[q] == cv[r]) {
          *err = "cell " + std::to_string(a) + " touches its own periodic image";
          return VX_ERR_DEGENERATE_SEEDS;
        }
    face_he[a] = h;
    for (int q = 0; q < m; ++q) {
      const int s = (start + q) % m, t = (start + q + 1) % m;
      const int32_t ox = ckx[t] - ckx[s], oy = cky[t] - cky[s];
      if (ox < -1 || ox > 1 || oy < -1 || oy > 1) {
        *err = "an edge spans more than one box copy";
        return VX_ERR_DEGENERATE_SEEDS;
      }
      int32_t* r = he + 8 * (h + q);
      r[0] = h + (q + m - 1) % m;
      r[1] = h + (q + 1) % m;
      r[2] = -1;
      r[3] = cv[s];
      r[4] = cv[t];
      r[5] = a;
      r[6] = ox;
      r[7] = oy;
    }
    h += m;
  }
  // Twins by (src, tgt, offset): the half-edges listed by source vertex
  // (counting sort), then the twin of s -> t is the half-edge out of t that
  // points back to s with the opposite offset.
  std::vector<int32_t> ostart(V + 1, 0), olist(HE);
  for (size_t q = 0; q < HE; ++q) ostart[he[8 * q + 3] + 1]++;
  for (int v = 0; v < V; ++v) ostart[v + 1] += ostart[v];
  {
    std::vector<int32_t> fill(ostart.begin(), ostart.end() - 1);
    for (size_t q = 0; q < HE; ++q) olist[fill[he[8 * q + 3]]++] = (int32_t)q;
  }
  auto same_dir = [&](int32_t p, int32_t q) {
    const int32_t *a = he + 8 * (size_t)p, *b = he + 8 * (size_t)q;
    return a[4] == b[4] && a[6] == b[6] && a[7] == b[7];
  };
  for (int v = 0; v < V; ++v)
    for (int32_t x = ostart[v]; x < ostart[v + 1]; ++x)
      for (int32_t y = x + 1; y < ostart[v + 1]; ++y)
        if (same_dir(olist[x], olist[y])) {
          *err = "duplicate half-edge";
          return VX_ERR_DEGENERATE_SEEDS;
        }
  for (size_t q = 0; q < HE; ++q) {
    int32_t* r = he + 8 * q;
    int32_t tw = -1;
    for (int32_t x = ostart[r[4]]; x < ostart[r[4] + 1] && tw < 0; ++x) {
      const int32_t* c = he + 8 * (size_t)olist[x];
      if (c[4] == r[3] && c[6] == -r[6] && c[7] == -r[7]) tw = olist[x];
    }
    if (tw < 0) {
      *err = "half-edge without twin";
      return VX_ERR_DEGENERATE_SEEDS;
    }
    r[2] = tw;
  }
  int32_t e = 0;
  for (size_t q = 0; q < HE; ++q) edge_id[q] = -1;
  for (size_t q = 0; q < HE; ++q) {
    const int32_t tw = he[8 * q + 2];
    if ((int32_t)q < tw) {
      edge_id[q] = edge_id[tw] = e++;
    }
  }
  // Nearly cocircular seeds: a Voronoi edge of (almost) zero length.
  double lmin2 = INFINITY;
  for (size_t q = 0; q < HE; ++q) {
    const int32_t* r = he + 8 * q;
    const double dx = vert[2 * r[4]] + r[6] * Lx - vert[2 * r[3]];
    const double dy = vert[2 * r[4] + 1] + r[7] * Ly - vert[2 * r[3] + 1];
    lmin2 = std::min(lmin2, dx * dx + dy * dy);
  }
  const double thr = 1e-9 * std::sqrt(Lx * Ly / n);
  if (std::sqrt(lmin2) < thr) {
    *err = "nearly cocircular seeds (a Voronoi edge of zero length)";
    return VX_ERR_DEGENERATE_SEEDS;
  }
  return VX_OK;
}

// Position of cell (x, y) of a 2^k x 2^k grid along the Hilbert curve:
// descend the quadrant tree, adding the number of cells in the quadrants the
// curve visits before this one and turning the frame so that every sub-square
// is traversed from its entry corner.
static uint64_t hilbert_index(uint32_t side, uint32_t x, uint32_t y) {
  uint64_t d = 0;
  for (uint32_t s = side >> 1; s > 0; s >>= 1) {
    const uint32_t rx = (x & s) ? 1u : 0u, ry = (y & s) ? 1u : 0u;
    d += (uint64_t)s * s * ((3u * rx) ^ ry);
    if (ry == 0) {
      if (rx == 1) {
        x = side - 1 - x;
        y = side - 1 - y;
      }
      const uint32_t t = x;
      x = y;
      y = t;
    }
  }
  return d;
}

void seed_order(const double* seeds, int n, double Lx, double Ly, int32_t* order) {
  const uint32_t side = 1u << 16;
  std::vector<std::pair<uint64_t, int32_t>> key(n);
  for (int i = 0; i < n; ++i) {
    const double fx = seeds[2 * i] / Lx, fy = seeds[2 * i + 1] / Ly;
    const uint32_t x = (uint32_t)std::min<double>(side - 1, std::max(0.0, fx * side));
    const uint32_t y = (uint32_t)std::min<double>(side - 1, std::max(0.0, fy * side));
    key[i] = {hilbert_index(side, x, y), i};
  }
  std::sort(key.begin(), key.end());
  for (int i = 0; i < n; ++i) order[i] = key[i].second;
}

}  // namespace vx
