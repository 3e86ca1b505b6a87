"""Oracle: periodic Voronoi tessellation -> canonical half-edge tables.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this.

Follows Methods, "Mesh initialization" and "Periodic mode": the seeds are
replicated into the eight neighbouring copies of the box, the tessellation of
the 3 x 3 replicated point set is computed with Qhull (``scipy.spatial``,
the library the paper uses), only the polygons of the primary seeds are kept,
and every half-edge whose target lies in another copy of the box gets that
copy as its offset (Methods, "System state and data structure": ``heTable``
columns prev, next, twin, source, target, face, offx, offy).

Qhull's Delaunay triangulation is used as the library step (it is the dual
that ``scipy.spatial.Voronoi`` is built from); every Voronoi vertex is the
circumcentre of one Delaunay triangle of the torus.

Canonical indexing (the paper does not fix one; both this oracle and the CUDA
library's host builder produce exactly this):

* face alpha is seed alpha;
* a vertex is a Delaunay triangle of the torus, written as three (seed,
  image-shift) corners in counter-clockwise order, translated so that its
  first corner has shift (0, 0); of the three rotations the lexicographically
  smallest tuple (a, b, sbx, sby, c, scx, scy) is the key; vertices are
  numbered in increasing key order;
* a vertex position is the circumcentre of its key triangle, wrapped into
  [0, Lx) x [0, Ly);
* the half-edges of face alpha are contiguous, faces in increasing order,
  each face's cycle counter-clockwise starting at its smallest vertex index;
* an undirected edge takes the rank of its smaller half-edge index as id.

A configuration is rejected as degenerate when a cell touches its own
periodic image (a vertex would repeat inside one face), when a cell's
vertices span more than one box copy (|offset| > 1), or when a Voronoi edge is
shorter than 1e-9 sqrt(Lx Ly / n) (four nearly cocircular seeds, where the
triangulation is not unique).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.spatial import Delaunay

HE_PREV, HE_NEXT, HE_TWIN, HE_SRC, HE_TGT, HE_FACE, HE_OFFX, HE_OFFY = range(8)

DEGENERATE_EDGE_FACTOR = 1e-9


class DegenerateSeeds(ValueError):
    pass


def _circumcentre(p, q, r):
    """Circumcentre of triangle (p, q, r), computed relative to p."""
    bx, by = q[0] - p[0], q[1] - p[1]
    cx, cy = r[0] - p[0], r[1] - p[1]
    d = 2.0 * (bx * cy - by * cx)
    b2 = bx * bx + by * by
    c2 = cx * cx + cy * cy
    ux = (cy * b2 - by * c2) / d
    uy = (bx * c2 - cx * b2) / d
    return (p[0] + ux, p[1] + uy)


def _canonical_key(corners):
    """corners: three (seed, sx, sy), CCW.  Returns (key, translation t) with
    the key the smallest normalised rotation; t is the integer shift that was
    subtracted from the corners to reach the key's frame."""
    best = None
    for r in range(3):
        rot = corners[r:] + corners[:r]
        a, ax, ay = rot[0]
        key = (a,
               rot[1][0], rot[1][1] - ax, rot[1][2] - ay,
               rot[2][0], rot[2][1] - ax, rot[2][2] - ay)
        if best is None or key < best[0]:
            best = (key, (ax, ay))
    return best


def build_periodic_voronoi(seeds, Lx, Ly):
    """Periodic Voronoi tessellation of ``seeds`` (n x 2) in [0,Lx) x [0,Ly).

    Returns a dict with
      vert   float64 [V, 2]   vertex positions (vertTable)
      he     int32   [HE, 8]  prev, next, twin, src, tgt, face, offx, offy
      face_he int32  [n]      first half-edge of each face
      edge_id int32  [HE]     undirected edge of each half-edge
    """
    seeds = np.asarray(seeds, dtype=np.float64)
    n = seeds.shape[0]
    if n < 3:
        raise DegenerateSeeds("need at least 3 seeds")
    L = (float(Lx), float(Ly))

    # 3 x 3 replication (Methods, "Mesh initialization").
    shifts = [(sx, sy) for sx in (-1, 0, 1) for sy in (-1, 0, 1)]
    pts = np.concatenate([seeds + np.array([sx * L[0], sy * L[1]]) for sx, sy in shifts])
    img_seed = np.tile(np.arange(n), len(shifts))
    img_sx = np.repeat([s[0] for s in shifts], n)
    img_sy = np.repeat([s[1] for s in shifts], n)

    tri = Delaunay(pts)
    simplices = tri.simplices

    def corner(p):
        return (int(img_seed[p]), int(img_sx[p]), int(img_sy[p]))

    def seed_pos(c):
        s, sx, sy = c
        return (seeds[s, 0] + sx * L[0], seeds[s, 1] + sy * L[1])

    # Every triangle of the torus has a representative touching the primary
    # copy; collect those, in CCW order, with their canonical keys.
    keys = {}
    incident = [[] for _ in range(n)]  # per primary seed: (key, t, corners)
    for simp in simplices:
        cs = [corner(p) for p in simp]
        if not any(c[1] == 0 and c[2] == 0 for c in cs):
            continue
        p0, p1, p2 = (seed_pos(c) for c in cs)
        orient = (p1[0] - p0[0]) * (p2[1] - p0[1]) - (p1[1] - p0[1]) * (p2[0] - p0[0])
        if orient < 0:
            cs = [cs[0], cs[2], cs[1]]
        key, t = _canonical_key(cs)
        keys[key] = True
        for c in cs:
            if c[1] == 0 and c[2] == 0:
                incident[c[0]].append((key, t))

    vkeys = sorted(keys)
    vindex = {k: i for i, k in enumerate(vkeys)}
    V = len(vkeys)

    # Vertex positions: circumcentre of the key triangle, wrapped into the box.
    vert = np.zeros((V, 2))
    wrap = np.zeros((V, 2), dtype=np.int64)
    for i, k in enumerate(vkeys):
        a, b, sbx, sby, c, scx, scy = k
        cc = _circumcentre(seed_pos((a, 0, 0)), seed_pos((b, sbx, sby)), seed_pos((c, scx, scy)))
        w = (math.floor(cc[0] / L[0]), math.floor(cc[1] / L[1]))
        vert[i] = (cc[0] - w[0] * L[0], cc[1] - w[1] * L[1])
        wrap[i] = w

    # Faces: the corners of cell alpha, sorted CCW by angle around seed alpha.
    # The representative touching alpha is the key triangle translated by t,
    # so a corner's unwrapped position in alpha's frame is vert + (wrap + t) L.
    faces = []
    for alpha in range(n):
        corners = []
        for key, t in incident[alpha]:
            v = vindex[key]
            k = (int(wrap[v, 0] + t[0]), int(wrap[v, 1] + t[1]))
            ux = vert[v, 0] + k[0] * L[0]
            uy = vert[v, 1] + k[1] * L[1]
            ang = math.atan2(uy - seeds[alpha, 1], ux - seeds[alpha, 0])
            corners.append((ang, v, k))
        corners.sort()
        vs = [c[1] for c in corners]
        if len(set(vs)) != len(vs):
            raise DegenerateSeeds(f"cell {alpha} touches its own periodic image")
        if len(vs) < 3:
            raise DegenerateSeeds(f"cell {alpha} has fewer than 3 vertices")
        start = int(np.argmin(vs))
        corners = corners[start:] + corners[:start]
        faces.append([(c[1], c[2]) for c in corners])

    HE = sum(len(f) for f in faces)
    he = np.zeros((HE, 8), dtype=np.int32)
    face_he = np.zeros(n, dtype=np.int32)
    h = 0
    for alpha, f in enumerate(faces):
        face_he[alpha] = h
        m = len(f)
        for i in range(m):
            (vs_, ks), (vt, kt) = f[i], f[(i + 1) % m]
            off = (kt[0] - ks[0], kt[1] - ks[1])
            if abs(off[0]) > 1 or abs(off[1]) > 1:
                raise DegenerateSeeds("an edge spans more than one box copy")
            he[h + i] = (h + (i - 1) % m, h + (i + 1) % m, -1, vs_, vt, alpha, off[0], off[1])
        h += m

    index = {}
    for i in range(HE):
        k = (int(he[i, HE_SRC]), int(he[i, HE_TGT]), int(he[i, HE_OFFX]), int(he[i, HE_OFFY]))
        if k in index:
            raise DegenerateSeeds("duplicate half-edge")
        index[k] = i
    for i in range(HE):
        k = (int(he[i, HE_TGT]), int(he[i, HE_SRC]), -int(he[i, HE_OFFX]), -int(he[i, HE_OFFY]))
        if k not in index:
            raise DegenerateSeeds("half-edge without twin")
        he[i, HE_TWIN] = index[k]

    edge_id = np.full(HE, -1, dtype=np.int32)
    e = 0
    for i in range(HE):
        j = int(he[i, HE_TWIN])
        if i < j:
            edge_id[i] = edge_id[j] = e
            e += 1

    # Nearly cocircular seeds: a Voronoi edge of (almost) zero length.
    d = vert[he[:, HE_TGT]] + he[:, HE_OFFX:HE_OFFY + 1] * np.array(L) - vert[he[:, HE_SRC]]
    lmin = float(np.sqrt((d * d).sum(axis=1)).min())
    if lmin < DEGENERATE_EDGE_FACTOR * math.sqrt(L[0] * L[1] / n):
        raise DegenerateSeeds("nearly cocircular seeds (a Voronoi edge of zero length)")

    if V != 2 * n or HE != 6 * n:
        raise DegenerateSeeds(f"not a 3-valent torus tessellation (V={V}, HE={HE}, n={n})")
    return dict(vert=vert, he=he, face_he=face_he, edge_id=edge_id, n=n, Lx=L[0], Ly=L[1])


def brute_force_delaunay(seeds, Lx, Ly):
    """Triangles of the torus Delaunay triangulation by the empty-circumcircle
    test over all triples of the 3 x 3 replicated seeds (O(n^4); tiny n only).
    Returns the set of canonical vertex keys."""
    seeds = np.asarray(seeds, dtype=np.float64)
    n = seeds.shape[0]
    pts, cs = [], []
    for sx in (-1, 0, 1):
        for sy in (-1, 0, 1):
            for s in range(n):
                pts.append((seeds[s, 0] + sx * Lx, seeds[s, 1] + sy * Ly))
                cs.append((s, sx, sy))
    # Points of a 5 x 5 replication are the witnesses of emptiness.
    wit = [(seeds[s, 0] + sx * Lx, seeds[s, 1] + sy * Ly)
           for sx in range(-2, 3) for sy in range(-2, 3) for s in range(n)]
    wit = np.asarray(wit)
    keys = set()
    P = len(pts)
    prim = [i for i in range(P) if cs[i][1] == 0 and cs[i][2] == 0]
    for i in prim:
        for j in range(P):
            if j == i:
                continue
            for k in range(j + 1, P):
                if k == i:
                    continue
                p, q, r = pts[i], pts[j], pts[k]
                orient = (q[0] - p[0]) * (r[1] - p[1]) - (q[1] - p[1]) * (r[0] - p[0])
                if abs(orient) < 1e-14:
                    continue
                c = _circumcentre(p, q, r)
                rad2 = (p[0] - c[0]) ** 2 + (p[1] - c[1]) ** 2
                d2 = (wit[:, 0] - c[0]) ** 2 + (wit[:, 1] - c[1]) ** 2
                if np.sum(d2 < rad2 * (1 - 1e-12)) > 0:
                    continue
                tri = [cs[i], cs[j], cs[k]] if orient > 0 else [cs[i], cs[k], cs[j]]
                keys.add(_canonical_key(tri)[0])
    return keys
