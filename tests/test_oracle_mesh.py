"""Pins of the oracle's periodic Voronoi builder (CPU only).

The oracle builder is checked against brute force (the empty-circumcircle
definition of the Delaunay triangulation, dual of the Voronoi diagram), the
regular honeycomb of a triangular lattice, the Voronoi property itself and
the combinatorial invariants of a 3-valent tessellation of the torus.
"""
import math

import numpy as np
import pytest

import vx_inputs as vi
from oracle import mesh, model
from oracle.mesh import HE_FACE, HE_NEXT, HE_OFFX, HE_OFFY, HE_PREV, HE_SRC, HE_TGT, HE_TWIN


def build(c):
    return mesh.build_periodic_voronoi(c["seeds"], c["Lx"], c["Ly"])


def check_half_edge_invariants(t):
    he = t["he"]
    HE = he.shape[0]
    h = np.arange(HE)
    assert np.array_equal(he[he[:, HE_NEXT], HE_PREV], h)
    assert np.array_equal(he[he[:, HE_TWIN], HE_TWIN], h)
    assert np.all(he[:, HE_TWIN] != h)
    assert np.array_equal(he[he[:, HE_TWIN], HE_SRC], he[:, HE_TGT])
    assert np.array_equal(he[he[:, HE_TWIN], HE_OFFX], -he[:, HE_OFFX])
    assert np.array_equal(he[he[:, HE_TWIN], HE_OFFY], -he[:, HE_OFFY])
    assert np.array_equal(he[he[:, HE_NEXT], HE_SRC], he[:, HE_TGT])
    assert np.array_equal(he[he[:, HE_NEXT], HE_FACE], he[:, HE_FACE])
    assert np.all(np.abs(he[:, HE_OFFX:]) <= 1)
    # 3-valent: every vertex is the source of exactly three half-edges.
    V = t["vert"].shape[0]
    assert np.all(np.bincount(he[:, HE_SRC], minlength=V) == 3)
    # Edge ids: both half-edges of an edge share it; ids cover 0..E-1.
    eid = t["edge_id"]
    assert np.array_equal(eid[he[:, HE_TWIN]], eid)
    assert sorted(set(eid.tolist())) == list(range(HE // 2))


@pytest.mark.parametrize("n,stream,aspect", [(12, 1, 1.0), (50, 2, 1.0), (100, 3, 2.5), (300, 4, 0.4)])
def test_counts_and_invariants(n, stream, aspect):
    c = vi.small_tissue(n, stream, aspect=aspect)
    t = build(c)
    V, HE = t["vert"].shape[0], t["he"].shape[0]
    assert V == 2 * n and HE == 6 * n            # Euler: chi = 0 on the torus
    check_half_edge_invariants(t)
    g = model.geometry(t["vert"], t)
    assert np.all(g["A"] > 0)
    assert abs(g["A"].sum() - c["Lx"] * c["Ly"]) < 1e-10 * c["Lx"] * c["Ly"]
    assert np.all(t["vert"] >= 0) and np.all(t["vert"][:, 0] < c["Lx"]) and np.all(t["vert"][:, 1] < c["Ly"])


def test_canonical_order():
    t = build(vi.small_tissue(60, 5))
    he, face_he = t["he"], t["face_he"]
    assert np.all(np.diff(he[:, HE_FACE]) >= 0)
    for a in range(t["n"]):
        h0 = face_he[a]
        hs = [h0]
        while he[hs[-1], HE_NEXT] != h0:
            hs.append(he[hs[-1], HE_NEXT])
        assert hs == list(range(h0, h0 + len(hs)))
        assert he[h0, HE_SRC] == min(he[hs, HE_SRC])
    rep = model.edge_rep(t)
    assert np.all(np.diff(rep) > 0)   # edge id = rank of its smaller half-edge


def test_voronoi_property():
    """Each vertex is equidistant from the seeds of its three cells and no
    seed image is closer (the definition of a Voronoi vertex)."""
    c = vi.small_tissue(80, 6)
    t = build(c)
    L = np.array([c["Lx"], c["Ly"]])
    seeds = c["seeds"]
    imgs = np.concatenate([seeds + np.array([sx, sy]) * L for sx in (-1, 0, 1) for sy in (-1, 0, 1)])
    he = t["he"]
    for v in range(t["vert"].shape[0]):
        x = t["vert"][v]
        faces = he[he[:, HE_SRC] == v, HE_FACE]
        d = np.sqrt(((imgs - x) ** 2).sum(axis=1))
        dmin = d.min()
        owner = np.nonzero(d < dmin * (1 + 1e-9))[0] % t["n"]
        assert sorted(set(owner.tolist())) == sorted(set(faces.tolist()))
    # every seed lies inside its own cell (polygon contains seed, CCW)
    for a in range(t["n"]):
        h0 = t["face_he"][a]
        hs = [h0]
        while he[hs[-1], HE_NEXT] != h0:
            hs.append(he[hs[-1], HE_NEXT])
        k = np.zeros(2)
        pts = []
        for h in hs:
            pts.append(t["vert"][he[h, HE_SRC]] + k * L)
            k = k + he[h, HE_OFFX:HE_OFFY + 1]
        pts = np.array(pts)
        s = seeds[a]
        s = s + L * np.round((pts[0] - s) / L)
        for i in range(len(pts)):
            e = pts[(i + 1) % len(pts)] - pts[i]
            w = s - pts[i]
            assert e[0] * w[1] - e[1] * w[0] > 0


@pytest.mark.parametrize("n,stream", [(5, 21), (7, 22), (9, 23), (12, 24)])
def test_brute_force_delaunay(n, stream):
    c = vi.small_tissue(n, stream)
    try:
        t = build(c)
    except mesh.DegenerateSeeds:
        pytest.skip("degenerate tiny tessellation")
    keys = mesh.brute_force_delaunay(c["seeds"], c["Lx"], c["Ly"])
    # reconstruct the keys of the built vertices from the faces around them
    he = t["he"]
    V = t["vert"].shape[0]
    assert len(keys) == V
    for v in range(V):
        faces = sorted(set(he[he[:, HE_SRC] == v, HE_FACE].tolist()))
        assert any(sorted({k[0], k[1], k[4]}) == faces for k in keys)


def test_honeycomb_closed_form():
    """Triangular lattice seeds give the regular honeycomb: every cell a
    hexagon of side s = a/sqrt(3), area (3 sqrt 3 / 2) s^2, perimeter 6 s."""
    seeds, Lx, Ly = vi.lattice_seeds(6, 8, a=1.0)
    t = mesh.build_periodic_voronoi(seeds, Lx, Ly)
    s = 1.0 / math.sqrt(3.0)
    g = model.geometry(t["vert"], t)
    assert np.all(np.bincount(t["he"][:, HE_FACE]) == 6)
    assert np.allclose(g["A"], 1.5 * math.sqrt(3.0) * s * s, rtol=1e-12)
    assert np.allclose(g["P"], 6 * s, rtol=1e-12)
    assert np.allclose(g["ell"], s, rtol=1e-12)


def test_degenerate_rejected():
    seeds, Lx, Ly = vi.lattice_seeds(4, 4, a=1.0, shift=(0.0, 0.0))
    # a square lattice: four cocircular seeds everywhere
    sq = np.array([(i + 0.25, j + 0.25) for i in range(5) for j in range(5)], dtype=float)
    with pytest.raises(mesh.DegenerateSeeds):
        mesh.build_periodic_voronoi(sq, 5.0, 5.0)
