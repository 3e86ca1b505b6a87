"""Pins of the oracle's energy, forces, Hessian and costs (CPU only).

Closed forms (regular hexagon, periodic honeycomb), invariants (areas tile
the box, each edge is in two perimeters, forces sum to zero, translation
invariance, relabelling through permuted seeds, Hessian symmetry and
translation null space), central finite
differences, and an independent area formula.  The last tests plant
plausible mistakes in the oracle and check that these pins catch them.
"""
import math

import numpy as np
import pytest

import vx_inputs as vi
from oracle import mesh, model
from oracle.mesh import HE_FACE, HE_NEXT, HE_OFFX, HE_OFFY, HE_SRC


def tissue(n=20, stream=31, p0=3.7, **kw):
    c = vi.small_tissue(n, stream, p0=p0, **kw)
    t = mesh.build_periodic_voronoi(c["seeds"], c["Lx"], c["Ly"])
    p = {k: c[k] for k in ("KA", "KP", "A0", "P0", "lam")}
    return c, t, p


def hetero(t, p, rng):
    """Per-cell parameters, so that every index of every term matters."""
    n = t["n"]
    q = dict(p)
    q["KA"] = rng.uniform(0.5, 2.0, n)
    q["KP"] = rng.uniform(0.5, 2.0, n)
    q["A0"] = rng.uniform(0.8, 1.2, n)
    q["P0"] = rng.uniform(3.4, 4.0, n)
    return q


def fd_forces(X, t, p, h=1e-6):
    F = np.zeros_like(X)
    for i in range(X.shape[0]):
        for c in range(2):
            Xp = X.copy(); Xp[i, c] += h
            Xm = X.copy(); Xm[i, c] -= h
            F[i, c] = -(model.energy(Xp, t, p) - model.energy(Xm, t, p)) / (2 * h)
    return F


def test_hexagon_and_honeycomb_closed_form():
    seeds, Lx, Ly = vi.lattice_seeds(4, 6, a=1.0)
    t = mesh.build_periodic_voronoi(seeds, Lx, Ly)
    n = t["n"]
    s = 1.0 / math.sqrt(3.0)
    KA, KP, A0, P0, lam = 1.3, 0.7, 0.9, 3.5, 0.04
    p = dict(KA=KA, KP=KP, A0=A0, P0=P0, lam=lam)
    A = 1.5 * math.sqrt(3.0) * s * s
    E = n * (KA * (A - A0) ** 2 + KP * (6 * s - P0) ** 2) + 3 * n * lam * s
    assert abs(model.energy(t["vert"], t, p) - E) < 1e-12 * E
    # a periodic honeycomb is in force balance for any parameters
    F = model.forces(t["vert"], t, p)
    assert np.abs(F).max() < 1e-12


@pytest.mark.parametrize("stream", [31, 32, 33])
def test_invariants(stream):
    c, t, p = tissue(40, stream)
    X = t["vert"]
    g = model.geometry(X, t)
    assert abs(g["A"].sum() - c["Lx"] * c["Ly"]) < 1e-11 * c["Lx"] * c["Ly"]
    rep = model.edge_rep(t)
    assert abs(g["P"].sum() - 2 * g["ell"][rep].sum()) < 1e-11 * g["P"].sum()
    q = hetero(t, p, np.random.default_rng(stream))
    F = model.forces(X, t, q)
    assert np.abs(F.sum(axis=0)).max() < 1e-12 * np.abs(F).max() * X.shape[0]
    shift = np.array([0.3, -0.7])
    assert abs(model.energy(X + shift, t, q) - model.energy(X, t, q)) < 1e-12 * abs(model.energy(X, t, q))
    assert np.abs(model.forces(X + shift, t, q) - F).max() < 1e-11 * np.abs(F).max()


def _match(P, Q, L):
    """Index map m with Q[m[i]] == P[i] (points wrapped into the box)."""
    key = lambda Z: [tuple(np.round(np.mod(z, L) / L * 1e9).astype(np.int64)) for z in Z]
    kq = {k: j for j, k in enumerate(key(Q))}
    return np.array([kq[k] for k in key(P)])


def test_relabelling_invariance():
    """Building from permuted seeds gives the same tissue under other labels:
    the same energy, areas and forces carried by the matching cells and
    vertices, with per-cell and per-edge parameters moved along."""
    c, t, p = tissue(40, 35)
    rng = np.random.default_rng(35)
    q = hetero(t, p, rng)
    q["lam"] = rng.uniform(0.02, 0.1, 3 * t["n"])
    pi = rng.permutation(t["n"])
    t2 = mesh.build_periodic_voronoi(c["seeds"][pi], c["Lx"], c["Ly"])
    L = np.array([c["Lx"], c["Ly"]])
    vm = _match(t["vert"], t2["vert"], L)            # vertex i -> vertex vm[i] of t2
    def mids(tt):
        rep = model.edge_rep(tt)
        d = model.geometry(tt["vert"], tt)["d"][rep]
        return tt["vert"][tt["he"][rep, HE_SRC]] + 0.5 * d
    em = _match(mids(t), mids(t2), L)               # edge e -> edge em[e] of t2
    q2 = {k: (v[pi] if np.ndim(v) else v) for k, v in q.items() if k != "lam"}
    lam2 = np.empty_like(q["lam"])
    lam2[em] = q["lam"]
    q2["lam"] = lam2
    E1, E2 = model.energy(t["vert"], t, q), model.energy(t2["vert"], t2, q2)
    assert abs(E1 - E2) < 1e-12 * abs(E1)
    A1, A2 = model.geometry(t["vert"], t)["A"], model.geometry(t2["vert"], t2)["A"]
    assert np.abs(A2 - A1[pi]).max() < 1e-12 * np.abs(A1).max()
    F1, F2 = model.forces(t["vert"], t, q), model.forces(t2["vert"], t2, q2)
    assert np.abs(F2[vm] - F1).max() < 1e-10 * np.abs(F1).max()


def test_area_independent_formula():
    """Shoelace areas equal the triangle-fan areas about each cell's seed."""
    c, t, p = tissue(30, 34)
    L = np.array([c["Lx"], c["Ly"]])
    he = t["he"]
    g = model.geometry(t["vert"], t)
    for a in range(t["n"]):
        h0 = t["face_he"][a]
        hs, h = [], h0
        while True:
            hs.append(h)
            h = he[h, HE_NEXT]
            if h == h0:
                break
        k = np.zeros(2)
        pts = []
        for h in hs:
            pts.append(t["vert"][he[h, HE_SRC]] + k * L)
            k = k + he[h, HE_OFFX:HE_OFFY + 1]
        pts = np.array(pts)
        s = c["seeds"][a] + L * np.round((pts[0] - c["seeds"][a]) / L)
        fan = 0.0
        for i in range(len(pts)):
            u, w = pts[i] - s, pts[(i + 1) % len(pts)] - s
            fan += 0.5 * abs(u[0] * w[1] - u[1] * w[0])
        assert abs(fan - g["A"][a]) < 1e-12 * g["A"][a]


@pytest.mark.parametrize("n,stream", [(8, 41), (14, 42), (20, 43)])
def test_forces_central_fd(n, stream):
    c, t, p = tissue(n, stream)
    q = hetero(t, p, np.random.default_rng(stream))
    q["lam"] = np.random.default_rng(stream + 1).uniform(0.0, 0.1, 3 * n)
    X = t["vert"]
    F = model.forces(X, t, q)
    Ffd = fd_forces(X, t, q)
    assert np.abs(F - Ffd).max() < 1e-7 * np.abs(F).max()


def test_hessian_fd_symmetry_nullspace():
    c, t, p = tissue(16, 44)
    q = hetero(t, p, np.random.default_rng(4))
    X = t["vert"]
    H = model.hessian(X, t, q, dense=True)
    assert np.abs(H - H.T).max() < 1e-12 * np.abs(H).max()
    V = X.shape[0]
    tx = np.tile([1.0, 0.0], V)
    ty = np.tile([0.0, 1.0], V)
    assert np.abs(H @ tx).max() < 1e-11 * np.abs(H).max()
    assert np.abs(H @ ty).max() < 1e-11 * np.abs(H).max()
    rng = np.random.default_rng(5)
    v = rng.standard_normal(X.shape)
    errs = []
    for h in (1e-4, 1e-5):
        fd = -(model.forces(X + h * v, t, q) - model.forces(X - h * v, t, q)) / (2 * h)
        errs.append(np.abs(model.hvp(X, t, q, v) - fd).max())
    # central FD error is O(h^2): a factor ~100 per decade of h
    assert errs[1] < 2e-2 * errs[0] + 1e-9
    assert errs[1] < 1e-5 * np.abs(model.hvp(X, t, q, v)).max()


def test_mixed_derivatives_fd():
    """(d^2E/dX dtheta)^T v against FD of d_theta E along v."""
    c, t, p = tissue(12, 45)
    q = hetero(t, p, np.random.default_rng(6))
    X = t["vert"]
    v = np.random.default_rng(7).standard_normal(X.shape)
    m = model.mixed_vjp(X, t, q, v)
    h = 1e-6
    dp, dm = model.dE_dtheta(X + h * v, t, q), model.dE_dtheta(X - h * v, t, q)
    for k in ("lam", "A0", "P0"):
        fd = (dp[k] - dm[k]) / (2 * h)
        assert np.abs(m[k] - fd).max() < 1e-6 * (np.abs(fd).max() + 1e-12)
    # d_theta E against FD of E in theta
    d = model.dE_dtheta(X, t, q)
    for k in ("A0", "P0"):
        for a in (0, 5):
            q1, q2 = dict(q), dict(q)
            q1[k] = q[k].copy(); q1[k][a] += h
            q2[k] = q[k].copy(); q2[k][a] -= h
            fd = (model.energy(X, t, q1) - model.energy(X, t, q2)) / (2 * h)
            assert abs(fd - d[k][a]) < 1e-6 * max(1.0, abs(fd))


def test_costs_fd():
    c, t, p = tissue(15, 46)
    X = t["vert"]
    rng = np.random.default_rng(8)
    Xt = X + 0.05 * rng.standard_normal(X.shape)
    C, G = model.cost_v2v(X, Xt, t)
    D = (X - Xt)
    assert abs(C - (D * D).sum() / (2 * X.shape[0])) < 1e-15
    # minimum image: shifting a target by a box period changes nothing
    Xt2 = Xt.copy(); Xt2[3, 0] += c["Lx"]
    assert abs(model.cost_v2v(X, Xt2, t)[0] - C) < 1e-15
    Ca, Ga = model.shape_tensor_anisotropy(X, t, (0.1, -0.05))
    h = 1e-6
    for i in (0, 7, 20):
        for k in range(2):
            Xp = X.copy(); Xp[i, k] += h
            Xm = X.copy(); Xm[i, k] -= h
            fd = (model.shape_tensor_anisotropy(Xp, t, (0.1, -0.05))[0]
                  - model.shape_tensor_anisotropy(Xm, t, (0.1, -0.05))[0]) / (2 * h)
            assert abs(fd - Ga[i, k]) < 1e-6 * np.abs(Ga).max()
    # a regular honeycomb is isotropic: q = 0
    seeds, Lx, Ly = vi.lattice_seeds(4, 6)
    th = mesh.build_periodic_voronoi(seeds, Lx, Ly)
    Ch, _ = model.shape_tensor_anisotropy(th["vert"], th, (0.0, 0.0))
    assert Ch < 1e-24


# ------------------------------------------------- planted mistakes (CPU)

def test_planted_dropped_offset_is_caught(monkeypatch):
    """Dropping the periodic offset in the edge vectors breaks the tiling
    invariant sum A = Lx Ly."""
    c, t, p = tissue(30, 47)
    orig = model.geometry

    def broken(X, tt):
        he = tt["he"].copy()
        he[:, HE_OFFX:HE_OFFY + 1] = 0
        t2 = dict(tt); t2["he"] = he
        t2.pop("_kcorner", None)
        return orig(X, t2)

    monkeypatch.setattr(model, "geometry", broken)
    g = model.geometry(t["vert"], t)
    assert abs(g["A"].sum() - c["Lx"] * c["Ly"]) > 1e-3


def test_planted_sign_error_is_caught(monkeypatch):
    """A sign error in the shoelace gradient fails the FD pin."""
    c, t, p = tissue(10, 48)
    orig = model.cell_gradients

    def broken(X, tt):
        g, dA, dP, u = orig(X, tt)
        return g, -dA, dP, u

    monkeypatch.setattr(model, "cell_gradients", broken)
    X = t["vert"]
    F = model.forces(X, t, p)
    assert np.abs(F - fd_forces(X, t, p)).max() > 1e-4 * np.abs(F).max()


def test_planted_wrong_edge_index_is_caught(monkeypatch):
    """Tensions attached to the wrong edges fail the FD pin."""
    c, t, p = tissue(10, 49)
    X = t["vert"]
    orig = model.edge_rep

    def broken(tt):
        return np.roll(orig(tt), 1)

    Ffd = fd_forces(X, t, p)
    monkeypatch.setattr(model, "edge_rep", broken)
    F = model.forces(X, t, p)
    assert np.abs(F - Ffd).max() > 1e-4 * np.abs(F).max()
