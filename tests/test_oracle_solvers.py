"""Pins of the oracle's minimisers, T1 transitions and equilibrium gradients.

The minimisers are checked for monotone energy (GD), convergence, recovery
of the honeycomb after a perturbation, and conservation of the centroid (the
forces sum to zero).  T1 rewiring is checked against the half-edge
invariants and the tiling identity sum A = Lx Ly.  The adjoint gradient is
checked against central finite differences of the outer cost with
re-minimisation, equilibrium propagation against the adjoint, and the
centred estimator's O(beta^2) error.  The dense adjoint's indefinite branch
(the eigen-solve MINRES is compared with) is checked by its residual, H lam
taken as a central difference of the forces.
"""
import math

import numpy as np
import pytest

import vx_inputs as vi
from oracle import mesh, model, solvers, topology
from oracle.mesh import HE_FACE, HE_TWIN

from test_oracle_mesh import check_half_edge_invariants


def tissue(n=20, stream=31, p0=3.7, lam_range=(0.02, 0.1)):
    c = vi.small_tissue(n, stream, p0=p0, lam_range=lam_range)
    t = mesh.build_periodic_voronoi(c["seeds"], c["Lx"], c["Ly"])
    p = {k: c[k] for k in ("KA", "KP", "A0", "P0", "lam")}
    return c, t, p


L_MIN = 5e-3


def honeycomb(m=6, k=6):
    seeds, Lx, Ly = vi.lattice_seeds(m, k, a=1.0)
    t = mesh.build_periodic_voronoi(seeds, Lx, Ly)
    A_hex = 1.5 * math.sqrt(3.0) / 3.0
    p = dict(KA=1.0, KP=1.0, A0=A_hex, P0=3.6 * math.sqrt(A_hex), lam=0.02)
    return t, p


def test_gd_energy_non_increasing():
    # a perturbed honeycomb: no edge approaches collapse, so a step below
    # 2 / (largest Hessian eigenvalue) decreases E at every iteration
    t, p = honeycomb()
    X0 = t["vert"] + 0.05 * np.random.default_rng(12).standard_normal(t["vert"].shape)
    o = solvers.MinOpts(method="gd", gd_lr=1e-2, tol=0.0, max_iter=400)
    r = solvers.relax(X0, t, p, o, trace_every=1)
    E = np.array(r.energy_trace)
    assert np.all(np.diff(E) <= 1e-14 * E[0])
    assert E[-1] < E[0]


def test_fire_converges_with_t1():
    c, t, p = tissue(40, 52)
    E0 = model.energy(t["vert"], t, p)
    o = solvers.MinOpts(tol=1e-9, max_iter=20000, dt0=0.01, dt_max=0.5)
    r = solvers.relax(t["vert"], t, p, o, l_min=L_MIN)
    assert r.converged and r.fmax < 1e-9
    assert model.energy(r.X, r.tissue, p) < E0
    check_half_edge_invariants(r.tissue)
    g = model.geometry(r.X, r.tissue)
    assert abs(g["A"].sum() - c["Lx"] * c["Ly"]) < 1e-10 * c["Lx"] * c["Ly"]
    assert g["ell"].min() > L_MIN


def test_centroid_conserved_without_t1():
    c, t, p = tissue(25, 53)
    o = solvers.MinOpts(tol=0.0, max_iter=200, dt0=0.01, dt_max=0.1)
    r = solvers.relax(t["vert"], t, p, o)
    assert np.abs(r.X.mean(axis=0) - t["vert"].mean(axis=0)).max() < 1e-13


def test_perturbed_honeycomb_relaxes_back():
    t, p = honeycomb()
    rng = np.random.default_rng(9)
    dX = 0.02 * rng.standard_normal(t["vert"].shape)
    r = solvers.relax(t["vert"] + dX, t, p, solvers.MinOpts(tol=1e-11, max_iter=50000, dt0=0.01))
    assert r.converged
    expect = t["vert"] + dX.mean(axis=0)
    assert np.abs(r.X - expect).max() < 1e-9


def test_t1_rewiring_invariants():
    c, t, p = tissue(40, 54)
    X = t["vert"]
    rep = model.edge_rep(t)
    he = t["he"]
    done = 0
    for e in range(0, rep.shape[0], 7):
        h = int(rep[e])
        out = topology.t1(X, t, h, 0.05)
        if out is None:
            continue
        Xn, tn = out
        check_half_edge_invariants(tn)
        g0, g1 = model.geometry(X, t), model.geometry(Xn, tn)
        assert abs(g1["A"].sum() - c["Lx"] * c["Ly"]) < 1e-10 * c["Lx"] * c["Ly"]
        s0 = np.bincount(he[:, HE_FACE], minlength=t["n"])
        s1 = np.bincount(tn["he"][:, HE_FACE], minlength=t["n"])
        C1, C2 = he[h, HE_FACE], he[he[h, HE_TWIN], HE_FACE]
        C3, C4 = tn["he"][tn["he"][h, HE_TWIN], HE_FACE], tn["he"][h, HE_FACE]
        assert s1[C1] == s0[C1] - 1 and s1[C2] == s0[C2] - 1
        assert s1[C3] == s0[C3] + 1 and s1[C4] == s0[C4] + 1
        assert abs(topology.edge_length(Xn, tn, h) - 0.05) < 1e-12
        # a second T1 on the new edge gives back the original adjacency
        back = topology.t1(Xn, tn, h, 0.05)
        if back is not None:
            assert np.array_equal(np.bincount(back[1]["he"][:, HE_FACE], minlength=t["n"]), s0)
        done += 1
    assert done >= 5
    # the stretch candidate keeps the midpoint and sets the length
    h = int(rep[3])
    Xs = topology.stretch(X, t, h, 0.123)
    assert abs(topology.edge_length(Xs, t, h) - 0.123) < 1e-12
    assert np.abs(Xs.sum(axis=0) - X.sum(axis=0)).max() < 1e-12


@pytest.fixture(scope="module")
def equilibrium():
    c, t, p = tissue(24, 55)
    o = solvers.MinOpts(tol=1e-11, max_iter=50000, dt0=0.01, dt_max=0.5)
    r = solvers.relax(t["vert"], t, p, o, l_min=L_MIN)
    assert r.converged
    return c, r.tissue, p, r.X


def test_adjoint_matches_fd(equilibrium):
    c, t, p, X = equilibrium
    rng = np.random.default_rng(10)
    Xt = X + 0.02 * rng.standard_normal(X.shape)
    cost = lambda Y: model.cost_v2v(Y, Xt, t)[0]
    _, G = model.cost_v2v(X, Xt, t)
    g, lam, info = solvers.adjoint_grad(X, t, p, G)
    assert info["pd"]
    edges = [0, 9, 33, 50]
    o = solvers.MinOpts(tol=1e-12, max_iter=100000, dt0=0.01, dt_max=0.5)
    fd = solvers.fd_grad_lambda(X, t, p, cost, edges, 1e-5, o)
    assert np.abs(g["lam"][edges] - fd).max() < 1e-5 * np.abs(fd).max()


def test_adjoint_zero_at_target(equilibrium):
    c, t, p, X = equilibrium
    _, G = model.cost_v2v(X, X, t)
    g, _, _ = solvers.adjoint_grad(X, t, p, G)
    assert max(np.abs(v).max() for v in g.values()) == 0.0


def test_ep_centered_second_order(equilibrium):
    """EP matches the adjoint, and its error falls ~4x when beta halves."""
    c, t, p, X = equilibrium
    rng = np.random.default_rng(11)
    Xt = X + 0.02 * rng.standard_normal(X.shape)
    gradC = lambda Y: model.cost_v2v(Y, Xt, t)[1]
    g_adj, _, _ = solvers.adjoint_grad(X, t, p, gradC(X))
    o = solvers.MinOpts(tol=1e-13, max_iter=100000, dt0=0.01, dt_max=0.5)
    errs = []
    for beta in (0.4, 0.2):
        g_ep, _ = solvers.ep_grad(X, t, p, gradC, beta, o, centered=True)
        errs.append(np.linalg.norm(g_ep["lam"] - g_adj["lam"]) / np.linalg.norm(g_adj["lam"]))
    assert errs[1] < 1e-2
    assert 2.5 < errs[0] / errs[1] < 5.5
    g_fw, _ = solvers.ep_grad(X, t, p, gradC, 0.05, o, centered=False)
    assert np.linalg.norm(g_fw["lam"] - g_adj["lam"]) / np.linalg.norm(g_adj["lam"]) < 5e-2


# --------------------------------------------- indefinite adjoint (Methods, "Implicit differentiation")

def _planted(func_name, old, new):
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(getattr(solvers, func_name)))
    assert src.count(old) == 1, f"{old!r} not found once in {func_name}"
    ns = dict(vars(solvers))
    exec(compile(src.replace(old, new), f"<planted {func_name}>", "exec"), ns)
    return ns[func_name]


def _indefinite_case():
    """A 40-cell Voronoi state at p0 = 4.4, not relaxed: its Hessian has
    negative eigenvalues on the translation-free subspace."""
    c = vi.small_tissue(40, 101, p0=4.4, lam_range=(0.02, 0.1))
    t = mesh.build_periodic_voronoi(c["seeds"], c["Lx"], c["Ly"])
    p = {k: c[k] for k in ("KA", "KP", "A0", "P0", "lam")}
    return t, p, t["vert"]


def _check_indefinite_solution(solve):
    """H lam = Pi b on the translation-free subspace, with H lam taken as a
    central difference of the forces (H = -dF/dX), which does not use the
    assembled Hessian, and lam free of translations."""
    t, p, X = _indefinite_case()
    b = np.random.default_rng(102).standard_normal(X.shape)
    lam, info = solve(X, t, p, b)
    assert not info["pd"] and info["min_eig"] < 0
    h = 1e-6 / np.abs(lam).max()
    Hl = -(model.forces(X + h * lam, t, p) - model.forces(X - h * lam, t, p)) / (2 * h)
    Pb = b - b.mean(axis=0)
    assert np.abs(lam.mean(axis=0)).max() < 1e-12 * np.abs(lam).max()
    assert np.linalg.norm(Hl - Pb) < 1e-6 * np.linalg.norm(Pb)


def test_adjoint_solve_on_an_indefinite_hessian():
    _check_indefinite_solution(solvers.adjoint_solve)


@pytest.mark.parametrize("old,new", [
    ("(U.T @ rhs) / w", "(U.T @ rhs) / np.abs(w)"),
    ("lam = U @ ((U.T @ rhs) / w)", "lam = -U @ ((U.T @ rhs) / w)"),
    ("lam = U @ ((U.T @ rhs) / w)", "lam = U.T @ ((U @ rhs) / w)"),
])
def test_indefinite_planted_mistakes_are_caught(old, new):
    with pytest.raises(AssertionError):
        _check_indefinite_solution(_planted("adjoint_solve", old, new))


def test_ep_forward_first_order(equilibrium, ep_grad=None):
    """The one-sided estimator's error against the adjoint falls ~2x when
    beta halves (first order in beta), and the centred one beats it at the
    same beta."""
    ep_grad = ep_grad or solvers.ep_grad
    c, t, p, X = equilibrium
    rng = np.random.default_rng(12)
    Xt = X + 0.02 * rng.standard_normal(X.shape)
    gradC = lambda Y: model.cost_v2v(Y, Xt, t)[1]
    g_adj, _, _ = solvers.adjoint_grad(X, t, p, gradC(X))
    o = solvers.MinOpts(tol=1e-13, max_iter=100000, dt0=0.01, dt_max=0.5)
    nrm = np.linalg.norm(g_adj["lam"])
    errs = []
    for beta in (0.2, 0.1):
        g_fw, _ = ep_grad(X, t, p, gradC, beta, o, centered=False)
        errs.append(np.linalg.norm(g_fw["lam"] - g_adj["lam"]) / nrm)
    assert 1.6 < errs[0] / errs[1] < 2.5
    g_c, _ = ep_grad(X, t, p, gradC, 0.1, o, centered=True)
    assert np.linalg.norm(g_c["lam"] - g_adj["lam"]) / nrm < 0.5 * errs[1]


@pytest.mark.parametrize("old,new", [
    ("return {k: (dp[k] - d0[k]) / beta for k in dp}, (rb,)",
     "return {k: (dp[k] - d0[k]) / (0.5 * beta) for k in dp}, (rb,)"),
    ("rb = nudged_relax(Xstar, t, p, cost_grad_fn, beta, opts)",
     "rb = nudged_relax(Xstar, t, p, cost_grad_fn, -beta, opts)"),
    ("dp, d0 = model.dE_dtheta(rb.X, t, p), model.dE_dtheta(Xstar, t, p)",
     "dp, d0 = model.dE_dtheta(rb.X, t, p), model.dE_dtheta(rb.X, t, p)"),
])
def test_ep_forward_planted_mistakes_are_caught(equilibrium, old, new):
    with pytest.raises(AssertionError):
        test_ep_forward_first_order(equilibrium, ep_grad=_planted("ep_grad", old, new))


# ------------------------------------- pure line tension (Results, "Energy functions")

def _line_tension_equilibrium(forces=None, monkeypatch=None):
    """Relax a perturbed honeycomb under pure, uniform line tension and
    return the largest |sum of the three unit edge vectors| over the
    vertices, computed from the geometry alone (0 at every vertex of a
    line-tension equilibrium: three 120-degree angles)."""
    from oracle.mesh import HE_OFFX, HE_OFFY, HE_SRC, HE_TGT
    if forces is not None:
        monkeypatch.setattr(model, "forces", forces)
    t, _ = honeycomb(6, 6)
    p = dict(KA=0.0, KP=0.0, A0=1.0, P0=1.0, lam=1.0)
    s = 1.0 / math.sqrt(3.0)
    X = t["vert"] + 0.05 * s * np.random.default_rng(5).standard_normal(t["vert"].shape)
    r = solvers.relax(X, t, p, solvers.MinOpts(tol=1e-11, max_iter=20000, dt0=0.01, dt_max=0.1))
    assert r.converged
    he, L = t["he"], np.array([t["Lx"], t["Ly"]])
    acc = np.zeros_like(r.X)
    for h in range(he.shape[0]):
        d = r.X[he[h, HE_TGT]] + he[h, [HE_OFFX, HE_OFFY]] * L - r.X[he[h, HE_SRC]]
        acc[he[h, HE_SRC]] += d / np.linalg.norm(d)
    return np.abs(acc).max()


def test_pure_line_tension_gives_120_degree_vertices():
    assert _line_tension_equilibrium() < 1e-9


def test_line_tension_planted_mistake_is_caught(monkeypatch):
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(model.forces))
    old = "gl = lam[:, None] * u[rep]"
    assert src.count(old) == 1
    ns = dict(vars(model))
    exec(compile(src.replace(old, "gl = lam[:, None] * u[he[rep, HE_NEXT]]"), "<planted forces>",
                 "exec"), ns)
    with pytest.raises(AssertionError):
        _line_tension_equilibrium(ns["forces"], monkeypatch)
