"""Pins of the oracle parts whose mistakes the invariant and FD pins cannot
see: the FIRE control flow, the GD step and stop rule, the T1 decision, the anisotropy magnitude and
the exit-time wrap (CPU only).

* FIRE (Bitzek, Koskinen, Gaehler, Moseler, Gumbsch, PRL 97, 170201, 2006).
  The oracle's force call is replaced by a scripted force, so every step of
  the state machine has a value that can be written down by hand:
  P = F.v; P > 0 mixes v with F (the identity when v is parallel to F) and,
  once more than N_min steps with P > 0 have followed the last reset, grows
  dt by f_inc (capped at dt_max) and shrinks alpha by f_alpha; P <= 0
  (including the first step, from rest) sets v = 0, dt = f_dec dt,
  alpha = alpha0; then v += dt F and x += dt v.
* GD and the stop rule (Methods, "Simulation engine"): x += eta F, and the
  solve stops once max|F| < tol has held for `patience` consecutive
  iterations (a force above tol restarts the count), checked on a scripted
  force sequence whose stopping iteration and final position are written
  out by hand.
* T1 (Methods, "T1 transitions").  With pure line tension only the four
  edges at the short edge's ends and the edge itself change between the two
  candidates.  For neighbours at distance w along the edge and h across it
  (both ends alike), the four edges have length sqrt((w - l/2)^2 + h^2)
  after the stretch and sqrt(w^2 + (h - l/2)^2) after the T1 (l = 1.5
  l_min), so the T1 is kept iff h > w.  A regular honeycomb has, for its
  vertical edges, w = s and h = s sqrt(3)/2 (the stretch wins); scaling y by
  1/2 gives w = s/2 (the T1 wins).
* Anisotropy.  A regular hexagon of circumradius s has S = (s^2/2) I; a
  tissue of regular hexagons mapped by a linear M has S = (s^2/2) M M^T in
  every cell, so q is fixed by M alone: diag(1, sigma) gives
  q = ((1 - sigma^2)/(1 + sigma^2), 0), the shear [[1, g], [0, 1]] gives
  q = (g^2, 2 g)/(2 + g^2).
* Wrap (Methods, "Periodic mode"): vertices back in the box, offsets fixed,
  every unwrapped edge vector, the energy and the forces unchanged.

Each pin is followed by a planted mistake (a one-token change in a copy of
the oracle's source) that the pin must catch.
"""
import inspect
import math
import textwrap

import numpy as np
import pytest

import vx_inputs as vi
from oracle import mesh, model, solvers, topology
from oracle.mesh import (HE_FACE, HE_NEXT, HE_OFFX, HE_OFFY, HE_PREV, HE_SRC, HE_TGT,
                         HE_TWIN)

from test_oracle_mesh import check_half_edge_invariants


def planted(module, func_name, old, new):
    """A copy of module.func_name with `old` replaced by `new` in its source,
    compiled in the module's namespace."""
    src = textwrap.dedent(inspect.getsource(getattr(module, func_name)))
    assert src.count(old) == 1, f"{old!r} not found once in {func_name}"
    ns = dict(vars(module))
    exec(compile(src.replace(old, new), f"<planted {func_name}>", "exec"), ns)
    return ns[func_name]


# --------------------------------------------------------------------- FIRE

DT0, DT_MAX, N_MIN, F_INC, F_DEC, ALPHA0, F_ALPHA = 1.0, 2.0, 5, 1.1, 0.5, 0.1, 0.99


def fire_opts(iters):
    return solvers.MinOpts(method="fire", tol=0.0, max_iter=iters, dt0=DT0, dt_max=DT_MAX,
                           n_min=N_MIN, f_inc=F_INC, f_dec=F_DEC, alpha0=ALPHA0, f_alpha=F_ALPHA)


def run_scripted(monkeypatch, script, minimize=None):
    """Run the oracle's FIRE on one vertex under the scripted forces
    script[k] (k = iteration); returns the positions x_0 .. x_K."""
    xs = []

    def forces(x, t, p):
        xs.append(x.copy())
        return np.array([script[min(len(xs) - 1, len(script) - 1)]], dtype=np.float64)

    monkeypatch.setattr(model, "forces", forces)
    fn = minimize or solvers.minimize
    r = fn(np.zeros((1, 2)), {}, {}, fire_opts(len(script)))
    xs.append(r.X.copy())   # final position (the call at iteration K saw it too)
    return np.array([x[0] for x in xs[:len(script) + 1]])


def expected_dt_constant_push(K):
    """dt of iterations 0..K-1 under a constant force: the first step (from
    rest, P = 0) resets dt to f_dec dt0; the next N_min + 1 steps have P > 0
    but at most N_min steps since the reset, so dt stays; from then on dt
    grows by f_inc per step up to dt_max."""
    d0 = F_DEC * DT0
    out = []
    for k in range(K):
        g = max(0, k - (N_MIN + 1))     # growth steps made up to iteration k
        out.append(min(d0 * F_INC ** g, DT_MAX))
    return out


def check_constant_push(xs, K):
    # F = (1, 0): v stays parallel to F, so the mix is the identity and
    # v_{k+1} = sum_{j <= k} dt_j, x_{k+1} - x_k = dt_k v_{k+1}.
    dt = expected_dt_constant_push(K)
    v = np.cumsum(dt)
    dx = np.array(dt) * v
    assert np.allclose(np.diff(xs[:, 0]), dx, rtol=1e-14, atol=0), (np.diff(xs[:, 0]), dx)
    assert np.all(xs[:, 1] == 0.0)


def test_fire_constant_push(monkeypatch):
    K = 24   # long enough for dt to reach dt_max (0.5 * 1.1^15 > 2)
    xs = run_scripted(monkeypatch, [(1.0, 0.0)] * K)
    check_constant_push(xs, K)
    # spot values written out: x_1 = 0.5^2, x_7 - x_6 = 0.5 * 3.5,
    # x_8 - x_7 = 0.55 * 4.05
    assert xs[1, 0] == 0.25
    assert abs((xs[7, 0] - xs[6, 0]) - 1.75) < 1e-14
    assert abs((xs[8, 0] - xs[7, 0]) - 0.55 * 4.05) < 1e-13


def check_reversal(xs, K, flip):
    # constant push for `flip` steps, then F = (-1, 0): P < 0 freezes v,
    # halves dt and restarts the N_min count; the next step has P > 0 again.
    dt = expected_dt_constant_push(flip)
    v = sum(dt)
    x = xs[flip, 0]
    d = F_DEC * dt[-1]
    exp = [x - d * d]                       # v = 0 + d (-1), x += d v
    exp.append(exp[-1] - d * (2 * d))       # v = -d - d, no growth yet
    assert v > 0
    assert np.allclose(xs[flip + 1:flip + 3, 0], exp, rtol=1e-14, atol=1e-14), (xs[flip + 1:flip + 3, 0], exp)


def test_fire_reset_on_reversal(monkeypatch):
    flip = 10
    K = flip + 2
    xs = run_scripted(monkeypatch, [(1.0, 0.0)] * flip + [(-1.0, 0.0)] * 2)
    check_constant_push(xs[:flip + 1], flip)
    check_reversal(xs, K, flip)


def check_mix(xs, flip):
    # F = (1, 0) for `flip` steps, then F = (1, 1): P = v_x > 0, so v is mixed
    # with the alpha of that moment, alpha0 f_alpha^g with g the growth steps
    # so far, before dt grows and alpha shrinks once more:
    # v' = (1 - a) (|v|, 0) + a |v| (1, 1)/sqrt(2), then v'' = v' + dt (1, 1).
    dt = expected_dt_constant_push(flip + 1)
    v = sum(dt[:flip])
    g = max(0, flip - (N_MIN + 2))      # growth at iterations N_min + 2 .. flip - 1
    a = ALPHA0 * F_ALPHA ** g
    d = dt[flip]
    vx = (1 - a) * v + a * v / math.sqrt(2.0) + d
    vy = a * v / math.sqrt(2.0) + d
    dx, dy = xs[flip + 1] - xs[flip]
    assert abs(dy - d * vy) < 1e-13 * abs(d * vy), (dy, d * vy)
    assert abs(dx - d * vx) < 1e-13 * abs(d * vx), (dx, d * vx)


def test_fire_mix_uses_current_alpha(monkeypatch):
    flip = 10
    xs = run_scripted(monkeypatch, [(1.0, 0.0)] * flip + [(1.0, 1.0)])
    check_mix(xs, flip)


@pytest.mark.parametrize("old,new,which", [
    ("if n_pos > opts.n_min:", "if n_pos >= opts.n_min:", "push"),        # N_min off by one
    ("if P > 0.0:", "if P >= 0.0:", "push"),                                # P = 0 counted as P > 0
    ("dt = dt * opts.f_dec", "dt = dt", "reversal"),                        # no dt cut on reset
    ("v = np.zeros_like(x)\n            dt", "v = v\n            dt", "reversal"),  # v not frozen
    ("v = (1.0 - alpha) * v + alpha * (vn / fn) * F", "v = (1.0 - alpha) * v + alpha * vn * F",
     "mix"),                                                                # unnormalised F
])
def test_fire_planted_mistakes_are_caught(monkeypatch, old, new, which):
    bad = planted(solvers, "minimize", old, new)
    with pytest.raises(AssertionError):
        if which == "push":
            check_constant_push(run_scripted(monkeypatch, [(1.0, 0.0)] * 24, bad), 24)
        elif which == "reversal":
            xs = run_scripted(monkeypatch, [(1.0, 0.0)] * 10 + [(-1.0, 0.0)] * 2, bad)
            check_reversal(xs, 12, 10)
        else:
            xs = run_scripted(monkeypatch, [(1.0, 0.0)] * 10 + [(1.0, 1.0)], bad)
            check_mix(xs, 10)


def test_fire_growth_then_alpha_order_planted(monkeypatch):
    """Growing dt and shrinking alpha before the mix (instead of after) is
    caught by the mixing pin."""
    src_old = ("            v = (1.0 - alpha) * v + alpha * (vn / fn) * F\n"
               "            if n_pos > opts.n_min:\n"
               "                dt = min(dt * opts.f_inc, opts.dt_max)\n"
               "                alpha = alpha * opts.f_alpha\n")
    src_new = ("            if n_pos > opts.n_min:\n"
               "                dt = min(dt * opts.f_inc, opts.dt_max)\n"
               "                alpha = alpha * opts.f_alpha\n"
               "            v = (1.0 - alpha) * v + alpha * (vn / fn) * F\n")
    bad = planted(solvers, "minimize", src_old, src_new)
    with pytest.raises(AssertionError):
        check_mix(run_scripted(monkeypatch, [(1.0, 0.0)] * 10 + [(1.0, 1.0)], bad), 10)


# ---------------------------------------------------- GD step and stop rule

def run_stop_rule(monkeypatch, fmax_seq, patience, minimize=None):
    """GD (eta = 0.25) on one vertex under the scripted forces (f_k, 0) with
    tol = 1; returns the result and the number of force evaluations."""
    calls = []

    def forces(x, t, p):
        calls.append(x.copy())
        return np.array([[fmax_seq[min(len(calls) - 1, len(fmax_seq) - 1)], 0.0]])

    monkeypatch.setattr(model, "forces", forces)
    o = solvers.MinOpts(method="gd", tol=1.0, patience=patience, max_iter=len(fmax_seq) + 5,
                        gd_lr=0.25)
    r = (minimize or solvers.minimize)(np.zeros((1, 2)), {}, {}, o)
    return r, len(calls)


STOP_SEQ = [2.0, 0.5, 0.5, 3.0, 0.5, 0.5, 0.5, 0.5]


def check_stop_rule(monkeypatch, minimize=None):
    # patience 3: below tol at iterations 1, 2, then 3.0 resets the count;
    # 4, 5, 6 make three in a row, so the solve stops at iteration 6 after
    # six GD steps x += 0.25 f: x = 0.25 (2 + 0.5 + 0.5 + 3 + 0.5 + 0.5)
    r, n = run_stop_rule(monkeypatch, STOP_SEQ, 3, minimize)
    assert r.converged and r.iters == 6 and n == 7
    assert r.X[0, 0] == 1.75 and r.X[0, 1] == 0.0
    # patience 1 stops at the first force below tol, after one step
    r, n = run_stop_rule(monkeypatch, STOP_SEQ, 1, minimize)
    assert r.converged and r.iters == 1 and n == 2 and r.X[0, 0] == 0.5


def test_gd_step_and_patience(monkeypatch):
    check_stop_rule(monkeypatch)


@pytest.mark.parametrize("old,new", [
    ("below = below + 1 if fmax < opts.tol else 0",
     "below = below + 1 if fmax < opts.tol else below"),
    ("if below >= opts.patience:", "if below > opts.patience:"),
    ("x = x + opts.gd_lr * F", "x = x - opts.gd_lr * F"),
])
def test_stop_rule_planted_mistakes_are_caught(monkeypatch, old, new):
    with pytest.raises(AssertionError):
        check_stop_rule(monkeypatch, planted(solvers, "minimize", old, new))


# ----------------------------------------------------------------------- T1

L_MIN = 0.02
L_SHORT = 0.5 * L_MIN
LINE = dict(KA=0.0, KP=0.0, A0=1.0, P0=1.0, lam=1.0)   # pure line tension


def honeycomb(sigma):
    """Regular honeycomb (side s = 1/sqrt(3)) with y scaled by sigma."""
    seeds, Lx, Ly = vi.lattice_seeds(6, 6, a=1.0)
    t = mesh.build_periodic_voronoi(seeds, Lx, Ly)
    t = dict(t)
    X = t["vert"].copy()
    X[:, 1] *= sigma
    t["Ly"] = Ly * sigma
    t["vert"] = X
    return t


def edge_vec(X, t, h):
    he = t["he"]
    L = np.array([t["Lx"], t["Ly"]])
    return X[he[h, HE_TGT]] + he[h, HE_OFFX:HE_OFFY + 1] * L - X[he[h, HE_SRC]]


def vertical_edges(t):
    rep = model.edge_rep(t)
    return [e for e, h in enumerate(rep) if abs(edge_vec(t["vert"], t, int(h))[0]) < 1e-9]


def shrink(X, t, h, ell):
    """The edge of h set to length ell about its midpoint (b in its frame)."""
    he = t["he"]
    L = np.array([t["Lx"], t["Ly"]])
    a, b = int(he[h, HE_SRC]), int(he[h, HE_TGT])
    d = edge_vec(X, t, h)
    u = d / np.linalg.norm(d)
    m = X[a] + 0.5 * d
    X = X.copy()
    X[a] = m - 0.5 * ell * u
    X[b] = m + 0.5 * ell * u - he[h, HE_OFFX:HE_OFFY + 1] * L
    return X, m, u


def t1_case(sigma, e=None):
    t = honeycomb(sigma)
    rep = model.edge_rep(t)
    e = vertical_edges(t)[0] if e is None else e
    h = int(rep[e])
    X, m, u = shrink(t["vert"], t, h, L_SHORT)
    return t, X, e, h, m, u


def check_decision(sigma, expect_t1, t1_pass=None):
    t, X, e, h, m, u = t1_case(sigma)
    run = t1_pass or topology.t1_pass
    Xn, tn, touched, n_t1, n_st = run(X, t, LINE, L_MIN)
    assert (n_t1, n_st) == ((1, 0) if expect_t1 else (0, 1))
    a, b = int(t["he"][h, HE_SRC]), int(t["he"][h, HE_TGT])
    assert sorted(touched) == sorted([a, b])
    d = edge_vec(Xn, tn, h)
    l_new = 1.5 * L_MIN
    assert abs(np.linalg.norm(d) - l_new) < 1e-12
    assert np.abs(Xn[a] + 0.5 * d - m).max() < 1e-12          # about the old midpoint
    perp = np.array([-u[1], u[0]])                                # into C1
    if expect_t1:
        assert abs(d @ u) < 1e-12                                 # orthogonal to the old edge
        assert np.abs(Xn[a] - (m + 0.5 * l_new * perp)).max() < 1e-12
        he0, he1 = t["he"], tn["he"]
        C1, C2 = he0[h, HE_FACE], he0[he0[h, HE_TWIN], HE_FACE]
        assert he1[h, HE_FACE] != C1 and he1[he1[h, HE_TWIN], HE_FACE] != C2
        check_half_edge_invariants(dict(tn, vert=Xn))
    else:
        assert abs(abs(d @ u) - l_new) < 1e-12                    # along the old edge
        assert np.array_equal(tn["he"], t["he"])
    # the choice agrees with the closed form h > w
    nb = [int(x) for x in (t["he"][t["he"][h, HE_PREV], HE_SRC], t["he"][t["he"][h, HE_NEXT], HE_TGT])]
    assert len(nb) == 2
    return Xn, tn


def test_t1_decision_stretch_wins_on_regular_honeycomb():
    # w = s = 1/sqrt(3), h = 1/2 < w
    check_decision(1.0, expect_t1=False)


def test_t1_decision_t1_wins_on_compressed_honeycomb():
    # y scaled by 1/2: w = s/2 < h = 1/2
    check_decision(0.5, expect_t1=True)


def test_t1_closed_form_energy_difference():
    """The oracle's two candidate energies differ by exactly the closed-form
    amount 4 [sqrt((w - l/2)^2 + h^2) - sqrt(w^2 + (h - l/2)^2)]."""
    l = 1.5 * L_MIN
    s = 1.0 / math.sqrt(3.0)
    for sigma in (1.0, 0.5, 0.8):
        t, X, e, h, m, u = t1_case(sigma)
        Xs = topology.stretch(X, t, h, l)
        Xt, tt = topology.t1(X, t, h, l)
        w, hh = sigma * s, 0.5
        expect = 4 * (math.sqrt((w - l / 2) ** 2 + hh ** 2) - math.sqrt(w ** 2 + (hh - l / 2) ** 2))
        got = model.energy(Xs, t, LINE) - model.energy(Xt, tt, LINE)
        assert abs(got - expect) < 1e-12, (sigma, got, expect)


def requeue_case(f_above):
    """Regular honeycomb, a vertical edge e shrunk below l_min and one of the
    four edges f at its ends shortened to 1.1 l_min (its far vertex moved
    towards the end of e).  The stretch of e (the stretch wins here: the
    three untouched neighbour edges favour it by ~0.1 l_min each, the
    shortened one favours the T1 by ~0.13 l_min) moves both ends of e
    outwards by l_min / 2, which takes f below l_min.  f_above selects f's id
    relative to e's."""
    t = honeycomb(1.0)
    he = t["he"]
    L = np.array([t["Lx"], t["Ly"]])
    rep = model.edge_rep(t)
    for e in vertical_edges(t):
        h = int(rep[e])
        hq = int(he[h, HE_TWIN])
        # (half-edge, True if its source is the far vertex)
        for g, far_is_src in ((int(he[h, HE_PREV]), True), (int(he[h, HE_NEXT]), False),
                              (int(he[hq, HE_NEXT]), False), (int(he[hq, HE_PREV]), True)):
            f = int(t["edge_id"][g])
            if (f > e) != f_above:
                continue
            X, m, u = shrink(t["vert"], t, h, L_SHORT)
            d = edge_vec(X, t, g)
            d1 = 1.1 * L_MIN * d / np.linalg.norm(d)
            s_g, t_g = int(he[g, HE_SRC]), int(he[g, HE_TGT])
            off = he[g, HE_OFFX:HE_OFFY + 1] * L
            if far_is_src:
                X[s_g] = X[t_g] + off - d1
            else:
                X[t_g] = X[s_g] + d1 - off
            assert abs(np.linalg.norm(edge_vec(X, t, g)) - 1.1 * L_MIN) < 1e-12
            return t, X, e, f, g
    raise AssertionError("no suitable edge pair")


def check_requeue(f_above, t1_pass=None):
    t, X, e, f, g = requeue_case(f_above)
    run = t1_pass or topology.t1_pass
    Xn, tn, touched, n_t1, n_st = run(X, t, LINE, L_MIN)
    assert n_st >= 1 and tn["edge_id"][g] == f
    rep = model.edge_rep(tn)
    lf = topology.edge_length(Xn, tn, int(rep[f]))
    if f_above:
        # f (id > e) became short while e was handled: same pass
        assert n_t1 + n_st == 2, (n_t1, n_st)
        assert lf >= L_MIN - 1e-12
    else:
        # f (id < e) was passed already: it stays short until the next pass
        assert n_t1 + n_st == 1, (n_t1, n_st)
        assert lf < L_MIN


@pytest.mark.parametrize("f_above", [True, False])
def test_t1_requeue_order(f_above):
    check_requeue(f_above)


@pytest.mark.parametrize("old,new,check", [
    ("if cand is not None and model.energy(cand[0], cand[1], p) < model.energy(Xs, t, p):",
     "if cand is not None and model.energy(cand[0], cand[1], p) > model.energy(Xs, t, p):",
     "decision"),                                                # reversed comparison
    ("            if f > e and edge_length(X, t, hh) < l_min:",
     "            if f < e and edge_length(X, t, hh) < l_min:", "requeue"),   # wrong re-queue side
    ("            if f > e and edge_length(X, t, hh) < l_min:",
     "            if False:", "requeue"),                       # no re-queue
    ("l_new = T1_STRETCH * l_min", "l_new = l_min", "decision"),  # wrong new length
])
def test_t1_planted_mistakes_are_caught(old, new, check):
    bad = planted(topology, "t1_pass", old, new)
    with pytest.raises(AssertionError):
        if check == "decision":
            check_decision(1.0, False, bad)
            check_decision(0.5, True, bad)
        else:
            check_requeue(True, bad)
            check_requeue(False, bad)


def test_t1_planted_off_centre_stretch_is_caught(monkeypatch):
    """A stretch that keeps a in place (instead of the midpoint) is caught."""
    bad = planted(topology, "stretch", "Xs[a] = mid - 0.5 * l_new * u", "Xs[a] = X[a]")
    monkeypatch.setattr(topology, "stretch", bad)
    with pytest.raises(AssertionError):
        check_decision(1.0, False)


# --------------------------------------------------------------- anisotropy

def mapped_honeycomb(M):
    """The honeycomb of lattice_seeds(4, 6) with its vertices mapped by M.
    M is diagonal, or a shear [[1, g], [0, 1]] with g Ly = j Lx (j integer),
    which keeps the rectangular box periodic: the offset (ox, oy) of a
    half-edge becomes (ox + j oy, oy) so that every edge vector maps by M."""
    seeds, Lx, Ly = vi.lattice_seeds(4, 6, a=1.0)
    t = dict(mesh.build_periodic_voronoi(seeds, Lx, Ly))
    M = np.asarray(M, dtype=np.float64)
    X = t["vert"] @ M.T
    he = t["he"].copy()
    if M[0, 1] != 0.0:
        j = M[0, 1] * Ly / Lx
        assert abs(j - round(j)) < 1e-12
        he[:, HE_OFFX] = he[:, HE_OFFX] + int(round(j)) * he[:, HE_OFFY]
    t["he"] = he
    t["Lx"], t["Ly"] = Lx * M[0, 0], Ly * M[1, 1]
    for k in ("_kcorner", "_faces", "_rep"):
        t.pop(k, None)
    return X, t


def q_closed_form(M):
    Q = np.asarray(M) @ np.asarray(M).T
    tr = Q[0, 0] + Q[1, 1]
    return np.array([(Q[0, 0] - Q[1, 1]) / tr, 2 * Q[0, 1] / tr])


def anisotropy_cases():
    seeds, Lx, Ly = vi.lattice_seeds(4, 6, a=1.0)
    g = Lx / Ly          # j = 1
    return [np.diag([1.0, 0.6]), np.diag([1.3, 1.0]), np.array([[1.0, g], [0.0, 1.0]])]


def check_anisotropy(fn):
    for M in anisotropy_cases():
        X, t = mapped_honeycomb(M)
        q = q_closed_form(M)
        C0, _ = fn(X, t, (0.0, 0.0))
        assert abs(C0 - (q @ q)) < 1e-12, (C0, q @ q)
        # C vanishes exactly at the closed-form q: both components pinned
        Cq, G = fn(X, t, tuple(q))
        assert Cq < 1e-24, (M, Cq)
        assert np.abs(G).max() < 1e-10


def test_anisotropy_closed_forms():
    # the shear case has q2 = 2 g/(2 + g^2) != 0
    M = anisotropy_cases()[2]
    assert abs(q_closed_form(M)[1]) > 0.3
    check_anisotropy(model.shape_tensor_anisotropy)


@pytest.mark.parametrize("old,new", [
    ("q1, q2 = (Qxx - Qyy) / T, 2.0 * Qxy / T", "q1, q2 = (Qyy - Qxx) / T, 2.0 * Qxy / T"),
    ("q1, q2 = (Qxx - Qyy) / T, 2.0 * Qxy / T", "q1, q2 = (Qxx - Qyy) / T, Qxy / T"),
    ("w = q - c[face]", "w = q"),
])
def test_anisotropy_planted_mistakes_are_caught(old, new):
    bad = planted(model, "shape_tensor_anisotropy", old, new)
    with pytest.raises(AssertionError):
        check_anisotropy(bad)


# --------------------------------------------------------------------- wrap

def check_wrap(X, t, p, wrap_fn):
    Xw, tw = wrap_fn(X, t)
    L = np.array([t["Lx"], t["Ly"]])
    assert np.all(Xw >= 0) and np.all(Xw <= L)
    assert np.all(np.abs(tw["he"][:, HE_OFFX:]) <= 1)
    check_half_edge_invariants(dict(tw, vert=Xw))
    # every unwrapped edge vector keeps its value
    for h in range(t["he"].shape[0]):
        assert np.abs(edge_vec(Xw, tw, h) - edge_vec(X, t, h)).max() < 1e-12 * L.max()
    E0, Ew = model.energy(X, t, p), model.energy(Xw, tw, p)
    assert abs(Ew - E0) < 1e-12 * abs(E0)
    F0 = model.forces(X, t, p)
    assert np.abs(model.forces(Xw, tw, p) - F0).max() < 1e-12 * np.abs(F0).max()
    # positions are equal modulo the box
    k = np.round((X - Xw) / L)
    assert np.abs(X - Xw - k * L).max() < 1e-12 * L.max()


def drifted(stream=61):
    """A small tissue whose vertices have drifted across the box edges by up
    to a few cells (a rigid shift plus small random moves: the unwrapped
    state a long relaxation leaves)."""
    c = vi.small_tissue(30, stream)
    t = mesh.build_periodic_voronoi(c["seeds"], c["Lx"], c["Ly"])
    p = {k: c[k] for k in ("KA", "KP", "A0", "P0", "lam")}
    rng = np.random.default_rng(stream)
    X = t["vert"] + np.array([1.37 * c["Lx"], -2.61 * c["Ly"]]) + 0.05 * rng.standard_normal(t["vert"].shape)
    return X, t, p


def test_wrap_keeps_geometry():
    X, t, p = drifted()
    check_wrap(X, t, p, topology.wrap)
    # the wrapped state is a fixed point
    Xw, tw = topology.wrap(X, t)
    Xw2, tw2 = topology.wrap(Xw, tw)
    assert np.array_equal(Xw2, Xw) and np.array_equal(tw2["he"], tw["he"])


def test_wrap_coordinate_edges():
    L = 1.0
    x = np.array([0.0, 1.0, -1e-300, -0.25, 2.0 - 1e-16, 3.5, -7.0])
    xw, k = topology.wrap_coordinate(x, L)
    assert np.all(xw >= 0) and np.all(xw < L)
    assert np.allclose(x - k * L, xw, atol=1e-15)


@pytest.mark.parametrize("old,new", [
    ("he[:, HE_OFFX] = he[:, HE_OFFX] + k[tgt, 0] - k[src, 0]",
     "he[:, HE_OFFX] = he[:, HE_OFFX] + k[src, 0] - k[tgt, 0]"),     # sign of the fix-up
    ("he[:, HE_OFFY] = he[:, HE_OFFY] + k[tgt, 1] - k[src, 1]",
     "he[:, HE_OFFY] = he[:, HE_OFFY]"),                             # offsets not updated
])
def test_wrap_planted_mistakes_are_caught(old, new):
    bad = planted(topology, "wrap", old, new)
    X, t, p = drifted()
    with pytest.raises(AssertionError):
        check_wrap(X, t, p, bad)
