"""Oracle: T1 transitions on the periodic half-edge tables.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this.

Methods, "T1 transitions": during each iteration the edges are checked one
after another; when an edge is shorter than l_min, two candidates are built,
(1) the edge stretched along its own direction and (2) the edge removed and
replaced by a new edge orthogonal to it (a T1 neighbour exchange), and the
candidate with the lower total energy is kept.

Readings of what the paper leaves open:

* both candidates give the edge the length l_new = T1_STRETCH * l_min,
  centred on the old midpoint;
* a T1 is not a candidate when either cell that would lose the edge is a
  triangle (it would become a two-sided polygon) or when the four cells
  around the edge are not distinct; the stretch is then kept;
* the edges are checked in increasing edge id, each against the positions
  left by the previous ones;
* the velocities of the two vertices of a modified edge are set to zero
  (done by the caller, which knows the minimiser state).

Naming, for the edge's half-edge h = a -> b and its twin h' = b -> a:
C1 = face(h) (left of a -> b), C2 = face(h'), p -> a = prev(h) in C1,
b -> y = next(h) in C1, z -> b = prev(h') in C2, a -> x = next(h') in C2,
C3 = the third cell at a, C4 = the third cell at b.  After the T1, a sits on
C1's side, joined to p and y; b on C2's side, joined to x and z; the new edge
a - b separates C3 from C4.

``wrap`` is the bookkeeping of Methods, "Periodic mode": every vertex is put
back into the primary box [0, Lx) x [0, Ly) and the offsets of the half-edges
are changed so that every unwrapped edge vector stays what it was.
"""
from __future__ import annotations

import numpy as np

from . import model
from .mesh import HE_FACE, HE_NEXT, HE_OFFX, HE_OFFY, HE_PREV, HE_SRC, HE_TGT, HE_TWIN

T1_STRETCH = 1.5


def _off(he, h):
    return he[h, HE_OFFX:HE_OFFY + 1].astype(np.int64)


def _set_off(he, h, k):
    he[h, HE_OFFX] = k[0]
    he[h, HE_OFFY] = k[1]


def face_size(he, h0):
    n, h = 0, h0
    while True:
        n += 1
        h = int(he[h, HE_NEXT])
        if h == h0:
            return n


def stretch(X, t, h, l_new):
    """Candidate 1: the edge of h stretched to l_new about its midpoint."""
    he = t["he"]
    L = np.array([t["Lx"], t["Ly"]])
    a, b = int(he[h, HE_SRC]), int(he[h, HE_TGT])
    ob = _off(he, h) * L
    d = X[b] + ob - X[a]
    u = d / np.sqrt(d @ d)
    mid = X[a] + 0.5 * d
    Xs = X.copy()
    Xs[a] = mid - 0.5 * l_new * u
    Xs[b] = mid + 0.5 * l_new * u - ob
    return Xs


def t1(X, t, h, l_new):
    """Candidate 2: T1 on the edge of h.  Returns (X, tissue) copies, or None
    when the T1 is not allowed."""
    he = t["he"].copy()
    face_he = t["face_he"].copy()
    L = np.array([t["Lx"], t["Ly"]])
    hq = int(he[h, HE_TWIN])
    a, b = int(he[h, HE_SRC]), int(he[h, HE_TGT])
    C1, C2 = int(he[h, HE_FACE]), int(he[hq, HE_FACE])
    hp1, hn1 = int(he[h, HE_PREV]), int(he[h, HE_NEXT])      # p -> a, b -> y
    hp2, hn2 = int(he[hq, HE_PREV]), int(he[hq, HE_NEXT])    # z -> b, a -> x
    ta_p, tb_y = int(he[hp1, HE_TWIN]), int(he[hn1, HE_TWIN])  # a -> p, y -> b
    tb_z, tx_a = int(he[hp2, HE_TWIN]), int(he[hn2, HE_TWIN])  # b -> z, x -> a
    C3, C4 = int(he[ta_p, HE_FACE]), int(he[tb_z, HE_FACE])
    if face_size(he, h) <= 3 or face_size(he, hq) <= 3:
        return None
    if len({C1, C2, C3, C4}) < 4:
        return None
    # Images of the neighbours in a's frame (stored X[v] = U_v - k_v L).
    k_b = _off(he, h)
    k_p = _off(he, ta_p)
    k_x = _off(he, hn2)
    k_y = k_b + _off(he, hn1)
    k_z = k_b + _off(he, tb_z)
    d = X[b] + k_b * L - X[a]
    ell = np.sqrt(d @ d)
    u = d / ell
    perp = np.array([-u[1], u[0]])  # points into C1
    mid = X[a] + 0.5 * d
    Xn = X.copy()
    Xn[a] = mid + 0.5 * l_new * perp
    Xn[b] = mid - 0.5 * l_new * perp   # b now stored in a's frame (k_b = 0)
    # Rewire.  C1: p -> a -> y.  C2: z -> b -> x.
    he[hp1, HE_NEXT], he[hn1, HE_PREV] = hn1, hp1
    he[hn1, HE_SRC] = a
    he[hp2, HE_NEXT], he[hn2, HE_PREV] = hn2, hp2
    he[hn2, HE_SRC] = b
    # C3: x -> b -> a -> p.  C4: y -> a -> b -> z.
    he[tx_a, HE_TGT] = b
    he[tx_a, HE_NEXT], he[hq, HE_PREV] = hq, tx_a
    he[hq, HE_NEXT], he[ta_p, HE_PREV] = ta_p, hq
    he[hq, HE_FACE] = C3
    he[tb_y, HE_TGT] = a
    he[tb_y, HE_NEXT], he[h, HE_PREV] = h, tb_y
    he[h, HE_NEXT], he[tb_z, HE_PREV] = tb_z, h
    he[h, HE_FACE] = C4
    # Offsets of every half-edge at a or b.
    zero = np.zeros(2, dtype=np.int64)
    for hh, k in ((ta_p, k_p), (hn1, k_y), (hn2, k_x), (tb_z, k_z), (h, zero)):
        _set_off(he, hh, k)
        _set_off(he, int(he[hh, HE_TWIN]), -k)
    if face_he[C1] == h:
        face_he[C1] = hn1
    if face_he[C2] == hq:
        face_he[C2] = hn2
    tn = dict(t)
    tn["he"], tn["face_he"] = he, face_he
    for key in ("_kcorner", "_faces", "_rep"):
        tn.pop(key, None)
    return Xn, tn


def edge_length(X, t, h):
    he = t["he"]
    L = np.array([t["Lx"], t["Ly"]])
    d = X[he[h, HE_TGT]] + _off(he, h) * L - X[he[h, HE_SRC]]
    return float(np.sqrt(d @ d))


def out_half_edges(he, h):
    """The three half-edges leaving src(h), h first."""
    h1 = int(he[int(he[h, HE_PREV]), HE_TWIN])
    h2 = int(he[int(he[h1, HE_PREV]), HE_TWIN])
    return (h, h1, h2)


def t1_pass(X, t, p, l_min):
    """Check the edges in increasing id against the current positions; apply
    the lower-energy candidate to every edge shorter than l_min.  Returns
    (X, tissue, touched vertices, number of T1s, number of stretches)."""
    l_new = T1_STRETCH * l_min
    rep = model.edge_rep(t)
    eid = t["edge_id"]
    ell = model.geometry(X, t)["ell"][rep]
    pending = set(int(e) for e in np.nonzero(ell < l_min)[0])
    touched, n_t1, n_st, e = [], 0, 0, -1
    while pending:
        e = min(pending)
        pending.discard(e)
        h = int(rep[e])
        if edge_length(X, t, h) >= l_min:
            continue
        he = t["he"]
        a, b = int(he[h, HE_SRC]), int(he[h, HE_TGT])
        touched += [a, b]
        Xs = stretch(X, t, h, l_new)
        cand = t1(X, t, h, l_new)
        if cand is not None and model.energy(cand[0], cand[1], p) < model.energy(Xs, t, p):
            X, t = cand
            n_t1 += 1
        else:
            X = Xs
            n_st += 1
        he = t["he"]
        for hh in out_half_edges(he, h) + out_half_edges(he, int(he[h, HE_TWIN])):
            f = int(eid[hh])
            if f > e and edge_length(X, t, hh) < l_min:
                pending.add(f)
    return X, t, touched, n_t1, n_st


def wrap_coordinate(x, L):
    """(x', k) with x' = x - k L in [0, L] and k an integer: k = floor(x / L),
    corrected by one period when the rounding of x / L or of x - k L left x'
    outside [0, L); a result that rounds to L is taken as 0."""
    k = np.floor(x / L)
    xw = x - k * L
    hi = xw >= L
    xw = np.where(hi, xw - L, xw)
    k = np.where(hi, k + 1, k)
    lo = xw < 0
    xw = np.where(lo, xw + L, xw)
    k = np.where(lo, k - 1, k)
    xw = np.where(xw >= L, 0.0, xw)
    return xw, k.astype(np.int64)


def wrap(X, t):
    """Wrap the vertices into the primary box and fix the offsets (Methods,
    "Periodic mode").  A vertex moved by -k_v L; a half-edge s -> t then
    needs the offset off + k_t - k_s for X[t] + off L - X[s] to keep its
    value.  Returns (X', tissue copy)."""
    he = t["he"].copy()
    Xw = np.empty_like(X)
    k = np.zeros(X.shape, dtype=np.int64)
    for c, L in ((0, t["Lx"]), (1, t["Ly"])):
        Xw[:, c], k[:, c] = wrap_coordinate(X[:, c], L)
    src, tgt = he[:, HE_SRC], he[:, HE_TGT]
    he[:, HE_OFFX] = he[:, HE_OFFX] + k[tgt, 0] - k[src, 0]
    he[:, HE_OFFY] = he[:, HE_OFFY] + k[tgt, 1] - k[src, 1]
    tn = dict(t)
    tn["he"] = he
    for key in ("_kcorner", "_faces", "_rep"):
        tn.pop(key, None)
    return Xw, tn
