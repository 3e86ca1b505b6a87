"""Oracle: energy, forces, Hessian and outer costs of the periodic vertex model.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this.

Plain FP64 numpy, written from the definitions:

* Energy (Methods, "Vertex model formulation", the E1 form with per-cell
  moduli, plus the E2 line-tension term on every edge):

      E(X) = sum_alpha K_A,alpha (A_alpha - A0_alpha)^2
           + sum_alpha K_P,alpha (P_alpha - P0_alpha)^2
           + sum_edges Lambda_e l_e

  The dimensionless E1 of Eq. (Energy1) is the special case K_A = 1/A0^2,
  K_P = 1/A0, Lambda = 0; E2 of Eq. (Energy2) is K_P = 0, K_A = K/2.
* A_alpha is the shoelace area and P_alpha the perimeter of the polygon of
  cell alpha; the polygon's corners are unwrapped with the heTable offsets
  (Methods, "Periodic mode"): a half-edge h runs from X[src] to
  X[tgt] + (offx Lx, offy Ly).
* Forces F = -grad_X E (Results, "Energy functions": the minimiser is driven
  by the gradient with respect to the vertex positions).
* Hessian H = grad^2_X E assembled explicitly from per-cell and per-edge
  blocks (used by implicit differentiation, Methods "Implicit
  differentiation").
* Outer costs: v2v (Methods, "Geometric vertex-to-vertex (v2v) cost") with
  minimum-image differences, and the mean cell-shape-tensor anisotropy.

A tissue is the dict returned by ``oracle.mesh.build_periodic_voronoi``.
Parameters are a dict with keys KA, KP, A0, P0 (scalar or per-cell array)
and lam (scalar or per-edge array).  Positions X are float64 [V, 2].
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import HE_FACE, HE_NEXT, HE_OFFX, HE_OFFY, HE_PREV, HE_SRC, HE_TGT, HE_TWIN


def _per_cell(v, n):
    v = np.asarray(v, dtype=np.float64)
    return np.full(n, float(v)) if v.ndim == 0 else v


def _per_edge(v, E):
    v = np.asarray(v, dtype=np.float64)
    return np.full(E, float(v)) if v.ndim == 0 else v


def params_arrays(t, p):
    n = t["n"]
    E = t["he"].shape[0] // 2
    return (_per_cell(p["KA"], n), _per_cell(p["KP"], n), _per_cell(p["A0"], n),
            _per_cell(p["P0"], n), _per_edge(p["lam"], E))


def corner_offsets(t):
    """Integer image of every half-edge's source corner relative to the first
    corner of its face (cumulative sum of the offsets along the face cycle)."""
    he = t["he"]
    HE = he.shape[0]
    k = np.zeros((HE, 2), dtype=np.int64)
    for h0 in t["face_he"]:
        h, acc = int(h0), np.zeros(2, dtype=np.int64)
        while True:
            k[h] = acc
            acc = acc + he[h, HE_OFFX:HE_OFFY + 1]
            h = int(he[h, HE_NEXT])
            if h == h0:
                break
        assert acc[0] == 0 and acc[1] == 0
    return k


def geometry(X, t):
    """Per half-edge local corner positions and edge vectors, per cell A, P.

    q[h]  = position of src(h) relative to the first corner of its face
    d[h]  = edge vector of h (target minus source, unwrapped)
    """
    he = t["he"]
    L = np.array([t["Lx"], t["Ly"]])
    if "_kcorner" not in t:
        t["_kcorner"] = corner_offsets(t)
    k = t["_kcorner"]
    face = he[:, HE_FACE]
    first_src = he[t["face_he"], HE_SRC]
    q = X[he[:, HE_SRC]] + k * L - X[first_src[face]]
    d = X[he[:, HE_TGT]] + he[:, HE_OFFX:HE_OFFY + 1] * L - X[he[:, HE_SRC]]
    qn = q + d  # position of tgt(h) in the same local frame
    n = t["n"]
    A = 0.5 * np.bincount(face, weights=q[:, 0] * qn[:, 1] - qn[:, 0] * q[:, 1], minlength=n)
    ell = np.sqrt((d * d).sum(axis=1))
    P = np.bincount(face, weights=ell, minlength=n)
    return dict(q=q, d=d, ell=ell, A=A, P=P)


def edge_rep(t):
    """For every undirected edge, its half-edge with the smaller index."""
    he = t["he"]
    E = he.shape[0] // 2
    rep = np.empty(E, dtype=np.int64)
    eid = t["edge_id"]
    for h in range(he.shape[0]):
        if h < he[h, HE_TWIN]:
            rep[eid[h]] = h
    return rep


def energy(X, t, p):
    KA, KP, A0, P0, lam = params_arrays(t, p)
    g = geometry(X, t)
    rep = edge_rep(t) if "_rep" not in t else t["_rep"]
    t["_rep"] = rep
    return float(np.sum(KA * (g["A"] - A0) ** 2) + np.sum(KP * (g["P"] - P0) ** 2)
                 + np.sum(lam * g["ell"][rep]))


def energy_terms(X, t, p):
    """(area term, perimeter term, line-tension term) of the energy."""
    KA, KP, A0, P0, lam = params_arrays(t, p)
    g = geometry(X, t)
    rep = edge_rep(t)
    return (float(np.sum(KA * (g["A"] - A0) ** 2)), float(np.sum(KP * (g["P"] - P0) ** 2)),
            float(np.sum(lam * g["ell"][rep])))


def cell_gradients(X, t):
    """Per half-edge h (corner src(h) of cell face(h)): dA/du and dP/du."""
    he = t["he"]
    g = geometry(X, t)
    q, d, ell = g["q"], g["d"], g["ell"]
    prev, nxt = he[:, HE_PREV], he[:, HE_NEXT]
    q_prev = q[prev]
    q_next = q[nxt]
    # Shoelace: dA/dx_k = (y_{k+1} - y_{k-1}) / 2, dA/dy_k = (x_{k-1} - x_{k+1}) / 2.
    dA = 0.5 * np.stack([q_next[:, 1] - q_prev[:, 1], q_prev[:, 0] - q_next[:, 0]], axis=1)
    u = d / ell[:, None]
    # P contains |u_next - u_k| (edge h) and |u_k - u_prev| (edge prev(h)).
    dP = u[prev] - u
    return g, dA, dP, u


def forces(X, t, p):
    """F = -grad_X E, float64 [V, 2]."""
    KA, KP, A0, P0, lam = params_arrays(t, p)
    he = t["he"]
    V = X.shape[0]
    g, dA, dP, u = cell_gradients(X, t)
    face = he[:, HE_FACE]
    cA = 2.0 * KA * (g["A"] - A0)
    cP = 2.0 * KP * (g["P"] - P0)
    grad = cA[face, None] * dA + cP[face, None] * dP
    rep = edge_rep(t)
    s, tt = he[rep, HE_SRC], he[rep, HE_TGT]
    gl = lam[:, None] * u[rep]  # d(Lambda l)/d(target) = +Lambda u, d/d(source) = -Lambda u
    G = np.zeros((V, 2))
    src = he[:, HE_SRC]
    for c in range(2):
        G[:, c] = (np.bincount(src, weights=grad[:, c], minlength=V)
                   + np.bincount(tt, weights=gl[:, c], minlength=V)
                   - np.bincount(s, weights=gl[:, c], minlength=V))
    return -G


def faces_list(t):
    he = t["he"]
    out = []
    for h0 in t["face_he"]:
        hs, h = [], int(h0)
        while True:
            hs.append(h)
            h = int(he[h, HE_NEXT])
            if h == h0:
                break
        out.append(hs)
    return out


def hessian(X, t, p, dense=False):
    """H = grad^2_X E assembled from per-cell 2m x 2m blocks and per-edge
    4 x 4 blocks.  Variables are ordered (x_0, y_0, x_1, y_1, ...)."""
    KA, KP, A0, P0, lam = params_arrays(t, p)
    he = t["he"]
    V = X.shape[0]
    g, dA, dP, u = cell_gradients(X, t)
    ell = g["ell"]
    rows, cols, vals = [], [], []

    def add_block(idx, B):
        ii = np.repeat(idx, len(idx))
        jj = np.tile(idx, len(idx))
        rows.append(ii)
        cols.append(jj)
        vals.append(B.ravel())

    def ell_hess(h):
        uh = u[h]
        return (np.eye(2) - np.outer(uh, uh)) / ell[h]

    if "_faces" not in t:
        t["_faces"] = faces_list(t)
    for alpha, hs in enumerate(t["_faces"]):
        m = len(hs)
        vs = he[hs, HE_SRC]
        idx = np.empty(2 * m, dtype=np.int64)
        idx[0::2] = 2 * vs
        idx[1::2] = 2 * vs + 1
        gA = dA[hs].ravel()
        gP = dP[hs].ravel()
        # Hessian of the shoelace area: d2A/dx_k dy_{k+1} = 1/2, d2A/dy_k dx_{k+1} = -1/2.
        HA = np.zeros((2 * m, 2 * m))
        for k in range(m):
            k1 = (k + 1) % m
            HA[2 * k, 2 * k1 + 1] += 0.5
            HA[2 * k1 + 1, 2 * k] += 0.5
            HA[2 * k + 1, 2 * k1] -= 0.5
            HA[2 * k1, 2 * k + 1] -= 0.5
        # Hessian of the perimeter: sum over the cell's edges of
        # [[M, -M], [-M, M]], M = (I - u u^T) / l.
        HP = np.zeros((2 * m, 2 * m))
        for k in range(m):
            k1 = (k + 1) % m
            M = ell_hess(hs[k])
            a, b = slice(2 * k, 2 * k + 2), slice(2 * k1, 2 * k1 + 2)
            HP[a, a] += M
            HP[b, b] += M
            HP[a, b] -= M
            HP[b, a] -= M
        B = (2.0 * KA[alpha] * (np.outer(gA, gA) + (g["A"][alpha] - A0[alpha]) * HA)
             + 2.0 * KP[alpha] * (np.outer(gP, gP) + (g["P"][alpha] - P0[alpha]) * HP))
        add_block(idx, B)
    rep = edge_rep(t)
    for e, h in enumerate(rep):
        s, tt = he[h, HE_SRC], he[h, HE_TGT]
        M = lam[e] * ell_hess(h)
        idx = np.array([2 * s, 2 * s + 1, 2 * tt, 2 * tt + 1])
        B = np.block([[M, -M], [-M, M]])
        add_block(idx, B)
    H = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(2 * V, 2 * V)).tocsr()
    return H.toarray() if dense else H


def hvp(X, t, p, Vdir):
    """Hessian-vector product H v, with v float64 [V, 2]."""
    H = hessian(X, t, p)
    return (H @ Vdir.reshape(-1)).reshape(-1, 2)


# ---------------------------------------------------------------- outer costs

def min_image(D, t):
    L = np.array([t["Lx"], t["Ly"]])
    return D - L * np.round(D / L)


def cost_v2v(X, Xt, t):
    """C = (1 / 2N) sum_i |x_i - x_target,i|^2 (Methods, v2v cost), N = V."""
    D = min_image(X - Xt, t)
    N = X.shape[0]
    return float((D * D).sum() / (2.0 * N)), D / N


def shape_tensor_anisotropy(X, t, q_target):
    """Mean cell-shape-tensor anisotropy cost and its gradient.

    S_alpha = (1/k) sum_i (r_i - c_alpha)(r_i - c_alpha)^T over the k corners
    of cell alpha (unwrapped in the cell's local frame, c_alpha their mean);
    Q = mean_alpha S_alpha; q = ((Qxx - Qyy) / tr Q, 2 Qxy / tr Q);
    C = |q - q_target|^2.
    """
    he = t["he"]
    n = t["n"]
    V = X.shape[0]
    g = geometry(X, t)
    q = g["q"]
    face = he[:, HE_FACE]
    cnt = np.bincount(face, minlength=n).astype(np.float64)
    c = np.stack([np.bincount(face, weights=q[:, i], minlength=n) for i in range(2)], axis=1) / cnt[:, None]
    w = q - c[face]
    Sxx = np.bincount(face, weights=w[:, 0] ** 2, minlength=n) / cnt
    Syy = np.bincount(face, weights=w[:, 1] ** 2, minlength=n) / cnt
    Sxy = np.bincount(face, weights=w[:, 0] * w[:, 1], minlength=n) / cnt
    Qxx, Qyy, Qxy = Sxx.mean(), Syy.mean(), Sxy.mean()
    T = Qxx + Qyy
    q1, q2 = (Qxx - Qyy) / T, 2.0 * Qxy / T
    C = (q1 - q_target[0]) ** 2 + (q2 - q_target[1]) ** 2
    r1, r2 = 2.0 * (q1 - q_target[0]), 2.0 * (q2 - q_target[1])
    Gxx = r1 * 2.0 * Qyy / T ** 2 + r2 * (-2.0 * Qxy / T ** 2)
    Gyy = r1 * (-2.0 * Qxx / T ** 2) + r2 * (-2.0 * Qxy / T ** 2)
    Gxy = r2 * 2.0 / T
    k = cnt[face]
    gx = (2.0 * Gxx * w[:, 0] + Gxy * w[:, 1]) / (n * k)
    gy = (2.0 * Gyy * w[:, 1] + Gxy * w[:, 0]) / (n * k)
    src = he[:, HE_SRC]
    grad = np.stack([np.bincount(src, weights=gx, minlength=V),
                     np.bincount(src, weights=gy, minlength=V)], axis=1)
    return float(C), grad


# ------------------------------------------------- parameter derivatives of E

def dE_dtheta(X, t, p):
    """Partial derivatives of E with respect to Lambda_e, A0_alpha, P0_alpha at
    fixed X (the quantities equilibrium propagation differences)."""
    KA, KP, A0, P0, lam = params_arrays(t, p)
    g = geometry(X, t)
    rep = edge_rep(t)
    return dict(lam=g["ell"][rep].copy(), A0=-2.0 * KA * (g["A"] - A0),
                P0=-2.0 * KP * (g["P"] - P0))


def mixed_vjp(X, t, p, lam_vec):
    """(d^2 E / dX dtheta)^T lam_vec for theta = (Lambda, A0, P0)."""
    KA, KP, A0, P0, lam = params_arrays(t, p)
    he = t["he"]
    n = t["n"]
    g, dA, dP, u = cell_gradients(X, t)
    rep = edge_rep(t)
    s, tt = he[rep, HE_SRC], he[rep, HE_TGT]
    out_lam = (u[rep] * (lam_vec[tt] - lam_vec[s])).sum(axis=1)
    face = he[:, HE_FACE]
    src = he[:, HE_SRC]
    dotA = np.bincount(face, weights=(dA * lam_vec[src]).sum(axis=1), minlength=n)
    dotP = np.bincount(face, weights=(dP * lam_vec[src]).sum(axis=1), minlength=n)
    return dict(lam=out_lam, A0=-2.0 * KA * dotA, P0=-2.0 * KP * dotP)
