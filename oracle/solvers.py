"""Oracle: inner minimisers and equilibrium gradients.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this.

* Gradient descent, X <- X - eta grad_X E (Methods, "Simulation engine"),
  halted when max_i |F_i| < tol held for ``patience`` consecutive checks or
  at ``max_iter`` (the paper's stopping rule).
* T1 transitions (Methods, "T1 transitions") are checked at the start of
  every iteration, before the force evaluation, when l_min is given; the
  velocities of the two vertices of every modified edge are set to zero.
* FIRE (Bitzek, Koskinen, Gaehler, Moseler, Gumbsch, "Structural relaxation
  made simple", PRL 97, 170201, 2006), unit masses, semi-implicit Euler MD
  step.  One iteration: evaluate F at x; test convergence; P = F.v; if P > 0
  mix v <- (1 - alpha) v + alpha |v| F/|F| and, once more than N_min steps
  have passed since the last reset, dt <- min(f_inc dt, dt_max) and
  alpha <- f_alpha alpha; otherwise v <- 0, dt <- f_dec dt, alpha <- alpha0;
  then v <- v + dt F, x <- x + dt v.
* Adjoint implicit differentiation (Methods, "Implicit differentiation"):
  grad_theta C = d_theta C - (d^2 E/dX dtheta)^T H^-1 grad_X C, with the
  linear system solved densely.  H has the two rigid translations in its
  null space, so the oracle solves (H + c t1 t1^T + c t2 t2^T) lam = Pi b,
  t_k the normalised translations, Pi the projection removing them.
* Equilibrium propagation (Methods, "Equilibrium propagation"): the centred
  estimator (1/beta)[d_theta E(X*_{+beta/2}) - d_theta E(X*_{-beta/2})] and
  the one-sided (1/beta)[d_theta E_aug(X*_beta) - d_theta E_aug(X*_0)], with
  the nudged equilibria minimising E + s C, warm-started from the free X*.
  The nudging force is -s Pi grad_X C, the translation-free part of the cost
  gradient: E does not see rigid translations, so E - (beta/2) C has no
  minimum along them when C (like v2v) is not translation invariant; the
  estimate is unchanged because the translations are in the null space of
  (d^2E/dX dtheta)^T.
* Central finite differences of the outer cost with re-minimisation (at
  fixed topology, like the nudged phases).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla

from . import model, topology


@dataclass
class MinOpts:
    method: str = "fire"          # "fire" or "gd"
    tol: float = 1e-8
    max_iter: int = 100_000
    patience: int = 1
    gd_lr: float = 1e-2
    dt0: float = 0.1
    dt_max: float = 1.0
    n_min: int = 5
    f_inc: float = 1.1
    f_dec: float = 0.5
    alpha0: float = 0.1
    f_alpha: float = 0.99


@dataclass
class MinResult:
    X: np.ndarray
    tissue: dict        # final topology (T1 transitions may have changed it)
    converged: bool
    iters: int          # number of position updates made
    fmax: float         # max_i |F_i| at the returned X
    n_t1: int = 0
    n_stretch: int = 0
    energy_trace: list = None


def minimize(X0, t, p, opts: MinOpts, l_min=None, extra_force=None, trace_every=0):
    """Relax X0 under E (plus ``extra_force(X)`` when given, e.g. -s grad C for
    a nudged phase).  T1 checks run each iteration when l_min is given."""
    x = np.array(X0, dtype=np.float64, copy=True)
    v = np.zeros_like(x)
    dt, alpha, n_pos, below = opts.dt0, opts.alpha0, 0, 0
    n_t1 = n_st = 0
    trace = []
    fmax = float("inf")
    for it in range(opts.max_iter + 1):
        if l_min is not None:
            x, t, touched, a, b = topology.t1_pass(x, t, p, l_min)
            n_t1 += a
            n_st += b
            if touched:
                v[touched] = 0.0
        F = model.forces(x, t, p)
        if extra_force is not None:
            F = F + extra_force(x)
        fmax = float(np.sqrt((F * F).sum(axis=1)).max())
        if trace_every and it % trace_every == 0:
            trace.append(model.energy(x, t, p))
        below = below + 1 if fmax < opts.tol else 0
        if below >= opts.patience:
            return MinResult(x, t, True, it, fmax, n_t1, n_st, trace)
        if it == opts.max_iter:
            break
        if opts.method == "gd":
            x = x + opts.gd_lr * F
            continue
        P = float((F * v).sum())
        if P > 0.0:
            vn = float(np.sqrt((v * v).sum()))
            fn = float(np.sqrt((F * F).sum()))
            v = (1.0 - alpha) * v + alpha * (vn / fn) * F
            if n_pos > opts.n_min:
                dt = min(dt * opts.f_inc, opts.dt_max)
                alpha = alpha * opts.f_alpha
            n_pos += 1
        else:
            v = np.zeros_like(x)
            dt = dt * opts.f_dec
            alpha = opts.alpha0
            n_pos = 0
        v = v + dt * F
        x = x + dt * v
    return MinResult(x, t, False, opts.max_iter, fmax, n_t1, n_st, trace)


def relax(X0, t, p, opts: MinOpts, l_min=None, **kw):
    return minimize(X0, t, p, opts, l_min=l_min, **kw)


# ------------------------------------------------------------------ adjoint

def translations(V):
    t1 = np.zeros(2 * V)
    t2 = np.zeros(2 * V)
    t1[0::2] = 1.0 / np.sqrt(V)
    t2[1::2] = 1.0 / np.sqrt(V)
    return t1, t2


def adjoint_solve(X, t, p, b):
    """Solve H lam = Pi b densely (b float64 [V, 2]).  Returns (lam, info)
    with info['min_eig'] the smallest eigenvalue of H restricted to
    translation-free vectors (None when the Cholesky factorisation succeeded
    without needing it)."""
    V = X.shape[0]
    H = model.hessian(X, t, p, dense=True)
    t1, t2 = translations(V)
    rhs = b.reshape(-1).copy()
    rhs -= t1 * (t1 @ rhs) + t2 * (t2 @ rhs)
    c = np.trace(H) / (2 * V)
    M = H + c * (np.outer(t1, t1) + np.outer(t2, t2))
    try:
        cf = sla.cho_factor(M)
        lam = sla.cho_solve(cf, rhs)
        info = dict(pd=True, min_eig=None)
    except np.linalg.LinAlgError:
        w, U = np.linalg.eigh(M)
        lam = U @ ((U.T @ rhs) / w)
        info = dict(pd=False, min_eig=float(w.min()))
    lam -= t1 * (t1 @ lam) + t2 * (t2 @ lam)
    return lam.reshape(-1, 2), info


def adjoint_grad(X, t, p, dCdX):
    """grad_theta C = -(d^2E/dX dtheta)^T H^-1 grad_X C (d_theta C = 0 for the
    built-in costs)."""
    lam, info = adjoint_solve(X, t, p, dCdX)
    m = model.mixed_vjp(X, t, p, lam)
    return {k: -v for k, v in m.items()}, lam, info


# ------------------------------------------------------ equilibrium propagation

def project_translations(G):
    """Pi G: G minus its mean over vertices (removes rigid translations)."""
    return G - G.mean(axis=0)


def nudged_relax(X0, t, p, cost_grad_fn, s, opts: MinOpts):
    """Minimise E + s C from X0 (cost_grad_fn(X) -> grad_X C) at fixed
    topology (no T1: the estimator differences two equilibria of one
    tissue), with the translation-free nudging force -s Pi grad_X C."""
    return minimize(X0, t, p, opts,
                    extra_force=lambda X: -s * project_translations(cost_grad_fn(X)))


def ep_grad(Xstar, t, p, cost_grad_fn, beta, opts: MinOpts, centered=True):
    if centered:
        rp = nudged_relax(Xstar, t, p, cost_grad_fn, +0.5 * beta, opts)
        rm = nudged_relax(Xstar, t, p, cost_grad_fn, -0.5 * beta, opts)
        dp, dm = model.dE_dtheta(rp.X, t, p), model.dE_dtheta(rm.X, t, p)
        return {k: (dp[k] - dm[k]) / beta for k in dp}, (rp, rm)
    rb = nudged_relax(Xstar, t, p, cost_grad_fn, beta, opts)
    dp, d0 = model.dE_dtheta(rb.X, t, p), model.dE_dtheta(Xstar, t, p)
    return {k: (dp[k] - d0[k]) / beta for k in dp}, (rb,)


# ------------------------------------------------------- finite differences

def fd_grad_lambda(Xstar, t, p, cost_fn, edges, h, opts: MinOpts):
    """Central FD of C(X*(Lambda +- h e_k)) for the listed edges, each side
    re-minimised from the free X*."""
    lam = np.array(model.params_arrays(t, p)[4])
    out = []
    for e in edges:
        vals = []
        for sgn in (+1.0, -1.0):
            q = dict(p)
            l2 = lam.copy()
            l2[e] += sgn * h
            q["lam"] = l2
            r = relax(Xstar, t, q, opts)
            vals.append(cost_fn(r.X))
        out.append((vals[0] - vals[1]) / (2.0 * h))
    return np.array(out)
