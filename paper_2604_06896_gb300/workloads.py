"""Workloads built on the library's calls: the rigidity-transition sweep and
the bilevel parameter-inference loop.

* rigidity_sweep (Results, "Inference of mechanical parameters from
  microscopy image": forward simulations of the solid-to-fluid transition
  as the target shape factor p0 grows; Fig. 3g left): many random periodic
  Voronoi tissues relaxed at every p0 of a grid, all tissues and all p0 in
  one batched launch (vx_minimize_batched), and the fraction of relaxations
  that end in a zero-energy state at each p0, with the sigmoid
  1 / (1 + exp(-(p0 - p*) / w)) fitted to it.
* infer_parameters (Methods, "Bilevel optimization framework" and "Outer
  optimisation"; the synthetic benchmark of Fig. 2): the outer loop
  min_theta C(X*(theta)) with X* = EquilibriumFn (vx_minimize forward, the
  implicit adjoint backward) and Adam on theta; C is the v2v cost.

The numerical work runs in the CUDA library; these functions arrange the
calls and reduce their results on the host.
"""
from __future__ import annotations

import math

import numpy as np


def rigidity_sweep(vx, seeds_list, box, p0_grid, energy_threshold=1e-6, dtype="f64",
                   opts=None, return_states=False):
    """Relax every tissue at every p0 of p0_grid in one batched launch.

    seeds_list: list of seed arrays (one tissue each) in a box (Lx, Ly) of
    area n A0 with A0 = 1; the energy is the dimensionless E1 of Eq.
    (Energy1) (K_A = K_P = 1, no line tension); FIRE with the T1 rule of
    Methods, "T1 transitions" (l_min = 5e-3).  A relaxation is a zero-energy
    state when its final energy per cell is below energy_threshold.  The
    default 1e-6 separates the two populations the relaxations end in: the
    floppy states keep meeting short edges (stretches and T1s, each a
    perturbation of order K_P l_min^2 = 2.5e-5 on a cell) and end between
    1e-11 and 1e-6 per cell, the rigid minima at 6e-6 per cell and above
    next to the transition.  Returns dict(p0, fraction, energies
    [len(p0), tissues], fit=(p_star, width), results) and, with
    return_states, the relaxed positions and topologies (tissue-major, p0
    minor: entry t * len(p0_grid) + j)."""
    import torch
    Lx, Ly = box
    meshes = [vx.vx_build_mesh(s, Lx, Ly) for s in seeds_list]
    T, G = len(meshes), len(p0_grid)
    b = vx.Batch([m for m in meshes for _ in range(G)], dtype)
    X = torch.tensor(np.concatenate([m["vert"] for m in meshes for _ in range(G)]),
                     dtype=torch.float64, device="cuda")
    P0 = np.array([p for _ in range(T) for p in p0_grid], dtype=np.float64)
    params = dict(KA=1.0, KP=1.0, A0=1.0, P0=P0, lam=0.0)
    o = dict(tol=1e-10, max_iter=50000, dt0=0.01, dt_max=0.5, l_min=5e-3)
    o.update(opts or {})
    rs = vx.vx_minimize_batched(b, X, params, **o)
    states = None
    if return_states:
        states = (b.split(X.cpu().numpy()), b.topologies())
    b.close()
    n = np.array([m["face_he"].shape[0] for m in meshes for _ in range(G)], dtype=np.float64)
    e = np.array([r.energy for r in rs]) / n
    energies = e.reshape(T, G).T
    frac = (energies < energy_threshold).mean(axis=1)
    out = dict(p0=np.asarray(p0_grid, dtype=np.float64), fraction=frac, energies=energies,
               fit=fit_sigmoid(np.asarray(p0_grid, dtype=np.float64), frac), results=rs)
    if states is not None:
        out["X"], out["topologies"] = states
    return out


def fit_sigmoid(x, y):
    """Least-squares fit of y = 1 / (1 + exp(-(x - x0) / w)); returns (x0, w)."""
    from scipy.optimize import curve_fit
    f = lambda x, x0, w: 1.0 / (1.0 + np.exp(-(x - x0) / w))
    i = int(np.argmin(np.abs(y - 0.5)))
    try:
        (x0, w), _ = curve_fit(f, x, y, p0=(x[i], 0.05), maxfev=10000)
    except Exception:
        x0, w = float(x[i]), float("nan")
    return float(x0), float(w)


def infer_parameters(vx, tissue, X0, target, base, theta0, which="P0", epochs=350, lr=1e-3,
                     inner=None, callback=None):
    """Adam on one parameter family (which = 'P0', 'A0' or 'lam') to fit the
    equilibrium to a target: C = (1 / 2V) sum |X*_i - target_i|^2 (minimum
    image).  Each epoch relaxes from X0 (the tissue's topology is restored
    first, so every epoch starts from the same state) and back-propagates
    through the implicit adjoint.  Returns (theta, cost history)."""
    import torch
    dev = "cuda"
    theta = torch.tensor(np.asarray(theta0, dtype=np.float64), device=dev, requires_grad=True)
    X0 = torch.as_tensor(np.asarray(X0, dtype=np.float64), device=dev)
    Xt = torch.as_tensor(np.asarray(target, dtype=np.float64), device=dev)
    L = torch.tensor([tissue.Lx, tissue.Ly], dtype=torch.float64, device=dev)
    n, E = tissue.n, tissue.E
    fixed = {k: torch.as_tensor(np.broadcast_to(np.asarray(base[k], dtype=np.float64),
                                                (E,) if k == "lam" else (n,)).copy(), device=dev)
             for k in ("lam", "A0", "P0")}
    opt = torch.optim.Adam([theta], lr=lr)
    o = dict(tol=1e-10, max_iter=20000, dt0=0.01, dt_max=0.5, l_min=5e-3, wrap=0)
    o.update(inner or {})
    hist = []
    for ep in range(epochs):
        vx.vx_tissue_restore(tissue)
        args = dict(fixed)
        args[which] = theta
        Xs = vx.EquilibriumFn.apply(X0, args["lam"], args["A0"], args["P0"], tissue,
                                    base["KA"], base["KP"], o)
        D = Xs - Xt
        D = D - L * torch.round(D / L)
        C = (D * D).sum() / (2.0 * Xs.shape[0])
        opt.zero_grad()
        C.backward()
        opt.step()
        hist.append(float(C.detach()))
        if callback:
            callback(ep, hist[-1], theta.detach())
    return theta.detach().cpu().numpy(), hist
