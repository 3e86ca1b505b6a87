"""The workloads built on the library: the rigidity-transition sweep and the
bilevel parameter inference (GPU)."""
import math

import numpy as np
import pytest

import vx_inputs as vi
from oracle import model as omodel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vx():
    import paper_2604_06896_gb300 as vx
    return vx


def test_rigidity_sweep(vx):
    """100 random 100-cell tissues relaxed at sixteen target shape indices in
    one batched launch (1,600 relaxations, FP64, FIRE + the T1 rule): the
    fraction of zero-energy states rises from 0 to 1 across the
    solid-to-fluid transition (Results, Fig. 3g left; the paper prints no
    threshold value).  Sampled relaxed states are checked against the
    oracle: the same energy at the returned positions and topology, and
    force balance where the GPU reports convergence."""
    from paper_2604_06896_gb300 import workloads
    n, T = 100, 100
    L = math.sqrt(n)
    seeds = [vi.uniform_seeds(n, L, L, vi.substream(7, i)) for i in range(T)]
    grid = np.round(np.arange(3.60, 4.21, 0.04), 2)
    out = workloads.rigidity_sweep(vx, seeds, (L, L), grid, return_states=True)
    p_star, w = out["fit"]
    frac = out["fraction"]
    med = np.median(out["energies"], axis=1)
    print("p0", out["p0"].tolist())
    print("fraction of zero-energy states", frac.tolist())
    print("median energy per cell", [f"{x:.1e}" for x in med])
    print(f"sigmoid fit: p* = {p_star:.3f}, width {w:.3f}")
    assert all(r.status in (0, 1) for r in out["results"])
    # solid side: none; fluid side: nearly all (a relaxation that stops just
    # after a stretch or T1 still carries that perturbation's energy)
    assert frac[0] == 0.0 and frac.max() > 0.95
    k = int(np.argmax(frac > 0.5))
    assert np.all(frac[k:] > 0.8)
    assert np.all(np.diff(frac[:k + 1]) > -0.1)
    # the energy of the minima falls as p0 approaches the transition
    assert np.all(np.diff(med[:k]) < 0)
    assert 3.8 < p_star < 4.1
    G = len(grid)
    for t, j in ((0, 0), (3, 6), (7, k), (11, G - 1)):
        q = t * G + j
        X, top, r = out["X"][q], out["topologies"][q], out["results"][q]
        prm = dict(KA=1.0, KP=1.0, A0=1.0, P0=float(grid[j]), lam=0.0)
        E = omodel.energy(X, dict(top, vert=X), prm)
        F = omodel.forces(X, dict(top, vert=X), prm)
        fo = float(np.sqrt((F * F).sum(axis=1)).max())
        print(f"tissue {t} p0 {grid[j]}: GPU E {r.energy:.6e} oracle {E:.6e}; fmax GPU {r.fmax:.1e} "
              f"oracle {fo:.1e}")
        assert abs(r.energy - E) <= 1e-10 * abs(E) + 1e-14
        if r.status == 0:
            assert fo < 1e-9

def test_infer_parameters_bilevel(vx):
    """The synthetic benchmark of the paper's Fig. 2 (N = 20 cells, box
    sqrt(N), Adam, T1 minimum length 5e-3): per-cell target shape indices
    inferred from a target equilibrium made with hidden ones, through the
    implicit adjoint.  The cost falls and the inferred parameters correlate
    with the hidden ones."""
    import torch
    from paper_2604_06896_gb300 import workloads
    n = 20
    c = vi.small_tissue(n, 105, p0=3.65)
    mesh = vx.vx_build_mesh(c["seeds"], c["Lx"], c["Ly"])
    rng = vi.SplitMix64(106)
    p0_hidden = rng.uniform(n, 3.55, 3.75)
    base = dict(KA=1.0, KP=1.0, A0=1.0, P0=3.65, lam=0.0)
    t = vx.Tissue(mesh, "f64")
    Xt = torch.tensor(mesh["vert"], dtype=torch.float64, device="cuda")
    r = vx.vx_minimize(t, Xt, dict(base, P0=p0_hidden), tol=1e-10, max_iter=20000, dt0=0.01,
                       dt_max=0.5, l_min=5e-3, wrap=0)
    assert r.converged
    vx.vx_tissue_restore(t)
    theta, hist = workloads.infer_parameters(vx, t, mesh["vert"], Xt.cpu().numpy(), base,
                                             np.full(n, 3.65), which="P0", epochs=350, lr=1e-3)
    corr = np.corrcoef(theta, p0_hidden)[0, 1]
    print(f"bilevel: cost {hist[0]:.3e} -> {hist[-1]:.3e}; Pearson {corr:.3f}; "
          f"max |p0 - p0*| {np.abs(theta - p0_hidden).max():.3f}")
    assert hist[-1] < 0.1 * hist[0]
    assert corr > 0.9
    t.close()
