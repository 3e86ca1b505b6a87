"""MINRES adjoint and forward sensitivities (Methods, "Implicit
differentiation") on the GPU against the oracle.

* On an indefinite Hessian (a 40-cell Voronoi state at p0 = 4.4: 75 negative
  eigenvalues) CG stops with VX_ERR_INDEFINITE, and MINRES reaches the
  oracle's solution (its dense eigendecomposition on the translation-free
  subspace).
* On a positive definite Hessian MINRES and CG give the same gradient.
* The forward form (one solve per parameter) gives the adjoint's numbers.
"""
import numpy as np
import pytest

import vx_inputs as vi
from oracle import mesh as omesh
from oracle import model as omodel
from oracle import solvers as osolv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vx():
    import paper_2604_06896_gb300 as vx
    return vx


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def indefinite_case():
    c = vi.small_tissue(40, 101, p0=4.4, lam_range=(0.02, 0.1))
    t = omesh.build_periodic_voronoi(c["seeds"], c["Lx"], c["Ly"])
    p = {k: c[k] for k in ("KA", "KP", "A0", "P0", "lam")}
    return c, t, p, t["vert"]


@pytest.mark.parametrize("dtype,rtol,tol", [("f64", 1e-12, 1e-6), ("f32", 1e-6, 1e-2)])
def test_minres_on_an_indefinite_hessian(vx, dtype, rtol, tol):
    """FP32 products (condition number ~2e4) limit the FP32 tissue to a
    residual of ~1e-6 and a solution error of ~1e-7 x 2e4."""
    c, t, p, X = indefinite_case()
    w = np.random.default_rng(102).standard_normal(X.shape)
    g_ref, _, info = osolv.adjoint_grad(X, t, p, w)
    assert not info["pd"] and info["min_eig"] < 0
    tis = vx.Tissue(t, dtype)
    with pytest.raises(vx.VxError, match="INDEFINITE"):
        vx.vx_equilibrium_grad(tis, X, p, dCdX=w, cg_rtol=rtol)
    g, r = vx.vx_equilibrium_grad(tis, X, p, dCdX=w, mode=vx.VX_ADJOINT_MINRES, cg_rtol=rtol,
                                  cg_max_iter=50000)
    errs = {k: rel(g[k].cpu().numpy(), g_ref[k]) for k in ("lam", "A0", "P0")}
    print(f"MINRES {dtype}: {r.cg_iters} iterations, residual {r.cg_rel_residual:.1e}, "
          f"min eig {info['min_eig']:.1f}; vs oracle {errs}")
    assert r.status == 0
    for k, e in errs.items():
        assert e < tol, k
    tis.close()


@pytest.fixture(scope="module")
def equilibrium():
    c = vi.small_tissue(120, 103, p0=3.7, lam_range=(0.02, 0.1))
    ref = omesh.build_periodic_voronoi(c["seeds"], c["Lx"], c["Ly"])
    p = {k: c[k] for k in ("KA", "KP", "A0", "P0", "lam")}
    r = osolv.relax(ref["vert"], ref, p, osolv.MinOpts(tol=1e-12, max_iter=100000, dt0=0.01,
                                                       dt_max=0.5), l_min=5e-3)
    assert r.converged
    Xt = r.X + 0.03 * np.random.default_rng(104).standard_normal(r.X.shape)
    return c, dict(r.tissue, vert=r.X), p, r.X, Xt


def test_minres_equals_cg_when_definite(vx, equilibrium):
    c, t, p, X, Xt = equilibrium
    tis = vx.Tissue(t, "f64")
    gc, rc = vx.vx_equilibrium_grad(tis, X, p, cost=vx.VX_COST_V2V, cost_data=Xt, cg_rtol=1e-13)
    gm, rm = vx.vx_equilibrium_grad(tis, X, p, cost=vx.VX_COST_V2V, cost_data=Xt,
                                    mode=vx.VX_ADJOINT_MINRES, cg_rtol=1e-13, cg_max_iter=50000)
    print(f"definite: CG {rc.cg_iters} it, MINRES {rm.cg_iters} it")
    assert rc.status == 0 and rm.status == 0
    assert abs(rm.cost - rc.cost) < 1e-14 * rc.cost
    for k in ("lam", "A0", "P0"):
        assert rel(gm[k].cpu().numpy(), gc[k].cpu().numpy()) < 1e-8, k
    tis.close()


@pytest.mark.parametrize("solver", ["cg", "minres"])
def test_sensitivity_equals_adjoint(vx, equilibrium, solver):
    """Forward sensitivities of twelve parameters (tensions, target areas,
    target perimeters) against the oracle's adjoint gradient."""
    c, t, p, X, Xt = equilibrium
    _, G = omodel.cost_v2v(X, Xt, t)
    g_ref, _, info = osolv.adjoint_grad(X, t, p, G)
    assert info["pd"]
    tis = vx.Tissue(t, "f64")
    kinds = [vx.VX_PARAM_LAMBDA] * 4 + [vx.VX_PARAM_A0] * 4 + [vx.VX_PARAM_P0] * 4
    idx = [0, 17, 101, 299, 3, 40, 77, 119, 5, 50, 88, 100]
    mode = vx.VX_ADJOINT_CG if solver == "cg" else vx.VX_ADJOINT_MINRES
    vals, st = vx.vx_sensitivity_grad(tis, X, p, G, kinds, idx, solver=mode, rtol=1e-13,
                                      max_iter=50000)
    ref = np.array([g_ref[{0: "lam", 1: "A0", 2: "P0"}[k]][i] for k, i in zip(kinds, idx)])
    print(f"sensitivities ({solver}): max rel err {np.abs(vals - ref).max() / np.abs(ref).max():.1e}")
    assert np.all(st == 0)
    assert np.abs(vals - ref).max() < 1e-8 * np.abs(ref).max()
    tis.close()
