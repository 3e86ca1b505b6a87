"""The 1,000-cell parameter-inference workload at full size.

Hidden tensions Lambda* give the target equilibrium X_target; trial tensions
give X*; the outer cost is v2v.  The GPU adjoint gradient with respect to
the 3,000 tensions is compared with the oracle's dense adjoint at the same
X* (FP64: 1e-8; FP32: 1e-4, the workload's bound), with equilibrium
propagation, and with central finite differences of the cost on the
workload's 20 edges (re-minimised with the FP64 GPU minimiser at fixed
topology; the oracle's adjoint is itself pinned against FD of the oracle).
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


@pytest.fixture(scope="module")
def c4(vx):
    import torch
    c = vi.tissue_c4()
    mesh = vx.vx_build_mesh(c["seeds"], c["Lx"], c["Ly"])
    base = dict(KA=c["KA"], KP=c["KP"], A0=c["A0"], P0=c["P0"])
    opts = dict(tol=1e-10, max_iter=200000, dt0=0.01, dt_max=0.5, l_min=5e-3)
    t = vx.Tissue(mesh, "f64")
    Xt = torch.tensor(mesh["vert"], dtype=torch.float64, device="cuda")
    r_t = vx.vx_minimize(t, Xt, dict(base, lam=c["lam_hidden"]), **opts)
    # the trial solve starts from the relaxed target state and its topology
    Xs = Xt.clone()
    r_s = vx.vx_minimize(t, Xs, dict(base, lam=c["lam"]), **opts)
    top = t.topology()
    top["vert"] = Xs.cpu().numpy()
    t.close()
    print(f"c4: target {r_t.status} {r_t.iters} it; trial {r_s.status} {r_s.iters} it")
    assert r_t.converged and r_s.converged
    return c, base, top, Xt.cpu().numpy(), Xs.cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_c4_adjoint_vs_oracle_ep_fd(vx, c4):
    import torch
    c, base, top, Xtgt, Xs = c4
    p = dict(base, lam=c["lam"])
    C, G = omodel.cost_v2v(Xs, Xtgt, top)
    g_ref, _, info = osolv.adjoint_grad(Xs, top, p, G)
    assert info["pd"]
    out = {}
    for dtype, tol, rtol in (("f64", 1e-8, 1e-12), ("f32", 1e-4, 1e-6)):
        t = vx.Tissue(top, dtype)
        g, r = vx.vx_equilibrium_grad(t, Xs, p, cost=vx.VX_COST_V2V, cost_data=Xtgt, cg_rtol=rtol)
        e = rel(g["lam"].cpu().numpy(), g_ref["lam"])
        print(f"c4 adjoint {dtype}: cg {r.cg_iters} it, rel res {r.cg_rel_residual:.1e}, vs oracle {e:.2e}")
        assert r.status == 0 and e < tol
        assert abs(r.cost - C) < 1e-10 * C
        out[dtype] = g["lam"].cpu().numpy()
        t.close()
    # equilibrium propagation (centred, beta = 1e-2 and 1e-3 as in the workload)
    t = vx.Tissue(top, "f64")
    for beta in (1e-2, 1e-3):
        g, r = vx.vx_equilibrium_grad(t, Xs, p, mode=vx.VX_EP_CENTERED, beta=beta,
                                      cost=vx.VX_COST_V2V, cost_data=Xtgt,
                                      inner=dict(tol=1e-13, max_iter=200000, dt0=0.01, dt_max=0.5))
        e = rel(g["lam"].cpu().numpy(), g_ref["lam"])
        print(f"c4 EP beta={beta}: nudged {r.nudged_iters}, vs adjoint {e:.2e}")
        assert r.status == 0 and e < 1e-2
    # central FD on the workload's 20 edges, re-minimised on the GPU (FP64);
    # h = 1e-4 keeps the re-minimisation noise (tol / h) below the O(h^2) error
    h = 1e-4
    lam = np.array(c["lam"])
    fd = []
    for e_ in c["fd_edges"]:
        vals = []
        for sgn in (1.0, -1.0):
            l2 = lam.copy()
            l2[e_] += sgn * h
            X = torch.tensor(Xs, dtype=torch.float64, device="cuda")
            r = vx.vx_minimize(t, X, dict(base, lam=l2), tol=1e-12, max_iter=200000, dt0=0.01,
                               dt_max=0.5)
            assert r.converged
            vals.append(omodel.cost_v2v(X.cpu().numpy(), Xtgt, top)[0])
        fd.append((vals[0] - vals[1]) / (2 * h))
    fd = np.array(fd)
    e = np.abs(out["f64"][c["fd_edges"]] - fd).max() / np.abs(fd).max()
    print(f"c4 FD on 20 edges: max rel err {e:.2e}")
    assert e < 1e-4
    t.close()
