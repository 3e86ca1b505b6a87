"""Batched adjoint gradients (every tissue of a batch in one persistent
launch) and the batched anisotropy cost, against the FP64 oracle at the same
equilibria and topologies: the oracle's cost and gradient (pinned against
finite differences in the oracle tests) and its dense adjoint.  Tolerances
as for the single-tissue adjoint: FP64 1e-8 relative (CG to rtol 1e-12),
FP32 1e-4 (the workload's bound for outer gradients)."""
import numpy as np
import pytest

import vx_inputs as vi
from oracle import mesh as omesh
from oracle import model as omodel
from oracle import solvers as osolv

pytestmark = pytest.mark.gpu

QT = (0.1, 0.0)


@pytest.fixture(scope="module")
def vx():
    import paper_2604_06896_gb300 as vx
    return vx


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def relaxed(vx):
    """Three tissues relaxed together by the FP64 batched minimiser (T1 on)."""
    import torch
    sizes, p0s = [120, 300, 600], [3.5, 3.55, 3.6]
    cs = [vi.small_tissue(n, 610 + k, p0=p0, lam_range=(0.02, 0.1))
          for k, (n, p0) in enumerate(zip(sizes, p0s))]
    meshes = [omesh.build_periodic_voronoi(c["seeds"], c["Lx"], c["Ly"]) for c in cs]
    b = vx.Batch(meshes, "f64")
    X = torch.tensor(np.concatenate([m["vert"] for m in meshes]), dtype=torch.float64,
                     device="cuda")
    lam = np.concatenate([c["lam"] for c in cs])
    params = dict(KA=1.0, KP=1.0, A0=1.0, P0=np.array(p0s), lam=torch.tensor(lam, device="cuda"))
    rs = vx.vx_minimize_batched(b, X, params, tol=1e-9, max_iter=200000, dt0=0.01, dt_max=0.5,
                                l_min=5e-3)
    for k, r in enumerate(rs):
        print(f"tissue {k} n={sizes[k]}: {r.iters} it, {r.n_t1} T1, fmax {r.fmax:.1e}")
        assert r.converged
    tops = b.topologies()
    Xs = b.split(X.cpu().numpy())
    ps = [dict(KA=1.0, KP=1.0, A0=1.0, P0=p0, lam=c["lam"]) for c, p0 in zip(cs, p0s)]
    yield b, X, params, tops, Xs, ps
    b.close()


def test_batch_aniso_cost_matches_oracle(vx, relaxed):
    b, X, params, tops, Xs, ps = relaxed
    C, G = vx.vx_batch_aniso_cost(b, X, QT)
    Gs = b.split(G.cpu().numpy())
    for k in range(b.count):
        C_ref, G_ref = omodel.shape_tensor_anisotropy(Xs[k], tops[k], QT)
        assert abs(C[k] - C_ref) < 1e-10 * abs(C_ref)
        assert rel(Gs[k], G_ref) < 1e-10


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-8), ("f32", 1e-4)])
def test_batch_adjoint_matches_oracle(vx, relaxed, dtype, tol):
    import torch
    b, X, params, tops, Xs, ps = relaxed
    C, G = vx.vx_batch_aniso_cost(b, X, QT)
    if dtype == "f64":
        bb = b  # its current topology is the relaxed one
    else:
        bb = vx.Batch([dict(t, vert=x) for t, x in zip(tops, Xs)], "f32")
    g, rs = vx.vx_equilibrium_grad_batched(bb, X, params, G,
                                           cg_rtol=1e-12 if dtype == "f64" else 1e-6)
    Gs = b.split(G.cpu().numpy())
    for k in range(b.count):
        g_ref, _, info = osolv.adjoint_grad(Xs[k], tops[k], ps[k], Gs[k])
        assert info["pd"]
        e0, e1 = b.ebase[k], b.ebase[k] + b.E[k]
        c0, c1 = b.cbase[k], b.cbase[k] + b.n[k]
        got = {"lam": g["lam"][e0:e1].cpu().numpy(), "A0": g["A0"][c0:c1].cpu().numpy(),
               "P0": g["P0"][c0:c1].cpu().numpy()}
        print(f"batched adjoint {dtype} tissue {k}: cg {rs[k].cg_iters} it, status "
              f"{rs[k].status}; " + ", ".join(f"{q} {rel(got[q], g_ref[q]):.2e}" for q in got))
        assert rs[k].status == 0
        for q in ("lam", "A0", "P0"):
            assert rel(got[q], g_ref[q]) < tol, (k, q)
    if bb is not b:
        bb.close()
    torch.cuda.synchronize()
