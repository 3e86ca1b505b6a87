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


def test_batch_grad_vs_oracle(vx):
    """vx_batch_grad on four small FP64 tissues (anisotropy cost, per-cell
    A0 and per-edge tensions as parameters): the free relaxation follows the
    oracle's (same T1 decisions and topology), and the adjoint and centred
    EP gradients of the one launch match the oracle's adjoint and EP at the
    oracle's equilibrium."""
    import torch
    sizes, p0s = [60, 150, 90, 220], [3.5, 3.6, 3.55, 3.65]
    cs = [vi.small_tissue(n, 620 + k, p0=p0, lam_range=(0.02, 0.1))
          for k, (n, p0) in enumerate(zip(sizes, p0s))]
    meshes = [omesh.build_periodic_voronoi(c["seeds"], c["Lx"], c["Ly"]) for c in cs]
    rng = np.random.default_rng(621)
    A0s = [rng.uniform(0.9, 1.1, n) for n in sizes]
    b = vx.Batch(meshes, "f64")
    X = torch.tensor(np.concatenate([m["vert"] for m in meshes]), dtype=torch.float64,
                     device="cuda")
    params = dict(KA=1.0, KP=1.0, A0=torch.tensor(np.concatenate(A0s), device="cuda"),
                  P0=np.array(p0s), lam=torch.tensor(np.concatenate([c["lam"] for c in cs]),
                                                     device="cuda"))
    free = dict(tol=1e-11, max_iter=100000, dt0=0.01, dt_max=0.5, l_min=5e-3, wrap=0)
    inner = dict(tol=1e-12, max_iter=100000, dt0=0.01, dt_max=0.5)
    beta = 0.2
    ga, ge, rs = vx.vx_batch_grad(b, X, params, vx.VX_COST_ANISO, QT, what=3, free=free,
                                  beta=beta, cg_rtol=1e-13, inner=inner)
    tops = b.topologies()
    Xs = b.split(X.cpu().numpy())
    for k in range(b.count):
        p = dict(KA=1.0, KP=1.0, A0=A0s[k], P0=p0s[k], lam=cs[k]["lam"])
        ro = osolv.relax(meshes[k]["vert"], meshes[k], p,
                         osolv.MinOpts(tol=1e-11, max_iter=100000, dt0=0.01, dt_max=0.5),
                         l_min=5e-3)
        fr, ra, re = rs[k]
        assert fr.converged and ro.converged
        assert (fr.n_t1, fr.n_stretch) == (ro.n_t1, ro.n_stretch)
        assert np.array_equal(tops[k]["he"], ro.tissue["he"])
        assert np.abs(Xs[k] - ro.X).max() < 1e-7
        t = ro.tissue
        gradC = lambda Y: omodel.shape_tensor_anisotropy(Y, t, QT)[1]
        C, G = omodel.shape_tensor_anisotropy(ro.X, t, QT)
        g_adj, _, info = osolv.adjoint_grad(ro.X, t, p, G)
        g_ep, _ = osolv.ep_grad(ro.X, t, p, gradC, beta, osolv.MinOpts(
            tol=1e-12, max_iter=100000, dt0=0.01, dt_max=0.5), centered=True)
        e0, e1 = b.ebase[k], b.ebase[k] + b.E[k]
        c0, c1 = b.cbase[k], b.cbase[k] + b.n[k]
        sl = {"lam": slice(e0, e1), "A0": slice(c0, c1), "P0": slice(c0, c1)}
        ea = {q: rel(ga[q][sl[q]].cpu().numpy(), g_adj[q]) for q in ("lam", "A0")}
        ee = {q: rel(ge[q][sl[q]].cpu().numpy(), g_ep[q]) for q in ("lam", "A0")}
        print(f"batch grad tissue {k} n={sizes[k]}: free {fr.iters} it {fr.n_t1} T1; cg "
              f"{ra.cg_iters}; EP {re.nudged_iters}; adjoint {ea}; EP {ee}")
        assert ra.status == 0 and re.status == 0
        assert abs(ra.cost - C) < 1e-9 * abs(C)
        for q in ("lam", "A0"):
            assert ea[q] < 1e-6, (k, q)
            assert ee[q] < 1e-6, (k, q)
    b.close()


@pytest.mark.parametrize("team,what", [("auto", 3), ("cluster", 1), ("resident", 1)])
def test_batch_grad_c5_full_size(vx, team, what):
    """The batched inverse-design workload at full size: 64 tissues of
    10,000 cells, FP32, anisotropy cost, per-cell A0 and per-edge tensions,
    free relaxation (T1 on, fixed budget), the adjoint and (what = 3)
    centred EP with FP64 nudged phases, in one launch: an 8-CTA cluster per
    tissue (the automatic choice for tissues this large), a 16-CTA cluster
    or one CTA per tissue (forced).  Checked on sampled tissues: the oracle's energy, max
    |F| and cost at the returned state agree with the GPU's, and the
    batched adjoint equals the single-tissue adjoint at the same state.
    EP's accuracy is not asserted here: the free relaxations stop at the
    iteration budget with max|F| of 1e-3 to 1e-1, while the nudge
    beta * grad C of the anisotropy cost is ~5e-8 per vertex, so the nudged
    phases measure the continued relaxation, not the nudge (EP against the
    adjoint at converged equilibria is asserted on smaller batches)."""
    import torch
    batch = vi.batch_c5()
    meshes = [vx.vx_build_mesh(c["seeds"], c["Lx"], c["Ly"]) for c in batch]
    b = vx.Batch(meshes, "f32")
    X = torch.tensor(np.concatenate([m["vert"] for m in meshes]), dtype=torch.float64,
                     device="cuda")
    lam = torch.tensor(np.concatenate([c["lam"] for c in batch]), device="cuda")
    A0 = torch.ones(int(b.n.sum()), dtype=torch.float64, device="cuda")
    params = dict(KA=1.0, KP=1.0, A0=A0, P0=3.7, lam=lam)
    free = dict(tol=1e-6, max_iter=10000, dt0=0.01, dt_max=0.5, l_min=5e-3, path=team)
    inner = dict(tol=1e-7, max_iter=5000, dt0=0.01, dt_max=0.5)
    ga, ge, rs = vx.vx_batch_grad(b, X, params, vx.VX_COST_ANISO, (0.1, 0.0), what=what,
                                  free=free, beta=1e-2, cg_rtol=1e-6, inner=inner, ep_f64=1)
    print(f"c5 ({team}): free", [r[0].status for r in rs].count(0), "converged of", b.count,
          "; iters", min(r[0].iters for r in rs), max(r[0].iters for r in rs),
          "; cg", min(r[1].cg_iters for r in rs), max(r[1].cg_iters for r in rs),
          "; EP", min(r[2].nudged_iters[0] for r in rs), max(r[2].nudged_iters[0] for r in rs))
    assert all(r[0].status in (0, 1) for r in rs)
    assert all(r[1].status == 0 for r in rs)
    if what & 2:
        assert all(r[2].status in (0, 1) and r[2].nudged_iters[0] > 0 for r in rs)
    tops = b.topologies()
    Xs = b.split(X.cpu().numpy())
    for k in (0, 37):
        p = dict(KA=1.0, KP=1.0, A0=1.0, P0=3.7, lam=batch[k]["lam"])
        top = dict(tops[k], vert=Xs[k])
        F = omodel.forces(Xs[k], top, p)
        fo = np.sqrt((F * F).sum(axis=1)).max()
        E = omodel.energy(Xs[k], top, p)
        fr, ra, re = rs[k]
        C, _ = omodel.shape_tensor_anisotropy(Xs[k], top, (0.1, 0.0))
        assert abs(fr.energy - E) < 1e-5 * abs(E)
        assert abs(fo - fr.fmax) < 1e-2 * fr.fmax + 1e-7
        assert abs(ra.cost - C) < 1e-8 * abs(C) + 1e-14
        t = vx.Tissue(top, "f32")
        g1, r1 = vx.vx_equilibrium_grad(t, Xs[k], p, cost=vx.VX_COST_ANISO,
                                        cost_data=np.array([0.1, 0.0]), cg_rtol=1e-6)
        t.close()
        e0, e1 = b.ebase[k], b.ebase[k] + b.E[k]
        ga_k = ga["lam"][e0:e1].cpu().numpy()
        e_single = rel(ga_k, g1["lam"].cpu().numpy())
        e_ep = rel(ge["lam"][e0:e1].cpu().numpy(), ga_k) if what & 2 else float("nan")
        print(f"c5 tissue {k}: free {fr.status} {fr.iters} it fmax {fr.fmax:.1e} (oracle {fo:.1e}); "
              f"batched vs single adjoint {e_single:.1e}; EP vs adjoint {e_ep:.1e}")
        assert e_single < 1e-3
    b.close()
