"""Batched minimiser (one persistent launch for many tissues) against the
FP64 oracle and against itself (graph replay is deterministic)."""
import numpy as np
import pytest

import vx_inputs as vi
from oracle import mesh as omesh
from oracle import model as omodel
from oracle import solvers as osolv

from test_oracle_mesh import check_half_edge_invariants

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vx():
    import paper_2604_06896_gb300 as vx
    return vx


def tissues(sizes, stream0, p0s):
    out = []
    for k, (n, p0) in enumerate(zip(sizes, p0s)):
        c = vi.small_tissue(n, stream0 + k, p0=p0, lam_range=(0.02, 0.1))
        m = omesh.build_periodic_voronoi(c["seeds"], c["Lx"], c["Ly"])
        out.append((c, m))
    return out


def soft_mode_bound(X, top, p, tol):
    """How far two relaxations that both stopped at max_i |F_i| < tol can
    end apart: each is within |F|_2 / lambda_min < tol sqrt(V) / lambda_min
    of the exact minimum (lambda_min: the smallest eigenvalue of the
    oracle's Hessian off the two rigid translations), so twice that."""
    H = omodel.hessian(X, top, p, dense=True)
    w = np.sort(np.linalg.eigvalsh(H))
    assert w[2] > 0
    return 2.0 * tol * np.sqrt(X.shape[0]) / w[2], w[2]


def test_batch_fp64_matches_oracle(vx):
    """FP64 batched relaxations (FIRE + T1) against the oracle: the same T1
    decisions and final topology, the same energy, and positions within the
    soft-mode bound.  The trajectories agree up to rounding order; over a
    long relaxation along soft modes a FIRE control decision (the sign of
    F.v near zero) eventually falls the other way, after which the two runs
    take different step sequences to the same minimum: the iteration counts
    then differ by a few per cent and the end points by up to
    tol sqrt(V) / lambda_min.  The single-tissue resident path on the same
    inputs shows the same drift (printed beside the batch's)."""
    import torch
    sizes = [30, 120, 45, 80, 200, 60, 150, 35]
    p0s = [3.6 + 0.03 * k for k in range(len(sizes))]
    ts = tissues(sizes, 500, p0s)
    b = vx.Batch([m for _, m in ts], "f64")
    X = torch.tensor(np.concatenate([m["vert"] for _, m in ts]), dtype=torch.float64, device="cuda")
    lam = np.concatenate([c["lam"] for c, _ in ts])
    params = dict(KA=1.0, KP=1.0, A0=1.0, P0=np.array(p0s), lam=torch.tensor(lam, device="cuda"))
    kw = dict(tol=1e-9, max_iter=50000, dt0=0.01, dt_max=0.5, l_min=5e-3, wrap=0)
    rs = vx.vx_minimize_batched(b, X, params, **kw)
    tops = b.topologies()
    Xs = b.split(X.cpu().numpy())
    for k, ((c, m), r) in enumerate(zip(ts, rs)):
        p = dict(KA=1.0, KP=1.0, A0=1.0, P0=p0s[k], lam=c["lam"])
        ro = osolv.relax(m["vert"], m, p, osolv.MinOpts(tol=1e-9, max_iter=50000, dt0=0.01,
                                                        dt_max=0.5), l_min=5e-3)
        t = vx.Tissue(m, "f64")
        Xk = torch.tensor(m["vert"], dtype=torch.float64, device="cuda")
        r1 = vx.vx_minimize(t, Xk, p, path="resident", **kw)
        t.close()
        bound, lmin = soft_mode_bound(ro.X, ro.tissue, p, 1e-9)
        d = np.abs(Xs[k] - ro.X).max()
        d1 = np.abs(Xk.cpu().numpy() - ro.X).max()
        print(f"tissue {k} n={sizes[k]}: batch {r.iters} it, single {r1.iters} it, oracle "
              f"{ro.iters} it ({r.n_t1} T1); |X - X_oracle| batch {d:.1e} single {d1:.1e}, "
              f"bound {bound:.1e} (lambda_min {lmin:.1e})")
        assert r.converged and ro.converged
        assert (r.n_t1, r.n_stretch) == (ro.n_t1, ro.n_stretch)
        assert np.array_equal(tops[k]["he"], ro.tissue["he"])
        assert abs(r.iters - ro.iters) <= max(2, 0.05 * ro.iters)
        assert abs(r.energy - omodel.energy(ro.X, ro.tissue, p)) < 1e-9 * abs(r.energy)
        assert d < bound
    b.close()


def test_batch_fp32_mixed_residency_and_replay(vx):
    """Tissues that fit shared memory and one that does not (global-memory
    residency) in the same launch; a second call after restoring the
    topology replays the captured graph and gives identical results."""
    import torch
    sizes = [300, 2500, 120, 800, 60, 1500]
    p0s = [3.7] * len(sizes)
    ts = tissues(sizes, 600, p0s)
    b = vx.Batch([m for _, m in ts], "f32")
    X0 = torch.tensor(np.concatenate([m["vert"] for _, m in ts]), dtype=torch.float64, device="cuda")
    lam = torch.tensor(np.concatenate([c["lam"] for c, _ in ts]), device="cuda")
    params = dict(KA=1.0, KP=1.0, A0=1.0, P0=3.7, lam=lam)
    kw = dict(tol=1e-6, max_iter=40000, dt0=0.01, dt_max=0.5, l_min=5e-3)
    X1 = X0.clone()
    r1 = vx.vx_minimize_batched(b, X1, params, **kw)
    tops = b.topologies()
    Xs = b.split(X1.cpu().numpy())
    for k, ((c, m), r) in enumerate(zip(ts, r1)):
        top = dict(tops[k])
        check_half_edge_invariants(dict(top, vert=Xs[k]))
        p = dict(KA=1.0, KP=1.0, A0=1.0, P0=3.7, lam=c["lam"])
        F = omodel.forces(Xs[k], top, p)
        fo = np.sqrt((F * F).sum(axis=1)).max()
        E = omodel.energy(Xs[k], top, p)
        print(f"tissue {k} n={sizes[k]}: status {r.status} it {r.iters} T1 {r.n_t1} fmax {r.fmax:.2e} oracle {fo:.2e}")
        assert r.status in (0, 1)
        assert abs(r.energy - E) < 1e-5 * abs(E)
        assert fo < 2e-6 + 2 * r.fmax
    vx.vx_batch_restore(b)
    X2 = X0.clone()
    r2 = vx.vx_minimize_batched(b, X2, params, **kw)
    assert [r.iters for r in r1] == [r.iters for r in r2]
    assert torch.equal(X1, X2)
    b.close()


def test_batch_autotune(vx):
    import torch
    sizes = [200, 400, 900, 150]
    ts = tissues(sizes, 700, [3.7] * 4)
    b = vx.Batch([m for _, m in ts], "f32")
    X = torch.tensor(np.concatenate([m["vert"] for _, m in ts]), dtype=torch.float64, device="cuda")
    lam = torch.tensor(np.concatenate([c["lam"] for c, _ in ts]), device="cuda")
    params = dict(KA=1.0, KP=1.0, A0=1.0, P0=3.7, lam=lam)
    kw = dict(tol=1e-6, max_iter=40000, dt0=0.01, dt_max=0.5, l_min=5e-3)
    X0 = X.clone()
    T, S = vx.vx_batch_autotune(b, X, params, probe_iters=100, **kw)
    assert T in (128, 256) and S > 0
    assert torch.equal(X, X0)   # probes do not move the caller's positions
    rs = vx.vx_minimize_batched(b, X, params, **kw)
    assert all(r.status in (0, 1) for r in rs)
    b.close()


def c3_sample(ns):
    """The tissues whose outputs the oracle recomputes: the smallest, the
    largest and every 64th."""
    ns = np.asarray(ns)
    return sorted({int(np.argmin(ns)), int(np.argmax(ns))} | set(range(0, len(ns), 64)))


def check_c3_outputs(batch, results, Xs, tops, sample):
    """On the sampled tissues: a solver status (converged or out of
    budget), the oracle's energy and max|F| at the returned state (positions
    and topology) as the GPU reported them, a valid periodic half-edge mesh,
    and areas that tile the box."""
    assert len(results) == len(batch)
    counts = np.bincount([r.status for r in results], minlength=10)
    print("c3 statuses (index = vx_status):", counts.tolist())
    for k in sample:
        c, r, X, top = batch[k], results[k], Xs[k], dict(tops[k])
        assert r.status in (0, 1), (k, r.status)
        t = dict(top, vert=X)
        check_half_edge_invariants(t)
        p = dict(KA=1.0, KP=1.0, A0=1.0, P0=c["P0"], lam=c["lam"])
        F = omodel.forces(X, t, p)
        fo = float(np.sqrt((F * F).sum(axis=1)).max())
        E = omodel.energy(X, t, p)
        A = omodel.geometry(X, t)["A"]
        print(f"c3 tissue {k} n={c['n']}: status {r.status} it {r.iters} T1 {r.n_t1} "
              f"fmax {r.fmax:.2e} oracle {fo:.2e} dE/E {abs(r.energy - E) / abs(E):.1e}")
        assert abs(A.sum() - c["Lx"] * c["Ly"]) < 1e-9 * c["Lx"] * c["Ly"]
        assert abs(r.energy - E) < 1e-5 * abs(E)
        assert fo < 2e-6 + 2 * r.fmax


def test_batch_c3_full_size(vx):
    """The batched forward workload at full size, in the launch the
    benchmark times: 512 tissues of 200-5,000 cells (7.5e5 cells), FP32,
    FIRE + T1 to max|F| < 1e-6 with a 20,000-iteration budget, small tissues
    on CTAs and large ones on 8-CTA clusters in one graph-replayed launch;
    sampled tissues checked against the oracle."""
    import torch
    batch = vi.batch_c3()
    meshes = [vx.vx_build_mesh(c["seeds"], c["Lx"], c["Ly"]) for c in batch]
    b = vx.Batch(meshes, "f32")
    X = torch.tensor(np.concatenate([m["vert"] for m in meshes]), dtype=torch.float64,
                     device="cuda")
    lam = torch.tensor(np.concatenate([c["lam"] for c in batch]), device="cuda")
    prm = dict(KA=1.0, KP=1.0, A0=1.0, P0=np.array([c["P0"] for c in batch]), lam=lam)
    rs = vx.vx_minimize_batched(b, X, prm, tol=1e-6, max_iter=20_000, dt0=0.01, dt_max=0.5,
                                l_min=5e-3)
    tops = b.topologies()
    Xs = b.split(X.cpu().numpy())
    print(f"c3: {sum(r.status == 0 for r in rs)} of {len(rs)} tissues converged")
    check_c3_outputs(batch, rs, Xs, tops, c3_sample([c["n"] for c in batch]))
    b.close()
