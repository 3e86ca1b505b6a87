"""Exit-time wrap (Methods, "Periodic mode") on the GPU against the oracle.

A tissue is started from positions shifted by several box lengths, so that
every vertex ends outside the box.  The same solve is run twice from the
same state: once with wrap off (the unwrapped result, the same bits on every
run) and once with wrap on.  The oracle's wrap of the unwrapped result must
equal the wrapped result bit for bit (positions and offsets), and the
energy and forces must be unchanged.
"""
import numpy as np
import pytest

import vx_inputs as vi
from oracle import mesh as omesh
from oracle import topology as otop

pytestmark = pytest.mark.gpu

SHIFT = np.array([1.37, -2.61])


@pytest.fixture(scope="module")
def vx():
    import paper_2604_06896_gb300 as vx
    return vx


def case(n, stream):
    c = vi.small_tissue(n, stream, lam_range=(0.02, 0.1))
    m = omesh.build_periodic_voronoi(c["seeds"], c["Lx"], c["Ly"])
    p = {k: c[k] for k in ("KA", "KP", "A0", "P0", "lam")}
    X0 = m["vert"] + SHIFT * np.array([c["Lx"], c["Ly"]])
    return c, m, p, X0


def run(vx, m, p, X0, dtype, wrap, **opts):
    import torch
    t = vx.Tissue(m, dtype)
    X = torch.tensor(X0, dtype=torch.float64, device="cuda")
    r = vx.vx_minimize(t, X, p, wrap=wrap, **opts)
    top = t.topology()
    return t, X, r, top


@pytest.mark.parametrize("path", ["resident", "cluster", "plain", "grid"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_wrap_matches_oracle(vx, path, dtype):
    c, m, p, X0 = case(400, 71)
    kw = dict(tol=0.0, max_iter=300, dt0=0.01, dt_max=0.5, l_min=5e-3, path=path)
    tu, Xu, ru, topu = run(vx, m, p, X0, dtype, 0, **kw)
    tw, Xw, rw, topw = run(vx, m, p, X0, dtype, 1, **kw)
    assert ru.status == rw.status == vx.capi.VX_NOT_CONVERGED
    assert (ru.iters, ru.n_t1, ru.n_stretch) == (rw.iters, rw.n_t1, rw.n_stretch)
    Xu_h, Xw_h = Xu.cpu().numpy(), Xw.cpu().numpy()
    L = np.array([c["Lx"], c["Ly"]])
    assert np.all(np.abs(Xu_h - Xu_h.mean(axis=0)).max() < 3 * L.max())
    assert np.all(Xu_h[:, 0] > c["Lx"])          # every vertex ended outside the box
    Xo, to = otop.wrap(Xu_h, dict(topu, vert=Xu_h))
    assert np.array_equal(Xw_h, Xo)
    assert np.array_equal(topw["he"], to["he"])
    assert np.all(Xw_h >= 0) and np.all(Xw_h < L)
    # energy and forces unchanged
    Fu, Eu = vx.vx_energy_forces(tu, Xu, p)
    Fw, Ew = vx.vx_energy_forces(tw, Xw, p)
    Fu, Fw = Fu.cpu().numpy(), Fw.cpu().numpy()
    if dtype == "f64":
        assert abs(Ew.item() - Eu.item()) < 1e-12 * abs(Eu.item())
        assert np.abs(Fw - Fu).max() < 1e-12 * np.abs(Fu).max()
    else:
        assert abs(Ew.item() - Eu.item()) < 1e-6 * abs(Eu.item())
        assert np.abs(Fw - Fu).max() < 1e-5 * np.abs(Fu).max()
    tu.close()
    tw.close()


def test_wrap_minimize_many(vx):
    """Several tissues in one launch are wrapped each with its own box."""
    import torch
    cases = [case(n, 72 + k) for k, n in enumerate((150, 3000, 90))]
    ts_u = [vx.Tissue(m, "f64") for _, m, _, _ in cases]
    ts_w = [vx.Tissue(m, "f64") for _, m, _, _ in cases]
    Xs_u = [torch.tensor(X0, dtype=torch.float64, device="cuda") for *_, X0 in cases]
    Xs_w = [x.clone() for x in Xs_u]
    ps = [p for _, _, p, _ in cases]
    kw = dict(tol=0.0, max_iter=200, dt0=0.01, dt_max=0.5, l_min=5e-3)
    vx.vx_minimize_many(ts_u, Xs_u, ps, wrap=0, **kw)
    vx.vx_minimize_many(ts_w, Xs_w, ps, wrap=1, **kw)
    for k in range(len(cases)):
        Xu = Xs_u[k].cpu().numpy()
        topu = ts_u[k].topology()
        Xo, to = otop.wrap(Xu, dict(topu, vert=Xu))
        assert np.array_equal(Xs_w[k].cpu().numpy(), Xo)
        assert np.array_equal(ts_w[k].topology()["he"], to["he"])
    for t in ts_u + ts_w:
        t.close()


def test_wrap_batched(vx):
    import torch
    cases = [case(n, 75 + k) for k, n in enumerate((120, 700, 60, 2500))]
    meshes = [m for _, m, _, _ in cases]
    X0 = np.concatenate([x for *_, x in cases])
    lam = torch.tensor(np.concatenate([c["lam"] for c, *_ in cases]), device="cuda")
    params = dict(KA=1.0, KP=1.0, A0=1.0, P0=3.7, lam=lam)
    kw = dict(tol=0.0, max_iter=200, dt0=0.01, dt_max=0.5, l_min=5e-3)
    out = {}
    for wrap in (0, 1):
        b = vx.Batch(meshes, "f64")
        X = torch.tensor(X0, dtype=torch.float64, device="cuda")
        vx.vx_minimize_batched(b, X, params, wrap=wrap, **kw)
        out[wrap] = (b.split(X.cpu().numpy()), b.topologies())
        b.close()
    for k in range(len(cases)):
        Xu, topu = out[0][0][k], out[0][1][k]
        Xo, to = otop.wrap(Xu, dict(topu, vert=Xu))
        assert np.array_equal(out[1][0][k], Xo)
        assert np.array_equal(out[1][1][k]["he"], to["he"])
