"""The boundary without allocation or host synchronisation: vx_minimize_async
and vx_equilibrium_grad_async recorded in a CUDA graph (with the topology
restore and the reset of X) and replayed, against the synchronous calls on
the same inputs.  The kernels are the same and deterministic, so the
replays must reproduce the synchronous results bit for bit."""
import numpy as np
import pytest

import vx_inputs as vi
from oracle import mesh as omesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vx():
    import paper_2604_06896_gb300 as vx
    return vx


def setup(n, stream):
    c = vi.small_tissue(n, stream, lam_range=(0.02, 0.1))
    m = omesh.build_periodic_voronoi(c["seeds"], c["Lx"], c["Ly"])
    p = {k: c[k] for k in ("KA", "KP", "A0", "P0", "lam")}
    Xt = m["vert"] + 0.02 * np.random.default_rng(stream).standard_normal(m["vert"].shape)
    return c, m, p, Xt


@pytest.mark.parametrize("path,n,dtype", [("resident", 300, "f32"), ("cluster", 1200, "f32"),
                                          ("resident", 200, "f64")])
@pytest.mark.parametrize("mode", ["adjoint", "ep"])
def test_minimize_and_gradient_replayed_from_a_graph(vx, path, n, dtype, mode):
    import torch
    c, m, p, Xt_h = setup(n, 95)
    mo = dict(tol=1e-6 if dtype == "f32" else 1e-10, max_iter=30000, dt0=0.01, dt_max=0.5,
              l_min=5e-3, path=path)
    go = dict(cost=vx.VX_COST_V2V, cg_rtol=1e-8, inner=dict(path=path, tol=1e-9, max_iter=20000))
    if mode == "ep":
        go.update(mode=vx.VX_EP_CENTERED, beta=0.2, ep_f64=1)
    t = vx.Tissue(m, dtype)
    X0 = torch.tensor(m["vert"], dtype=torch.float64, device="cuda")
    Xt = torch.tensor(Xt_h, dtype=torch.float64, device="cuda")
    # synchronous reference
    X = X0.clone()
    r_ref = vx.vx_minimize(t, X, p, **mo)
    g_ref, rg_ref = vx.vx_equilibrium_grad(t, X, p, cost_data=Xt, **go)
    X_ref = X.clone()
    assert r_ref.path_used == {"resident": vx.VX_PATH_RESIDENT, "cluster": vx.VX_PATH_CLUSTER}[path]
    # the same work recorded in a graph: restore, reset, relax, gradient
    prm = vx.Params(t, p)
    rmin = vx.result_buffer("min")
    rgrad = vx.result_buffer("grad", pinned=True)
    g = {k: torch.empty_like(v) for k, v in g_ref.items()}
    X = X0.clone()

    def work():
        vx.vx_tissue_restore(t)
        X.copy_(X0)
        vx.vx_minimize_async(t, X, prm, rmin, **mo)
        vx.vx_equilibrium_grad_async(t, X, prm, g, rgrad, cost_data=Xt, **go)

    work()                       # first calls outside the capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            work()
    for rep in range(2):
        X.fill_(float("nan"))
        for v in g.values():
            v.fill_(float("nan"))
        graph.replay()
        r = vx.read_result(rmin, "min")
        rg = vx.read_result(rgrad, "grad")
        assert torch.equal(X, X_ref), rep
        for k in g:
            assert torch.equal(g[k], g_ref[k]), (rep, k)
        assert (r.status, r.iters, r.n_t1, r.n_stretch, r.path_used) == \
            (r_ref.status, r_ref.iters, r_ref.n_t1, r_ref.n_stretch, r_ref.path_used)
        assert r.fmax == r_ref.fmax and r.energy == r_ref.energy
        assert (rg.status, rg.cg_iters, rg.nudged_iters) == \
            (rg_ref.status, rg_ref.cg_iters, rg_ref.nudged_iters)
        assert rg.cost == rg_ref.cost
    print(f"{path} {dtype} {mode}: {r.iters} iterations, {r.n_t1} T1; gradient {rg}")
    t.close()


def test_async_rejects_host_polled_paths(vx):
    import torch
    c, m, p, Xt = setup(100, 96)
    t = vx.Tissue(m, "f64")
    X = torch.tensor(m["vert"], dtype=torch.float64, device="cuda")
    buf = vx.result_buffer("min")
    for path in ("plain", "grid"):
        with pytest.raises(vx.VxError, match="INVALID_ARG"):
            vx.vx_minimize_async(t, X, p, buf, path=path)
    t.close()
