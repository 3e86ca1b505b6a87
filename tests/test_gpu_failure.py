"""Failure detection on the GPU without a fault: the GRID path's barrier
waits are bounded, so a team member that never arrives ends the wait with
VX_ERR_TIMEOUT after the limit, and the context stays usable."""
import time

import numpy as np
import pytest

import vx_inputs as vi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vx():
    import paper_2604_06896_gb300 as vx
    return vx


def test_grid_barrier_all_present(vx):
    st, per = vx.vx_grid_barrier_selftest(16, absent_rank=-1, rounds=50, wait_s=1.0)
    assert st == vx.capi.VX_OK
    assert np.all(per == vx.capi.VX_OK)


@pytest.mark.parametrize("absent", [0, 5])
def test_grid_barrier_wait_runs_out(vx, absent):
    t0 = time.perf_counter()
    st, per = vx.vx_grid_barrier_selftest(8, absent_rank=absent, rounds=4, wait_s=0.2)
    dt = time.perf_counter() - t0
    assert st == vx.capi.VX_ERR_TIMEOUT
    assert per[absent] == -1
    assert np.all(np.delete(per, absent) == vx.capi.VX_ERR_TIMEOUT)
    assert dt < 5.0
    # the context is still usable: a small relaxation on the grid path
    import torch
    c = vi.small_tissue(300, 88, lam_range=(0.02, 0.1))
    mesh = vx.vx_build_mesh(c["seeds"], c["Lx"], c["Ly"])
    p = {k: c[k] for k in ("KA", "KP", "A0", "P0", "lam")}
    t = vx.Tissue(mesh, "f32")
    X = torch.tensor(mesh["vert"], dtype=torch.float64, device="cuda")
    r = vx.vx_minimize(t, X, p, tol=1e-6, max_iter=20000, dt0=0.01, dt_max=0.5, l_min=5e-3,
                       path="grid")
    assert r.converged
    t.close()


def test_grid_barrier_rejects_bad_arguments(vx):
    with pytest.raises(vx.VxError, match="INVALID_ARG"):
        vx.vx_grid_barrier_selftest(4, absent_rank=4)
    with pytest.raises(vx.VxError, match="INVALID_ARG"):
        vx.vx_grid_barrier_selftest(4, wait_s=100.0)
