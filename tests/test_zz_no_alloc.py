"""vx_energy_forces_noalloc: the entry point for callers that cannot
allocate device memory (stream captures with a frozen pool, plugins with a
fixed memory budget, real-time loops).  It takes the topology tables in the
caller's device memory and keeps its scratch in one static device array, so
it must give what the handle-based vx_energy_forces gives, call after call
(the array keeps the previous call's contents; what must start at zero is
cleared by every call).

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import vx_inputs as vi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vx():
    import paper_2604_06896_gb300 as vx
    return vx


def noalloc(vx, mesh, X, params):
    import torch
    from paper_2604_06896_gb300 import _capi

    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    he, fh, eid = dev(mesh["he"]), dev(mesh["face_he"]), dev(mesh["edge_id"])
    n = int(mesh["face_he"].shape[0])
    prm, keep = vx.make_params(params, n, 3 * n)
    F = torch.empty((2 * n, 2), dtype=torch.float64, device="cuda")
    E = torch.empty(1, dtype=torch.float64, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = _capi.vx_energy_forces_noalloc(he.data_ptr(), fh.data_ptr(), eid.data_ptr(), n,
                                        mesh["Lx"], mesh["Ly"], X.data_ptr(), C.byref(prm),
                                        F.data_ptr(), E.data_ptr(), st.data_ptr(), stream)
    torch.cuda.synchronize()
    return rc, F.cpu().numpy(), E.item(), int(st.item())


def case(vx, n, stream):
    c = vi.small_tissue(n, stream)
    mesh = vx.vx_build_mesh(c["seeds"], c["Lx"], c["Ly"])
    rng = np.random.default_rng(stream)
    params = dict(KA=rng.uniform(0.5, 2.0, n), KP=1.3, A0=rng.uniform(0.8, 1.2, n), P0=3.6,
                  lam=c["lam"])
    return mesh, params


@pytest.mark.parametrize("n,stream", [(100, 901), (2000, 902)])
def test_noalloc_matches_energy_forces_twice(vx, n, stream):
    import torch
    mesh, params = case(vx, n, stream)
    X = torch.tensor(mesh["vert"], dtype=torch.float64, device="cuda")
    t = vx.Tissue(mesh, "f64")
    F_ref, E_ref = vx.vx_energy_forces(t, X, params)
    F_ref, E_ref = F_ref.cpu().numpy(), E_ref.item()
    t.close()
    scale = np.abs(F_ref).max()
    for call in range(2):
        rc, F, E, st = noalloc(vx, mesh, X, params)
        assert rc == 0 and st == 0, (call, rc, st)
        assert np.abs(F - F_ref).max() < 1e-12 * scale, call
        assert abs(E - E_ref) < 1e-12 * abs(E_ref), call


def test_noalloc_rejects_oversized_tissue(vx):
    from paper_2604_06896_gb300 import _capi
    prm = _capi.vx_params()
    rc = _capi.vx_energy_forces_noalloc(C.c_void_p(16), C.c_void_p(16), C.c_void_p(16), 40000,
                                        1.0, 1.0, C.c_void_p(16), C.byref(prm), None, None,
                                        C.c_void_p(16), None)
    assert rc == _capi.VX_ERR_INVALID_ARG
    assert "32768" in _capi.vx_last_error().decode()
