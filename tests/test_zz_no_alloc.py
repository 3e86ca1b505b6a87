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


class NoAllocCall:
    """Device copies of a mesh's tables, its parameters and output buffers,
    and the raw C-ABI call on torch's current stream."""

    def __init__(self, vx, mesh, X, params, forces=True):
        import torch
        dev = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
        self.he, self.fh, self.eid = dev(mesh["he"]), dev(mesh["face_he"]), dev(mesh["edge_id"])
        self.n = int(mesh["face_he"].shape[0])
        self.Lx, self.Ly = mesh["Lx"], mesh["Ly"]
        self.X = X
        self.prm, self.keep = vx.make_params(params, self.n, 3 * self.n)
        self.F = torch.empty((2 * self.n, 2), dtype=torch.float64, device="cuda") if forces else None
        self.E = torch.empty(1, dtype=torch.float64, device="cuda")
        self.st = torch.full((1,), -1, dtype=torch.int32, device="cuda")

    def __call__(self):
        import torch
        from paper_2604_06896_gb300 import _capi
        stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        return _capi.vx_energy_forces_noalloc(
            self.he.data_ptr(), self.fh.data_ptr(), self.eid.data_ptr(), self.n, self.Lx, self.Ly,
            self.X.data_ptr(), C.byref(self.prm),
            self.F.data_ptr() if self.F is not None else None, self.E.data_ptr(),
            self.st.data_ptr(), stream)

    def results(self):
        import torch
        torch.cuda.synchronize()
        F = self.F.cpu().numpy() if self.F is not None else None
        return F, self.E.item(), int(self.st.item())


def noalloc(vx, mesh, X, params):
    call = NoAllocCall(vx, mesh, X, params)
    rc = call()
    F, E, st = call.results()
    return rc, F, E, st


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


def reference(vx, mesh, X, params):
    t = vx.Tissue(mesh, "f64")
    F_ref, E_ref = vx.vx_energy_forces(t, X, params)
    F_ref, E_ref = F_ref.cpu().numpy(), E_ref.item()
    t.close()
    return F_ref, E_ref


def test_noalloc_replayed_from_a_cuda_graph(vx):
    """A caller that cannot allocate typically records the call into a CUDA
    graph: one call first (it looks up the scratch array's address on this
    device), then a capture, then replays."""
    import torch
    mesh, params = case(vx, 600, 903)
    X = torch.tensor(mesh["vert"], dtype=torch.float64, device="cuda")
    F_ref, E_ref = reference(vx, mesh, X, params)
    call = NoAllocCall(vx, mesh, X, params)
    assert call() == 0
    call.results()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            rc = call()
    assert rc == 0
    for rep in range(2):
        call.F.fill_(float("nan"))
        call.E.fill_(float("nan"))
        g.replay()
        F, E, st = call.results()
        assert st == 0, rep
        assert np.abs(F - F_ref).max() < 1e-12 * np.abs(F_ref).max(), rep
        assert abs(E - E_ref) < 1e-12 * abs(E_ref), rep


def test_noalloc_energy_only(vx):
    import torch
    mesh, params = case(vx, 300, 904)
    X = torch.tensor(mesh["vert"], dtype=torch.float64, device="cuda")
    F_ref, E_ref = reference(vx, mesh, X, params)
    call = NoAllocCall(vx, mesh, X, params, forces=False)
    assert call() == 0
    _, E, st = call.results()
    assert st == 0 and abs(E - E_ref) < 1e-12 * abs(E_ref)


@pytest.mark.parametrize("forces", [True, False])
def test_noalloc_flags_a_vertex_that_is_not_3_valent(vx, forces):
    """One half-edge's source moved to another valid vertex: counts 4 and 2,
    every index still in range.  Status bit 1, with or without forces."""
    import torch
    mesh, params = case(vx, 200, 905)
    bad = dict(mesh)
    he = mesh["he"].copy()
    h = 17
    old = int(he[h, 3])
    he[h, 3] = (old + 5) % (he.shape[0] // 3)
    assert he[h, 3] != old
    bad["he"] = he
    X = torch.tensor(mesh["vert"], dtype=torch.float64, device="cuda")
    call = NoAllocCall(vx, bad, X, params, forces=forces)
    assert call() == 0
    _, E, st = call.results()
    assert st & 1, st


def test_noalloc_flags_an_index_out_of_range(vx):
    """A target index beyond the vertices: status bit 2, no access outside
    the caller's buffers (the kernels check before they load)."""
    import torch
    mesh, params = case(vx, 200, 906)
    bad = dict(mesh)
    he = mesh["he"].copy()
    he[23, 4] = 2 * 200 + 7
    bad["he"] = he
    X = torch.tensor(mesh["vert"], dtype=torch.float64, device="cuda")
    call = NoAllocCall(vx, bad, X, params)
    assert call() == 0
    _, E, st = call.results()
    assert st & 2, st
    # the next, valid call on the same scratch is clean again
    good = NoAllocCall(vx, mesh, X, params)
    assert good() == 0
    F, E, st = good.results()
    F_ref, E_ref = reference(vx, mesh, X, params)
    assert st == 0 and np.abs(F - F_ref).max() < 1e-12 * np.abs(F_ref).max()
