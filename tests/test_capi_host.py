"""C ABI without a GPU: the library loads, exports every symbol vx.h
declares (and the Python binding offers each under the same name),
validates arguments, and its host mesh builder reproduces the
oracle's topology bit for bit."""
import os
import re

import numpy as np
import pytest

import vx_inputs as vi
from oracle import mesh as omesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def vx():
    import paper_2604_06896_gb300 as vx
    return vx


def test_exports_every_declared_symbol(vx):
    hdr = open(os.path.join(ROOT, "include", "vx.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)   # declarations only, not comments
    declared = set(re.findall(r"\b(vx_[a-z_0-9]+)\s*\(", hdr))
    declared -= {"vx_status"}
    from paper_2604_06896_gb300 import _capi
    for name in declared:
        assert hasattr(_capi.lib, name), name
    assert declared == set(_capi.EXPORTED)
    assert _capi.vx_version().decode().startswith("vx ")


# Entry points whose Python form is a method or a helper of the handle
# classes (Tissue, Batch) or a defaults filler used by the option builders.
_HANDLE_LEVEL = {"vx_last_error", "vx_tissue_destroy", "vx_tissue_sizes", "vx_tissue_topology",
                 "vx_batch_destroy", "vx_batch_sizes", "vx_batch_topology",
                 "vx_min_opts_default", "vx_grad_opts_default"}


def test_binding_has_every_entry_point(vx):
    """The Python binding offers each C entry point under the same name."""
    from paper_2604_06896_gb300 import _capi
    for name in set(_capi.EXPORTED) - _HANDLE_LEVEL:
        assert name in vx.__all__ and callable(getattr(vx, name)), name


def test_noalloc_binding_refuses_host_tensors(vx):
    """No CPU path: host tensors are refused before anything is called."""
    import torch
    n = 10
    he = torch.zeros((6 * n, 8), dtype=torch.int32)
    fh = torch.zeros(n, dtype=torch.int32)
    eid = torch.zeros(6 * n, dtype=torch.int32)
    X = torch.zeros((2 * n, 2), dtype=torch.float64)
    st = torch.zeros(1, dtype=torch.int32)
    p = dict(KA=1.0, KP=1.0, A0=1.0, P0=3.7, lam=0.0)
    with pytest.raises(ValueError, match="CUDA tensor"):
        vx.vx_energy_forces_noalloc(he, fh, eid, 1.0, 1.0, X, p, status=st)


@pytest.mark.parametrize("n,stream,aspect", [(10, 61, 1.0), (37, 62, 1.0), (100, 63, 1.0),
                                             (250, 64, 2.0), (500, 65, 0.5), (1000, 66, 1.0)])
def test_mesh_bit_exact_vs_oracle(vx, n, stream, aspect):
    c = vi.small_tissue(n, stream, aspect=aspect)
    try:
        ref = omesh.build_periodic_voronoi(c["seeds"], c["Lx"], c["Ly"])
    except omesh.DegenerateSeeds:
        with pytest.raises(vx.VxError):
            vx.vx_build_mesh(c["seeds"], c["Lx"], c["Ly"])
        return
    got = vx.vx_build_mesh(c["seeds"], c["Lx"], c["Ly"])
    assert np.array_equal(got["he"], ref["he"])
    assert np.array_equal(got["face_he"], ref["face_he"])
    assert np.array_equal(got["edge_id"], ref["edge_id"])
    L = max(c["Lx"], c["Ly"])
    assert np.abs(got["vert"] - ref["vert"]).max() < 1e-12 * L


def test_mesh_bit_exact_many_seed_sets(vx):
    """1,000 random seed sets of 3..60 cells (tiny tessellations where the
    3 x 3 replication and cells touching their own image are common)."""
    rng = vi.SplitMix64(67)
    agree = rejected = 0
    for k in range(1000):
        n = 3 + int(rng.next_u64(1)[0] % np.uint64(58))
        c = vi.small_tissue(n, 10_000 + k)
        try:
            ref = omesh.build_periodic_voronoi(c["seeds"], c["Lx"], c["Ly"])
        except omesh.DegenerateSeeds:
            ref = None
        try:
            got = vx.vx_build_mesh(c["seeds"], c["Lx"], c["Ly"])
        except vx.VxError:
            got = None
        # both sides reject the same (degenerate) seed sets
        assert (ref is None) == (got is None), (k, n, ref is None, got is None)
        if ref is None:
            rejected += 1
            continue
        assert np.array_equal(got["he"], ref["he"]), (k, n)
        assert np.array_equal(got["edge_id"], ref["edge_id"])
        agree += 1
    assert agree > 700


def test_mesh_degenerate_verdicts_agree(vx):
    """Adversarial seed sets: coincident seeds and cocircular quadruples on
    coarse grids, square lattices (every Delaunay triangle ambiguous) and
    seeds crowded into a strip.  Both builders refuse the same sets and give
    the same tables and positions for the others."""
    rng = np.random.default_rng(0)
    seen = set()
    for k in range(150):
        n = int(rng.integers(4, 80))
        Lx, Ly = float(rng.uniform(1, 3)), float(rng.uniform(1, 3))
        if k % 3 == 0:
            g = int(rng.integers(3, 9))
            s = np.stack([rng.integers(0, g, n) * Lx / g, rng.integers(0, g, n) * Ly / g], 1)
        elif k % 3 == 1:
            m = int(np.ceil(np.sqrt(n)))
            i = np.arange(n)
            s = np.stack([(i % m + 0.5) * Lx / m, (i // m % m + 0.5) * Ly / m], 1)
        else:
            s = np.stack([rng.uniform(0, 0.2 * Lx, n), rng.uniform(0, Ly, n)], 1)
        try:
            ref = omesh.build_periodic_voronoi(s, Lx, Ly)
        except omesh.DegenerateSeeds:
            ref = None
        try:
            got = vx.vx_build_mesh(s, Lx, Ly)
        except vx.VxError:
            got = None
        assert (ref is None) == (got is None), (k, n)
        seen.add(ref is None)
        if ref is not None:
            for key in ("he", "face_he", "edge_id", "vert"):
                assert np.array_equal(got[key], ref[key]), (k, key)
    assert seen == {True, False}


@pytest.mark.parametrize("case", ["c2", "c2_hilbert", "n5000"])
def test_mesh_bit_exact_full_size(vx, case):
    """The 10,000-cell tissue the benchmark builds (in the given seed order
    and in Hilbert order, as the benchmark does) and a 5,000-cell tissue."""
    if case.startswith("c2"):
        c = vi.tissue_c2(3.7)
        seeds = c["seeds"]
        if case == "c2_hilbert":
            seeds = seeds[vx.vx_seed_order(seeds, c["Lx"], c["Ly"])]
    else:
        c = vi.small_tissue(5000, 69)
        seeds = c["seeds"]
    got = vx.vx_build_mesh(seeds, c["Lx"], c["Ly"])
    ref = omesh.build_periodic_voronoi(seeds, c["Lx"], c["Ly"])
    assert np.array_equal(got["he"], ref["he"])
    assert np.array_equal(got["face_he"], ref["face_he"])
    assert np.array_equal(got["edge_id"], ref["edge_id"])
    assert np.abs(got["vert"] - ref["vert"]).max() < 1e-12 * max(c["Lx"], c["Ly"])


def test_mesh_c1_and_honeycomb(vx):
    c = vi.tissue_c1()
    got = vx.vx_build_mesh(c["seeds"], 1.0, 1.0)
    ref = omesh.build_periodic_voronoi(c["seeds"], 1.0, 1.0)
    assert np.array_equal(got["he"], ref["he"])
    seeds, Lx, Ly = vi.lattice_seeds(8, 6)
    got = vx.vx_build_mesh(seeds, Lx, Ly)
    ref = omesh.build_periodic_voronoi(seeds, Lx, Ly)
    assert np.array_equal(got["he"], ref["he"])


def test_mesh_invalid_arguments(vx):
    with pytest.raises(vx.VxError, match="INVALID_ARG"):
        vx.vx_build_mesh(np.zeros((2, 2)), 1.0, 1.0)
    with pytest.raises(vx.VxError, match="INVALID_ARG"):
        vx.vx_build_mesh(np.array([[0.5, 0.5], [1.5, 0.2], [0.1, 0.1]]), 1.0, 1.0)
    with pytest.raises(vx.VxError, match="INVALID_ARG"):
        vx.vx_build_mesh(np.random.default_rng(0).uniform(size=(10, 2)), -1.0, 1.0)
    sq = np.array([(i + 0.25, j + 0.25) for i in range(5) for j in range(5)], dtype=float)
    with pytest.raises(vx.VxError, match="DEGENERATE"):
        vx.vx_build_mesh(sq, 5.0, 5.0)


def test_seed_order_is_a_locality_permutation(vx):
    """A permutation; building from the reordered seeds gives the same
    tissue (oracle, bit-exact on the relabelled seeds) with spatially
    coherent numbering (consecutive cells are close)."""
    c = vi.small_tissue(2000, 68)
    order = vx.vx_seed_order(c["seeds"], c["Lx"], c["Ly"])
    assert sorted(order.tolist()) == list(range(2000))
    s2 = c["seeds"][order]
    got = vx.vx_build_mesh(s2, c["Lx"], c["Ly"])
    ref = omesh.build_periodic_voronoi(s2, c["Lx"], c["Ly"])
    assert np.array_equal(got["he"], ref["he"])
    step = lambda s: np.median(np.sqrt((np.diff(s, axis=0) ** 2).sum(axis=1)))
    assert step(s2) < 0.2 * step(c["seeds"])
    # the areas are a permutation of the unordered tissue's areas
    from oracle import model as omodel
    a0 = omodel.geometry(ref["vert"], ref)["A"]
    r1 = omesh.build_periodic_voronoi(c["seeds"], c["Lx"], c["Ly"])
    a1 = omodel.geometry(r1["vert"], r1)["A"]
    assert np.allclose(a0, a1[order], rtol=1e-12)


def _create(he, face_he, edge_id, n, Lx, Ly, dtype=0):
    """vx_tissue_create through the raw ABI; the table checks run on the host
    before any device call, so malformed tables are refused without a GPU."""
    import ctypes as C
    from paper_2604_06896_gb300 import _capi
    he = np.ascontiguousarray(he, dtype=np.int32)
    fh = np.ascontiguousarray(face_he, dtype=np.int32)
    eid = np.ascontiguousarray(edge_id, dtype=np.int32)
    h = C.c_void_p()
    st = _capi.vx_tissue_create(he.ctypes.data, fh.ctypes.data, eid.ctypes.data, n, he.shape[0],
                                Lx, Ly, dtype, None, C.byref(h))
    return st, _capi.vx_last_error().decode()


def _malformed_cases(m):
    """(name, he, face_he, edge_id, expected message) from one valid mesh."""
    he, fh, eid = m["he"], m["face_he"], m["edge_id"]
    HE = he.shape[0]
    out = []
    a = he.copy(); a[3, 1] = HE
    out.append(("next out of range", a, fh, eid, "index out of range"))
    a = he.copy(); a[5, 5] = m["n"]
    out.append(("face out of range", a, fh, eid, "face out of range"))
    a = he.copy(); a[7, 6] = 2
    out.append(("offset 2", a, fh, eid, "offsets must be in"))
    e = eid.copy(); e[4] = HE // 2
    out.append(("edge id out of range", he, fh, e, "edge_id out of range"))
    a = he.copy(); a[9, 2] = 9
    out.append(("twin of itself", a, fh, eid, "twin is not an involution"))
    # a half-edge whose offset is not the negated offset of its twin's
    h = int(np.nonzero(he[:, 6] != 0)[0][0])
    a = he.copy(); a[h, 6] = 0
    out.append(("twin offsets", a, fh, eid, "twin offsets must be negated"))
    # the offsets of one edge changed on both half-edges: twins agree, the
    # two faces' offset sums no longer vanish
    h = int(np.nonzero((he[:, 6] == 0) & (he[:, 7] == 0))[0][0])
    a = he.copy(); a[h, 7] = 1; a[he[h, 2], 7] = -1
    out.append(("face offsets", a, fh, eid, "do not cancel"))
    # prev pointers of two half-edges exchanged
    a = he.copy(); a[[0, 10], 0] = a[[10, 0], 0]
    out.append(("prev(next(h))", a, fh, eid, "prev(next(h)) != h"))
    # edge ids of two half-edges of different edges exchanged
    h2 = next(q for q in range(1, HE) if eid[q] != eid[0] and he[0, 2] != q)
    e = eid.copy(); e[[0, h2]] = e[[h2, 0]]
    out.append(("edge ids", he, fh, e, "twins must share an edge id"))
    f = fh.copy(); f[0] = fh[1]
    out.append(("face_he", he, f, eid, "face_he[0]"))
    return out


def test_tissue_create_refuses_malformed_tables(vx):
    c = vi.small_tissue(20, 64)
    m = vx.vx_build_mesh(c["seeds"], c["Lx"], c["Ly"])
    for name, he, fh, eid, msg in _malformed_cases(m):
        st, err = _create(he, fh, eid, m["n"], m["Lx"], m["Ly"])
        assert st == 2 and msg in err, (name, st, err)
    st, err = _create(m["he"][:-6], m["face_he"], m["edge_id"][:-6], m["n"], m["Lx"], m["Ly"])
    assert st == 2 and "6 n half-edges" in err
    st, err = _create(m["he"], m["face_he"], m["edge_id"], m["n"], m["Lx"], m["Ly"], dtype=7)
    assert st == 2 and "dtype" in err
    st, err = _create(m["he"], m["face_he"], m["edge_id"], m["n"], 0.0, m["Ly"])
    assert st == 2 and "box" in err


def test_option_defaults_through_the_binding(vx):
    """The defaults the library fills in reach Python field by field (the
    ctypes structs match vx.h's layout), and FIRE's constants are the
    oracle's (Bitzek et al.: N_min 5, f_inc 1.1, f_dec 0.5, alpha0 0.1,
    f_alpha 0.99), which the same-trajectory parity tests rely on."""
    import ctypes as C
    from oracle import solvers
    from paper_2604_06896_gb300 import _capi
    o = _capi.vx_min_opts()
    _capi.vx_min_opts_default(C.byref(o))
    assert (o.method, o.tol, o.patience, o.max_iter, o.gd_lr) == (vx.VX_FIRE, 1e-8, 1, 100000, 1e-2)
    assert (o.dt0, o.dt_max, o.l_min, o.path, o.check_every) == (0.01, 0.5, 0.0, vx.VX_PATH_AUTO, 50)
    assert (o.wrap, o.refine_tol) == (1, 0.0) and not o.edge_events
    ref = solvers.MinOpts()
    assert (o.n_min, o.f_inc, o.f_dec, o.alpha0, o.f_alpha) == \
        (ref.n_min, ref.f_inc, ref.f_dec, ref.alpha0, ref.f_alpha)
    g = _capi.vx_grad_opts()
    _capi.vx_grad_opts_default(C.byref(g))
    assert (g.mode, g.beta, g.cg_rtol, g.cg_max_iter, g.cost) == \
        (vx.VX_ADJOINT_CG, 1e-3, 1e-10, 20000, vx.VX_COST_NONE)
    assert not g.cost_data and g.ep_f64 == 1
    assert (g.inner.tol, g.inner.n_min, g.inner.wrap) == (1e-10, 5, 1)


def test_batch_create_names_the_malformed_tissue(vx):
    """vx_batch_create checks every member's tables on the host before any
    device allocation and names the first member it refuses."""
    import ctypes as C
    from paper_2604_06896_gb300 import _capi
    ms = []
    for n, st in ((60, 65), (40, 66), (30, 67)):
        c = vi.small_tissue(n, st)
        ms.append(vx.vx_build_mesh(c["seeds"], c["Lx"], c["Ly"]))
    bad = _malformed_cases(ms[1])[0]            # next out of range
    tables = [(m["he"], m["face_he"], m["edge_id"]) for m in ms]
    tables[1] = bad[1:4]
    n = np.array([m["n"] for m in ms], dtype=np.int32)
    box = np.ascontiguousarray([[m["Lx"], m["Ly"]] for m in ms], dtype=np.float64)
    he, fh, eid = (np.ascontiguousarray(np.concatenate([t[i] for t in tables]), dtype=np.int32)
                   for i in range(3))
    h = C.c_void_p()
    st = _capi.vx_batch_create(3, n.ctypes.data, box.ctypes.data, he.ctypes.data, fh.ctypes.data,
                               eid.ctypes.data, 1, None, C.byref(h))
    err = _capi.vx_last_error().decode()
    assert st == 2 and err.startswith("tissue 1: ") and "index out of range" in err
    assert h.value is None
