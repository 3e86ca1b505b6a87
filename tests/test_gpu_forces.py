"""Energy and forces: CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: FP64 path 1e-12 relative (rounding order only).  FP32 path:
every force term is a product of O(1) factors each carrying a few units of
float rounding (u = 6e-8) and the hi/lo position differences are exact to
one rounding, so |dF_i| <= ~20 u max_i |F_i|; the test allows 2e-6 of the
largest force.  Energy: 1e-5 relative for FP32 (the bound the workload
states), 1e-12 for FP64.
"""
import numpy as np
import pytest

import vx_inputs as vi
from oracle import mesh as omesh
from oracle import model as omodel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vx():
    import paper_2604_06896_gb300 as vx
    return vx


def case(name):
    if name == "c1":
        c = vi.tissue_c1()
    elif name == "c2":
        c = vi.tissue_c2(3.7)
    elif name == "rect":
        c = vi.small_tissue(300, 71, aspect=2.7)
    elif name == "tiny":
        c = vi.small_tissue(12, 72)
    else:
        c = vi.small_tissue(400, 73)
    ref = omesh.build_periodic_voronoi(c["seeds"], c["Lx"], c["Ly"])
    p = {k: c[k] for k in ("KA", "KP", "A0", "P0", "lam")}
    return c, ref, p


def hetero(ref, p, seed):
    rng = np.random.default_rng(seed)
    n = ref["n"]
    q = dict(p)
    q["KA"] = p["KA"] * rng.uniform(0.5, 2.0, n)
    q["KP"] = p["KP"] * rng.uniform(0.5, 2.0, n)
    q["A0"] = p["A0"] * rng.uniform(0.8, 1.2, n)
    q["P0"] = p["P0"] * rng.uniform(0.9, 1.1, n)
    return q


def run(vx, ref, p, dtype, X=None):
    import torch
    t = vx.Tissue(ref, dtype)
    Xn = ref["vert"] if X is None else X
    Xd = torch.tensor(Xn, dtype=torch.float64, device="cuda")
    F, E = vx.vx_energy_forces(t, Xd, p)
    torch.cuda.synchronize()
    out = F.cpu().numpy(), E.item()
    t.close()
    return out


@pytest.mark.parametrize("name", ["c1", "rect", "tiny", "rand"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("het", [False, True])
def test_forces_energy_parity(vx, name, dtype, het):
    c, ref, p = case(name)
    if het:
        p = hetero(ref, p, 5)
    F, E = run(vx, ref, p, dtype)
    Fr = omodel.forces(ref["vert"], ref, p)
    Er = omodel.energy(ref["vert"], ref, p)
    ftol = 1e-12 if dtype == "f64" else 2e-6
    etol = 1e-12 if dtype == "f64" else 1e-5
    err = np.abs(F - Fr).max() / np.abs(Fr).max()
    print(f"{name} {dtype} het={het}: force rel err {err:.2e}, energy rel err {abs(E - Er) / abs(Er):.2e}")
    assert err < ftol
    assert abs(E - Er) < etol * abs(Er)


def test_honeycomb_balance(vx):
    seeds, Lx, Ly = vi.lattice_seeds(10, 12)
    ref = omesh.build_periodic_voronoi(seeds, Lx, Ly)
    p = dict(KA=1.3, KP=0.7, A0=0.9, P0=3.5, lam=0.04)
    for dtype in ("f64", "f32"):
        F, E = run(vx, ref, p, dtype)
        assert np.abs(F).max() < (1e-12 if dtype == "f64" else 1e-6)
        Er = omodel.energy(ref["vert"], ref, p)
        assert abs(E - Er) < 1e-6 * Er


def test_full_size_c2(vx):
    """10,000-cell tissue at the launch size of the workload."""
    c, ref, p = case("c2")
    F, E = run(vx, ref, p, "f32")
    Fr = omodel.forces(ref["vert"], ref, p)
    Er = omodel.energy(ref["vert"], ref, p)
    assert np.abs(F - Fr).max() < 2e-6 * np.abs(Fr).max()
    assert abs(E - Er) < 1e-5 * abs(Er)
    # sum of forces vanishes
    assert np.abs(F.sum(axis=0)).max() < 1e-4 * np.abs(F).max()


def test_translation_invariance_gpu(vx):
    c, ref, p = case("rand")
    F0, E0 = run(vx, ref, p, "f32")
    F1, E1 = run(vx, ref, p, "f32", ref["vert"] + np.array([0.37, -1.21]))
    assert np.abs(F1 - F0).max() < 2e-6 * np.abs(F0).max()
    assert abs(E1 - E0) < 1e-6 * abs(E0)


def test_bad_arguments(vx):
    import torch
    c, ref, p = case("tiny")
    t = vx.Tissue(ref, "f64")
    X = torch.tensor(ref["vert"], dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        vx.vx_energy_forces(t, X[:-1], p)
    bad = dict(p)
    bad["KA"] = float("nan")
    with pytest.raises(vx.VxError, match="INVALID_ARG"):
        vx.vx_energy_forces(t, X, bad)
    broken = dict(ref)
    he = ref["he"].copy()
    he[0, 2] = he[1, 2]
    broken["he"] = he
    with pytest.raises(vx.VxError, match="INVALID_ARG"):
        vx.Tissue(broken, "f64")
    t.close()
