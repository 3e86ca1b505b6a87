"""GB300-native periodic vertex model (VertAX hot path) — Python binding.

The names follow the C ABI of ``include/vx.h``.  This module only marshals
arguments: torch tensors (float64, contiguous, on the current CUDA device)
are passed to the CUDA library as raw device pointers on torch's current
stream.  There is no CPU fallback; importing fails when ``libvx.so`` has not
been built.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _capi as capi
from ._capi import (VX_ADJOINT_CG, VX_ADJOINT_MINRES, VX_COST_ANISO, VX_COST_NONE,  # noqa: F401
                    VX_COST_V2V, VX_EP_CENTERED, VX_EP_FORWARD, VX_F32, VX_F64, VX_FIRE, VX_GD,
                    VX_GRAD_ADJOINT, VX_GRAD_EP, VX_PARAM_A0, VX_PARAM_LAMBDA, VX_PARAM_P0,
                    VX_PATH_AUTO, VX_PATH_CLUSTER, VX_PATH_GRID, VX_PATH_PLAIN, VX_PATH_RESIDENT,
                    VxError)

__all__ = ["vx_build_mesh", "vx_seed_order", "vx_tissue_create", "vx_tissue_restore", "Tissue",
           "vx_energy_forces", "vx_energy_forces_noalloc", "vx_hessian_vector", "vx_minimize",
           "vx_minimize_async", "vx_minimize_many", "vx_equilibrium_grad",
           "vx_equilibrium_grad_async", "vx_sensitivity_grad", "Batch", "vx_batch_create",
           "vx_batch_restore", "vx_minimize_batched", "vx_batch_autotune",
           "vx_equilibrium_grad_batched", "vx_batch_grad", "vx_batch_aniso_cost",
           "vx_grid_barrier_selftest", "vx_version", "EquilibriumFn", "VxError"]


def _torch():
    import torch
    return torch


def _stream():
    torch = _torch()
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _dev_f64(x, shape=None):
    torch = _torch()
    if not torch.is_tensor(x):
        x = torch.as_tensor(np.asarray(x, dtype=np.float64))
    x = x.to(device="cuda", dtype=torch.float64).contiguous()
    if shape is not None and tuple(x.shape) != tuple(shape):
        raise ValueError(f"expected shape {shape}, got {tuple(x.shape)}")
    return x


# ---------------------------------------------------------------- mesh

def vx_build_mesh(seeds, Lx, Ly):
    """Periodic Voronoi tessellation of the seeds (host; see vx.h).
    Returns dict(vert [2n,2] f64, he [6n,8] i32, face_he [n] i32,
    edge_id [6n] i32, n, Lx, Ly) as numpy arrays."""
    s = np.ascontiguousarray(np.asarray(seeds, dtype=np.float64))
    n = s.shape[0]
    vert = np.zeros((2 * n, 2), dtype=np.float64)
    he = np.zeros((6 * n, 8), dtype=np.int32)
    face_he = np.zeros(n, dtype=np.int32)
    edge_id = np.zeros(6 * n, dtype=np.int32)
    st = capi.vx_build_mesh(s.ctypes.data, n, float(Lx), float(Ly), vert.ctypes.data,
                            he.ctypes.data, face_he.ctypes.data, edge_id.ctypes.data)
    capi.check(st, "vx_build_mesh")
    return dict(vert=vert, he=he, face_he=face_he, edge_id=edge_id, n=n, Lx=float(Lx),
                Ly=float(Ly))


def vx_seed_order(seeds, Lx, Ly):
    """Hilbert-curve order of the seeds (see vx.h); build from seeds[order]
    for spatially ordered cell, vertex and edge numbering."""
    s = np.ascontiguousarray(np.asarray(seeds, dtype=np.float64))
    order = np.zeros(s.shape[0], dtype=np.int32)
    capi.check(capi.vx_seed_order(s.ctypes.data, s.shape[0], float(Lx), float(Ly),
                                  order.ctypes.data), "vx_seed_order")
    return order


# ------------------------------------------------------------ parameters

def make_params(p, n=None, E=None):
    """vx_params from a dict with KA, KP, A0, P0 (scalar or per-cell) and lam
    (scalar or per-edge).  Returns (struct, tensors kept alive)."""
    keep = []
    out = capi.vx_params()
    for key, fp, fs, size in (("KA", "KA", "KA_s", n), ("KP", "KP", "KP_s", n),
                              ("A0", "A0", "A0_s", n), ("P0", "P0", "P0_s", n),
                              ("lam", "lambda_", "lambda_s", E)):
        v = p[key]
        if np.ndim(v) == 0 and not (hasattr(v, "dim") and v.dim() > 0):
            setattr(out, fp, None)
            setattr(out, fs, float(v))
        else:
            t = _dev_f64(v)
            if size is not None and t.numel() != size:
                raise ValueError(f"{key}: expected {size} values, got {t.numel()}")
            keep.append(t)
            setattr(out, fp, t.data_ptr())
            setattr(out, fs, 0.0)
    return out, keep


@dataclass
class MinResult:
    status: int
    iters: int
    n_t1: int
    n_stretch: int
    n_short_edges: int
    n_inverted: int
    fmax: float
    energy: float
    path_used: int
    force_evals: int

    @property
    def converged(self):
        return self.status == capi.VX_OK


def min_opts(**kw):
    o = capi.vx_min_opts()
    capi.vx_min_opts_default(C.byref(o))
    for k, v in kw.items():
        if k == "method" and isinstance(v, str):
            v = {"fire": VX_FIRE, "gd": VX_GD}[v]
        if k == "path" and isinstance(v, str):
            v = {"auto": VX_PATH_AUTO, "resident": VX_PATH_RESIDENT, "plain": VX_PATH_PLAIN,
                 "cluster": VX_PATH_CLUSTER, "grid": VX_PATH_GRID}[v]
        if k == "edge_events" and v is not None and hasattr(v, "data_ptr"):
            v = v.data_ptr()    # a device int32 [E, 2] tensor
        if not hasattr(o, k):
            raise TypeError(f"unknown minimiser option {k}")
        setattr(o, k, v)
    return o


# ----------------------------------------------------------------- tissue

class Tissue:
    """A tissue handle (vx_tissue): device topology plus workspace."""

    def __init__(self, mesh, dtype="f64"):
        he = np.ascontiguousarray(mesh["he"], dtype=np.int32)
        face_he = np.ascontiguousarray(mesh["face_he"], dtype=np.int32)
        edge_id = np.ascontiguousarray(mesh["edge_id"], dtype=np.int32)
        self.n = int(face_he.shape[0])
        self.HE = int(he.shape[0])
        self.V, self.E = self.HE // 3, self.HE // 2
        self.Lx, self.Ly = float(mesh["Lx"]), float(mesh["Ly"])
        self.dtype = {"f64": VX_F64, "f32": VX_F32}[dtype] if isinstance(dtype, str) else dtype
        h = C.c_void_p()
        _torch().cuda.init()
        st = capi.vx_tissue_create(he.ctypes.data, face_he.ctypes.data, edge_id.ctypes.data,
                                   self.n, self.HE, self.Lx, self.Ly, self.dtype, _stream(),
                                   C.byref(h))
        capi.check(st, "vx_tissue_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            capi.vx_tissue_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def topology(self):
        he = np.zeros((self.HE, 8), dtype=np.int32)
        face_he = np.zeros(self.n, dtype=np.int32)
        edge_id = np.zeros(self.HE, dtype=np.int32)
        capi.check(capi.vx_tissue_topology(self.handle, he.ctypes.data, face_he.ctypes.data,
                                           edge_id.ctypes.data), "vx_tissue_topology")
        return dict(he=he, face_he=face_he, edge_id=edge_id, n=self.n, Lx=self.Lx, Ly=self.Ly)


def vx_tissue_create(mesh, dtype="f64"):
    return Tissue(mesh, dtype)


def vx_tissue_restore(t: Tissue):
    """Put back the topology the tissue had at creation (asynchronous)."""
    capi.check(capi.vx_tissue_restore(t.handle, _stream()), "vx_tissue_restore")


def vx_hessian_vector(t: Tissue, X, params, v):
    """H v at X (device f64 [V,2] tensors)."""
    torch = _torch()
    X = _dev_f64(X, (t.V, 2))
    v = _dev_f64(v, (t.V, 2))
    prm, keep = make_params(params, t.n, t.E)
    Hv = torch.empty((t.V, 2), dtype=torch.float64, device="cuda")
    capi.check(capi.vx_hessian_vector(t.handle, _ptr(X), C.byref(prm), _ptr(v), _ptr(Hv),
                                      _stream()), "vx_hessian_vector")
    return Hv


def vx_energy_forces(t: Tissue, X, params, forces=True, energy=True):
    """(F [V,2] f64 or None, E [1] f64 or None) at X, on the current stream."""
    torch = _torch()
    X = _dev_f64(X, (t.V, 2))
    prm, keep = make_params(params, t.n, t.E)
    F = torch.empty((t.V, 2), dtype=torch.float64, device="cuda") if forces else None
    E = torch.empty(1, dtype=torch.float64, device="cuda") if energy else None
    st = capi.vx_energy_forces(t.handle, _ptr(X), C.byref(prm), _ptr(F), _ptr(E), _stream())
    capi.check(st, "vx_energy_forces")
    return F, E


def vx_minimize(t: Tissue, X, params, **opts):
    """Relax X (device f64 [V,2], updated in place) to force balance."""
    if not (hasattr(X, "is_cuda") and X.is_cuda and X.dtype == _torch().float64
            and X.is_contiguous()):
        raise TypeError("X must be a contiguous float64 CUDA tensor (updated in place)")
    prm, keep = make_params(params, t.n, t.E)
    o = min_opts(**opts)
    r = capi.vx_min_result()
    st = capi.vx_minimize(t.handle, _ptr(X), C.byref(prm), C.byref(o), C.byref(r), _stream())
    capi.check(st, "vx_minimize")
    return MinResult(r.status, r.iters, r.n_t1, r.n_stretch, r.n_short_edges, r.n_inverted,
                     r.fmax, r.energy, r.path_used, r.force_evals)


def result_buffer(kind="min", pinned=False):
    """A buffer for the result struct of vx_minimize_async (kind "min") or
    vx_equilibrium_grad_async ("grad"): a uint8 tensor on the device, or in
    pinned host memory."""
    torch = _torch()
    n = C.sizeof(capi.vx_min_result if kind == "min" else capi.vx_grad_result)
    if pinned:
        return torch.zeros(n, dtype=torch.uint8, pin_memory=True)
    return torch.zeros(n, dtype=torch.uint8, device="cuda")


def read_result(buf, kind="min"):
    """The MinResult / GradResult held in a result_buffer (synchronises)."""
    torch = _torch()
    torch.cuda.synchronize()
    raw = bytes(buf.cpu().numpy().tobytes())
    if kind == "min":
        x = capi.vx_min_result.from_buffer_copy(raw)
        return MinResult(x.status, x.iters, x.n_t1, x.n_stretch, x.n_short_edges, x.n_inverted,
                         x.fmax, x.energy, x.path_used, x.force_evals)
    x = capi.vx_grad_result.from_buffer_copy(raw)
    return GradResult(x.status, x.cg_iters, x.cg_rel_residual, x.cost, tuple(x.nudged_iters))


class Params:
    """vx_params built once (device copies kept alive), for calls that are
    recorded in a CUDA graph."""

    def __init__(self, t, p):
        self.struct, self.keep = make_params(p, t.n, t.E)


def vx_minimize_async(t: Tissue, X, params, result, **opts):
    """vx_minimize without host synchronisation (see vx.h): the GPU writes
    the result into `result` (a result_buffer("min")).  params: a dict or a
    Params (use Params inside a CUDA graph capture)."""
    prm = params if isinstance(params, Params) else Params(t, params)
    o = min_opts(**opts)
    st = capi.vx_minimize_async(t.handle, _ptr(X), C.byref(prm.struct), C.byref(o),
                                C.c_void_p(result.data_ptr()), _stream())
    capi.check(st, "vx_minimize_async")
    return prm


def vx_equilibrium_grad_async(t: Tissue, Xstar, params, g, result, dCdX=None, mode=VX_ADJOINT_CG,
                              beta=1e-3, cg_rtol=1e-10, cg_max_iter=20000, cost=VX_COST_NONE,
                              cost_data=None, inner=None, ep_f64=1):
    """vx_equilibrium_grad without host synchronisation (see vx.h): the
    gradients go to the device tensors g["lam"], g["A0"], g["P0"] (each may
    be missing) and the GPU writes the result into `result` (a
    result_buffer("grad")).  Xstar, dCdX and cost_data must be device
    float64 tensors already (nothing is copied)."""
    prm = params if isinstance(params, Params) else Params(t, params)
    o = capi.vx_grad_opts()
    capi.vx_grad_opts_default(C.byref(o))
    o.mode, o.beta, o.cg_rtol, o.cg_max_iter, o.cost = mode, beta, cg_rtol, cg_max_iter, cost
    o.ep_f64 = ep_f64
    if cost_data is not None:
        o.cost_data = cost_data.data_ptr()
    if inner is not None:
        o.inner = min_opts(**inner)
    st = capi.vx_equilibrium_grad_async(t.handle, _ptr(Xstar), C.byref(prm.struct), _ptr(dCdX),
                                        C.byref(o), _ptr(g.get("lam")), _ptr(g.get("A0")),
                                        _ptr(g.get("P0")), C.c_void_p(result.data_ptr()),
                                        _stream())
    capi.check(st, "vx_equilibrium_grad_async")
    return prm


def vx_minimize_many(tissues, Xs, params, **opts):
    """Relax several tissues in one launch (see vx.h).  Xs: list of device
    f64 [V_k, 2] tensors updated in place; params: one dict per tissue (or
    one dict for all).  Returns a list of MinResult."""
    count = len(tissues)
    if isinstance(params, dict):
        params = [params] * count
    for X in Xs:
        if not (hasattr(X, "is_cuda") and X.is_cuda and X.dtype == _torch().float64
                and X.is_contiguous()):
            raise TypeError("every X must be a contiguous float64 CUDA tensor")
    keep = []
    parr = (capi.vx_params * count)()
    for k, (t, p) in enumerate(zip(tissues, params)):
        prm, kk = make_params(p, t.n, t.E)
        parr[k] = prm
        keep.append(kk)
    hs = (C.c_void_p * count)(*[t.handle.value for t in tissues])
    xs = (C.c_void_p * count)(*[X.data_ptr() for X in Xs])
    o = min_opts(**opts)
    r = (capi.vx_min_result * count)()
    st = capi.vx_minimize_many(hs, count, xs, parr, C.byref(o), r, _stream())
    capi.check(st, "vx_minimize_many")
    return [MinResult(x.status, x.iters, x.n_t1, x.n_stretch, x.n_short_edges, x.n_inverted,
                      x.fmax, x.energy, x.path_used, x.force_evals) for x in r]


@dataclass
class GradResult:
    status: int
    cg_iters: int
    cg_rel_residual: float
    cost: float
    nudged_iters: tuple


def vx_equilibrium_grad(t: Tissue, Xstar, params, dCdX=None, mode=VX_ADJOINT_CG, beta=1e-3,
                        cg_rtol=1e-10, cg_max_iter=20000, cost=VX_COST_NONE, cost_data=None,
                        inner=None, ep_f64=1):
    """Gradient of the outer cost at the equilibrium X* with respect to
    (Lambda, A0, P0).  Returns (dict of device f64 tensors, GradResult)."""
    torch = _torch()
    Xstar = _dev_f64(Xstar, (t.V, 2))
    prm, keep = make_params(params, t.n, t.E)
    o = capi.vx_grad_opts()
    capi.vx_grad_opts_default(C.byref(o))
    o.mode, o.beta, o.cg_rtol, o.cg_max_iter, o.cost = mode, beta, cg_rtol, cg_max_iter, cost
    o.ep_f64 = ep_f64
    cd = None
    if cost_data is not None:
        cd = _dev_f64(cost_data)
        o.cost_data = cd.data_ptr()
    if inner is not None:
        o.inner = min_opts(**inner)
    dc = _dev_f64(dCdX, (t.V, 2)) if dCdX is not None else None
    g = {k: torch.empty(m, dtype=torch.float64, device="cuda")
         for k, m in (("lam", t.E), ("A0", t.n), ("P0", t.n))}
    r = capi.vx_grad_result()
    st = capi.vx_equilibrium_grad(t.handle, _ptr(Xstar), C.byref(prm), _ptr(dc), C.byref(o),
                                  _ptr(g["lam"]), _ptr(g["A0"]), _ptr(g["P0"]), C.byref(r),
                                  _stream())
    capi.check(st, "vx_equilibrium_grad")
    return g, GradResult(r.status, r.cg_iters, r.cg_rel_residual, r.cost, tuple(r.nudged_iters))


def vx_sensitivity_grad(t: Tissue, Xstar, params, dCdX, kinds, indices, solver=VX_ADJOINT_CG,
                        rtol=1e-10, max_iter=20000):
    """Forward-mode implicit differentiation (see vx.h): dC/dtheta for the
    listed parameters (kinds: VX_PARAM_LAMBDA / A0 / P0; indices: edge or
    cell ids), one linear solve each.  Returns (values, statuses) as numpy
    arrays."""
    Xstar = _dev_f64(Xstar, (t.V, 2))
    dCdX = _dev_f64(dCdX, (t.V, 2))
    prm, keep = make_params(params, t.n, t.E)
    k = np.ascontiguousarray(kinds, dtype=np.int32)
    ix = np.ascontiguousarray(indices, dtype=np.int32)
    out = np.zeros(k.size, dtype=np.float64)
    st = np.zeros(k.size, dtype=np.int32)
    capi.check(capi.vx_sensitivity_grad(t.handle, _ptr(Xstar), C.byref(prm), _ptr(dCdX), k.size,
                                        k.ctypes.data, ix.ctypes.data, solver, rtol, max_iter,
                                        out.ctypes.data, st.ctypes.data, _stream()),
               "vx_sensitivity_grad")
    return out, st


def _make_equilibrium_fn():
    torch = _torch()

    class EquilibriumFn(torch.autograd.Function):
        """X* = argmin_X E(X; Lambda, A0, P0) as a differentiable function.

        forward: vx_minimize from X0.  backward: the implicit adjoint, i.e.
        vx_equilibrium_grad(ADJOINT_CG) with dC/dX* = grad_output.  Gradients
        flow to lam (per edge), A0 and P0 (per cell); X0 gets none (X* does
        not depend on the starting point within its basin).
        """

        @staticmethod
        def forward(ctx, X0, lam, A0, P0, tissue, KA, KP, opts):
            X = X0.detach().clone().contiguous()
            params = dict(KA=KA, KP=KP, A0=A0.detach(), P0=P0.detach(), lam=lam.detach())
            res = vx_minimize(tissue, X, params, **(opts or {}))
            ctx.tissue, ctx.KA, ctx.KP = tissue, KA, KP
            ctx.save_for_backward(X, lam.detach(), A0.detach(), P0.detach())
            ctx.result = res
            return X

        @staticmethod
        def backward(ctx, gX):
            X, lam, A0, P0 = ctx.saved_tensors
            params = dict(KA=ctx.KA, KP=ctx.KP, A0=A0, P0=P0, lam=lam)
            g, _ = vx_equilibrium_grad(ctx.tissue, X, params, dCdX=gX.contiguous())
            return None, g["lam"], g["A0"], g["P0"], None, None, None, None

    return EquilibriumFn


class _Lazy:
    _fn = None

    def __getattr__(self, k):
        if _Lazy._fn is None:
            _Lazy._fn = _make_equilibrium_fn()
        return getattr(_Lazy._fn, k)


EquilibriumFn = _Lazy()


# ----------------------------------------------------------------- batches

class Batch:
    """Many tissues solved in one persistent launch (vx_batch)."""

    def __init__(self, meshes, dtype="f32"):
        self.count = len(meshes)
        self.n = np.array([int(m["face_he"].shape[0]) for m in meshes], dtype=np.int32)
        self.V = 2 * self.n
        self.E = 3 * self.n
        self.vbase = np.concatenate([[0], np.cumsum(self.V)[:-1]]).astype(np.int64)
        self.cbase = np.concatenate([[0], np.cumsum(self.n)[:-1]]).astype(np.int64)
        self.ebase = np.concatenate([[0], np.cumsum(self.E)[:-1]]).astype(np.int64)
        box = np.ascontiguousarray([[m["Lx"], m["Ly"]] for m in meshes], dtype=np.float64)
        self.box = box
        he = np.ascontiguousarray(np.concatenate([m["he"] for m in meshes]), dtype=np.int32)
        face_he = np.ascontiguousarray(np.concatenate([m["face_he"] for m in meshes]), dtype=np.int32)
        edge_id = np.ascontiguousarray(np.concatenate([m["edge_id"] for m in meshes]), dtype=np.int32)
        self.dtype = {"f64": VX_F64, "f32": VX_F32}[dtype] if isinstance(dtype, str) else dtype
        _torch().cuda.init()
        h = C.c_void_p()
        st = capi.vx_batch_create(self.count, self.n.ctypes.data, box.ctypes.data, he.ctypes.data,
                                  face_he.ctypes.data, edge_id.ctypes.data, self.dtype, _stream(),
                                  C.byref(h))
        capi.check(st, "vx_batch_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            capi.vx_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def split(self, X):
        return [X[b:b + v] for b, v in zip(self.vbase, self.V)]

    def topologies(self):
        """Current per-tissue topologies (list of dicts, input format)."""
        HE = int(6 * self.n.sum())
        he = np.zeros((HE, 8), dtype=np.int32)
        face_he = np.zeros(int(self.n.sum()), dtype=np.int32)
        edge_id = np.zeros(HE, dtype=np.int32)
        capi.check(capi.vx_batch_topology(self.handle, he.ctypes.data, face_he.ctypes.data,
                                          edge_id.ctypes.data), "vx_batch_topology")
        out, h0 = [], 0
        for k in range(self.count):
            n = int(self.n[k])
            out.append(dict(he=he[h0:h0 + 6 * n], face_he=face_he[self.cbase[k]:self.cbase[k] + n],
                            edge_id=edge_id[h0:h0 + 6 * n], n=n, Lx=self.box[k, 0],
                            Ly=self.box[k, 1]))
            h0 += 6 * n
        return out


def make_batch_params(p, b: Batch):
    """vx_batch_params from a dict: each of KA, KP, A0, P0, lam is a scalar,
    a per-tissue list/array of length count ('per tissue'), or a device
    array over all cells / edges of the batch."""
    keep = []
    out = capi.vx_batch_params()
    for key, fp, ft, fs, tot in (("KA", "KA", "KA_t", "KA_s", int(b.n.sum())),
                                 ("KP", "KP", "KP_t", "KP_s", int(b.n.sum())),
                                 ("A0", "A0", "A0_t", "A0_s", int(b.n.sum())),
                                 ("P0", "P0", "P0_t", "P0_s", int(b.n.sum())),
                                 ("lam", "lambda_", "lambda_t", "lambda_s", int(b.E.sum()))):
        v = p[key]
        setattr(out, fp, None)
        setattr(out, ft, None)
        setattr(out, fs, 0.0)
        if np.ndim(v) == 0 and not (hasattr(v, "dim") and v.dim() > 0):
            setattr(out, fs, float(v))
        elif (hasattr(v, "numel") and v.numel() == tot) or (not hasattr(v, "numel") and np.size(v) == tot
                                                          and tot != b.count):
            t = _dev_f64(v)
            keep.append(t)
            setattr(out, fp, t.data_ptr())
        else:
            a = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
            if a.size != b.count:
                raise ValueError(f"{key}: expected a scalar, {b.count} per-tissue values or {tot}")
            keep.append(a)
            setattr(out, ft, a.ctypes.data)
    return out, keep


def vx_batch_create(meshes, dtype="f32"):
    return Batch(meshes, dtype)


def vx_batch_restore(b: Batch):
    capi.check(capi.vx_batch_restore(b.handle, _stream()), "vx_batch_restore")


def vx_minimize_batched(b: Batch, X, params, **opts):
    """Relax every tissue of the batch (X: device f64 [sum V, 2], in place).
    Returns a list of MinResult."""
    if not (hasattr(X, "is_cuda") and X.is_cuda and X.dtype == _torch().float64
            and X.is_contiguous()):
        raise TypeError("X must be a contiguous float64 CUDA tensor (updated in place)")
    prm, keep = make_batch_params(params, b)
    o = min_opts(**opts)
    r = (capi.vx_min_result * b.count)()
    st = capi.vx_minimize_batched(b.handle, _ptr(X), C.byref(prm), C.byref(o), r, _stream())
    capi.check(st, "vx_minimize_batched")
    return [MinResult(x.status, x.iters, x.n_t1, x.n_stretch, x.n_short_edges, x.n_inverted,
                      x.fmax, x.energy, x.path_used, x.force_evals) for x in r]


def vx_batch_aniso_cost(b: Batch, X, q_target):
    """Anisotropy cost of every tissue: (host array [count] of C, device f64
    [sum V, 2] of grad_X C)."""
    torch = _torch()
    Vt, Et, nt = int(b.V.sum()), int(b.E.sum()), int(b.n.sum())
    X = _dev_f64(X, (Vt, 2))
    qt = _dev_f64(np.asarray(q_target, dtype=np.float64).reshape(2))
    C_ = np.zeros(b.count, dtype=np.float64)
    G = torch.empty((Vt, 2), dtype=torch.float64, device="cuda")
    st = capi.vx_batch_aniso_cost(b.handle, _ptr(X), _ptr(qt), C_.ctypes.data, _ptr(G), _stream())
    capi.check(st, "vx_batch_aniso_cost")
    return C_, G


def vx_equilibrium_grad_batched(b: Batch, Xstar, params, dCdX, cg_rtol=1e-10, cg_max_iter=20000):
    """Adjoint gradients of every tissue of the batch at X* (device f64
    [sum V, 2]) for the outer-cost gradient dCdX (same shape).  Returns
    (dict of device f64 tensors lam [sum E], A0 [sum n], P0 [sum n], list of
    GradResult)."""
    torch = _torch()
    Vt, Et, nt = int(b.V.sum()), int(b.E.sum()), int(b.n.sum())
    Xstar = _dev_f64(Xstar, (Vt, 2))
    dCdX = _dev_f64(dCdX, (Vt, 2))
    prm, keep = make_batch_params(params, b)
    g = {k: torch.empty(m, dtype=torch.float64, device="cuda")
         for k, m in (("lam", Et), ("A0", nt), ("P0", nt))}
    r = (capi.vx_grad_result * b.count)()
    st = capi.vx_equilibrium_grad_batched(b.handle, _ptr(Xstar), C.byref(prm), _ptr(dCdX), cg_rtol,
                                          cg_max_iter, _ptr(g["lam"]), _ptr(g["A0"]),
                                          _ptr(g["P0"]), r, _stream())
    if st not in (capi.VX_OK, capi.VX_ERR_INDEFINITE):
        capi.check(st, "vx_equilibrium_grad_batched")
    return g, [GradResult(x.status, x.cg_iters, x.cg_rel_residual, x.cost, tuple(x.nudged_iters))
               for x in r]


def vx_batch_grad(b: Batch, X, params, cost, cost_data, what=3, free=None, mode=VX_EP_CENTERED,
                  beta=1e-3, cg_rtol=1e-10, cg_max_iter=20000, inner=None, ep_f64=1,
                  strict=True):
    """The batched gradient workload in one launch (see vx.h): relax every
    tissue (X: device f64 [sum V, 2], updated in place to X*), then the
    adjoint (what & 1) and / or EP (what & 2) gradients of the built-in
    cost.  Returns (adjoint dict, EP dict of device f64 tensors lam / A0 /
    P0, list of (MinResult, adjoint GradResult, EP GradResult)).  A tissue
    whose free relaxation ends in non-finite forces or an inconsistent
    topology raises VxError unless strict=False, in which case the
    per-tissue statuses report it."""
    torch = _torch()
    if not (hasattr(X, "is_cuda") and X.is_cuda and X.dtype == torch.float64
            and X.is_contiguous()):
        raise TypeError("X must be a contiguous float64 CUDA tensor (updated in place)")
    Vt, Et, nt = int(b.V.sum()), int(b.E.sum()), int(b.n.sum())
    prm, keep = make_batch_params(params, b)
    fo = min_opts(**(free or {}))
    go = capi.vx_grad_opts()
    capi.vx_grad_opts_default(C.byref(go))
    go.mode, go.beta, go.cg_rtol, go.cg_max_iter, go.cost = mode, beta, cg_rtol, cg_max_iter, cost
    go.ep_f64 = ep_f64
    cd = _dev_f64(cost_data)
    go.cost_data = cd.data_ptr()
    if inner is not None:
        go.inner = min_opts(**inner)
    mk = lambda: {k: torch.empty(m, dtype=torch.float64, device="cuda")
                  for k, m in (("lam", Et), ("A0", nt), ("P0", nt))}
    ga = mk() if what & capi.VX_GRAD_ADJOINT else {}
    ge = mk() if what & capi.VX_GRAD_EP else {}
    r = (capi.vx_batch_grad_result * b.count)()
    st = capi.vx_batch_grad(b.handle, _ptr(X), C.byref(prm), C.byref(fo), C.byref(go), what,
                            _ptr(ga.get("lam")), _ptr(ga.get("A0")), _ptr(ga.get("P0")),
                            _ptr(ge.get("lam")), _ptr(ge.get("A0")), _ptr(ge.get("P0")), r,
                            _stream())
    per_tissue = (capi.VX_ERR_INDEFINITE, capi.VX_ERR_NONFINITE, capi.VX_ERR_TOPOLOGY)
    if st != capi.VX_OK and (strict and st != capi.VX_ERR_INDEFINITE or st not in per_tissue):
        capi.check(st, "vx_batch_grad")
    out = []
    for x in r:
        f = x.free
        out.append((MinResult(f.status, f.iters, f.n_t1, f.n_stretch, f.n_short_edges,
                              f.n_inverted, f.fmax, f.energy, f.path_used, f.force_evals),
                    GradResult(x.adjoint.status, x.adjoint.cg_iters, x.adjoint.cg_rel_residual,
                               x.adjoint.cost, tuple(x.adjoint.nudged_iters)),
                    GradResult(x.ep.status, x.ep.cg_iters, x.ep.cg_rel_residual, x.ep.cost,
                               tuple(x.ep.nudged_iters))))
    return ga, ge, out


def vx_grid_barrier_selftest(ctas, absent_rank=-1, rounds=8, wait_s=0.25):
    """Bounded-wait check of the GRID barrier (see vx.h).  Returns (status,
    per-CTA statuses)."""
    out = np.zeros(ctas, dtype=np.int32)
    st = capi.vx_grid_barrier_selftest(ctas, absent_rank, rounds, wait_s, out.ctypes.data,
                                       _stream())
    if st not in (capi.VX_OK, capi.VX_ERR_TIMEOUT):
        capi.check(st, "vx_grid_barrier_selftest")
    return st, out


def _dev_tensor(name, x, dtype, shape):
    torch = _torch()
    if not torch.is_tensor(x) or not x.is_cuda:
        raise ValueError(f"{name}: expected a CUDA tensor (the caller's device memory)")
    if x.dtype != dtype or not x.is_contiguous() or tuple(x.shape) != tuple(shape):
        raise ValueError(f"{name}: expected a contiguous {dtype} tensor of shape {tuple(shape)}, "
                         f"got {x.dtype} {tuple(x.shape)}")
    return x


def vx_energy_forces_noalloc(he, face_he, edge_id, Lx, Ly, X, params, F=None, E=None,
                             status=None):
    """vx_energy_forces without a vx_tissue and without any allocation by the
    library (see vx.h).  he int32 [6n, 8], face_he int32 [n], edge_id int32
    [6n] and X float64 [2n, 2] are CUDA tensors the caller owns; F float64
    [2n, 2], E float64 [1] and status int32 [1] are CUDA outputs (F and E may
    be None).  Asynchronous on torch's current stream: status (table checks,
    see vx.h) is written by the GPU.  Per-cell or per-edge parameters are
    passed as CUDA float64 tensors of n or 3n values."""
    torch = _torch()
    if not torch.is_tensor(face_he):
        raise ValueError("face_he: expected a CUDA tensor (the caller's device memory)")
    n = int(face_he.shape[0])
    _dev_tensor("face_he", face_he, torch.int32, (n,))
    _dev_tensor("he", he, torch.int32, (6 * n, 8))
    _dev_tensor("edge_id", edge_id, torch.int32, (6 * n,))
    _dev_tensor("X", X, torch.float64, (2 * n, 2))
    if F is not None:
        _dev_tensor("F", F, torch.float64, (2 * n, 2))
    if E is not None:
        _dev_tensor("E", E, torch.float64, (1,))
    if status is None:
        raise ValueError("status: an int32 [1] CUDA tensor is required")
    _dev_tensor("status", status, torch.int32, (1,))
    for k in ("KA", "KP", "A0", "P0", "lam"):
        v = params[k]
        if torch.is_tensor(v) and v.dim() > 0:
            _dev_tensor(k, v, torch.float64, (3 * n,) if k == "lam" else (n,))
    prm, keep = make_params(params, n, 3 * n)
    st = capi.vx_energy_forces_noalloc(he.data_ptr(), face_he.data_ptr(), edge_id.data_ptr(), n,
                                       float(Lx), float(Ly), X.data_ptr(), C.byref(prm), _ptr(F),
                                       _ptr(E), status.data_ptr(), _stream())
    capi.check(st, "vx_energy_forces_noalloc")


def vx_version():
    return capi.vx_version().decode()


def vx_batch_autotune(b: Batch, X, params, probe_iters=200, **opts):
    prm, keep = make_batch_params(params, b)
    o = min_opts(**opts)
    T = C.c_int32()
    S = C.c_int32()
    st = capi.vx_batch_autotune(b.handle, _ptr(X), C.byref(prm), C.byref(o), probe_iters,
                                C.byref(T), C.byref(S), _stream())
    capi.check(st, "vx_batch_autotune")
    return T.value, S.value
