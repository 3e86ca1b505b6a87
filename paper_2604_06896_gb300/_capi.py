"""ctypes binding of libvx.so: the C structs of vx.h and the raw entry points.

Argument marshalling only.  Every computation runs in the CUDA library; if
the library is missing this module raises ImportError (there is no CPU
fallback).
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvx.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python -c 'import __graft_entry__ as g; g.build()')")

lib = C.CDLL(LIB_PATH)

VX_OK, VX_NOT_CONVERGED, VX_ERR_INVALID_ARG, VX_ERR_DEGENERATE_SEEDS, VX_ERR_CUDA, VX_ERR_OOM, \
    VX_ERR_INDEFINITE, VX_ERR_TIMEOUT, VX_ERR_NONFINITE, VX_ERR_TOPOLOGY = range(10)
VX_F64, VX_F32 = 0, 1
VX_FIRE, VX_GD = 0, 1
VX_ADJOINT_CG, VX_EP_CENTERED, VX_EP_FORWARD, VX_ADJOINT_MINRES = 0, 1, 2, 3
VX_PARAM_LAMBDA, VX_PARAM_A0, VX_PARAM_P0 = 0, 1, 2
VX_COST_NONE, VX_COST_V2V, VX_COST_ANISO = 0, 1, 2
VX_PATH_AUTO, VX_PATH_RESIDENT, VX_PATH_PLAIN, VX_PATH_CLUSTER, VX_PATH_GRID = 0, 1, 2, 3, 4

STATUS_NAMES = {0: "VX_OK", 1: "VX_NOT_CONVERGED", 2: "VX_ERR_INVALID_ARG",
                3: "VX_ERR_DEGENERATE_SEEDS", 4: "VX_ERR_CUDA", 5: "VX_ERR_OOM",
                6: "VX_ERR_INDEFINITE", 7: "VX_ERR_TIMEOUT", 8: "VX_ERR_NONFINITE",
                9: "VX_ERR_TOPOLOGY"}

P_d = C.POINTER(C.c_double)
P_i32 = C.POINTER(C.c_int32)


class vx_params(C.Structure):
    _fields_ = [("KA", C.c_void_p), ("KP", C.c_void_p), ("A0", C.c_void_p), ("P0", C.c_void_p),
                ("lambda_", C.c_void_p),
                ("KA_s", C.c_double), ("KP_s", C.c_double), ("A0_s", C.c_double),
                ("P0_s", C.c_double), ("lambda_s", C.c_double)]


class vx_min_opts(C.Structure):
    _fields_ = [("method", C.c_int32), ("tol", C.c_double), ("patience", C.c_int32),
                ("max_iter", C.c_int32), ("gd_lr", C.c_double), ("dt0", C.c_double),
                ("dt_max", C.c_double), ("n_min", C.c_int32), ("f_inc", C.c_double),
                ("f_dec", C.c_double), ("alpha0", C.c_double), ("f_alpha", C.c_double),
                ("l_min", C.c_double), ("path", C.c_int32), ("check_every", C.c_int32),
                ("wrap", C.c_int32), ("edge_events", C.c_void_p), ("refine_tol", C.c_double)]


class vx_min_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("n_t1", C.c_int32),
                ("n_stretch", C.c_int32), ("n_short_edges", C.c_int32), ("n_inverted", C.c_int32),
                ("fmax", C.c_double), ("energy", C.c_double), ("path_used", C.c_int32),
                ("force_evals", C.c_int32)]


class vx_grad_opts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("beta", C.c_double), ("cg_rtol", C.c_double),
                ("cg_max_iter", C.c_int32), ("cost", C.c_int32), ("cost_data", C.c_void_p),
                ("inner", vx_min_opts), ("ep_f64", C.c_int32)]


class vx_grad_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("cg_iters", C.c_int32), ("cg_rel_residual", C.c_double),
                ("cost", C.c_double), ("nudged_iters", C.c_int32 * 2)]


class vx_batch_params(C.Structure):
    _fields_ = [("KA", C.c_void_p), ("KP", C.c_void_p), ("A0", C.c_void_p), ("P0", C.c_void_p),
                ("lambda_", C.c_void_p),
                ("KA_t", C.c_void_p), ("KP_t", C.c_void_p), ("A0_t", C.c_void_p),
                ("P0_t", C.c_void_p), ("lambda_t", C.c_void_p),
                ("KA_s", C.c_double), ("KP_s", C.c_double), ("A0_s", C.c_double),
                ("P0_s", C.c_double), ("lambda_s", C.c_double)]


def _sig(name, res, *args):
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = list(args)
    return f


vx_last_error = _sig("vx_last_error", C.c_char_p)
vx_version = _sig("vx_version", C.c_char_p)
vx_build_mesh = _sig("vx_build_mesh", C.c_int, C.c_void_p, C.c_int32, C.c_double, C.c_double,
                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p)
vx_seed_order = _sig("vx_seed_order", C.c_int, C.c_void_p, C.c_int32, C.c_double, C.c_double,
                     C.c_void_p)
vx_tissue_create = _sig("vx_tissue_create", C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                        C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_int32, C.c_void_p,
                        C.POINTER(C.c_void_p))
vx_tissue_destroy = _sig("vx_tissue_destroy", C.c_int, C.c_void_p)
vx_tissue_sizes = _sig("vx_tissue_sizes", C.c_int, C.c_void_p, P_i32, P_i32, P_i32, P_i32)
vx_tissue_topology = _sig("vx_tissue_topology", C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                          C.c_void_p)
vx_tissue_restore = _sig("vx_tissue_restore", C.c_int, C.c_void_p, C.c_void_p)
vx_hessian_vector = _sig("vx_hessian_vector", C.c_int, C.c_void_p, C.c_void_p,
                         C.POINTER(vx_params), C.c_void_p, C.c_void_p, C.c_void_p)
vx_energy_forces = _sig("vx_energy_forces", C.c_int, C.c_void_p, C.c_void_p,
                        C.POINTER(vx_params), C.c_void_p, C.c_void_p, C.c_void_p)
vx_min_opts_default = _sig("vx_min_opts_default", None, C.POINTER(vx_min_opts))
vx_minimize = _sig("vx_minimize", C.c_int, C.c_void_p, C.c_void_p, C.POINTER(vx_params),
                   C.POINTER(vx_min_opts), C.POINTER(vx_min_result), C.c_void_p)
vx_minimize_many = _sig("vx_minimize_many", C.c_int, C.POINTER(C.c_void_p), C.c_int32,
                        C.POINTER(C.c_void_p), C.POINTER(vx_params), C.POINTER(vx_min_opts),
                        C.POINTER(vx_min_result), C.c_void_p)
vx_grad_opts_default = _sig("vx_grad_opts_default", None, C.POINTER(vx_grad_opts))
vx_equilibrium_grad = _sig("vx_equilibrium_grad", C.c_int, C.c_void_p, C.c_void_p,
                           C.POINTER(vx_params), C.c_void_p, C.POINTER(vx_grad_opts), C.c_void_p,
                           C.c_void_p, C.c_void_p, C.POINTER(vx_grad_result), C.c_void_p)

vx_energy_forces_noalloc = _sig("vx_energy_forces_noalloc", C.c_int, C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_int32, C.c_double, C.c_double, C.c_void_p,
                                C.POINTER(vx_params), C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_void_p)
vx_sensitivity_grad = _sig("vx_sensitivity_grad", C.c_int, C.c_void_p, C.c_void_p,
                           C.POINTER(vx_params), C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                           C.c_int32, C.c_double, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p)
vx_minimize_async = _sig("vx_minimize_async", C.c_int, C.c_void_p, C.c_void_p,
                         C.POINTER(vx_params), C.POINTER(vx_min_opts), C.c_void_p, C.c_void_p)
vx_equilibrium_grad_async = _sig("vx_equilibrium_grad_async", C.c_int, C.c_void_p, C.c_void_p,
                                 C.POINTER(vx_params), C.c_void_p, C.POINTER(vx_grad_opts),
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p)
vx_grid_barrier_selftest = _sig("vx_grid_barrier_selftest", C.c_int, C.c_int32, C.c_int32,
                                C.c_int32, C.c_double, C.c_void_p, C.c_void_p)
vx_batch_create = _sig("vx_batch_create", C.c_int, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                       C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_void_p))
vx_batch_destroy = _sig("vx_batch_destroy", C.c_int, C.c_void_p)
vx_batch_restore = _sig("vx_batch_restore", C.c_int, C.c_void_p, C.c_void_p)
vx_batch_sizes = _sig("vx_batch_sizes", C.c_int, C.c_void_p, P_i32, P_i32, P_i32, P_i32)
vx_batch_topology = _sig("vx_batch_topology", C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                         C.c_void_p)
vx_minimize_batched = _sig("vx_minimize_batched", C.c_int, C.c_void_p, C.c_void_p,
                           C.POINTER(vx_batch_params), C.POINTER(vx_min_opts),
                           C.c_void_p, C.c_void_p)
vx_batch_autotune = _sig("vx_batch_autotune", C.c_int, C.c_void_p, C.c_void_p,
                         C.POINTER(vx_batch_params), C.POINTER(vx_min_opts), C.c_int32,
                         P_i32, P_i32, C.c_void_p)

vx_equilibrium_grad_batched = _sig("vx_equilibrium_grad_batched", C.c_int, C.c_void_p, C.c_void_p,
                                   C.POINTER(vx_batch_params), C.c_void_p, C.c_double, C.c_int32,
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p)
class vx_batch_grad_result(C.Structure):
    _fields_ = [("free", vx_min_result), ("adjoint", vx_grad_result), ("ep", vx_grad_result)]


VX_GRAD_ADJOINT, VX_GRAD_EP = 1, 2
vx_batch_grad = _sig("vx_batch_grad", C.c_int, C.c_void_p, C.c_void_p, C.POINTER(vx_batch_params),
                     C.POINTER(vx_min_opts), C.POINTER(vx_grad_opts), C.c_int32, C.c_void_p,
                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                     C.c_void_p)
vx_batch_aniso_cost = _sig("vx_batch_aniso_cost", C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                           C.c_void_p, C.c_void_p, C.c_void_p)

EXPORTED = ["vx_last_error", "vx_version", "vx_build_mesh", "vx_seed_order", "vx_tissue_create",
            "vx_tissue_destroy", "vx_tissue_sizes", "vx_tissue_topology", "vx_tissue_restore",
            "vx_hessian_vector", "vx_energy_forces",
            "vx_min_opts_default", "vx_minimize", "vx_minimize_many", "vx_grad_opts_default",
            "vx_equilibrium_grad",
            "vx_batch_create", "vx_batch_destroy", "vx_batch_restore", "vx_batch_sizes",
            "vx_batch_topology", "vx_energy_forces_noalloc", "vx_grid_barrier_selftest",
            "vx_minimize_async", "vx_equilibrium_grad_async", "vx_batch_grad",
            "vx_sensitivity_grad",
            "vx_minimize_batched", "vx_batch_autotune", "vx_equilibrium_grad_batched",
            "vx_batch_aniso_cost"]


class VxError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = vx_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


def check(status, where):
    if status not in (VX_OK, VX_NOT_CONVERGED):
        raise VxError(status, where)
    return status
