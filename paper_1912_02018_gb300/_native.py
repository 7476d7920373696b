"""ctypes declarations of the C ABI in include/lbm.h (argument marshalling only).

Loading fails loudly if liblbm.so has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_ESTATE = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "LBM_OK", -1: "LBM_EINVAL", -2: "LBM_ENOMEM", -3: "LBM_ECUDA", -4: "LBM_EUNSTABLE",
                -5: "LBM_ETIMEOUT", -6: "LBM_ESTATE"}
LBM_STORE_F64, LBM_STORE_F32, LBM_STORE_F16S = 0, 1, 2
STORAGE = {"f64": LBM_STORE_F64, "f32": LBM_STORE_F32, "f16s": LBM_STORE_F16S}
FIELD_BITS = {"rho": 1, "ux": 2, "uy": 4, "T": 8, "psi": 16, "solid": 32, "Fx": 64, "Fy": 128}

# every symbol include/lbm.h declares
EXPORTS = ("lbm_create", "lbm_step", "lbm_sync", "lbm_wall_heat_flux", "lbm_reset_heat_flux", "lbm_fields",
           "lbm_get_state", "lbm_set_state", "lbm_info", "lbm_profile", "lbm_profile_read", "lbm_last_error",
           "lbm_destroy", "lbm_wall_heat_flux_noalloc", "lbm_batch_create", "lbm_batch_step", "lbm_batch_tune",
           "lbm_batch_graph", "lbm_batch_domain", "lbm_batch_destroy", "lbm_adjoint_window", "lbm_adjoint_step",
           "lbm_get_state_native", "lbm_set_state_native", "lbm_inject_fault", "lbm_stage_state_native",
           "lbm_take_staged")
LBM_FAULT_STARVE_COLLIDE, LBM_FAULT_STARVE_ENERGY = 1, 2


class Domain(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("periodic_x", C.c_int32), ("walls", C.c_int32)]


class Cylinder(C.Structure):
    _fields_ = [("xc", C.c_double), ("yc", C.c_double), ("D", C.c_double), ("superheat_Tc", C.c_double),
                ("rho_solid", C.c_double), ("wall_dT", C.POINTER(C.c_double)), ("n_wall", C.c_int32),
                ("reserved", C.c_int32)]


LBM_COLL_CM, LBM_COLL_BGK = 0, 1


class Params(C.Structure):
    _fields_ = [("a", C.c_double), ("b", C.c_double), ("R", C.c_double), ("acentric", C.c_double),
                ("G", C.c_double), ("sigma", C.c_double), ("Tr_sat", C.c_double), ("Re", C.c_double),
                ("u_in", C.c_double), ("nu_l", C.c_double), ("nu_ratio", C.c_double), ("Pr_l", C.c_double),
                ("Pr_v", C.c_double), ("c_v", C.c_double), ("g", C.c_double), ("outlet_U", C.c_double),
                ("warmup_steps", C.c_int64), ("energy", C.c_int32), ("storage", C.c_int32),
                ("compute_f64", C.c_int32), ("psi_mode", C.c_int32), ("seed", C.c_uint64),
                ("noise_amp", C.c_double), ("body_fx", C.c_double), ("collision", C.c_int32),
                ("reserved", C.c_int32)]


class Init(C.Structure):
    _fields_ = [("rho", C.c_void_p), ("drho", C.c_void_p), ("ux", C.c_void_p), ("uy", C.c_void_p),
                ("T", C.c_void_p)]


class WindowGrad(C.Structure):
    _fields_ = [("J", C.c_double), ("dJ_dsuperheat", C.c_double), ("dJ_du_in", C.c_double),
                ("dJ_dwall_dT", C.POINTER(C.c_double)), ("dJ_dTw", C.POINTER(C.c_double))]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class Info(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("Tc", "pc", "T_sat", "T_wall", "rho_l", "rho_v", "p_sat", "h_fg", "nu_l",
                                          "nu_v", "alpha_l", "alpha_v", "lambda_v", "g", "outlet_U")] + [
        ("steps", C.c_int64), ("n_boundary", C.c_int64), ("kernel_launches", C.c_int64),
        ("device_bytes", C.c_int64)]


_LIB = None


def lib():
    """The loaded liblbm.so with argument types set; raises if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run paper_1912_02018_gb300/nvcc_build.py (no CPU fallback exists)")
    L = C.CDLL(LIB_PATH)
    vp, dp, i64 = C.c_void_p, C.POINTER(C.c_double), C.c_int64
    L.lbm_create.argtypes = [C.POINTER(Domain), C.POINTER(Cylinder), C.POINTER(Params), C.POINTER(Init),
                             C.POINTER(Allocator), vp, C.POINTER(vp)]
    L.lbm_step.argtypes = [vp, i64]
    L.lbm_sync.argtypes = [vp]
    L.lbm_wall_heat_flux.argtypes = [vp, dp, dp, dp, dp, C.POINTER(i64)]
    L.lbm_reset_heat_flux.argtypes = [vp]
    L.lbm_fields.argtypes = [vp, C.c_uint32, vp, C.c_size_t, C.c_int]
    L.lbm_get_state.argtypes = [vp, vp, vp, vp, C.POINTER(i64)]
    L.lbm_set_state.argtypes = [vp, vp, vp, vp, i64]
    L.lbm_get_state_native.argtypes = [vp, vp, vp, vp, C.POINTER(i64)]
    L.lbm_set_state_native.argtypes = [vp, vp, vp, vp, i64]
    L.lbm_stage_state_native.argtypes = [vp, vp, vp, vp, i64]
    L.lbm_take_staged.argtypes = [vp]
    L.lbm_info.argtypes = [vp, C.POINTER(Info)]
    L.lbm_inject_fault.argtypes = [vp, C.c_int32]
    L.lbm_profile.argtypes = [vp, C.c_int]
    L.lbm_profile_read.argtypes = [vp, C.POINTER(C.c_char_p), C.POINTER(i64), dp, C.c_int32,
                                   C.POINTER(C.c_int32)]
    L.lbm_last_error.argtypes = [vp]
    L.lbm_last_error.restype = C.c_char_p
    L.lbm_wall_heat_flux_noalloc.argtypes = [C.POINTER(Domain), C.POINTER(Cylinder), C.POINTER(Params), vp, vp,
                                             vp, vp]
    L.lbm_destroy.argtypes = [vp]
    L.lbm_destroy.restype = None
    L.lbm_batch_create.argtypes = [C.c_int32, C.POINTER(Domain), C.POINTER(Cylinder), C.POINTER(Params),
                                   C.POINTER(Allocator), vp, C.POINTER(vp)]
    L.lbm_batch_step.argtypes = [vp, i64]
    L.lbm_batch_tune.argtypes = [vp, C.c_int32, C.POINTER(C.c_int32)]
    L.lbm_batch_graph.argtypes = [vp, C.c_int]
    L.lbm_batch_domain.argtypes = [vp, C.c_int32, C.POINTER(vp)]
    L.lbm_adjoint_window.argtypes = [vp, i64, C.c_int32, C.POINTER(WindowGrad)]
    L.lbm_adjoint_step.argtypes = [vp, vp, vp, vp, C.c_double, vp, vp, vp, vp, dp]
    L.lbm_batch_destroy.argtypes = [vp]
    L.lbm_batch_destroy.restype = None
    for name in EXPORTS:
        if name not in ("lbm_last_error", "lbm_destroy", "lbm_batch_destroy"):
            getattr(L, name).restype = C.c_int
    _LIB = L
    return L


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int, handle=None):
    if status != LBM_OK:
        msg = lib().lbm_last_error(handle).decode(errors="replace")
        raise LbmError(status, msg)
