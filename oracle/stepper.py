"""ctypes wrapper of the C oracle stepper (TEST INFRASTRUCTURE ONLY).

Derives the run constants from a synthetic_inputs.Case exactly as Sec. II.C and
Sec. IV.A of Saito et al. (arXiv:1912.02018) state them (see derive_params), then
drives lbm_oracle.c.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import build as _build
from .thermo import PR


class OrcParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("periodic_x", C.c_int32), ("energy", C.c_int32),
        ("warmup", C.c_int64),
        ("xc", C.c_double), ("yc", C.c_double), ("D", C.c_double),
        ("a", C.c_double), ("b", C.c_double), ("R", C.c_double), ("kappa", C.c_double), ("Tc", C.c_double),
        ("G", C.c_double), ("sigma", C.c_double),
        ("T_sat", C.c_double), ("T_wall", C.c_double),
        ("rho_l", C.c_double), ("rho_v", C.c_double), ("rho_s", C.c_double),
        ("nu_l", C.c_double), ("nu_v", C.c_double), ("alpha_l", C.c_double), ("alpha_v", C.c_double),
        ("c_v", C.c_double),
        ("g", C.c_double), ("u_in", C.c_double), ("U_out", C.c_double),
        ("n_wall", C.c_int32), ("walls", C.c_int32), ("wall_dT", C.POINTER(C.c_double)),
        ("body_fx", C.c_double),
        ("collision", C.c_int32), ("reserved", C.c_int32),
        ("wall_q", C.c_double),
    ]


_LIB = None


def load():
    global _LIB
    if _LIB is None:
        lib = C.CDLL(_build.build())
        P = C.POINTER(OrcParams)
        dp = C.POINTER(C.c_double)
        lib.orc_create.restype = C.c_void_p
        lib.orc_create.argtypes = [P, dp, dp, dp, dp]
        lib.orc_destroy.argtypes = [C.c_void_p]
        lib.orc_step.argtypes = [C.c_void_p, C.c_int64]
        lib.orc_get_field.argtypes = [C.c_void_p, C.c_int, dp]
        lib.orc_get_f.argtypes = [C.c_void_p, dp]
        lib.orc_get_side.argtypes = [C.c_void_p, dp]
        lib.orc_set_state.argtypes = [C.c_void_p, dp, dp, dp, C.c_int64]
        lib.orc_steps.restype = C.c_int64
        lib.orc_steps.argtypes = [C.c_void_p]
        lib.orc_n_boundary.restype = C.c_int
        lib.orc_n_boundary.argtypes = [C.c_void_p]
        lib.orc_boundary.argtypes = [C.c_void_p, C.POINTER(C.c_int), dp, dp]
        lib.orc_link_fractions.argtypes = [C.c_void_p, dp]
        lib.orc_heat_flux.argtypes = [C.c_void_p, dp]
        lib.orc_p_eos.restype = C.c_double
        lib.orc_p_eos.argtypes = [P, C.c_double, C.c_double]
        lib.orc_dpdT.restype = C.c_double
        lib.orc_dpdT.argtypes = [P, C.c_double, C.c_double]
        lib.orc_psi.restype = C.c_double
        lib.orc_psi.argtypes = [P, C.c_double, C.c_double]
        lib.orc_lambda.restype = C.c_double
        lib.orc_lambda.argtypes = [P, C.c_double]
        lib.orc_nu.restype = C.c_double
        lib.orc_nu.argtypes = [P, C.c_double]
        lib.orc_feq.argtypes = [C.c_double, C.c_double, C.c_double, dp]
        lib.orc_matrix_M.argtypes = [dp]
        lib.orc_matrix_N.argtypes = [C.c_double, C.c_double, dp]
        lib.orc_invert9.restype = C.c_int
        lib.orc_invert9.argtypes = [dp, dp]
        lib.orc_collide_node.argtypes = [dp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                         C.c_double, C.c_double, C.c_int, dp, dp, dp, dp, dp]
        lib.orc_energy_rhs_fields.argtypes = [P, dp, dp, dp, dp, dp]
        lib.orc_interaction_force.argtypes = [P, dp, dp, dp]
        _LIB = lib
    return _LIB


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _c(a, n):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    assert a.size == n
    return a


@dataclass
class Derived:
    """Constants the oracle derives from a Case."""
    eos: PR
    Tc: float
    T_sat: float
    T_wall: float
    rho_l: float
    rho_v: float
    nu_l: float
    nu_v: float
    alpha_l: float
    alpha_v: float
    g: float
    U_out: float
    lambda_v: float


_MAXWELL_CACHE: dict = {}


def derive(case) -> tuple[OrcParams, Derived]:
    """Run constants from the raw case, as the paper sets them.

    Tc from the EOS constants (Sec. II.C); T_sat = Tr_sat Tc; T_w = T_sat + superheat;
    rho_l, rho_v by Maxwell at T_sat (Sec. III.D); nu_l = u_in D / Re and
    nu_v = nu_l / eta; alpha = nu / Pr per phase; g from u_in / sqrt(g D) = 4
    (Sec. IV.A); convective-outlet speed U = u_in.
    """
    eos = PR(case.a, case.b, case.R, case.acentric)
    Tc = eos.Tc
    T_sat = case.Tr_sat * Tc
    T_wall = T_sat + case.superheat_Tc * Tc
    key = (case.a, case.b, case.R, case.acentric, case.Tr_sat)
    if key not in _MAXWELL_CACHE:
        _MAXWELL_CACHE[key] = eos.maxwell(T_sat)
    rho_v, rho_l, _ = _MAXWELL_CACHE[key]
    nu_l = case.nu_l if case.nu_l > 0 else case.u_in * case.D / case.Re
    nu_v = nu_l / case.nu_ratio
    alpha_l = nu_l / case.Pr_l
    alpha_v = nu_v / case.Pr_v
    g = case.g if case.g >= 0 else (case.u_in * case.u_in / (16.0 * case.D) if case.D > 0 else 0.0)
    U_out = case.U_out if case.U_out >= 0 else case.u_in
    p = OrcParams(
        nx=case.nx, ny=case.ny, periodic_x=case.periodic_x, energy=case.energy, warmup=case.warmup,
        xc=case.xc, yc=case.yc, D=case.D, a=case.a, b=case.b, R=case.R, kappa=eos.kappa, Tc=Tc,
        G=case.G, sigma=case.sigma, T_sat=T_sat, T_wall=T_wall, rho_l=rho_l, rho_v=rho_v,
        rho_s=case.rho_s if case.rho_s > 0 else rho_l,
        nu_l=nu_l, nu_v=nu_v, alpha_l=alpha_l, alpha_v=alpha_v, c_v=case.c_v,
        g=g, u_in=case.u_in, U_out=U_out, walls=int(getattr(case, "walls", 0)),
        body_fx=float(getattr(case, "body_fx", 0.0)), collision=int(getattr(case, "collision", 0)),
        wall_q=float(getattr(case, "wall_q", 0.5)))
    knots = np.ascontiguousarray(getattr(case, "wall_dT", ()) or (), dtype=np.float64)
    if knots.size:
        p.n_wall = knots.size
        p.wall_dT = knots.ctypes.data_as(C.POINTER(C.c_double))
        p._keep = knots  # the knots must outlive the structure
    d = Derived(eos, Tc, T_sat, T_wall, rho_l, rho_v, nu_l, nu_v, alpha_l, alpha_v, g, U_out,
                rho_v * case.c_v * alpha_v)
    return p, d


class Oracle:
    """FP64 CPU stepper for one Case.

    Initial state: rho = (rho if given else rho_l) + drho, u = (ux, uy) if given else
    (u_in, 0), T = T if given else T_sat; populations f* = f^eq(rho, u).
    Arrays are (ny, nx) with node id = y*nx + x.
    """

    FIELDS = ("rho", "ux", "uy", "T", "psi", "solid")

    def __init__(self, case, drho=None, rho=None, ux=None, uy=None, T=None):
        self.lib = load()
        self.case = case
        self.params, self.derived = derive(case)
        n = case.nx * case.ny
        self.n_nodes = n
        r = _c(rho, n)
        if drho is not None:
            base = r if r is not None else np.full(n, self.derived.rho_l)
            r = base + _c(drho, n)
        self._keep = [r, _c(ux, n), _c(uy, n), _c(T, n)]
        self.h = self.lib.orc_create(C.byref(self.params), *[_ptr(a) for a in self._keep])

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.orc_destroy(h)
            self.h = None

    def step(self, n: int = 1):
        self.lib.orc_step(self.h, int(n))
        return self

    @property
    def steps(self) -> int:
        return int(self.lib.orc_steps(self.h))

    def field(self, name: str) -> np.ndarray:
        out = np.empty(self.n_nodes)
        self.lib.orc_get_field(self.h, self.FIELDS.index(name), _ptr(out))
        return out.reshape(self.case.ny, self.case.nx)

    def fields(self) -> dict:
        return {k: self.field(k) for k in ("rho", "ux", "uy", "T", "psi")}

    def populations(self) -> np.ndarray:
        out = np.empty(9 * self.n_nodes)
        self.lib.orc_get_f(self.h, _ptr(out))
        return out.reshape(9, self.case.ny, self.case.nx)

    def side(self) -> np.ndarray:
        out = np.empty(3 * self.case.ny)
        self.lib.orc_get_side(self.h, _ptr(out))
        return out.reshape(3, self.case.ny)

    def set_state(self, f=None, T=None, side=None, n=None):
        keep = [_c(f, 9 * self.n_nodes), _c(T, self.n_nodes), _c(side, 3 * self.case.ny)]
        self.lib.orc_set_state(self.h, *[_ptr(a) for a in keep], int(self.steps if n is None else n))

    def boundary(self):
        nb = self.lib.orc_n_boundary(self.h)
        node = np.empty(nb, dtype=np.int32)
        bx = np.empty(nb)
        by = np.empty(nb)
        self.lib.orc_boundary(self.h, node.ctypes.data_as(C.POINTER(C.c_int)), _ptr(bx), _ptr(by))
        return node, bx, by

    def link_fractions(self) -> np.ndarray:
        out = np.empty(9 * self.n_nodes)
        self.lib.orc_link_fractions(self.h, _ptr(out))
        return out.reshape(self.case.ny, self.case.nx, 9)

    def heat_flux(self) -> dict:
        out = np.empty(4)
        self.lib.orc_heat_flux(self.h, _ptr(out))
        cnt = int(out[3])
        mean = out[1] / cnt if cnt else 0.0
        var = max(out[2] / cnt - mean * mean, 0.0) if cnt else 0.0
        d = self.derived
        dT = d.T_wall - d.T_sat
        nu = mean * self.case.D / (d.lambda_v * dT) if (cnt and dT > 0) else 0.0
        return {"q_now": out[0], "q_mean": mean, "q_std": var ** 0.5, "count": cnt, "nu_mean": nu,
                "q_sum": out[1], "q_sumsq": out[2]}


def collide_node(f, Fx, Fy, Fmx, Fmy, psi, omega, sigma, bgk=0):
    """The C oracle's one-node collision, CM or (bgk=1) BGK (for definition-level tests)."""
    lib = load()
    M = np.empty(81)
    lib.orc_matrix_M(_ptr(M))
    Minv = np.empty(81)
    lib.orc_invert9(_ptr(M), _ptr(Minv))
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty(9)
    r = C.c_double()
    u = C.c_double()
    v = C.c_double()
    lib.orc_collide_node(_ptr(f), Fx, Fy, Fmx, Fmy, psi, omega, sigma, int(bgk), _ptr(Minv), _ptr(out),
                         C.byref(r), C.byref(u), C.byref(v))
    return out, r.value, u.value, v.value


def matrix_N(ux, uy) -> np.ndarray:
    out = np.empty(81)
    load().orc_matrix_N(ux, uy, _ptr(out))
    return out.reshape(9, 9)


def matrix_M() -> np.ndarray:
    out = np.empty(81)
    load().orc_matrix_M(_ptr(out))
    return out.reshape(9, 9)


def feq(rho, ux, uy) -> np.ndarray:
    out = np.empty(9)
    load().orc_feq(rho, ux, uy, _ptr(out))
    return out


def energy_rhs(case, rho, ux, uy, T) -> np.ndarray:
    p, _ = derive(case)
    n = case.nx * case.ny
    arrs = [_c(a, n) for a in (rho, ux, uy, T)]
    out = np.empty(n)
    load().orc_energy_rhs_fields(C.byref(p), *[_ptr(a) for a in arrs], _ptr(out))
    return out.reshape(case.ny, case.nx)


def interaction_force(case, psi):
    p, _ = derive(case)
    n = case.nx * case.ny
    ps = _c(psi, n)
    fx = np.empty(n)
    fy = np.empty(n)
    load().orc_interaction_force(C.byref(p), _ptr(ps), _ptr(fx), _ptr(fy))
    return fx.reshape(case.ny, case.nx), fy.reshape(case.ny, case.nx)


def eos_funcs(case):
    """The C oracle's p_EOS, (dp/dT)_rho, psi, lambda and nu for a case."""
    p, _ = derive(case)
    lib = load()
    return {
        "p": lambda r, T: lib.orc_p_eos(C.byref(p), r, T),
        "dpdT": lambda r, T: lib.orc_dpdT(C.byref(p), r, T),
        "psi": lambda r, T: lib.orc_psi(C.byref(p), r, T),
        "lambda": lambda r: lib.orc_lambda(C.byref(p), r),
        "nu": lambda r: lib.orc_nu(C.byref(p), r),
    }
