"""CPU checks of the C-ABI library: it builds, loads and exports every declared symbol,
and it rejects invalid parameters on the host before touching the GPU."""
import ctypes as C
import os
import re

import pytest

from paper_1912_02018_gb300 import _native as N
from paper_1912_02018_gb300 import build as build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build_lib()
    return N.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbm_create", "lbm_step", "lbm_wall_heat_flux", "lbm_fields"):
        assert required in names
    assert set(names) == set(N.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_struct_sizes_match_header_layout():
    assert C.sizeof(N.Domain) == 16
    assert C.sizeof(N.Cylinder) == 56
    assert C.sizeof(N.Params) == 16 * 8 + 8 + 16 + 16 + 8 + 8
    assert C.sizeof(N.Init) == 40
    assert C.sizeof(N.Info) == 15 * 8 + 4 * 8
    assert C.sizeof(N.WindowGrad) == 3 * 8 + 2 * 8


def test_adjoint_entry_points_reject_null_context(lib):
    g = N.WindowGrad()
    assert lib.lbm_adjoint_window(None, 10, 5, C.byref(g)) == N.LBM_EINVAL
    assert lib.lbm_adjoint_step(None, None, None, None, 0.0, None, None, None, None, None) == N.LBM_EINVAL


def _create(lib, dom, cyl, prm):
    h = C.c_void_p()
    st = lib.lbm_create(C.byref(dom), C.byref(cyl), C.byref(prm), None, None, None, C.byref(h))
    return st, h


def _good():
    dom = N.Domain(128, 64, 0, 0)
    cyl = N.Cylinder(32.0, 32.0, 16.0, 0.05, 0.0)
    prm = N.Params(a=2 / 49, b=2 / 21, R=1.0, acentric=0.344, G=-1.0, sigma=0.38, Tr_sat=0.86, Re=30.0,
                   u_in=0.05, nu_l=0.0, nu_ratio=1.0, Pr_l=0.862, Pr_v=1.5, c_v=11.0, g=-1.0, outlet_U=-1.0,
                   warmup_steps=0, energy=1, storage=N.LBM_STORE_F32, compute_f64=0, psi_mode=0, seed=0,
                   noise_amp=1e-4)
    return dom, cyl, prm


@pytest.mark.parametrize("what", ["small", "storage", "G", "Tr", "cyl_inlet", "cyl_wide", "nu", "psi_mode",
                                  "walls_bits", "wall_periodic", "collision", "reserved"])
def test_invalid_parameters_are_rejected_on_the_host(lib, what):
    dom, cyl, prm = _good()
    if what == "small":
        dom.nx = 4
    elif what == "storage":
        prm.compute_f64 = 1
    elif what == "G":
        prm.G = 0.5
    elif what == "Tr":
        prm.Tr_sat = 1.2
    elif what == "cyl_inlet":
        cyl.xc = 8.0
    elif what == "cyl_wide":
        cyl.D = 62.0
    elif what == "psi_mode":
        prm.psi_mode = 3
    elif what == "walls_bits":
        dom.walls = 4
    elif what == "wall_periodic":
        dom.walls, dom.periodic_x = 1, 1  # a wall at x = 0 replaces the inlet of a non-periodic domain
    elif what == "collision":
        prm.collision = 2
    elif what == "reserved":
        prm.reserved = 1
    elif what == "nu":
        prm.Re = 0.0  # nu_l = 0 and no Reynolds number: no valid relaxation rate
    st, h = _create(lib, dom, cyl, prm)
    assert st == N.LBM_EINVAL
    assert not h.value
    assert lib.lbm_last_error(None)


def test_null_handles_are_rejected(lib):
    assert lib.lbm_step(None, 1) == N.LBM_EINVAL
    assert lib.lbm_sync(None) == N.LBM_EINVAL
    assert lib.lbm_inject_fault(None, N.LBM_FAULT_STARVE_COLLIDE) == N.LBM_EINVAL
    assert lib.lbm_stage_state_native(None, None, None, None, -1) == N.LBM_EINVAL
    assert lib.lbm_take_staged(None) == N.LBM_EINVAL
    lib.lbm_destroy(None)


@pytest.mark.parametrize("what", ["collision", "psi_mode", "storage"])
def test_batch_takes_the_cm_collision_and_default_precision_only(lib, what):
    # checked on the host before any domain is created
    dom, cyl, prm = _good()
    if what == "collision":
        prm.collision = N.LBM_COLL_BGK
    elif what == "psi_mode":
        prm.psi_mode = 1
    else:
        prm.storage = N.LBM_STORE_F16S
    h = C.c_void_p()
    st = lib.lbm_batch_create(1, C.byref(dom), C.byref(cyl), C.byref(prm), None, None, C.byref(h))
    assert st == N.LBM_EINVAL
    assert not h.value
