"""The allocation-free wall heat flux (lbm_wall_heat_flux_noalloc) against the context's own.

Callers that cannot allocate device memory (a fixed pool from an outer framework, or a hook
where allocating would synchronise the device) use this entry point: it takes the fields
from the caller and keeps its working sums in a fixed array inside the library.  It must
reproduce what lbm_wall_heat_flux reports for the same fields.  This file is collected
last so that a run stopping at the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_02018_gb300 import _native as N
    from paper_1912_02018_gb300 import build

    build()
    torch.cuda.set_device(0)
    return N


def _structs(N, case):
    dom = N.Domain(case.nx, case.ny, case.periodic_x, 0)
    cyl = N.Cylinder(case.xc, case.yc, case.D, case.superheat_Tc, case.rho_s)
    prm = N.Params(a=case.a, b=case.b, R=case.R, acentric=case.acentric, G=case.G, sigma=case.sigma,
                   Tr_sat=case.Tr_sat, Re=case.Re, u_in=case.u_in, nu_l=case.nu_l, nu_ratio=case.nu_ratio,
                   Pr_l=case.Pr_l, Pr_v=case.Pr_v, c_v=case.c_v, g=case.g, outlet_U=case.U_out,
                   warmup_steps=case.warmup, energy=case.energy, storage=N.LBM_STORE_F64, compute_f64=1,
                   psi_mode=0, seed=case.seed, noise_amp=case.noise_amp)
    return dom, cyl, prm


@pytest.mark.parametrize("case", [si.SMALL, si.SMALL.replace(nx=96, ny=48, D=12.0, xc=24.3, yc=23.6, nu_ratio=2.0),
                                  si.cylinder_case(1024, 512, 64.0, Re=300.0, superheat_Tc=0.1),
                                  si.SMALL.replace(periodic_x=1)],
                         ids=["128x64_D16", "96x48_D12_offgrid", "1024x512_D64_2048_tiles", "128x64_periodic_x"])
def test_noalloc_heat_flux_matches_context_sample_on_two_calls(lib, case):
    import torch

    from paper_1912_02018_gb300 import Sim

    N = lib
    sim = Sim.from_case(case, f64=True).step(5)
    dom, cyl, prm = _structs(N, case)
    q_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        # the context samples q from the temperature entering a step and that step's density
        T_in, _ = sim.fields_device(("T",))
        sim.step(1)
        rho, _ = sim.fields_device(("rho",))
        q_ref = sim.heat_flux()["q_now"]
        q_dev.fill_(np.nan)
        st = N.lib().lbm_wall_heat_flux_noalloc(C.byref(dom), C.byref(cyl), C.byref(prm), T_in.data_ptr(),
                                                rho.data_ptr(), q_dev.data_ptr(), C.c_void_p(stream))
        assert st == N.LBM_OK, f"call {call}: status {st}"
        torch.cuda.synchronize()
        q = float(q_dev.item())
        assert abs(q - q_ref) <= 1e-12 * abs(q_ref), f"call {call}: {q} vs {q_ref}"
        sim.step(3)


def test_noalloc_rejects_lattices_beyond_its_scratch(lib):
    import torch

    N = lib
    case = si.cylinder_case(4096, 2080, 64.0)  # 128 x 260 tiles of 32 x 8 > 32,768
    dom, cyl, prm = _structs(N, case)
    buf = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = N.lib().lbm_wall_heat_flux_noalloc(C.byref(dom), C.byref(cyl), C.byref(prm), buf.data_ptr(),
                                            buf.data_ptr(), buf.data_ptr(), None)
    assert st == N.LBM_EINVAL
