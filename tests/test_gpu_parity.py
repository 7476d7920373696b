"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars (from the method's precision targets): the FP64 build within 1e-12 relative on
every field; FP32 within 1e-5 relative on rho and T after 200 steps.  The relative
error of a field is max |gpu - oracle| / max |oracle| over fluid nodes.
"""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import Oracle

pytestmark = pytest.mark.gpu

FIELDS = ("rho", "ux", "uy", "T", "psi")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    from oracle import build as ob
    from paper_1912_02018_gb300 import build

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build()
    ob.build()
    torch.cuda.set_device(0)


def Sim():
    from paper_1912_02018_gb300 import Sim as S

    return S


def rel(a, b, fluid):
    a, b = a[fluid], b[fluid]
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def pair(case, steps, f64, init=None):
    init = dict(init or {})
    if "drho" not in init and "rho" not in init:
        init["drho"] = case.drho()
    sim = Sim().from_case(case, f64=f64, init=init)
    sim.step(steps)
    ref = Oracle(case, **init).step(steps)
    return sim, ref


def assert_fields(sim, ref, tol, names=FIELDS):
    """Relative error per field; the velocity components are scaled by the largest velocity
    magnitude (the velocity is one vector field), every other field by its own maximum."""
    got = sim.fields()
    fluid = ref.field("solid") == 0
    speed = np.hypot(ref.field("ux"), ref.field("uy"))[fluid].max()
    errs = {}
    for k in names:
        if k in ("ux", "uy"):
            errs[k] = np.abs(got[k] - ref.field(k))[fluid].max() / speed
        else:
            errs[k] = rel(got[k], ref.field(k), fluid)
    tols = tol if isinstance(tol, dict) else {k: tol for k in names}
    bad = {k: v for k, v in errs.items() if not v <= tols[k]}
    assert not bad, f"relative errors {errs}"
    return errs


def test_fp64_parity_1000_steps_plain_method_case():
    case = si.SMALL  # 128x64, D=16 at (32,32), superheat 0.05 Tc, Re=30
    sim, ref = pair(case, 1000, True)
    assert_fields(sim, ref, 1e-12)
    f, T, side, n = sim.get_state()
    fluid = ref.field("solid") == 0
    fr = ref.populations()
    assert n == 1000
    assert np.abs(f[:, fluid] - fr[:, fluid]).max() / np.abs(fr).max() < 1e-12
    assert np.abs(side - ref.side()).max() / np.abs(ref.side()).max() < 1e-12
    hg, hr = sim.heat_flux(), ref.heat_flux()
    assert hg["count"] == hr["count"] == 1000
    assert abs(hg["q_mean"] - hr["q_mean"]) <= 1e-12 * abs(hr["q_mean"])
    assert abs(hg["q_now"] - hr["q_now"]) <= 1e-12 * abs(hr["q_now"])
    assert abs(hg["nu_mean"] - hr["nu_mean"]) <= 1e-11 * abs(hr["nu_mean"])


def test_fp32_parity_200_steps_plain_method_case():
    case = si.SMALL
    sim, ref = pair(case, 200, False)
    errs = assert_fields(sim, ref, {"rho": 1e-5, "T": 1e-5}, names=("rho", "T"))
    fluid = ref.field("solid") == 0
    got = sim.fields()
    for k in ("ux", "uy", "psi"):
        errs[k] = rel(got[k], ref.field(k), fluid)
    assert errs["ux"] < 1e-3 and errs["uy"] < 1e-3 and errs["psi"] < 1e-5, errs
    hg, hr = sim.heat_flux(), ref.heat_flux()
    assert abs(hg["q_mean"] - hr["q_mean"]) <= 1e-3 * abs(hr["q_mean"])


def test_force_planes_are_those_of_the_last_collision():
    # lbm_fields' FX, FY: F_m of Eq. (interForce) from the psi the collision used, plus gravity
    # (Sec. IV.A); the FP64 build against the oracle's force on the same psi and rho fields
    from oracle import stepper

    case = si.SMALL
    sim = Sim().from_case(case, f64=True, init={"drho": case.drho()})
    z = sim.fields(("Fx", "Fy"))
    assert not z["Fx"].any() and not z["Fy"].any()  # no collision yet
    sim.step(30)
    got = sim.fields(("rho", "psi", "solid", "Fx", "Fy"))
    fx, fy = stepper.interaction_force(case, got["psi"])
    _, d = stepper.derive(case)
    fx = fx - (got["rho"] - d.rho_l) * d.g
    fluid = got["solid"] == 0
    scale = np.hypot(fx, fy)[fluid].max()
    assert scale > 0
    assert np.abs(got["Fx"] - fx)[fluid].max() <= 1e-12 * scale
    assert np.abs(got["Fy"] - fy)[fluid].max() <= 1e-12 * scale
    assert not got["Fx"][~fluid].any() and not got["Fy"][~fluid].any()
    # a warm-up step applies no force
    warm = Sim().from_case(case.replace(warmup=5), f64=False).step(3)
    w = warm.fields(("Fx", "Fy"))
    assert not w["Fx"].any() and not w["Fy"].any()


def test_fp32_parity_200_steps_on_mostly_staged_tiles():
    # 512 x 256, D = 32, Re = 300: 82% of the collision tiles and 77% of the energy tiles are
    # staged by TMA, so the staged interior code paths carry the 200-step FP32 bar
    case = si.ADJOINT
    sim, ref = pair(case, 200, False)
    assert_fields(sim, ref, {"rho": 1e-5, "T": 1e-5}, names=("rho", "T"))
    fluid = ref.field("solid") == 0
    got = sim.fields(("psi",))
    assert rel(got["psi"], ref.field("psi"), fluid) < 1e-5


@pytest.mark.parametrize("storage,tol", [("f64", 1e-5), ("f16s", 2e-4)])
def test_fp32_compute_with_other_population_storage(storage, tol):
    # FP32 arithmetic with populations stored as FP64 or as shifted FP16 (h = f - w rho_l)
    case = si.SMALL
    init = {"drho": case.drho()}
    sim = Sim().from_case(case, f64=False, storage=storage, init=init).step(200)
    ref = Oracle(case, **init).step(200)
    fluid = ref.field("solid") == 0
    got = sim.fields(("rho", "T"))
    errs = {k: rel(got[k], ref.field(k), fluid) for k in ("rho", "T")}
    assert max(errs.values()) < tol, errs


def test_shifted_fp16_state_round_trip():
    case = si.SMALL
    a = Sim().from_case(case, storage="f16s").step(10)
    f, T, side, n = a.get_state()
    b = Sim().from_case(case, storage="f16s")
    b.set_state(f, T, side, n)
    f2, T2, side2, n2 = b.get_state()
    assert np.array_equal(f, f2) and np.array_equal(T, T2) and n2 == n


def _two_phase_periodic():
    c = si.Case(nx=40, ny=24, D=0.0, xc=0.0, yc=0.0, periodic_x=1, g=3e-5, u_in=0.0, nu_l=0.1,
                superheat_Tc=0.0, noise_amp=0.0, name="periodic_two_phase")
    rho = 3.4 + 0.6 * si.uniform_pm1(11, 40 * 24).reshape(24, 40)
    return c, {"rho": rho, "ux": np.zeros((24, 40)), "uy": np.zeros((24, 40))}


EDGE_CASES = {
    "ragged_37x13_no_cylinder": (si.Case(nx=37, ny=13, D=0.0, xc=0.0, yc=0.0, Re=30.0, nu_l=0.04), None),
    "minimal_5x5": (si.Case(nx=5, ny=5, D=0.0, xc=0.0, yc=0.0, nu_l=0.05), None),
    "off_grid_cylinder_70x27": (si.Case(nx=70, ny=27, D=9.4, xc=20.3, yc=11.7, Re=40.0, superheat_Tc=0.08), None),
    "periodic_two_phase": _two_phase_periodic(),
    "single_phase_G0": (si.SMALL.replace(G=0.0, sigma=0.0), None),
    "warmup_30": (si.SMALL.replace(warmup=30), None),
    "viscosity_ratio_2": (si.SMALL.replace(nu_ratio=2.0, Pr_v=1.0), None),
    "no_energy": (si.SMALL.replace(energy=0), None),
    "wall_profile_7_knots": (si.SMALL.replace(wall_dT=(0.0, 0.03, -0.02, 0.05, 0.01, -0.04, 0.02)), None),
}


@pytest.mark.parametrize("name", sorted(EDGE_CASES))
def test_fp64_parity_edge_cases(name):
    case, init = EDGE_CASES[name]
    sim, ref = pair(case, 60, True, init=init)
    assert_fields(sim, ref, 1e-12)
    hg, hr = sim.heat_flux(), ref.heat_flux()
    assert hg["count"] == hr["count"]
    if hr["count"]:
        assert abs(hg["q_mean"] - hr["q_mean"]) <= 1e-12 * max(abs(hr["q_mean"]), 1e-300)


@pytest.mark.parametrize("name", ["ragged_37x13_no_cylinder", "off_grid_cylinder_70x27", "periodic_two_phase"])
def test_fp32_parity_edge_cases(name):
    case, init = EDGE_CASES[name]
    sim, ref = pair(case, 60, False, init=init)
    assert_fields(sim, ref, {"rho": 1e-5, "T": 1e-5}, names=("rho", "T"))


@pytest.mark.parametrize("case", [si.PAPER_SHAPED.replace(warmup=0), si.PRECISION.replace(warmup=0)],
                         ids=lambda c: c.name)
def test_fp32_full_size_first_steps_match_oracle(case):
    # the benchmark's workloads at full size, two steps from the seeded state, every node
    sim, ref = pair(case, 2, False)
    assert_fields(sim, ref, {"rho": 1e-6, "T": 1e-6, "psi": 1e-6}, names=("rho", "T", "psi"))
    fluid = ref.field("solid") == 0
    got = sim.fields(("ux", "uy"))
    umax = np.abs(ref.field("ux")[fluid]).max()
    for k in ("ux", "uy"):
        assert np.abs(got[k][fluid] - ref.field(k)[fluid]).max() < 1e-5 * umax


def test_fp32_rest_state_stays_exactly_at_rest_at_full_size():
    c = si.Case(nx=1536, ny=768, D=0.0, xc=0.0, yc=0.0, periodic_x=1, g=0.0, u_in=0.0, nu_l=0.02, noise_amp=0.0)
    sim = Sim().from_case(c, f64=False, init={"ux": np.zeros((768, 1536)), "uy": np.zeros((768, 1536))})
    sim.step(20)
    f = sim.fields(("ux", "uy", "T"))
    assert np.all(f["ux"] == 0) and np.all(f["uy"] == 0)
    assert np.ptp(f["T"]) == 0


def test_fp64_mass_conservation_periodic():
    case, init = _two_phase_periodic()
    sim = Sim().from_case(case, f64=True, init=init)
    m0 = init["rho"].sum()
    for _ in range(4):
        sim.step(50)
        assert abs(sim.fields(("rho",))["rho"].sum() - m0) / m0 < 1e-13


def test_psi_from_the_energy_pass_equals_the_psi_pass():
    # a restored state makes the next step run the psi pass; stepping on without a restore takes
    # psi from the previous step's energy pass: both must give the same bits
    case = si.SMALL
    for f64 in (True, False):
        a = Sim().from_case(case, f64=f64).step(7)
        f, T, side, n = a.get_state()
        b = Sim().from_case(case, f64=f64)
        b.set_state(f, T, side, n)
        a.step(1)
        b.step(1)
        fa, fb = a.fields(), b.fields()
        for k in FIELDS:
            assert np.array_equal(fa[k], fb[k]), (f64, k)


@pytest.mark.parametrize("f64,storage,periodic_x", [(False, "f32", 0), (True, "f64", 0), (False, "f32", 1),
                                                    (False, "f16s", 0), (False, "f64", 0)])
def test_tma_staged_and_plain_collision_tiles_agree_bitwise(monkeypatch, f64, storage, periodic_x):
    # interior collision tiles copy their pull window and psi tile into shared memory with TMA;
    # LBM_TMA=0 (read at creation) makes every tile load from global memory: same bits
    case = si.Case(nx=256, ny=96, D=24.0, xc=64.0, yc=48.0, Re=300.0, superheat_Tc=0.1, periodic_x=periodic_x,
                   name="256x96_D24")
    out = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("LBM_TMA", flag)
        s = Sim().from_case(case, f64=f64, storage=storage).step(40)
        out[flag] = (s.fields(), s.get_state()[0], s.heat_flux()["q_mean"])
    for k in FIELDS:
        assert np.array_equal(out["1"][0][k], out["0"][0][k]), k
    assert np.array_equal(out["1"][1], out["0"][1])
    assert out["1"][2] == out["0"][2]


@pytest.mark.parametrize("f64,storage", [(False, "f32"), (True, "f64"), (False, "f16s")])
def test_dependent_launches_give_the_same_bits(monkeypatch, f64, storage):
    # the collision and energy passes are launched as programmatic dependents of the kernel
    # before them (from the second step of a call on, the collision copies its populations while
    # the previous energy pass ends); LBM_PDL=0 (read at creation) launches them plainly: same
    # bits through the warm-up (collisions back to back), the switch-on, one-step calls with reads
    # in between, and a restore
    case = si.Case(nx=1024, ny=384, D=48.0, xc=256.0, yc=192.0, Re=300.0, superheat_Tc=0.1, warmup=25,
                   name="1024x384_D48")
    out = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("LBM_PDL", flag)
        s = Sim().from_case(case, f64=f64, storage=storage).step(60)
        mid = s.fields()
        for _ in range(5):
            s.step(1)
        st = s.get_state_native()
        s.step(30)
        s.set_state_native(*st)
        s.step(20)
        out[flag] = (mid, s.fields(), s.get_state_native()[0], s.heat_flux()["q_mean"])
    for k in FIELDS:
        assert np.array_equal(out["1"][0][k], out["0"][0][k]), k
        assert np.array_equal(out["1"][1][k], out["0"][1][k]), k
    assert np.array_equal(out["1"][2], out["0"][2])
    assert out["1"][3] == out["0"][3]


@pytest.mark.parametrize("f64,storage", [(False, "f32"), (True, "f64"), (False, "f16s")])
def test_staged_restore_matches_the_synchronous_one(f64, storage):
    # lbm_stage_state_native copies a state on the context's copy stream while the context
    # steps; lbm_take_staged swaps it in.  Against lbm_set_state_native: same bits after the
    # restore, with the copy overlapping steps of another state, and repeated takes of the same
    # host arrays (pinned torch tensors); then the step counter and outlet rows kept
    import torch

    case = si.SMALL.replace(warmup=5)
    a = Sim().from_case(case, f64=f64, storage=storage).step(30)
    st = a.get_state_native()
    a.step(7)
    ref = Sim().from_case(case, f64=f64, storage=storage)
    ref.set_state_native(*st)
    ref.step(12)
    want = (ref.fields(), ref.get_state_native())
    f_h, T_h = torch.from_numpy(st[0]).pin_memory(), torch.from_numpy(st[1]).pin_memory()
    for rep in range(3):
        a.stage_state_native(f_h, T_h, st[2], st[3])
        a.step(3)  # the current state steps while the staged one is copied
        a.take_staged().step(12)
        got = (a.fields(), a.get_state_native())
        for k in FIELDS:
            assert np.array_equal(got[0][k], want[0][k]), (rep, k)
        for x, y in zip(got[1], want[1]):
            assert np.array_equal(x, y), rep
    # outlet rows kept (side None) and steps kept (-1): the counter continues from the take
    n0 = a.get_state_native()[3]
    a.stage_state_native(st[0], st[1]).take_staged()
    assert a.get_state_native()[3] == n0
    assert np.array_equal(a.get_state_native()[1], st[1])
    from paper_1912_02018_gb300._native import LbmError
    with pytest.raises(LbmError, match="ESTATE"):
        a.take_staged()


def test_checkpoint_restart_is_bit_exact():
    case = si.SMALL
    drho = case.drho()
    a = Sim().from_case(case, f64=True, init={"drho": drho}).step(30)
    f, T, side, n = a.get_state()
    a.step(20)
    b = Sim().from_case(case, f64=True, init={"drho": drho})
    b.set_state(f, T, side, n)
    b.step(20)
    fa, fb = a.fields(), b.fields()
    for k in FIELDS:
        assert np.array_equal(fa[k], fb[k]), k


@pytest.mark.parametrize("f64,storage", [(True, "f64"), (False, "f32"), (False, "f16s"), (False, "f64")])
def test_native_checkpoint_round_trip_is_bit_exact(f64, storage):
    case = si.SMALL
    a = Sim().from_case(case, f64=f64, storage=storage).step(12)
    f, T, side, n = a.get_state_native()
    a.step(5)
    b = Sim().from_case(case, f64=f64, storage=storage)
    b.set_state_native(f, T, side, n)
    b.step(5)
    assert b.info()["steps"] == n + 5
    fa, fb = a.get_state_native(), b.get_state_native()
    for x, y in zip(fa[:3], fb[:3]):
        assert np.array_equal(x, y)
    # the double form of the same state agrees value for value
    fd, Td, sd, _ = a.get_state()
    assert np.array_equal(fa[1].astype(np.float64), Td)
    if storage != "f16s":
        assert np.array_equal(fa[0].astype(np.float64), fd)


def test_torch_allocator_and_cudamalloc_agree():
    case = si.SMALL
    init = {"drho": case.drho()}
    a = Sim().from_case(case, f64=False, init=init, torch_alloc=True).step(25)
    b = Sim().from_case(case, f64=False, init=init, torch_alloc=False).step(25)
    for k, v in a.fields().items():
        assert np.array_equal(v, b.fields()[k]), k


@pytest.mark.parametrize("psi_mode", [0, 1, 2], ids=["double_float", "ieee_fp64", "fp32"])
def test_fp32_psi_modes_match_oracle(psi_mode):
    case = si.SMALL
    init = {"drho": case.drho()}
    sim = Sim().from_case(case, f64=False, init=init, psi_mode=psi_mode).step(1)
    ref = Oracle(case, **init).step(1)
    fluid = ref.field("solid") == 0
    got = sim.fields(("psi", "rho", "T"))
    # one step: rho differs from the oracle by the FP32 rounding of the pull only, so psi shows
    # the evaluation error itself (FP32 storage: 2^-24 ~ 6e-8 relative per rounding)
    tol = 3e-7 if psi_mode != 2 else 1e-6
    assert rel(got["psi"], ref.field("psi"), fluid) < tol
    assert rel(got["rho"], ref.field("rho"), fluid) < 1e-6


def test_library_default_noise_matches_seeded_input_generator():
    case = si.SMALL.replace(seed=5, noise_amp=3e-4)
    a = Sim().from_case(case, f64=True)  # the library draws SplitMix64(seed) itself
    b = Sim().from_case(case, f64=True, init={"drho": case.drho()})
    assert np.array_equal(a.fields(("rho",))["rho"], b.fields(("rho",))["rho"])


def test_profile_counts_launches():
    case = si.SMALL
    sim = Sim().from_case(case, f64=False)
    sim.profile(True)
    sim.step(10)
    prof = sim.profile_read()
    # psi of every later step comes from the energy pass of the step before
    assert prof["k_rho_psi"][0] == 1 and prof["k_collide"][0] == 10 and prof["k_energy"][0] == 10
    assert all(v[1] >= 0 for v in prof.values())
    info = sim.info()
    assert info["steps"] == 10 and info["kernel_launches"] >= 21
