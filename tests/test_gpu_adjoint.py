"""The CUDA adjoint against the FP64 gradient oracle and against central differences.

One reverse step (lbm_adjoint_step) must equal the vector-Jacobian product that reverse-mode
autograd of the oracle's step gives for the same seeds; the checkpointed window
(lbm_adjoint_window) must give the oracle's gradient of the time-averaged wall heat flux
(Sec. IV.B), and agree with central differences of the CUDA forward within 1e-4.
"""
import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu


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


def _fixed(case):
    from paper_1912_02018_gb300.adjoint import fixed_transport

    return case.replace(**fixed_transport(case, f64=True))


SUB = si.cylinder_case(64, 32, 8.0, Re=300.0, superheat_Tc=0.05,
                       wall_dT=tuple(0.01 * si.uniform_pm1(3, 200)), name="64x32_D8_Re300")
SMALL = si.Case(nx=48, ny=24, D=8.0, xc=12.0, yc=12.0, Re=300.0, superheat_Tc=0.05,
                wall_dT=tuple(0.01 * si.uniform_pm1(7, 16)), name="48x24_D8")


def _spun_up(case, steps, f64=True):
    from paper_1912_02018_gb300 import Sim

    s = Sim.from_case(case, f64=f64).step(steps)
    return s.get_state()


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


@pytest.fixture(scope="module")
def small_state():
    case = _fixed(SMALL)
    return case, _spun_up(case, 60)


@pytest.mark.parametrize("seeds", ["q", "T", "f", "side", "all"])
def test_one_reverse_step_matches_oracle_vjp(small_state, seeds):
    import torch

    from oracle.gradient import GradientOracle
    from paper_1912_02018_gb300 import Sim

    case, (f, T, side, n) = small_state
    go = GradientOracle(case)
    solid = go.solid_np.reshape(case.ny, case.nx)
    rs = np.random.default_rng(5)
    fb = rs.standard_normal((9, case.ny, case.nx)) * (~solid) if seeds in ("f", "all") else np.zeros((9, case.ny, case.nx))
    Tb = rs.standard_normal((case.ny, case.nx)) if seeds in ("T", "all") else np.zeros((case.ny, case.nx))
    sb = rs.standard_normal((3, case.ny)) if seeds in ("side", "all") else np.zeros((3, case.ny))
    qw = 0.7 if seeds in ("q", "all") else 0.0
    # the oracle's vector-Jacobian product by autograd
    fs = torch.tensor(f.reshape(9, -1), dtype=torch.float64, requires_grad=True)
    Tt = torch.tensor(T.reshape(-1), dtype=torch.float64, requires_grad=True)
    st = torch.tensor(side, dtype=torch.float64, requires_grad=True)
    ui = torch.tensor(case.u_in, dtype=torch.float64, requires_grad=True)
    Tw = go.wall_T(torch.tensor(case.superheat_Tc, dtype=torch.float64),
                   torch.tensor(case.wall_dT, dtype=torch.float64)).detach().requires_grad_(True)
    f1, T1, s1, q = go.step(fs, Tt, st, ui, Tw)
    L = (f1 * torch.tensor(fb.reshape(9, -1))).sum() + (T1 * torch.tensor(Tb.reshape(-1))).sum() + \
        (s1 * torch.tensor(sb)).sum() + qw * q
    L.backward()
    sim = Sim.from_case(case, f64=True)
    sim.set_state(f, T, side, n)
    got = sim.adjoint_step(fb, Tb, sb, qw)
    ref_f = fs.grad.numpy().reshape(9, case.ny, case.nx)
    ref_T = Tt.grad.numpy().reshape(case.ny, case.nx)
    ref_Tw = np.where(solid, Tw.grad.numpy().reshape(case.ny, case.nx), 0.0)
    errs = {"f": _rel(got["f"], ref_f), "T": _rel(got["T"], ref_T), "side": _rel(got["side"], st.grad.numpy()),
            "Tw": _rel(got["Tw"], ref_Tw),
            "u_in": abs(got["u_in"] - float(ui.grad)) / max(abs(float(ui.grad)), 1e-300)}
    scale = {"f": np.abs(ref_f).max(), "T": np.abs(ref_T).max(), "Tw": np.abs(ref_Tw).max(),
             "u_in": abs(float(ui.grad))}
    bad = {k: v for k, v in errs.items() if not v < 1e-10 and scale.get(k, 1.0) > 0}
    assert not bad, (errs, scale)


def test_window_fp64_matches_oracle_gradient(small_state):
    from oracle.gradient import GradientOracle
    from paper_1912_02018_gb300 import Sim

    case, (f, T, side, n) = small_state
    ref = GradientOracle(case).gradient(f, T, side, 24)
    sim = Sim.from_case(case, f64=True)
    sim.set_state(f, T, side, n)
    got = sim.adjoint_window(24, ckpt_every=10)  # segments of 10, 10 and 4 steps
    assert got["J"] == pytest.approx(ref["J"], rel=1e-12)
    assert got["superheat"] == pytest.approx(ref["superheat"], rel=1e-9)
    assert got["u_in"] == pytest.approx(ref["u_in"], rel=1e-9)
    assert _rel(got["wall_dT"], ref["wall_dT"]) < 1e-9
    assert sim.info()["steps"] == n + 24


def _window_J(case, state, n, f64=True):
    from paper_1912_02018_gb300 import Sim

    f, T, side, steps = state
    s = Sim.from_case(case, f64=f64)
    solid = s.fields(("solid",))["solid"] == 1
    s.set_state(f, np.where(solid, s.fields(("T",))["T"], T), side, steps)
    s.reset_heat_flux()
    s.step(n)
    return s.heat_flux()["q_mean"]


@pytest.fixture(scope="module")
def sub_case():
    case = _fixed(SUB)
    return case, _spun_up(case, 200)


def test_window_on_64x32_matches_oracle_and_central_differences(sub_case):
    from oracle.gradient import GradientOracle
    from paper_1912_02018_gb300 import Sim

    case, state = sub_case
    f, T, side, n = state
    nw = 100
    sim = Sim.from_case(case, f64=True)
    sim.set_state(f, T, side, n)
    got = sim.adjoint_window(nw, ckpt_every=20)
    ref = GradientOracle(case).gradient(f, T, side, nw)
    assert got["superheat"] == pytest.approx(ref["superheat"], rel=1e-9)
    assert got["u_in"] == pytest.approx(ref["u_in"], rel=1e-9)
    assert _rel(got["wall_dT"], ref["wall_dT"]) < 1e-9
    h = 1e-4
    fd = (_window_J(case.replace(superheat_Tc=case.superheat_Tc + h), state, nw) -
          _window_J(case.replace(superheat_Tc=case.superheat_Tc - h), state, nw)) / (2 * h)
    assert got["superheat"] == pytest.approx(fd, rel=1e-4)
    fd = (_window_J(case.replace(u_in=case.u_in + h), state, nw) -
          _window_J(case.replace(u_in=case.u_in - h), state, nw)) / (2 * h)
    assert got["u_in"] == pytest.approx(fd, rel=1e-4)
    kn = np.array(case.wall_dT)
    for k in np.argsort(-np.abs(got["wall_dT"]))[:3]:
        p, m = kn.copy(), kn.copy()
        p[k] += h
        m[k] -= h
        fd = (_window_J(case.replace(wall_dT=tuple(p)), state, nw) -
              _window_J(case.replace(wall_dT=tuple(m)), state, nw)) / (2 * h)
        assert got["wall_dT"][k] == pytest.approx(fd, rel=1e-4), k


def test_fp32_adjoint_against_fp64_adjoint(sub_case):
    from paper_1912_02018_gb300 import Sim

    case, (f, T, side, n) = sub_case
    out = {}
    for f64 in (True, False):
        sim = Sim.from_case(case, f64=f64)
        sim.set_state(f, T, side, n)
        out[f64] = sim.adjoint_window(100, ckpt_every=20)
    a, b = out[False], out[True]
    errs = {k: abs(a[k] - b[k]) / abs(b[k]) for k in ("J", "superheat", "u_in")}
    errs["wall_dT"] = _rel(a["wall_dT"], b["wall_dT"])
    assert max(errs.values()) < 1e-3, errs


@pytest.mark.parametrize("f64", [True, False])
def test_window_gradient_is_the_same_with_plain_launches(monkeypatch, f64):
    # the window's forward pass steps with programmatic dependent launches (LBM_PDL=0 at creation
    # launches plainly), its checkpoints then seed the recompute: the same gradient bits, on a
    # lattice of many blocks per pass
    from paper_1912_02018_gb300 import Sim

    case = _fixed(si.cylinder_case(256, 128, 16.0, Re=300.0, superheat_Tc=0.05,
                                   wall_dT=tuple(0.01 * si.uniform_pm1(5, 200)), name="256x128_D16"))
    state = _spun_up(case, 200, f64=f64)
    out = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("LBM_PDL", flag)
        sim = Sim.from_case(case, f64=f64)
        sim.set_state(*state)
        out[flag] = sim.adjoint_window(60, ckpt_every=20)
    for k in ("J", "superheat", "u_in"):
        assert out["1"][k] == out["0"][k], k
    assert np.array_equal(np.asarray(out["1"]["wall_dT"]), np.asarray(out["0"]["wall_dT"]))


def test_torch_autograd_function_gives_the_window_gradient(sub_case):
    import torch

    from paper_1912_02018_gb300.adjoint import heat_flux_window
    from paper_1912_02018_gb300 import Sim

    case, state = sub_case
    sh = torch.tensor(case.superheat_Tc, dtype=torch.float64, requires_grad=True)
    ui = torch.tensor(case.u_in, dtype=torch.float64, requires_grad=True)
    kn = torch.tensor(case.wall_dT, dtype=torch.float64, requires_grad=True)
    J = heat_flux_window(case, state, 40, ckpt_every=20, superheat=sh, u_in=ui, wall_dT=kn, f64=True,
                         fixed={})
    (3.0 * J).backward()
    sim = Sim.from_case(case, f64=True)
    sim.set_state(*state)
    g = sim.adjoint_window(40, ckpt_every=20)
    assert float(J.detach()) == pytest.approx(g["J"], rel=1e-14)
    assert float(sh.grad) == pytest.approx(3.0 * g["superheat"], rel=1e-14)
    assert float(ui.grad) == pytest.approx(3.0 * g["u_in"], rel=1e-14)
    assert np.allclose(kn.grad.numpy(), 3.0 * g["wall_dT"], rtol=1e-14, atol=0)


def test_full_size_window_512x256_against_central_differences():
    # the adjoint workload: 512 x 256, D = 32, Re = 300, 200 knots, a 500-step window checkpointed
    # every 50 steps from the state after a 2000-step spin-up; FP64 adjoint against central
    # differences (h = 1e-4) of the FP64 forward, and the FP32 adjoint against the FP64 one
    from paper_1912_02018_gb300 import Sim

    case = _fixed(si.ADJOINT.replace(wall_dT=tuple(0.01 * si.uniform_pm1(9, 200))))
    state = _spun_up(case, 2000)
    nw = 500
    out = {}
    for f64 in (True, False):
        sim = Sim.from_case(case, f64=f64)
        sim.set_state(*state)
        out[f64] = sim.adjoint_window(nw, ckpt_every=50)
        sim.close()
    got = out[True]
    h = 1e-4
    checks = {"superheat": ("superheat_Tc", case.superheat_Tc), "u_in": ("u_in", case.u_in)}
    for key, (field, v) in checks.items():
        fd = (_window_J(case.replace(**{field: v + h}), state, nw) -
              _window_J(case.replace(**{field: v - h}), state, nw)) / (2 * h)
        assert got[key] == pytest.approx(fd, rel=1e-4), key
    kn = np.array(case.wall_dT)
    for k in np.argsort(-np.abs(got["wall_dT"]))[:3]:
        p, m = kn.copy(), kn.copy()
        p[k] += h
        m[k] -= h
        fd = (_window_J(case.replace(wall_dT=tuple(p)), state, nw) -
              _window_J(case.replace(wall_dT=tuple(m)), state, nw)) / (2 * h)
        assert got["wall_dT"][k] == pytest.approx(fd, rel=1e-4), k
    # the FP32 build: its forward J is 1.2e-4 from the FP64 one (wall temperature rounding over the
    # window), and its gradients (measured 1.3e-4 to 2.2e-4 from the FP64 adjoint) inherit that
    a = out[False]
    errs = {k: abs(a[k] - got[k]) / abs(got[k]) for k in ("J", "superheat", "u_in")}
    errs["wall_dT"] = _rel(a["wall_dT"], got["wall_dT"])
    assert max(errs.values()) < 5e-4, errs
