"""Pins of the FP64 gradient oracle (oracle/gradient.py).

Its forward step must reproduce the C oracle, and its reverse-mode gradient of the
time-averaged wall heat flux (Sec. IV.B) must match central finite differences of the C
oracle's own objective, with nu_l, g and the outlet speed held fixed while u_in moves.
"""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import Oracle, derive
from oracle.gradient import GradientOracle


def _case(**kw):
    base = dict(Re=300.0, superheat_Tc=0.05, wall_dT=tuple(0.01 * si.uniform_pm1(7, 16)))
    base.update(kw)
    return si.Case(nx=48, ny=24, D=8.0, xc=12.0, yc=12.0, **base)


def _fixed(case):
    """The case with nu_l, g and U_out explicit, so that u_in enters only through the inlet."""
    _, d = derive(case)
    return case.replace(nu_l=d.nu_l, g=d.g, U_out=d.U_out)


def _window_J(case, state, n):
    """Objective of the C oracle; the window starts with the solid nodes at this case's T_w."""
    f, T, side = state
    o = Oracle(case, drho=case.drho())
    solid = o.field("solid") == 1
    o.set_state(f, np.where(solid, o.field("T"), T), side, 10 ** 6)
    before = o.heat_flux()["q_sum"]
    o.step(n)
    return (o.heat_flux()["q_sum"] - before) / n


@pytest.fixture(scope="module")
def spun_up():
    case = _fixed(_case())
    o = Oracle(case, drho=case.drho()).step(60)
    return case, (o.populations(), o.field("T"), o.side())


def test_forward_matches_c_oracle(spun_up):
    import torch

    case, (f, T, side) = spun_up
    go = GradientOracle(case)
    n = 15
    with torch.no_grad():
        J, (fs, Tn, sn) = go.objective(f, T, side, n, torch.tensor(case.superheat_Tc, dtype=torch.float64),
                                       torch.tensor(case.u_in, dtype=torch.float64),
                                       torch.tensor(case.wall_dT, dtype=torch.float64))
    o = Oracle(case, drho=case.drho())
    o.set_state(f, T, side, 10 ** 6)
    o.step(n)
    fr = o.populations().reshape(9, -1)
    assert np.abs(fs.numpy() - fr).max() <= 1e-12 * np.abs(fr).max()
    assert np.abs(Tn.numpy() - o.field("T").reshape(-1)).max() <= 1e-12 * np.abs(T).max()
    assert np.abs(sn.numpy() - o.side()).max() <= 1e-12 * np.abs(o.side()).max()
    assert abs(float(J) - o.heat_flux()["q_mean"]) <= 1e-12 * abs(float(J))


def test_gradient_matches_central_differences_of_the_c_oracle(spun_up):
    case, state = spun_up
    n = 12
    g = GradientOracle(case).gradient(*state, n)
    assert g["J"] == pytest.approx(_window_J(case, state, n), rel=1e-12)
    h = 1e-6

    def fd(**kw_pm):
        (k, v), = kw_pm.items()
        plus = _window_J(case.replace(**{k: v(+h)}), state, n)
        minus = _window_J(case.replace(**{k: v(-h)}), state, n)
        return (plus - minus) / (2 * h)

    d_sh = fd(superheat_Tc=lambda e: case.superheat_Tc + e)
    d_u = fd(u_in=lambda e: case.u_in + e)
    assert g["superheat"] == pytest.approx(d_sh, rel=1e-6)
    assert g["u_in"] == pytest.approx(d_u, rel=1e-6)
    kn = np.array(case.wall_dT)
    for k in np.argsort(-np.abs(g["wall_dT"]))[:3]:
        def knot(e, k=k):
            v = kn.copy()
            v[k] += e
            return tuple(v)

        assert g["wall_dT"][k] == pytest.approx(fd(wall_dT=knot), rel=1e-6), k
    # the knot weights of every solid node sum to one
    assert g["wall_dT"].sum() == pytest.approx(g["superheat"], rel=1e-12)


def test_knots_that_reach_no_fluid_stencil_have_zero_gradient(spun_up):
    # with 64 knots on a D = 8 cylinder some knot intervals hold only nodes deeper than the
    # radius-2 stencils reach (or none at all)
    case = _fixed(_case(wall_dT=(0.0,) * 64))
    o = Oracle(case, drho=case.drho()).step(30)
    g = GradientOracle(case).gradient(o.populations(), o.field("T"), o.side(), 4)
    zero = g["wall_dT"] == 0.0
    assert zero.any() and (~zero).any()
