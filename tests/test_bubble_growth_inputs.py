"""Inputs of the bubble-growth driver (App. D): the superheated liquid is started at the density where
the Peng-Robinson pressure at T_sat + dT equals p_sat(T_sat), which keeps the bubble; started at
rho_l(T_sat) instead, the liquid is over-pressured and the bubble collapses (both on the oracle)."""
import math

import numpy as np

import synthetic_inputs as si
from oracle import Oracle, stepper


def _setup(N):
    from paper_1912_02018_gb300 import bubble_growth as bg

    case = bg.paper_case(N)
    c = si.Case(**{k: getattr(case, k) for k in ("nx", "ny", "D", "xc", "yc", "periodic_x", "a", "b", "R", "acentric",
                                                  "G", "sigma", "Tr_sat", "superheat_Tc", "u_in", "nu_l", "nu_ratio",
                                                  "Pr_l", "Pr_v", "c_v", "g", "U_out", "warmup", "energy",
                                                  "noise_amp")})
    _, d = stepper.derive(c)
    info = {"Tc": d.Tc, "T_sat": d.T_sat, "T_wall": d.T_wall, "rho_l": d.rho_l, "rho_v": d.rho_v,
            "p_sat": d.eos.p(d.rho_l, d.T_sat)}
    return bg, case, c, d, info


def test_superheated_liquid_sits_at_the_saturation_pressure():
    bg, case, c, d, info = _setup(64)
    rl = bg.superheated_liquid_density(case, info)
    assert abs(d.eos.p(rl, d.T_wall) - info["p_sat"]) < 1e-13
    assert d.eos.dp_drho(rl, d.T_wall) > 0 and d.eos.spinodals(d.T_wall)[1] < rl < d.rho_l


def test_initial_fields_and_radius():
    bg, case, c, d, info = _setup(96)
    rho, T, rl = bg.initial_fields(case, info, R0=15.0)
    assert rho.shape == (96, 96)
    assert abs(bg.radius(rho, 0.5 * (d.rho_l + d.rho_v)) - 15.0) < 0.5
    # the tanh profile leaves a 6e-6 share of the liquid value at the centre (2 R0 / width = 6)
    assert abs(rho[0, 0] - rl) < 1e-9 and abs(rho[48, 48] - d.rho_v) < 1e-5 * rl
    assert abs(T[0, 0] - d.T_wall) < 1e-12 and abs(T[48, 48] - d.T_sat) < 1e-5 * (d.T_wall - d.T_sat)


def test_bubble_survives_only_with_the_saturated_liquid_start():
    bg, case, c, d, info = _setup(96)
    mid = 0.5 * (d.rho_l + d.rho_v)
    rho, T, rl = bg.initial_fields(case, info, R0=15.0)
    z = np.zeros_like(rho)
    kept = Oracle(c, rho=rho, T=T, ux=z, uy=z).step(600)
    assert bg.radius(kept.field("rho"), mid) > 13.0
    naive = np.where(rho > mid, d.rho_l, rho)  # the liquid at rho_l(T_sat) instead
    lost = Oracle(c, rho=naive, T=T, ux=z, uy=z).step(600)
    assert bg.radius(lost.field("rho"), mid) < 5.0
