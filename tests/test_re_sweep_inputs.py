"""Inputs of the Reynolds-number and superheat sweep driver (re_sweep.py), checked on the CPU:
the 4 x 4 grid, the viscosity from Re at the inlet speed, the warm-up of 5 D / u_in steps, the
cylinder at (W/4, H/2), distinct seeds, and the oracle's derived constants for one case."""
import numpy as np

from oracle import stepper
from paper_1912_02018_gb300 import re_sweep


def test_grid_and_warmup():
    cs = re_sweep.cases()
    assert len(cs) == 16
    assert sorted({c.Re for c in cs}) == [30.0, 300.0, 3000.0, 30000.0]
    assert sorted({c.superheat_Tc for c in cs}) == [0.02, 0.05, 0.10, 0.20]
    assert all(c.nx == 1536 and c.ny == 768 and c.D == 96.0 and (c.xc, c.yc) == (384.0, 384.0) for c in cs)
    assert all(c.warmup == 9600 for c in cs)
    assert len({c.seed for c in cs}) == 16


def test_derived_viscosity_and_gravity():
    c = re_sweep.cases()[5]  # Re = 300, superheat 0.05 Tc
    _, d = stepper.derive(c)
    assert np.isclose(d.nu_l, 0.05 * 96.0 / 300.0, rtol=1e-15)
    assert np.isclose(d.g, 0.05 ** 2 / (16.0 * 96.0), rtol=1e-15)
    assert np.isclose(d.T_wall - d.T_sat, 0.05 * d.Tc, rtol=1e-12)
