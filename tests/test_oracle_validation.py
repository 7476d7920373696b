"""Pins of the oracle's flat walls and body force against the Poiseuille closed form (Sec. III.C).

Halfway bounce-back on flat walls (link fraction 1/2) with the uniform force F_x = 8 nu U0 / L^2
must converge to u_x = 4 U0 y' (L - y') / L^2 at second order in the channel width (the paper
reports 2.04), with no transverse velocity and uniform density.
"""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import Oracle


def _steady(L):
    case = si.poiseuille_case(L)
    rho = np.ones((case.ny, case.nx))
    zero = np.zeros_like(rho)
    o = Oracle(case, rho=rho, ux=zero, uy=zero)
    o.step(int(8 * L * L / (1.0 / 6.0)))  # eight diffusion times L^2 / nu
    return case, o


def test_poiseuille_converges_at_second_order():
    errs = []
    for L in (8, 16, 32):
        case, o = _steady(L)
        u = o.field("ux")[1:case.ny - 1].mean(axis=1)
        ref = si.poiseuille_profile(L)
        errs.append(np.linalg.norm(u - ref) / np.linalg.norm(ref))
        assert np.abs(o.field("uy")).max() < 1e-13
        assert np.ptp(o.field("ux")[1:case.ny - 1], axis=1).max() < 1e-14  # uniform along x
        assert np.abs(o.field("rho")[1:case.ny - 1] - 1.0).max() < 1e-9
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((orders > 1.95) & (orders < 2.05)), (errs, orders)
    assert errs[1] < 2.5e-3, errs


def test_flat_walls_give_halfway_links_and_wall_normals():
    case = si.Case(nx=12, ny=9, D=0.0, xc=0.0, yc=0.0, walls=3, G=0.0, energy=0, u_in=0.0, nu_l=1.0 / 6.0,
                   g=0.0, noise_amp=0.0)
    o = Oracle(case)
    solid = o.field("solid")
    assert np.all(solid[:, 0] == 1) and np.all(solid[0] == 1) and np.all(solid[-1] == 1)
    assert solid[1:-1, 1:].sum() == 0
    q = o.link_fractions()
    assert set(np.unique(q[q >= 0])) == {0.5}
    nodes, nx_, ny_ = o.boundary()
    xs, ys = nodes % case.nx, nodes // case.nx
    # rows next to the y-walls face +y / -y, the column next to the x-wall faces +x
    assert np.all(ny_[ys == 1] == 1.0) and np.all(ny_[ys == case.ny - 2] == -1.0)
    mid = (xs == 1) & (ys > 1) & (ys < case.ny - 2)
    assert mid.any() and np.all(nx_[mid] == 1.0) and np.all(ny_[mid] == 0.0)
