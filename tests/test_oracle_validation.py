"""Pins of the oracle's flat walls, body force and phase change against closed forms.

Poiseuille (Sec. III.C): halfway bounce-back on flat walls (link fraction 1/2) with the uniform
force F_x = 8 nu U0 / L^2 must converge to u_x = 4 U0 y' (L - y') / L^2 at second order in the
channel width (the paper reports 2.04), with no transverse velocity and uniform density.
Stefan (Sec. III.E): a vapour film on a heated wall grows as Welch's 2 beta sqrt(alpha_v t).
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


def _welch_beta(St):
    from scipy import optimize, special

    return optimize.brentq(lambda b: b * np.exp(b * b) * special.erf(b) - St / np.sqrt(np.pi), 1e-9, 5.0,
                           xtol=1e-14)


@pytest.mark.slow
@pytest.mark.parametrize("Tr,dT", [(0.86, 0.010), (0.86, 0.023), (0.90, 0.010)])
def test_stefan_film_grows_as_welch(Tr, dT):
    # Sec. III.E with the readings of the workloads: G = -2 (sigma = 0.38 at Maxwell coexistence),
    # alpha_v = 0.1, a vapour-wetting wall (rho_s = rho_v), a liquid diffusivity a tenth of the
    # vapour's (the paper states only alpha_v), a 15-node initial film (5 nodes are about one
    # interface width and do not survive), outlet speed 0.2.  The film thickness y_i grows as
    # 2 beta sqrt(alpha_v t); the paper's three cases land within 15% of Welch's beta.
    from oracle.thermo import PR

    eos = PR(3.0 / 49.0, 2.0 / 21.0, 1.0, 0.344)
    Ts = Tr * eos.Tc
    rv, rl, _ = eos.maxwell(Ts)
    alpha_v = 0.1
    c = si.Case(nx=101, ny=5, D=0.0, xc=0.0, yc=0.0, walls=1, a=3.0 / 49.0, G=-2.0, sigma=0.38, Tr_sat=Tr,
                superheat_Tc=dT / eos.Tc, u_in=0.0, nu_l=1.5 * alpha_v, nu_ratio=1.0, Pr_v=1.5, Pr_l=15.0, U_out=0.2,
                rho_s=rv, g=0.0, noise_amp=0.0, name="stefan")
    x = np.arange(c.nx, dtype=float)
    rho = np.tile(rv + (rl - rv) * 0.5 * (1.0 + np.tanh((x - 15.0) / 2.0)), (c.ny, 1))
    o = Oracle(c, rho=rho, ux=np.zeros_like(rho), uy=np.zeros_like(rho))
    mid = 0.5 * (rl + rv)
    t, y = [], []
    for k in range(20):
        o.step(1000)
        r = o.field("rho").mean(axis=0)
        j = int(np.argmax(r[1:] > mid)) + 1
        t.append((k + 1) * 1000.0)
        y.append((j - 1) + (mid - r[j - 1]) / (r[j] - r[j - 1]) - 0.5)
    slope = np.polyfit(t[6:], np.square(y[6:]), 1)[0]
    beta = np.sqrt(slope / (4.0 * alpha_v))
    beta_w = _welch_beta(11.0 * dT / eos.h_fg(Ts))
    assert y[-1] > y[0] + 5.0  # the film grows
    assert abs(beta / beta_w - 1.0) < 0.15, (beta, beta_w)
