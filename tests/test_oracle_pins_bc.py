"""Pins of the oracle's boundary substitutions and of the conductive part of Eq. (energy) against
closed forms and an independent reference, each chosen so that the plausible mistake fails.

- Linear interpolated bounce-back (Bouzidi 2001), the wall condition of Sec. IV.A: with the flat
  walls' surface placed a fraction q of a link from the last fluid row, Poiseuille flow (Sec. III.C)
  converges at second order to the closed form with the wall at its true position, through the
  q < 1/2 branch (q = 0.2) and the q >= 1/2 branch (q = 0.7); halfway bounce-back, which puts the
  wall half a link away, converges only at first order to that profile.
- Convective outlet (Lou 2013), the outlet of Sec. IV.A: a vortex carried out through x = nx-1
  leaves the flow upstream as it would in a domain twice as long; a zero-gradient outlet, or the
  convective law with its weights swapped, reflects it.
- grad(lambda) . grad(T) in Eq. (energy): with a smooth density field (so lambda varies) and
  u = 0, the right-hand side converges at second order to the analytic div(lambda grad T) / (rho c_v).
"""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import Oracle, stepper


# ---------------------------------------------------------------- Bouzidi (Sec. IV.A) on offset flat walls

def _offset_poiseuille(L, q, wall_q, nu=1.0 / 6.0, U0=0.01):
    """Steady u_x at the fluid rows 1..L of a channel whose wall surfaces lie at y = 1 - q and
    y = L + q (width W = L - 1 + 2q), driven by F_x = 8 nu U0 / W^2, with the oracle's flat walls
    at link fraction wall_q; returns the relative L2 error against 4 U0 y'(W - y') / W^2."""
    W = L - 1 + 2.0 * q
    c = si.poiseuille_case(L, U0=U0, nu=nu).replace(body_fx=8.0 * nu * U0 / W ** 2, wall_q=wall_q)
    rho = np.ones((c.ny, c.nx))
    zero = np.zeros_like(rho)
    o = Oracle(c, rho=rho, ux=zero, uy=zero).step(int(8 * W * W / nu))  # eight diffusion times
    u = o.field("ux")[1:c.ny - 1].mean(axis=1)
    yp = np.arange(1, L + 1) - (1.0 - q)
    ref = 4.0 * U0 * yp * (W - yp) / W ** 2
    assert np.abs(o.field("uy")).max() < 1e-13
    return np.linalg.norm(u - ref) / np.linalg.norm(ref)


def test_flat_wall_link_fraction_is_the_option():
    c = si.Case(nx=10, ny=8, D=0.0, xc=0.0, yc=0.0, walls=2, periodic_x=1, G=0.0, energy=0, u_in=0.0,
                nu_l=1.0 / 6.0, g=0.0, noise_amp=0.0, wall_q=0.3)
    q = Oracle(c).link_fractions()
    assert set(np.unique(q[q >= 0])) == {0.3}
    # links into the walls from the first and last fluid rows only: 3 per node per wall
    assert (q[1] >= 0).sum() == 3 * c.nx and (q[c.ny - 2] >= 0).sum() == 3 * c.nx


@pytest.mark.slow
@pytest.mark.parametrize("q", [0.2, 0.7])
def test_bouzidi_offset_walls_converge_at_second_order(q):
    errs = np.array([_offset_poiseuille(L, q, q) for L in (8, 16, 32)])
    orders = np.log2(errs[:-1] / errs[1:])
    assert np.all((orders > 1.85) & (orders < 2.25)), (errs, orders)
    assert errs[-1] < 4e-3, errs
    # halfway bounce-back puts the wall at y = 1/2 instead: first order against the true profile
    hb = np.array([_offset_poiseuille(L, q, 0.5) for L in (16, 32)])
    assert hb[-1] > 10 * errs[-1] and np.log2(hb[0] / hb[1]) < 1.2, hb


# ---------------------------------------------------------------- convective outlet (Sec. IV.A)

def _vortex_run(nx, ny, L, U_out, u_in=0.1, nu=0.01, uv=0.02, r0=6.0, steps=1200, every=100):
    """A single-phase uniform stream u_in with a Gaussian vortex (peak swirl uv, radius r0, in
    pressure balance) started 30 nodes before x = L - 1; returns (u_x, u_y) on the columns
    x < L - 1 every `every` steps."""
    c = si.Case(nx=nx, ny=ny, D=0.0, xc=0.0, yc=0.0, periodic_x=0, G=0.0, sigma=0.0, energy=0, u_in=u_in,
                nu_l=nu, g=0.0, noise_amp=0.0, U_out=U_out)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    dx, dy = x - (L - 30.0), y - ny / 2.0
    r2 = dx * dx + dy * dy
    s = uv / r0 * np.exp(0.5 * (1.0 - r2 / r0 ** 2))  # u_theta = uv (r / r0) exp((1 - r^2 / r0^2) / 2)
    rho = 1.0 - 1.5 * uv * uv * np.e * np.exp(-r2 / r0 ** 2)  # dp/dr = u_theta^2 / r, p = rho / 3
    o = Oracle(c, rho=rho, ux=u_in - s * dy, uy=s * dx)
    out = []
    for _ in range(steps // every):
        o.step(every)
        out.append((o.field("ux")[:, :L - 1], o.field("uy")[:, :L - 1]))
    return out


@pytest.mark.slow
def test_convective_outlet_lets_a_vortex_leave_as_a_longer_domain_does():
    L, ny, uv = 96, 64, 0.02
    ref = _vortex_run(2 * L, ny, L, -1.0)  # the same flow with the outlet L nodes further downstream

    def worst(U_out):
        got = _vortex_run(L, ny, L, U_out)
        return max(max(np.abs(a[0] - b[0]).max(), np.abs(a[1] - b[1]).max()) for a, b in zip(got, ref)) / uv

    # U = u_in (the reading of the outlet speed): measured 1.6% of the vortex's swirl
    assert worst(-1.0) < 0.03
    # a zero-gradient outlet (U -> infinity) and swapped weights (U -> 1/U) reflect the vortex (36%)
    assert worst(1e9) > 0.2
    assert worst(1.0 / 0.1) > 0.2


# ---------------------------------------------------------------- grad(lambda) . grad(T) (Eq. energy)

def _rhs_error(n):
    c = si.Case(nx=n, ny=n, D=0.0, xc=0.0, yc=0.0, periodic_x=1, G=-2.0, energy=1, u_in=0.0, nu_l=0.1,
                g=0.0, noise_amp=0.0, Pr_l=0.862, Pr_v=1.5)
    _, d = stepper.derive(c)
    k = 2.0 * np.pi / n
    y, x = np.mgrid[0:n, 0:n].astype(float)
    # density strictly between the phases (no clipping of the phase fraction), so lambda is smooth
    A = 0.3 * (d.rho_l - d.rho_v)
    rho = 0.5 * (d.rho_l + d.rho_v) + A * np.sin(k * x + 0.4) * np.cos(k * y + 0.2)
    rx = A * k * np.cos(k * x + 0.4) * np.cos(k * y + 0.2)
    ry = -A * k * np.sin(k * x + 0.4) * np.sin(k * y + 0.2)
    B = 0.01
    T = d.T_sat + B * np.cos(k * x + 1.1) * np.sin(2 * k * y + 0.7)
    Tx = -B * k * np.sin(k * x + 1.1) * np.sin(2 * k * y + 0.7)
    Ty = 2 * B * k * np.cos(k * x + 1.1) * np.cos(2 * k * y + 0.7)
    lapT = -5 * B * k * k * np.cos(k * x + 1.1) * np.sin(2 * k * y + 0.7)
    # lambda = rho c_v alpha(phi), alpha linear in phi = (rho - rho_v) / (rho_l - rho_v)
    da = d.alpha_l - d.alpha_v
    phi = (rho - d.rho_v) / (d.rho_l - d.rho_v)
    lam = rho * c.c_v * (d.alpha_v + phi * da)
    dlam = c.c_v * (d.alpha_v + phi * da) + rho * c.c_v * da / (d.rho_l - d.rho_v)
    ref = (lam * lapT + dlam * (rx * Tx + ry * Ty)) / (rho * c.c_v)  # div(lambda grad T) / (rho c_v)
    zero = np.zeros_like(rho)
    got = stepper.energy_rhs(c, rho, zero, zero, T)
    return np.abs(got - ref).max() / np.abs(ref).max()


def test_conduction_with_variable_conductivity_converges_at_second_order():
    errs = np.array([_rhs_error(n) for n in (32, 64, 128)])
    orders = np.log2(errs[:-1] / errs[1:])
    # measured 0.0285, 0.0072, 0.0018; without the grad(lambda) . grad(T) term the error stays at 0.21
    assert np.all(orders > 1.9), (errs, orders)
    assert errs[-1] < 3e-3, errs
