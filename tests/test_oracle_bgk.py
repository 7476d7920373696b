"""Pins of the oracle's BGK operator, the comparison collision of Sec. III.B (double shear layer):
single-rate relaxation on the same fourth-order Hermite equilibrium (Eq. equi) and forcing
(Eq. forcingTerm) as the central-moment collision of Sec. II.A."""
import numpy as np

import synthetic_inputs as si
from oracle import Oracle, cm_defs, stepper

rng = np.random.default_rng(7)


def random_node():
    rho = rng.uniform(0.4, 6.6)
    u0 = rng.uniform(-0.15, 0.15, 2)
    f = cm_defs.feq(rho, *u0) * (1 + rng.uniform(-0.05, 0.05, 9))
    Fx, Fy = rng.uniform(-5e-3, 5e-3, 2)
    return rho, f, Fx, Fy


def test_oracle_bgk_equals_population_space_definition():
    # the C oracle goes through central moments (K = omega I); the definition is in population space
    for _ in range(20):
        rho, f, Fx, Fy = random_node()
        omega = rng.uniform(0.3, 1.99)
        a, ra, uxa, uya = stepper.collide_node(f, Fx, Fy, Fx, Fy, 2.0, omega, 0.38, bgk=1)
        b, rb, uxb, uyb = cm_defs.collide_bgk_direct(f, Fx, Fy, omega)
        assert np.allclose(a, b, rtol=0, atol=1e-14 * rho)
        assert abs(ra - rb) < 1e-14 * rho and abs(uxa - uxb) < 1e-15 and abs(uya - uyb) < 1e-15


def test_bgk_and_cm_coincide_at_unit_relaxation_rate():
    # omega = 1 relaxes every central moment at rate 1 in both operators: f* = f^eq + F_i / 2
    for _ in range(10):
        rho, f, Fx, Fy = random_node()
        a = stepper.collide_node(f, Fx, Fy, Fx, Fy, 2.0, 1.0, 0.0, bgk=1)[0]
        b = stepper.collide_node(f, Fx, Fy, Fx, Fy, 2.0, 1.0, 0.0, bgk=0)[0]
        assert np.allclose(a, b, rtol=0, atol=2e-15 * rho)


def test_bgk_differs_from_cm_only_outside_the_shear_moments():
    # both relax k4, k5 at omega; BGK also relaxes the other non-conserved moments at omega
    rho, f, Fx, Fy = random_node()
    omega = 1.6
    a, _, ux, uy = stepper.collide_node(f, Fx, Fy, Fx, Fy, 2.0, omega, 0.0, bgk=1)
    b = stepper.collide_node(f, Fx, Fy, Fx, Fy, 2.0, omega, 0.0, bgk=0)[0]
    T = cm_defs.T_matrix(ux, uy)
    ka, kb = T @ a, T @ b
    assert np.allclose(ka[:3], kb[:3], rtol=0, atol=1e-14 * rho)
    assert np.allclose(ka[4:6], kb[4:6], rtol=0, atol=1e-14 * rho)
    assert np.abs(ka[[3, 6, 7, 8]] - kb[[3, 6, 7, 8]]).max() > 1e-6 * rho


def test_bgk_conserves_mass_and_gives_half_force_momentum():
    for _ in range(10):
        rho, f, Fx, Fy = random_node()
        fs, r, ux, uy = stepper.collide_node(f, Fx, Fy, Fx, Fy, 2.0, 1.3, 0.38, bgk=1)
        assert abs(fs.sum() - f.sum()) < 1e-14 * rho
        assert abs(fs @ cm_defs.CX - (r * ux + Fx / 2)) < 1e-14 * rho
        assert abs(fs @ cm_defs.CY - (r * uy + Fy / 2)) < 1e-14 * rho


def test_bgk_equilibrium_is_a_fixed_point():
    rho, ux, uy = 2.5, 0.12, -0.07
    fe = cm_defs.feq(rho, ux, uy)
    fs = stepper.collide_node(fe, 0.0, 0.0, 0.0, 0.0, 2.0, 1.7, 0.0, bgk=1)[0]
    assert np.allclose(fs, fe, rtol=0, atol=1e-15 * rho)


def test_bgk_taylor_green_decay_matches_closed_form():
    n, nu, u0, t = 64, 0.02, 1e-3, 1000
    k = 2 * np.pi / n
    c = si.Case(nx=n, ny=n, D=0.0, xc=0.0, yc=0.0, periodic_x=1, g=0.0, u_in=0.0, noise_amp=0.0,
                G=0.0, sigma=0.0, energy=0, nu_l=nu, collision=1)
    y, x = np.mgrid[0:n, 0:n].astype(float)
    ux = u0 * np.sin(k * x) * np.cos(k * y)
    uy = -u0 * np.cos(k * x) * np.sin(k * y)
    o = Oracle(c, rho=np.ones((n, n)), ux=ux, uy=uy).step(t)
    amp = (o.field("ux") * ux).sum() / (ux * ux).sum()
    assert abs(amp / np.exp(-2 * nu * k * k * t) - 1) < 5e-3


def test_shear_layer_input_is_the_printed_initial_condition():
    L, Ma = 64, 0.3
    ux, uy = si.shear_layer_velocity(L, Ma)
    u0 = Ma / np.sqrt(3.0)
    # the layers sit at y/L = 1/4 and 3/4 (u_x changes sign there), u_x is +-u0 tanh(20) at y/L = 1/2, 0
    assert ux[16, 0] == 0.0 and abs(ux[48, 5]) < 1e-16
    assert np.isclose(ux[32, 0], u0 * np.tanh(20.0)) and np.isclose(ux[0, 0], -u0 * np.tanh(20.0))
    assert np.isclose(uy[0, 0], u0 * 0.05) and np.isclose(uy[3, 16], 0.0, atol=1e-17)
    c = si.shear_layer_case(L, Ma, collision=1)
    o = Oracle(c, rho=np.ones((L, L)), ux=ux, uy=uy)
    assert np.allclose(o.field("ux"), ux, rtol=0, atol=1e-15) and np.allclose(o.field("uy"), uy, rtol=0, atol=1e-15)
    assert np.isclose(stepper.derive(c)[1].nu_l, u0 * L / 3.0e4)
