"""Pins of the oracle's CM algebra against what the paper and mathematics fix.

Sec. II.A and App. A of Saito et al. (arXiv:1912.02018): the raw-moment matrix M,
the shift matrix N = T M^{-1}, the equilibrium and forcing central moments, and the
collision Eq. (collision) in its matrix form.
"""
import json
import os

import numpy as np
import pytest

from oracle import cm_defs, stepper

GOLD = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(1234)


def test_M_matches_printed_matrix():
    printed = np.loadtxt(os.path.join(GOLD, "M_matrix_appA.txt"))
    assert np.array_equal(stepper.matrix_M(), printed)
    assert np.array_equal(cm_defs.M_matrix(), printed)


@pytest.mark.parametrize("k", range(6))
def test_printed_N_equals_T_Minv(k):
    ux, uy = rng.uniform(-0.3, 0.3, 2)
    N_def = cm_defs.T_matrix(ux, uy) @ np.linalg.inv(cm_defs.M_matrix())
    assert np.allclose(stepper.matrix_N(ux, uy), N_def, atol=1e-14, rtol=0)


def test_N_inverse_is_N_of_minus_u():
    ux, uy = 0.17, -0.08
    prod = stepper.matrix_N(ux, uy) @ stepper.matrix_N(-ux, -uy)
    assert np.allclose(prod, np.eye(9), atol=1e-15)


def test_T_times_reconstruction_is_identity():
    # T(u) M^{-1} N(-u) = I: the two-step reconstruction inverts the CM transform
    for _ in range(5):
        ux, uy = rng.uniform(-0.3, 0.3, 2)
        A = cm_defs.T_matrix(ux, uy) @ np.linalg.inv(stepper.matrix_M()) @ stepper.matrix_N(-ux, -uy)
        assert np.allclose(A, np.eye(9), atol=1e-14)


def test_equilibrium_central_moments_match_paper():
    gold = json.load(open(os.path.join(GOLD, "paper_constants.json")))["k_eq"]["value"]
    assert gold == ["rho", 0, 0, "2rho/3", 0, 0, 0, 0, "rho/9"]
    for _ in range(5):
        rho = rng.uniform(0.3, 7.0)
        ux, uy = rng.uniform(-0.2, 0.2, 2)
        k = cm_defs.T_matrix(ux, uy) @ cm_defs.feq(rho, ux, uy)
        assert np.allclose(k, [rho, 0, 0, 2 * rho / 3, 0, 0, 0, 0, rho / 9], atol=1e-14 * rho)


def test_forcing_central_moments_match_paper():
    for _ in range(5):
        Fx, Fy = rng.uniform(-1e-2, 1e-2, 2)
        ux, uy = rng.uniform(-0.2, 0.2, 2)
        R = cm_defs.T_matrix(ux, uy) @ cm_defs.huang_force(Fx, Fy, ux, uy)
        assert np.allclose(R, [0, Fx, Fy, 0, 0, 0, Fy / 3, Fx / 3, 0], atol=1e-16)


def test_hermite_equilibrium_equals_product_form():
    # Textbook: the full-Hermite D2Q9 equilibrium factorises into 1-D parts with
    # <1>=1, <c>=u, <c^2>=1/3+u^2.
    def one_d(c, u):
        return np.where(c == 0, 2 / 3 - u * u, (1 / 3 + u * u + c * u) / 2)

    for _ in range(5):
        rho = rng.uniform(0.3, 7.0)
        ux, uy = rng.uniform(-0.3, 0.3, 2)
        prod = rho * one_d(cm_defs.CX, ux) * one_d(cm_defs.CY, uy)
        assert np.allclose(stepper.feq(rho, ux, uy), prod, rtol=1e-14, atol=0)
        assert np.allclose(cm_defs.feq(rho, ux, uy), prod, rtol=1e-14, atol=0)


@pytest.mark.parametrize("sigma", [0.0, 0.38])
def test_oracle_collision_equals_direct_definition(sigma):
    for _ in range(20):
        rho = rng.uniform(0.4, 6.6)
        u0 = rng.uniform(-0.1, 0.1, 2)
        f = cm_defs.feq(rho, *u0) * (1 + rng.uniform(-0.05, 0.05, 9))
        Fx, Fy, Fmx, Fmy = rng.uniform(-5e-3, 5e-3, 4)
        psi = rng.uniform(1.0, 4.0)
        omega = rng.uniform(0.3, 1.9)
        a, ra, uxa, uya = stepper.collide_node(f, Fx, Fy, Fmx, Fmy, psi, omega, sigma)
        b, rb, uxb, uyb = cm_defs.collide_direct(f, Fx, Fy, Fmx, Fmy, psi, omega, sigma)
        assert np.allclose(a, b, rtol=0, atol=1e-14 * rho)
        assert abs(ra - rb) < 1e-14 * rho and abs(uxa - uxb) < 1e-15 and abs(uya - uyb) < 1e-15


def test_collision_conserves_mass_and_gives_half_force_momentum():
    for _ in range(10):
        rho = rng.uniform(0.4, 6.6)
        f = cm_defs.feq(rho, 0.05, -0.02) * (1 + rng.uniform(-0.05, 0.05, 9))
        Fx, Fy = rng.uniform(-5e-3, 5e-3, 2)
        fs, r, ux, uy = stepper.collide_node(f, Fx, Fy, Fx, Fy, 2.0, 1.2, 0.38)
        assert abs(r - f.sum()) < 1e-14 * rho
        assert abs(fs.sum() - r) < 1e-14 * rho
        # k1* = Fx/2 in the central frame  <=>  sum f* c = rho u + F/2
        assert abs(fs @ cm_defs.CX - (r * ux + Fx / 2)) < 1e-14 * rho
        assert abs(fs @ cm_defs.CY - (r * uy + Fy / 2)) < 1e-14 * rho


def test_post_collision_moments_match_eq_postColl2():
    rho = 5.0
    f = cm_defs.feq(rho, 0.03, 0.01) * (1 + rng.uniform(-0.05, 0.05, 9))
    Fx, Fy, Fmx, Fmy, psi, omega, sigma = 1e-3, -2e-3, 7e-4, -3e-4, 2.5, 1.4, 0.38
    fs, rho, ux, uy = stepper.collide_node(f, Fx, Fy, Fmx, Fmy, psi, omega, sigma)
    T = cm_defs.T_matrix(ux, uy)
    k = T @ f
    ks = T @ fs
    alpha = sigma / psi ** 2
    Fm2 = Fmx ** 2 + Fmy ** 2
    expect = [rho, Fx / 2, Fy / 2, 2 * rho / 3 + 2 * alpha * Fm2, (1 - omega) * k[4], (1 - omega) * k[5],
              Fy / 6, Fx / 6, rho / 9 + 2 / 3 * alpha * Fm2]
    assert np.allclose(ks, expect, atol=1e-14 * rho, rtol=0)


def test_sigma_zero_reduces_to_original_forcing():
    f = cm_defs.feq(3.0, 0.02, 0.0) * (1 + rng.uniform(-0.02, 0.02, 9))
    a = stepper.collide_node(f, 1e-3, 0, 1e-3, 0, 2.0, 1.0, 0.0)[0]
    b = stepper.collide_node(f, 1e-3, 0, 5.0, 5.0, 2.0, 1.0, 0.0)[0]  # F_m only enters through sigma
    assert np.array_equal(a, b)
