"""The double-shear-layer driver (Sec. III.B) builds the same inputs as the seeded workload
description the oracle tests use, and its kinetic energy is the plain sum rho |u|^2 / 2."""
import numpy as np

import synthetic_inputs as si


def test_shear_layer_driver_inputs_match_the_workload_description():
    from paper_1912_02018_gb300 import shear_layer

    a = si.shear_layer_velocity(96, 0.6)
    b = shear_layer.initial_velocity(96, 0.6)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    c, d = si.shear_layer_case(96, 0.6, collision=1), shear_layer.paper_case(96, 0.6, collision=1)
    for k in ("nx", "ny", "periodic_x", "G", "energy", "nu_l", "g", "collision"):
        assert getattr(c, k) == getattr(d, k), k


def test_kinetic_energy_is_the_plain_sum():
    from paper_1912_02018_gb300 import shear_layer

    rng = np.random.default_rng(3)
    f = {k: rng.uniform(0.5, 1.5, (7, 9)) for k in ("rho", "ux", "uy")}
    expect = sum(0.5 * f["rho"][j, i] * (f["ux"][j, i] ** 2 + f["uy"][j, i] ** 2) for j in range(7) for i in range(9))
    assert abs(shear_layer.kinetic_energy(f) - expect) < 1e-12 * expect
