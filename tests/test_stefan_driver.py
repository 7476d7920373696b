"""Host parts of the Stefan driver (Sec. III.E): Welch's beta and the interface tracking."""
import math

import numpy as np
from scipy import optimize, special

from oracle.thermo import PR


def test_welch_beta_solves_the_transcendental_equation():
    from paper_1912_02018_gb300.stefan import welch_beta

    eos = PR(3.0 / 49.0, 2.0 / 21.0, 1.0, 0.344)
    for Tr, dT in ((0.86, 0.010), (0.86, 0.023), (0.90, 0.010)):
        St = 11.0 * dT / eos.h_fg(Tr * eos.Tc)
        ref = optimize.brentq(lambda b: b * np.exp(b * b) * special.erf(b) - St / np.sqrt(np.pi), 1e-9, 5.0, xtol=1e-15)
        assert abs(welch_beta(St) - ref) < 1e-12
    # small-Stefan limit: beta ~ sqrt(St / 2)
    assert abs(welch_beta(1e-6) / math.sqrt(0.5e-6) - 1) < 1e-5


def test_interface_position_of_a_tanh_film():
    from paper_1912_02018_gb300.stefan import interface_position

    x = np.arange(60, dtype=float)
    for xi in (5.0, 7.3, 20.6):
        prof = 0.4 + 6.0 * 0.5 * (1 + np.tanh((x - xi) / 2.0))
        # the crossing of the mid density is at x = xi exactly; linear interpolation errs by < 0.01 node
        assert abs(interface_position(prof, 0.4 + 3.0) - (xi - 0.5)) < 1e-2
