"""Host side of the boiling-curve driver: the film-boiling correlations of the paper's appendix
and the paper-shaped domain of Sec. IV.A."""
import numpy as np

from paper_1912_02018_gb300 import boiling_curve as bc


def _slope(f, Ja):
    h = 1e-6
    return (np.log(f(Ja * (1 + h))) - np.log(f(Ja * (1 - h)))) / (np.log1p(h) - np.log1p(-h))


def test_mode1_and_mode2_scale_as_the_appendix_states():
    for Ja in (0.05, 0.2, 0.7):
        assert abs(_slope(lambda j: bc.mode1(2.7, 1.0, 30.0, 1.5, j), Ja) + 0.5) < 1e-6
        assert abs(_slope(lambda j: bc.mode2(0.537, 17.0, 1.0, 30.0, 1.5, j), Ja) + 0.25) < 1e-6
    # Nu ~ eta^1/2 Re^1/2 in both modes; gamma^1/4 and Pr^1/4 in Mode 2, Pr^1/2 in Mode 1
    assert np.isclose(bc.mode2(1.0, 16.0, 4.0, 9.0, 16.0, 1.0), 2.0 * 2.0 * 3.0 * 2.0)
    assert np.isclose(bc.mode1(1.0, 4.0, 9.0, 16.0, 1.0 / 4.0), 2.0 * 3.0 * 4.0 * 2.0)


def test_bromley_uses_the_effective_latent_heat():
    # h' = h_fg (1 + 0.4 Ja)^2: at small Ja Bromley is Mode 1 with C = 2.7; at Ja = 0.5 the
    # effective Jacob number is 0.5 / 1.2^2
    assert np.isclose(bc.bromley(1.0, 30.0, 1.5, 1e-9), bc.mode1(2.7, 1.0, 30.0, 1.5, 1e-9), rtol=1e-8)
    assert np.isclose(bc.bromley(1.0, 30.0, 1.5, 0.5), bc.mode1(2.7, 1.0, 30.0, 1.5, 0.5 / 1.44))
    c = bc.correlations(17.0, 1.0, 30.0, 1.5, 0.2)
    assert set(c) == {"bromley_2.7", "epstein_hauser_0.537", "epstein_hauser_1.13", "ito_0.46", "ito_0.48",
                      "ito_0.51"}
    assert np.isclose(c["epstein_hauser_1.13"] / c["epstein_hauser_0.537"], 1.13 / 0.537)


def test_paper_case_is_the_sec_iv_a_domain():
    c = bc.paper_case(0.010, 30.0, seed=1)
    assert (c.nx, c.ny, c.D, c.xc, c.yc) == (1350, 600, 30.0, 270.0, 300.0)
    Tc = 0.0778 * (3.0 / 49.0) / (0.4572 * (2.0 / 21.0))
    assert abs(Tc - 0.1094) < 5e-5  # the T_c the paper prints for a = 3/49, b = 2/21, R = 1 (Sec. II.C)
    assert np.isclose(c.superheat_Tc * Tc, 0.010)
    assert c.warmup == 3000 and c.u_in == 0.05 and c.Re == 30.0 and c.Pr_v == 1.5 and c.c_v == 11.0
