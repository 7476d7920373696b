"""Peng-Robinson thermodynamics of the boiling model, in plain FP64 numpy/scipy.

TEST INFRASTRUCTURE ONLY: part of the oracle that the CUDA path is checked
against; only the tests, the smoke check and the benchmark's CPU-baseline leg may
import it.

Follows Sec. II.C of Saito et al. (arXiv:1912.02018):
  * Eq. (eos): p = rho R T / (1 - b rho) - a phi(T) rho^2 / (1 + 2 b rho - b^2 rho^2),
    phi(T) = [1 + kappa (1 - sqrt(T/Tc))]^2,
    kappa = 0.37464 + 1.54226 w - 0.26992 w^2 (w = acentric factor);
  * the critical constants from a = 0.4572 R^2 Tc^2 / pc and b = 0.0778 R Tc / pc;
  * coexistence densities by Maxwell's equal-area rule "by numerical integration
    of the EOS" (Sec. III.D);
  * the latent heat h_fg "from the EOS" (Sec. IV.A), read as Clausius-Clapeyron
    h_fg = T (1/rho_v - 1/rho_l) dp_sat/dT.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

from scipy import integrate, optimize


@dataclass(frozen=True)
class PR:
    a: float
    b: float
    R: float = 1.0
    acentric: float = 0.344

    @property
    def kappa(self) -> float:
        w = self.acentric
        return 0.37464 + 1.54226 * w - 0.26992 * w * w

    @property
    def Tc(self) -> float:
        # from a/b = (0.4572/0.0778) R Tc
        return 0.0778 * self.a / (0.4572 * self.b * self.R)

    @property
    def pc(self) -> float:
        return 0.0778 * self.R * self.Tc / self.b

    def phi(self, T: float) -> float:
        s = 1.0 + self.kappa * (1.0 - math.sqrt(T / self.Tc))
        return s * s

    def p(self, rho: float, T: float) -> float:
        b = self.b
        return rho * self.R * T / (1.0 - b * rho) - self.a * self.phi(T) * rho * rho / (
            1.0 + 2.0 * b * rho - b * b * rho * rho)

    def dp_drho(self, rho: float, T: float) -> float:
        b = self.b
        den = 1.0 + 2.0 * b * rho - b * b * rho * rho
        rep = self.R * T / (1.0 - b * rho) ** 2
        att = self.a * self.phi(T) * (2.0 * rho * den - rho * rho * (2.0 * b - 2.0 * b * b * rho)) / den ** 2
        return rep - att

    def dp_dT(self, rho: float, T: float) -> float:
        """(dp/dT) at fixed rho, by differentiating Eq. (eos)."""
        b = self.b
        s = 1.0 + self.kappa * (1.0 - math.sqrt(T / self.Tc))
        dphi = -self.kappa * s / math.sqrt(T * self.Tc)
        return rho * self.R / (1.0 - b * rho) - self.a * dphi * rho * rho / (
            1.0 + 2.0 * b * rho - b * b * rho * rho)

    def rho_c(self) -> float:
        """Density of the inflection point of p(rho) at Tc."""
        T = self.Tc
        h = 1e-5

        def d2(r):
            return (self.dp_drho(r + h, T) - self.dp_drho(r - h, T)) / (2 * h)

        return optimize.brentq(d2, 0.5 / self.b * 0.05, 0.9 / self.b, xtol=1e-14)

    def spinodals(self, T: float) -> tuple[float, float]:
        """Densities where dp/drho = 0 (vapour-side max and liquid-side min of p)."""
        grid = [(k + 0.5) / 4000.0 * (1.0 / self.b) for k in range(4000)]
        vals = [self.dp_drho(r, T) for r in grid]
        roots = []
        for k in range(len(grid) - 1):
            if vals[k] * vals[k + 1] < 0.0:
                roots.append(optimize.brentq(lambda r: self.dp_drho(r, T), grid[k], grid[k + 1], xtol=1e-15))
        if len(roots) != 2:
            raise ValueError(f"no two-phase region at T={T}")
        return roots[0], roots[1]

    def maxwell(self, T: float) -> tuple[float, float, float]:
        """(rho_v, rho_l, p_sat) by the equal-area rule int (p - p_s) dv = 0, v = 1/rho."""
        ra, rb = self.spinodals(T)
        p_hi = self.p(ra, T)
        p_lo = max(self.p(rb, T), 1e-10 * p_hi)

        def branches(ps):
            rv = optimize.brentq(lambda r: self.p(r, T) - ps, 0.0, ra, xtol=1e-15, rtol=1e-15)
            rl = optimize.brentq(lambda r: self.p(r, T) - ps, rb, (1.0 - 1e-12) / self.b, xtol=1e-15, rtol=1e-15)
            return rv, rl

        def area(ps):
            rv, rl = branches(ps)
            val, _ = integrate.quad(lambda r: (self.p(r, T) - ps) / (r * r), rv, rl,
                                    epsabs=1e-15, epsrel=1e-13, limit=400)
            return val

        lo = p_lo + 1e-14 * (p_hi - p_lo)
        hi = p_hi - 1e-14 * (p_hi - p_lo)
        ps = optimize.brentq(area, lo, hi, xtol=1e-16, rtol=1e-15, maxiter=500)
        rv, rl = branches(ps)
        return rv, rl, ps

    def h_fg(self, T: float, rel_step: float = 1e-5) -> float:
        """Latent heat from Clausius-Clapeyron with a central difference of p_sat(T)."""
        h = rel_step * T
        dps = (self.maxwell(T + h)[2] - self.maxwell(T - h)[2]) / (2 * h)
        rv, rl, _ = self.maxwell(T)
        return T * (1.0 / rv - 1.0 / rl) * dps
