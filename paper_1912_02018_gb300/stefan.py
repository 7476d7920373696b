"""Stefan problem (Sec. III.E): the interface of a vapour film on a heated wall against Welch's law.

The paper's pseudo one-dimensional domain (5 x 100, the wall at one end, the outflow of Sec. IV.A
at the other) is laid out along x: the column x = 0 is a flat wall (halfway bounce-back, held at
T_w = T_sat + dT), the rows are periodic in y, x = nx-1 is the convective outlet.  A vapour film
of thickness xi0 lies on the wall; alpha_v = 0.1.  The interface position y_i(t)
(where the y-averaged density crosses (rho_l + rho_v)/2, measured from the wall surface at
x = 1/2) is compared with y_i = 2 beta (alpha_v t)^(1/2), beta the root of
    beta exp(beta^2) erf(beta) = c_p dT / (h_fg sqrt(pi)),
through the slope of y_i^2 against t over the last two thirds of the run (4 beta^2 alpha_v).
Readings the paper leaves open are options, with defaults under which the oracle's beta lies within
12% of Welch's for the paper's three cases: G = -2, the wall's psi density rho_s = rho_v (a
vapour-wetting wall), a liquid diffusivity a tenth of the vapour's (Pr_l = 15 at eta = 1), an
initial film of 15 nodes (the paper's 5 is about one interface width here and does not survive),
outlet speed 0.2.

    python -m paper_1912_02018_gb300.stefan --Tr 0.86 --dT 0.010 --steps 20000

Prints one JSON document.  Lattice units.
"""
from __future__ import annotations

import argparse
import json
import math
import time
from types import SimpleNamespace

import numpy as np

from .sim import Sim


def welch_beta(St):
    """Root of beta exp(beta^2) erf(beta) = St / sqrt(pi) (monotonic in beta >= 0), by bisection."""
    target = St / math.sqrt(math.pi)
    lo, hi = 0.0, 1.0
    while hi * math.exp(hi * hi) * math.erf(hi) < target:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid * math.exp(mid * mid) * math.erf(mid) < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def paper_case(Tr=0.86, dT=0.010, nx=101, ny=5, alpha_v=0.1, G=-2.0, Pr_l=15.0, Pr_v=1.5, U_out=0.2, rho_s=-1.0,
               a=3.0 / 49.0, b=2.0 / 21.0, R=1.0):
    """dT in lattice temperature units; rho_s < 0 means rho_v (set once the coexistence is known)."""
    Tc = 0.0778 * a / (0.4572 * b * R)  # Peng-Robinson critical temperature (Sec. II.C)
    nu = alpha_v * Pr_v
    return SimpleNamespace(
        nx=nx, ny=ny, D=0.0, xc=0.0, yc=0.0, periodic_x=0, walls=1, superheat_Tc=dT / Tc, rho_s=rho_s, a=a, b=b, R=R,
        acentric=0.344, G=G, sigma=0.38, Tr_sat=Tr, Re=30.0, u_in=0.0, nu_l=nu, nu_ratio=1.0, Pr_l=Pr_l, Pr_v=Pr_v,
        c_v=11.0, g=0.0, U_out=U_out, warmup=0, energy=1, seed=0, noise_amp=0.0, psi_mode=0, wall_dT=(),
        body_fx=0.0, collision=0)


def interface_position(profile, mid):
    """Distance from the wall surface (x = 1/2) to where the y-averaged density first crosses mid,
    linearly interpolated between nodes; profile[0] is the wall column."""
    p = np.asarray(profile, dtype=np.float64)
    j = int(np.argmax(p[1:] > mid)) + 1
    if not p[j] > mid:
        return float("nan")
    return (j - 1) + (mid - p[j - 1]) / (p[j] - p[j - 1]) - 0.5


def initial_density(case, rv, rl, xi0=15.0, width=2.0):
    """The film: rho_v at the wall rising to rho_l through a tanh of half-width `width` at xi0."""
    x = np.arange(case.nx, dtype=np.float64)
    return np.tile(rv + (rl - rv) * 0.5 * (1.0 + np.tanh((x - xi0) / width)), (case.ny, 1))


def run(Tr=0.86, dT=0.010, steps=20000, every=500, xi0=15.0, width=2.0, f64=False, **kw):
    case = paper_case(Tr, dT, **kw)
    probe = Sim.from_case(SimpleNamespace(**{**vars(case), "rho_s": 0.0}), f64=f64)
    info = probe.info()
    probe.close()
    rv, rl = info["rho_v"], info["rho_l"]
    if case.rho_s < 0:
        case.rho_s = rv
    rho = initial_density(case, rv, rl, xi0, width)
    sim = Sim.from_case(case, f64=f64, init={"rho": rho, "ux": np.zeros_like(rho), "uy": np.zeros_like(rho)})
    mid = 0.5 * (rl + rv)
    t, y = [], []
    t0 = time.perf_counter()
    for k in range(steps // every):
        sim.step(every)
        t.append((k + 1) * every)
        y.append(interface_position(sim.fields(("rho",))["rho"].mean(axis=0), mid))
    seconds = time.perf_counter() - t0
    sim.close()
    beta = welch_beta(case.c_v * dT / info["h_fg"])
    h = len(t) // 3
    ok = np.isfinite(y[h:]).all() and len(t) - h >= 2
    slope = float(np.polyfit(np.array(t[h:], float), np.array(y[h:]) ** 2, 1)[0]) if ok else float("nan")
    alpha_v = case.nu_l / case.Pr_v
    beta_num = math.sqrt(slope / (4.0 * alpha_v)) if slope > 0 else 0.0
    return {"Tr": Tr, "dT": dT, "G": case.G, "rho_s": case.rho_s, "rho_v": rv, "rho_l": rl, "Pr_l": case.Pr_l,
            "U_out": case.U_out, "xi0": xi0, "width": width,
            "h_fg": info["h_fg"], "beta_welch": beta, "beta_sim": beta_num, "t": t, "y_i": y, "seconds": seconds}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--Tr", type=float, default=0.86)
    ap.add_argument("--dT", type=float, default=0.010)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--xi0", type=float, default=15.0)
    ap.add_argument("--G", type=float, default=-2.0)
    ap.add_argument("--Pr-l", type=float, default=15.0)
    ap.add_argument("--U-out", type=float, default=0.2)
    ap.add_argument("--rho-s", type=float, default=-1.0, help="density of the wall's psi (< 0: rho_v)")
    ap.add_argument("--f64", action="store_true")
    a = ap.parse_args()
    print(json.dumps(run(a.Tr, a.dT, a.steps, xi0=a.xi0, f64=a.f64, G=a.G, Pr_l=a.Pr_l, U_out=a.U_out,
                         rho_s=a.rho_s)))


if __name__ == "__main__":
    main()
