"""Bubble growth in a superheated liquid against the Plesset-Zwick law (App. D).

A vapour bubble of radius R0 = 15 sits at the centre of an N x N lattice (N = 1000 in the paper)
of liquid superheated by dT = 0.04 T_c; the paper compares R(t) with
    R(t) = (12 alpha_l / pi)^(1/2) Ja t^(1/2),   Ja = rho_l c_p dT / (rho_v h_fg),
for alpha_l = 5.8e-2 (agreement) and 5.8e-5 (the thermal layer is not resolved).  Setup readings
(the paper shows the setup as a figure only): periodic in y; the column x = 0 is the Zou-He
inlet at zero speed (T held at T_sat there) and x = N-1 a convective outlet at the sound speed,
so the liquid the bubble displaces can leave; no gravity; c_p = c_v = 11, T_r = 0.86, a = 3/49,
nu_l = alpha_l Pr_l, eta = 1.  Initial state: the bubble at rho_v(T_sat) and T_sat inside a
tanh interface of width 5; the liquid at T_sat + dT and at the density where the Peng-Robinson
pressure equals p_sat(T_sat) (a liquid at rho_l(T_sat) and T_sat + dT is over-pressured and
crushes the bubble).  R(t) is the radius of the area where rho < (rho_l + rho_v)/2; the growth
constant is the slope of R^2 against t over the second half of the run, against (12/pi)
alpha_l Ja^2.

    python -m paper_1912_02018_gb300.bubble_growth --N 1000 --steps 20000

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


def paper_case(N=1000, dT_Tc=0.04, alpha_l=5.8e-2, G=-2.0, a=3.0 / 49.0, b=2.0 / 21.0, R=1.0, Tr=0.86,
               Pr_l=0.862, Pr_v=1.5):
    return SimpleNamespace(
        nx=N, ny=N, D=0.0, xc=0.0, yc=0.0, periodic_x=0, walls=0, superheat_Tc=dT_Tc, rho_s=0.0, a=a, b=b, R=R,
        acentric=0.344, G=G, sigma=0.38, Tr_sat=Tr, Re=30.0, u_in=0.0, nu_l=alpha_l * Pr_l, nu_ratio=1.0,
        Pr_l=Pr_l, Pr_v=Pr_v, c_v=11.0, g=0.0, U_out=1.0 / math.sqrt(3.0), warmup=0, energy=1, seed=0, noise_amp=0.0,
        psi_mode=0, wall_dT=(), body_fx=0.0, collision=0)


def pr_pressure(case, rho, T, Tc):
    """Peng-Robinson pressure of Eq. (eos) (host-side setup of the initial liquid only)."""
    w = case.acentric
    kappa = 0.37464 + 1.54226 * w - 0.26992 * w * w
    phi = (1.0 + kappa * (1.0 - math.sqrt(T / Tc))) ** 2
    return rho * case.R * T / (1.0 - case.b * rho) - case.a * phi * rho * rho / (
        1.0 + 2.0 * case.b * rho - case.b * case.b * rho * rho)


def superheated_liquid_density(case, info):
    """The liquid-branch density at which p_EOS(rho, T_sat + dT) = p_sat(T_sat): Newton's method from
    rho_l(T_sat), where the pressure is above p_sat and decreases monotonically towards the root."""
    T, p0, Tc = info["T_wall"], info["p_sat"], info["Tc"]
    r = info["rho_l"]
    for _ in range(100):
        f = pr_pressure(case, r, T, Tc) - p0
        h = 1e-6 * r
        df = (pr_pressure(case, r + h, T, Tc) - pr_pressure(case, r - h, T, Tc)) / (2 * h)
        if not df > 0:
            raise ValueError("left the liquid branch: the superheat is beyond the liquid spinodal")
        step = f / df
        r -= step
        if abs(step) < 1e-14 * r:
            return r
    raise ValueError("no convergence")


def initial_fields(case, info, R0=15.0, width=5.0):
    """rho and T of the initial state, shape (ny, nx); inside the bubble rho_v(T_sat) and T_sat."""
    rl = superheated_liquid_density(case, info)
    y, x = np.mgrid[0:case.ny, 0:case.nx].astype(np.float64)
    r = np.hypot(x - case.nx / 2, y - case.ny / 2)
    s = 0.5 * (1.0 + np.tanh(2.0 * (r - R0) / width))  # 0 in the bubble, 1 in the liquid
    rho = info["rho_v"] + (rl - info["rho_v"]) * s
    T = info["T_sat"] + (info["T_wall"] - info["T_sat"]) * s
    return rho, T, rl


def radius(rho, mid):
    return math.sqrt(float((rho < mid).sum()) / math.pi)


def run(N=1000, steps=20000, every=500, dT_Tc=0.04, alpha_l=5.8e-2, G=-2.0, R0=15.0, f64=False):
    case = paper_case(N, dT_Tc, alpha_l, G)
    probe = Sim.from_case(SimpleNamespace(**{**vars(case), "nx": 16, "ny": 16}), f64=f64)
    info = probe.info()
    probe.close()
    rho, T, rl = initial_fields(case, info, R0)
    sim = Sim.from_case(case, f64=f64, init={"rho": rho, "T": T, "ux": np.zeros_like(rho), "uy": np.zeros_like(rho)})
    mid = 0.5 * (info["rho_l"] + info["rho_v"])
    t, R = [0], [radius(rho, mid)]
    t0 = time.perf_counter()
    for k in range(steps // every):
        sim.step(every)
        t.append((k + 1) * every)
        R.append(radius(sim.fields(("rho",))["rho"], mid))
    seconds = time.perf_counter() - t0
    sim.close()
    Ja = info["rho_l"] * case.c_v * dT_Tc * info["Tc"] / (info["rho_v"] * info["h_fg"])
    C2 = 12.0 / math.pi * alpha_l * Ja * Ja
    h = len(t) // 2
    slope = float(np.polyfit(np.array(t[h:], float), np.array(R[h:]) ** 2, 1)[0]) if len(t) - h >= 2 else float("nan")
    return {"N": N, "steps": steps, "dT_Tc": dT_Tc, "alpha_l": alpha_l, "G": G, "R0": R0, "rho_l_superheated": rl,
            "Ja": Ja, "plesset_zwick_R2_slope": C2, "R2_slope": slope, "slope_ratio": slope / C2, "t": t, "R": R,
            "seconds": seconds, "mlups": N * N * steps / seconds / 1e6}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--N", type=int, default=1000)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--every", type=int, default=500)
    ap.add_argument("--dT", type=float, default=0.04, help="superheat as a fraction of T_c")
    ap.add_argument("--alpha-l", type=float, default=5.8e-2)
    ap.add_argument("--G", type=float, default=-2.0)
    ap.add_argument("--f64", action="store_true")
    a = ap.parse_args()
    print(json.dumps(run(a.N, a.steps, a.every, a.dT, a.alpha_l, a.G, f64=a.f64)))


if __name__ == "__main__":
    main()
