"""Boiling curve and film-boiling Nusselt numbers on the paper's geometry (Sec. IV).

Runs the superheat sweep of Sec. IV.B on the CUDA path.  The domain of Sec. IV.A, W x H = 20D x
45D = 600 x 1350 with the flow along H, is laid out with the flow along +x: nx = 1350, ny = 600,
cylinder D = 30 at 0.2 H downstream of the inlet and W / 2 across; a = 3/49 (so h_fg = 0.572),
T_r = 0.86, u_l = 0.05, Re = 30 or 30000 (nu_l = u_l D / Re), g from u_l / sqrt(g D) = 4,
Pr_v = 1.5, c_p = c_v = 11, 3000 warm-up steps without force and energy equation.  The domains
of one Reynolds number step together in one batch (lbm_batch_*).  The wall heat flux is averaged
over the second half of the run after the warm-up (the quasi-steady state), giving the boiling
curve q(dT) with its standard deviation and Nu = q D / (lambda_v dT), Ja = c_p dT / h_fg.

Beside each point the film-boiling correlations of the paper's appendix (saturated form):
Mode 1, Bromley et al. with C = 2.7 and the effective latent heat h' = h_fg (1 + 0.4 Ja)^2;
Mode 2, Epstein-Hauser with C = 0.537 (theory) and 1.13 (fit), Ito et al. with C = 0.46, 0.48,
0.51; with gamma = rho_l / rho_v, eta = nu_l / nu_v, Re = u_l D / nu_l, Pr = nu_v / alpha_v.

    python -m paper_1912_02018_gb300.boiling_curve --Re 30 --steps 100000
    python -m paper_1912_02018_gb300.boiling_curve --Re 30000 --Pr-v 1.5e-3   # low-Prandtl study, Sec. IV.C

Prints one JSON document.  Lattice units.
"""
from __future__ import annotations

import argparse
import json
import time
from types import SimpleNamespace

import numpy as np

from ._native import LbmError
from .sim import Batch


def mode1(C, eta, Re, Pr, Ja):
    """Mode 1 film-boiling correlation: Nu = C eta^1/2 Re^1/2 Pr^1/2 Ja^-1/2."""
    return C * np.sqrt(eta) * np.sqrt(Re) * np.sqrt(Pr) / np.sqrt(Ja)


def mode2(C, gamma, eta, Re, Pr, Ja):
    """Mode 2 film-boiling correlation: Nu = C gamma^1/4 eta^1/2 Re^1/2 Pr^1/4 Ja^-1/4."""
    return C * gamma ** 0.25 * np.sqrt(eta) * np.sqrt(Re) * Pr ** 0.25 / Ja ** 0.25


def bromley(eta, Re, Pr, Ja, C=2.7):
    """Bromley et al. at high flow (u_l / sqrt(g D) > 2): Mode 1 with c_p dT / h' in place of Ja,
    h' = h_fg (1 + 0.4 c_p dT / h_fg)^2 the effective latent heat."""
    return mode1(C, eta, Re, Pr, Ja / (1.0 + 0.4 * Ja) ** 2)


def correlations(gamma, eta, Re, Pr, Ja) -> dict:
    return {
        "bromley_2.7": bromley(eta, Re, Pr, Ja),
        "epstein_hauser_0.537": mode2(0.537, gamma, eta, Re, Pr, Ja),
        "epstein_hauser_1.13": mode2(1.13, gamma, eta, Re, Pr, Ja),
        "ito_0.46": mode2(0.46, gamma, eta, Re, Pr, Ja),
        "ito_0.48": mode2(0.48, gamma, eta, Re, Pr, Ja),
        "ito_0.51": mode2(0.51, gamma, eta, Re, Pr, Ja),
    }


def paper_case(dT, Re, seed, a=3.0 / 49.0, b=2.0 / 21.0, R=1.0, D=30.0, u_l=0.05, Tr=0.86, warmup=3000, rho_s=0.0,
               Pr_l=0.862, Pr_v=1.5):
    """One domain of the sweep; dT in lattice temperature units; rho_s the density that sets the
    solid's psi (0: rho_l, a liquid-wetting wall; the paper does not state it); Pr_l, Pr_v the
    Prandtl numbers (Pr_v = 1.5e-3 for the low-Prandtl study of Sec. IV.C)."""
    Tc = 0.0778 * a / (0.4572 * b * R)  # Peng-Robinson critical temperature (Sec. II.C)
    H, W = 45.0 * D, 20.0 * D
    return SimpleNamespace(
        nx=int(H), ny=int(W), D=D, xc=0.2 * H, yc=0.5 * W, periodic_x=0, walls=0, superheat_Tc=dT / Tc, rho_s=rho_s,
        a=a, b=b, R=R, acentric=0.344, G=-2.0, sigma=0.38, Tr_sat=Tr, Re=Re, u_in=u_l, nu_l=0.0, nu_ratio=1.0,
        Pr_l=Pr_l, Pr_v=Pr_v, c_v=11.0, g=-1.0, U_out=-1.0, warmup=warmup, energy=1, seed=seed, noise_amp=1e-4,
        psi_mode=0, wall_dT=(), body_fx=0.0)


def run(Re, dTs, steps, warmup=3000, rho_s=0.0, Pr_l=0.862, Pr_v=1.5):
    """A domain whose state turns non-finite is reported as such (status), the others go on."""
    cases = [paper_case(dT, Re, seed=k + 1, warmup=warmup, rho_s=rho_s, Pr_l=Pr_l, Pr_v=Pr_v)
             for k, dT in enumerate(dTs)]
    b = Batch(cases)
    status = ["ok"] * len(cases)
    t0 = time.perf_counter()
    first = warmup + (steps - warmup) // 2
    b.step(first)
    for i in range(len(cases)):
        try:
            b.domain(i).reset_heat_flux()  # average over the second half of the post-warm-up run
        except LbmError as e:
            status[i] = f"failed before step {first}: {e}"
    b.step(steps - first)
    b._torch.cuda.current_stream().synchronize()
    seconds = time.perf_counter() - t0
    info = b.domain(0).info()
    gamma = info["rho_l"] / info["rho_v"]
    eta = info["nu_l"] / info["nu_v"]
    Pr = info["nu_v"] / info["alpha_v"]
    c_p = cases[0].c_v
    points = []
    for i, dT in enumerate(dTs):
        Ja = c_p * dT / info["h_fg"]
        point = {"dT": dT, "Ja": Ja, "status": status[i], "correlations": correlations(gamma, eta, Re, Pr, Ja)}
        if status[i] == "ok":
            try:
                hf = b.domain(i).heat_flux()
                point.update(q_mean=hf["q_mean"], q_std=hf["q_std"], Nu=hf["nu_mean"], samples=hf["count"])
            except LbmError as e:
                point["status"] = f"failed after step {first}: {e}"
        points.append(point)
    nodes = sum(c.nx * c.ny for c in cases)
    b.close()
    return {"Re": Re, "steps": steps, "warmup": warmup, "domain": [cases[0].nx, cases[0].ny], "D": cases[0].D,
            "rho_s": rho_s if rho_s > 0 else info["rho_l"], "Pr_l": Pr_l, "Pr_v": Pr_v,
            "gamma": gamma, "eta": eta, "Pr": Pr, "h_fg": info["h_fg"], "lambda_v": info["lambda_v"],
            "seconds": seconds, "mlups": nodes * steps / seconds / 1e6, "points": points}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--Re", type=float, default=30.0)
    ap.add_argument("--steps", type=int, default=100000)
    ap.add_argument("--warmup", type=int, default=3000)
    ap.add_argument("--rho-s", type=float, default=0.0, help="density of the solid's psi (0: rho_l)")
    ap.add_argument("--Pr-l", type=float, default=0.862, help="liquid Prandtl number")
    ap.add_argument("--Pr-v", type=float, default=1.5, help="vapour Prandtl number (1.5e-3: the low-Prandtl study)")
    ap.add_argument("--dT", type=float, nargs="*", default=[round(0.005 * k, 3) for k in range(1, 14)],
                    help="superheats in lattice units (default 0.005 .. 0.065, the paper's range)")
    a = ap.parse_args()
    print(json.dumps(run(a.Re, a.dT, a.steps, a.warmup, a.rho_s, a.Pr_l, a.Pr_v)))


if __name__ == "__main__":
    main()
