"""Double shear layer (Sec. III.B): stability of the CM collision against the BGK operator.

A periodic L x L single-phase fluid (G = 0, T held fixed) starts from two tanh shear layers at
y/L = 1/4 and 3/4 (width 1/kappa, kappa = 80) with a transverse sine perturbation of relative
amplitude delta = 0.05; u0 = Ma c_s, nu = u0 L / Re, L = 512, Re = 3e4, Ma = 0.1, 0.3, 0.6.
The paper follows the kinetic energy E(t) = sum rho |u|^2 / 2, normalised by E(0), over
t / t0 with t0 = L / u0, for the CM collision and for the BGK operator on the same
fourth-order Hermite equilibrium: the two agree at Ma 0.1 and 0.3, and BGK blows up near
t / t0 = 0.66 at Ma 0.6 while the CM collision does not.  Both operators run on the CUDA
path (lbm_params.collision); a run whose state turns non-finite or whose density turns
non-positive is reported with the interval in which that happened.

    python -m paper_1912_02018_gb300.shear_layer --Ma 0.1 0.3 0.6 --t-end 2

Prints one JSON document.  Lattice units.
"""
from __future__ import annotations

import argparse
import json
import time
from types import SimpleNamespace

import numpy as np

from ._native import LbmError
from .sim import Sim


def paper_case(L=512, Ma=0.1, Re=3.0e4, collision=0):
    u0 = Ma / np.sqrt(3.0)
    return SimpleNamespace(
        nx=L, ny=L, D=0.0, xc=0.0, yc=0.0, periodic_x=1, walls=0, superheat_Tc=0.0, rho_s=0.0, G=0.0, sigma=0.0,
        energy=0, u_in=0.0, nu_l=u0 * L / Re, nu_ratio=1.0, g=0.0, noise_amp=0.0, warmup=0, body_fx=0.0,
        collision=collision, seed=0)


def initial_velocity(L, Ma, kappa=80.0, delta=0.05):
    """(u_x, u_y) of Sec. III.B at the nodes (x, y), 0 <= x, y < L, shape (L, L)."""
    u0 = Ma / np.sqrt(3.0)
    y, x = np.mgrid[0:L, 0:L].astype(np.float64) / L
    ux = np.where(y <= 0.5, u0 * np.tanh(kappa * (y - 0.25)), u0 * np.tanh(kappa * (0.75 - y)))
    uy = u0 * delta * np.sin(2.0 * np.pi * (x + 0.25))
    return ux, uy


def kinetic_energy(fields) -> float:
    return float(0.5 * (fields["rho"] * (fields["ux"] ** 2 + fields["uy"] ** 2)).sum())


def run(L=512, Ma=0.1, Re=3.0e4, collision=0, t_end=2.0, samples=40, f64=False):
    """E(t)/E(0) at `samples` equally spaced t/t0 in (0, t_end]; status "ok" or the interval of t/t0
    in which the run became unstable."""
    case = paper_case(L, Ma, Re, collision)
    ux, uy = initial_velocity(L, Ma)
    sim = Sim.from_case(case, f64=f64, init={"rho": np.ones((L, L)), "ux": ux, "uy": uy})
    t0 = L / (Ma / np.sqrt(3.0))
    E0 = kinetic_energy(sim.fields(("rho", "ux", "uy")))
    times, energy, status = [], [], "ok"
    done, t_prev = 0, 0.0
    t_start = time.perf_counter()
    for k in range(1, samples + 1):
        t = t_end * k / samples
        n = int(round(t * t0)) - done
        try:
            sim.step(n)
            done += n
            E = kinetic_energy(sim.fields(("rho", "ux", "uy"))) / E0
        except LbmError as e:
            status = f"unstable between t/t0 = {t_prev:.3f} and {t:.3f}: {e}"
            break
        if not np.isfinite(E):
            status = f"unstable between t/t0 = {t_prev:.3f} and {t:.3f}: kinetic energy {E}"
            break
        times.append(done / t0)
        energy.append(E)
        t_prev = t
    seconds = time.perf_counter() - t_start
    sim.close()
    return {"L": L, "Ma": Ma, "Re": Re, "collision": "bgk" if collision else "cm", "t0": t0, "steps": done,
            "status": status, "t_over_t0": times, "E_over_E0": energy, "seconds": seconds,
            "mlups": L * L * done / seconds / 1e6 if seconds > 0 else 0.0}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--L", type=int, default=512)
    ap.add_argument("--Re", type=float, default=3.0e4)
    ap.add_argument("--Ma", type=float, nargs="*", default=[0.1, 0.3, 0.6])
    ap.add_argument("--t-end", type=float, default=2.0)
    ap.add_argument("--samples", type=int, default=40)
    ap.add_argument("--f64", action="store_true")
    a = ap.parse_args()
    runs = [run(a.L, Ma, a.Re, op, a.t_end, a.samples, a.f64) for Ma in a.Ma for op in (0, 1)]
    print(json.dumps({"runs": runs}))


if __name__ == "__main__":
    main()
