"""Population-storage precision study on one GPU.

Runs one workload with populations stored as FP64, FP32 and shifted FP16 (all with FP32
arithmetic, psi in double-float, heat flux accumulated in FP64) and with the FP64 build as
the reference, and reports, at checkpoints, the relative max-norm error of rho, T and |u|
against the reference, and the time-averaged wall Nusselt number of each run.

    python -m paper_1912_02018_gb300.precision_study --nx 2048 --ny 1024 --D 128 --Re 30000 \\
        --superheat 0.2 --steps 50000 --every 10000 --warmup 12800

Prints one JSON document.  Lattice units; the cylinder sits at (nx/4, ny/2).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from .sim import Sim


def run(nx, ny, D, Re, superheat, steps, every, warmup, seed=0, noise=1e-4):
    common = dict(D=D, xc=nx / 4.0, yc=ny / 2.0, Re=Re, superheat_Tc=superheat, warmup=warmup, seed=seed,
                  noise_amp=noise)
    variants = {"f64_build": dict(f64=True), "f64_store": dict(storage="f64"), "f32_store": dict(storage="f32"),
                "f16s_store": dict(storage="f16s")}
    sims = {k: Sim(nx, ny, **common, **v) for k, v in variants.items()}
    out = {"workload": dict(nx=nx, ny=ny, D=D, Re=Re, superheat_Tc=superheat, steps=steps, warmup=warmup),
           "checkpoints": [], "seconds": {}}
    done = 0
    avg_started = False
    while done < steps:
        n = min(every, steps - done)
        for k, s in sims.items():
            t = time.perf_counter()
            s.step(n).sync()
            out["seconds"][k] = out["seconds"].get(k, 0.0) + time.perf_counter() - t
        done += n
        if not avg_started and done >= warmup + (steps - warmup) // 2:
            for s in sims.values():
                s.reset_heat_flux()  # average over the second half of the post-warm-up run
            avg_started = True
        ref = sims["f64_build"].fields(("rho", "ux", "uy", "T", "solid"))
        fluid = ref["solid"] == 0
        speed = np.hypot(ref["ux"], ref["uy"])[fluid].max()
        cp = {"step": done}
        for k, s in sims.items():
            if k == "f64_build":
                continue
            f = s.fields(("rho", "ux", "uy", "T"))
            cp[k] = {
                "rho": float(np.abs(f["rho"] - ref["rho"])[fluid].max() / np.abs(ref["rho"][fluid]).max()),
                "T": float(np.abs(f["T"] - ref["T"])[fluid].max() / np.abs(ref["T"][fluid]).max()),
                "u": float(np.hypot(f["ux"] - ref["ux"], f["uy"] - ref["uy"])[fluid].max() / speed),
            }
        out["checkpoints"].append(cp)
    out["nusselt"] = {k: s.heat_flux() for k, s in sims.items()}
    nref = out["nusselt"]["f64_build"]["nu_mean"]
    out["nusselt_drift"] = {k: (v["nu_mean"] - nref) / nref if nref else None for k, v in out["nusselt"].items()}
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--nx", type=int, default=2048)
    ap.add_argument("--ny", type=int, default=1024)
    ap.add_argument("--D", type=float, default=128.0)
    ap.add_argument("--Re", type=float, default=30000.0)
    ap.add_argument("--superheat", type=float, default=0.2)
    ap.add_argument("--steps", type=int, default=50000)
    ap.add_argument("--every", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=12800)
    a = ap.parse_args()
    print(json.dumps(run(a.nx, a.ny, a.D, a.Re, a.superheat, a.steps, a.every, a.warmup)))


if __name__ == "__main__":
    main()
