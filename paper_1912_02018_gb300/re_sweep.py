"""Reynolds-number and superheat sweep of the time-averaged wall Nusselt number on a 1536 x 768
domain with a cylinder of D = 96 (the set-up of Sec. IV.A at 3.2 times the paper's D = 30).

The 16 cases are Re in {30, 300, 3000, 30000}, set by the liquid viscosity nu_l = u_in D / Re at
u_in = 0.05, times wall superheat in {0.02, 0.05, 0.10, 0.20} T_c.  Constants as in the
benchmark workloads: a = 2/49, b = 2/21, T_r = 0.86, G = -2, sigma = 0.38, Pr_l = 0.862,
Pr_v = 1.5, c_v = 11, eta = 1, g from u_in / sqrt(g D) = 4, cylinder at (W/4, H/2) = (384, 384).
Each run starts from saturated liquid with the seeded density perturbation, takes round(5 D /
u_in) = 9600 warm-up steps without force and energy equation (Sec. IV.A), and averages the wall
heat flux over the second half of its steps (the quasi-steady window, Sec. IV.B):
Nu = <q> D / (lambda_v dT).

The FP32 build steps all 16 domains as one batch (lbm_batch_*).  --f64 I J ... repeats cases I,
J, ... (indices into the Re-major list) with the FP64 build, also as one batch, and reports the
relative drift of the FP32 <Nu> against the FP64 one.  A domain whose state turns non-finite is
reported as unstable with the step range in which that happened.

    python -m paper_1912_02018_gb300.re_sweep --steps 200000 --f64 4 5 6 7

Prints one JSON document.  Lattice units.
"""
from __future__ import annotations

import argparse
import json
import time
from types import SimpleNamespace

from ._native import LbmError
from .sim import Batch

RE = (30.0, 300.0, 3000.0, 30000.0)
SUPERHEAT_TC = (0.02, 0.05, 0.10, 0.20)


def sweep_case(Re, superheat_Tc, seed, nx=1536, ny=768, D=96.0, u_in=0.05):
    """One domain of the sweep (the fields of a workload description, as Sim.from_case reads them)."""
    return SimpleNamespace(
        nx=nx, ny=ny, D=D, xc=nx / 4.0, yc=ny / 2.0, periodic_x=0, walls=0, superheat_Tc=superheat_Tc, rho_s=0.0,
        a=2.0 / 49.0, b=2.0 / 21.0, R=1.0, acentric=0.344, G=-2.0, sigma=0.38, Tr_sat=0.86, Re=Re, u_in=u_in,
        nu_l=0.0, nu_ratio=1.0, Pr_l=0.862, Pr_v=1.5, c_v=11.0, g=-1.0, U_out=-1.0,
        warmup=int(round(5.0 * D / u_in)), energy=1, seed=seed, noise_amp=1e-4, psi_mode=0, wall_dT=(),
        body_fx=0.0)


def cases():
    return [sweep_case(Re, sh, seed=1 + 4 * i + j) for i, Re in enumerate(RE) for j, sh in enumerate(SUPERHEAT_TC)]


def run_batch(cs, steps, f64, chunk):
    """Step the domains of cs together; returns one record per domain and the run's MLUPS.  Each
    record carries the history of the wall heat flux: the mean of the samples of every chunk of
    steps after the warm-up (from the running sums the library keeps)."""
    b = Batch(cs, f64=f64)
    first = cs[0].warmup + (steps - cs[0].warmup) // 2
    status = ["ok"] * len(cs)
    hist = [[] for _ in cs]
    last = [(0.0, 0) for _ in cs]  # running sum and count of the samples since the last reset
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        n = min(chunk, steps - done, first - done if done < first else steps - done)
        b.step(n)
        done += n
        for i in range(len(cs)):
            if status[i] != "ok":
                continue
            try:
                d = b.domain(i)
                hf = d.heat_flux()
                tot, cnt = hf["q_mean"] * hf["count"], hf["count"]
                if cnt > last[i][1]:
                    hist[i].append([done, (tot - last[i][0]) / (cnt - last[i][1])])
                last[i] = (tot, cnt)
                if done == first:
                    d.reset_heat_flux()  # average over the second half of the run
                    last[i] = (0.0, 0)
            except LbmError as e:
                status[i] = f"unstable between steps {done - n} and {done}: {e}"
    b._torch.cuda.current_stream().synchronize()
    seconds = time.perf_counter() - t0
    out = []
    for i in range(len(cs)):
        rec = {"Re": cs[i].Re, "superheat_Tc": cs[i].superheat_Tc, "status": status[i], "q_history": hist[i]}
        if status[i] == "ok":
            hf = b.domain(i).heat_flux()
            rec.update(Nu_mean=hf["nu_mean"], q_mean=hf["q_mean"], q_std=hf["q_std"], samples=hf["count"])
        out.append(rec)
    nodes = sum(c.nx * c.ny for c in cs)
    b.close()
    return out, nodes * steps / seconds / 1e6, seconds


def run(steps, f64_cases=(), chunk=5000):
    cs = cases()
    fp32, mlups, secs = run_batch(cs, steps, False, chunk)
    res = {"domain": [cs[0].nx, cs[0].ny], "D": cs[0].D, "steps": steps, "warmup": cs[0].warmup,
           "window": [cs[0].warmup + (steps - cs[0].warmup) // 2, steps], "fp32_batch_mlups": mlups,
           "fp32_seconds": secs, "cases": fp32}
    if f64_cases:
        sel = [cs[i] for i in f64_cases]
        fp64, mlups64, secs64 = run_batch(sel, steps, True, chunk)
        res.update(fp64_batch_mlups=mlups64, fp64_seconds=secs64)
        for i, r in zip(f64_cases, fp64):
            rec = res["cases"][i]
            rec["fp64"] = r
            if rec["status"] == "ok" and r["status"] == "ok" and r["Nu_mean"] != 0:
                rec["fp32_vs_fp64_Nu"] = rec["Nu_mean"] / r["Nu_mean"] - 1.0
    return res


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--steps", type=int, default=200000)
    ap.add_argument("--f64", type=int, nargs="*", default=[], help="case indices to repeat with the FP64 build")
    ap.add_argument("--chunk", type=int, default=5000, help="steps between status checks (and heat-flux history points)")
    a = ap.parse_args()
    print(json.dumps(run(a.steps, tuple(a.f64), a.chunk)))


if __name__ == "__main__":
    main()
