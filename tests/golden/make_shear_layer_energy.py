"""Writes shear_layer_energy_L512.json: the FP64 oracle's normalised kinetic energy E(t)/E(0) of the
double shear layer of Sec. III.B (L = 512, Re = 3e4, Ma = 0.1, 0.3, 0.6) for the CM collision and
the BGK operator, at t/t0 = 0.1, 0.2, ..., 1.0 (t0 = L / u0, step counts rounded to the nearest
integer), with the interval in which a run became unstable.  Calls only the oracle; about 15
minutes on 8 cores.

    python tests/golden/make_shear_layer_energy.py
"""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", ".."))
import synthetic_inputs as si  # noqa: E402
from oracle import Oracle  # noqa: E402

L, RE, SAMPLES = 512, 3.0e4, 10


def energy(o):
    r, a, b = o.field("rho"), o.field("ux"), o.field("uy")
    return float(0.5 * (r * (a * a + b * b)).sum())


def main():
    runs = []
    for Ma in (0.1, 0.3, 0.6):
        ux, uy = si.shear_layer_velocity(L, Ma)
        t0 = L / (Ma / np.sqrt(3.0))
        for op in (0, 1):
            o = Oracle(si.shear_layer_case(L, Ma, RE, collision=op), rho=np.ones((L, L)), ux=ux, uy=uy)
            E0 = float(0.5 * (ux * ux + uy * uy).sum())
            t, E, status, done = [], [], "ok", 0
            for k in range(1, SAMPLES + 1):
                n = int(round(k / SAMPLES * t0)) - done
                o.step(n)
                done += n
                e = energy(o) / E0
                r = o.field("rho")
                if not np.isfinite(e) or not (r.min() > 0):
                    status = f"unstable between t/t0 = {(k - 1) / SAMPLES:.1f} and {k / SAMPLES:.1f}"
                    break
                t.append(done / t0)
                E.append(e)
            runs.append({"Ma": Ma, "collision": "bgk" if op else "cm", "t_over_t0": t, "E_over_E0": E,
                         "status": status})
            print(runs[-1]["Ma"], runs[-1]["collision"], status, flush=True)
    out = {"source": "FP64 oracle (oracle/lbm_oracle.c), tests/golden/make_shear_layer_energy.py",
           "L": L, "Re": RE, "runs": runs}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "shear_layer_energy_L512.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
