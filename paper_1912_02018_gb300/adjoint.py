"""torch.autograd face of the adjoint window (lbm_adjoint_window in include/lbm.h).

heat_flux_window(...) returns J, the mean wall heat flux (Sec. IV.B) over a window of n steps
from a given state, as a 0-d tensor whose backward gives dJ/d(superheat_Tc, u_in, wall_dT)
from the library's discrete adjoint (checkpoint every ckpt_every steps, recompute between).
The forward and the reverse pass both run in the CUDA library; this module only marshals.
"""
from __future__ import annotations

import numpy as np
import torch

from .sim import Sim


def fixed_transport(case, f64=False) -> dict:
    """nu_l, g and the outlet speed the library derives for `case`, as explicit parameters, so
    that u_in then enters only through the inlet condition."""
    s = Sim.from_case(case.replace(wall_dT=()) if getattr(case, "wall_dT", ()) else case, f64=f64)
    info = s.info()
    s.close()
    return {"nu_l": info["nu_l"], "g": info["g"], "U_out": info["outlet_U"]}


class HeatFluxWindow(torch.autograd.Function):
    """J(superheat, u_in, wall_dT) over a window; backward from the adjoint window."""

    @staticmethod
    def forward(ctx, superheat, u_in, wall_dT, spec):
        case = spec["case"].replace(superheat_Tc=float(superheat), u_in=float(u_in),
                                    wall_dT=tuple(float(v) for v in wall_dT.detach().cpu().reshape(-1)),
                                    **spec["fixed"])
        f, T, side, steps = spec["state"]
        sim = Sim.from_case(case, f64=spec["f64"])
        sim.set_state(f, T, side, steps)
        g = sim.adjoint_window(spec["n"], spec["ckpt_every"])
        sim.close()
        ctx.grads = (g["superheat"], g["u_in"], np.asarray(g["wall_dT"]))
        ctx.knot_shape = wall_dT.shape
        return torch.tensor(g["J"], dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        dsh, du, dk = ctx.grads
        gk = torch.as_tensor(dk, dtype=torch.float64).reshape(ctx.knot_shape) * gJ
        return gJ * dsh, gJ * du, gk, None


def heat_flux_window(case, state, n, ckpt_every=50, superheat=None, u_in=None, wall_dT=None, f64=False,
                     fixed=None):
    """J as a differentiable tensor.  state = (f*, T, side, steps) as Sim.get_state returns it;
    superheat, u_in, wall_dT: tensors (requires_grad as wanted) or None for the case's values;
    fixed: explicit nu_l, g, U_out (default: the values derived for `case`)."""
    superheat = torch.as_tensor(case.superheat_Tc if superheat is None else superheat, dtype=torch.float64)
    u_in = torch.as_tensor(case.u_in if u_in is None else u_in, dtype=torch.float64)
    wall_dT = torch.as_tensor(case.wall_dT if wall_dT is None else wall_dT, dtype=torch.float64)
    spec = {"case": case, "state": state, "n": int(n), "ckpt_every": int(ckpt_every), "f64": bool(f64),
            "fixed": fixed if fixed is not None else fixed_transport(case, f64)}
    return HeatFluxWindow.apply(superheat, u_in, wall_dT, spec)
