"""The experiment drivers' own bookkeeping (set-up, sampling, fits), run end to end with the FP64
oracle standing in for the CUDA context: a stand-in with the calls the drivers make (from_case,
info, step, fields, close).  The CUDA path itself is held to the oracle by the GPU parity tests."""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import Oracle, stepper


class OracleSim:
    """Sim's driver-facing calls over the oracle (test infrastructure)."""

    def __init__(self, case, init=None):
        fields = {k: getattr(case, k) for k in si.Case.__dataclass_fields__ if hasattr(case, k)}
        fields["wall_dT"] = tuple(fields.get("wall_dT", ()) or ())
        self.case = si.Case(**fields)
        _, self.d = stepper.derive(self.case)
        init = dict(init or {})
        if not any(k in init for k in ("rho", "drho")):
            init["drho"] = self.case.drho()
        self.o = Oracle(self.case, **init)

    @classmethod
    def from_case(cls, case, f64=False, init=None, **kw):
        return cls(case, init)

    def info(self):
        d = self.d
        return {"Tc": d.Tc, "T_sat": d.T_sat, "T_wall": d.T_wall, "rho_l": d.rho_l, "rho_v": d.rho_v,
                "p_sat": d.eos.p(d.rho_l, d.T_sat), "h_fg": d.eos.h_fg(d.T_sat), "nu_l": d.nu_l, "nu_v": d.nu_v,
                "alpha_v": d.alpha_v, "lambda_v": d.lambda_v}

    def step(self, n=1):
        self.o.step(n)
        return self

    def fields(self, names=("rho", "ux", "uy", "T", "psi")):
        return {k: self.o.field(k) for k in names}

    def close(self):
        pass


@pytest.mark.slow
def test_stefan_driver_on_the_oracle_gives_welch_beta(monkeypatch):
    from paper_1912_02018_gb300 import stefan

    monkeypatch.setattr(stefan, "Sim", OracleSim)
    out = stefan.run(0.86, 0.023, steps=20000, every=1000)
    assert out["y_i"][-1] > out["y_i"][0] + 5.0
    assert abs(out["beta_sim"] / out["beta_welch"] - 1.0) < 0.15, out["beta_sim"]


def test_bubble_growth_driver_on_the_oracle(monkeypatch):
    from paper_1912_02018_gb300 import bubble_growth

    monkeypatch.setattr(bubble_growth, "Sim", OracleSim)
    out = bubble_growth.run(N=96, steps=600, every=200)
    assert len(out["R"]) == 4 and abs(out["R"][0] - 15.0) < 0.5 and out["R"][-1] > 13.0
    assert out["plesset_zwick_R2_slope"] > 0 and np.isfinite(out["R2_slope"])


def test_shear_layer_driver_on_the_oracle(monkeypatch):
    from paper_1912_02018_gb300 import shear_layer

    monkeypatch.setattr(shear_layer, "Sim", OracleSim)
    out = shear_layer.run(64, 0.3, 5000.0, 1, t_end=0.2, samples=2)
    assert out["status"] == "ok" and len(out["E_over_E0"]) == 2
    # the same run straight on the oracle
    ux, uy = si.shear_layer_velocity(64, 0.3)
    c = si.shear_layer_case(64, 0.3, Re=5000.0, collision=1)
    o = Oracle(c, rho=np.ones((64, 64)), ux=ux, uy=uy).step(out["steps"])
    r, a, b = o.field("rho"), o.field("ux"), o.field("uy")
    E = 0.5 * (r * (a * a + b * b)).sum() / (0.5 * (ux * ux + uy * uy).sum())
    assert abs(out["E_over_E0"][-1] - E) < 1e-12
