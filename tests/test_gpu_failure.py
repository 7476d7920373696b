"""Failure detection on the GPU path, made without a GPU fault.

- A non-finite population written on the host (through lbm_set_state) is latched by the
  collision and reported as LBM_EUNSTABLE by the next synchronising call.
- The bounded waits of the TMA-staged tiles: the test hook lbm_inject_fault makes every staged
  tile of one pass arm its barrier without issuing a copy (nothing is ever in flight), so its
  short bounded wait runs out; the next synchronising call reports LBM_ETIMEOUT naming the pass.
In both cases a restored state clears the latch and the context then steps exactly like a fresh
context started from the same state (fields and the heat-flux sample bit-equal).
"""
import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu

CASE = si.SMALL  # 128 x 64, D = 16: 12 TMA-staged collision tiles and 4 staged energy tiles (FP32)
FIELDS = ("rho", "ux", "uy", "T", "psi")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    from paper_1912_02018_gb300 import build

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build()
    torch.cuda.set_device(0)


def _same_as_fresh(sim, state, steps, native):
    """Step `sim` and a fresh context from `state`; both must give the same bits."""
    from paper_1912_02018_gb300 import Sim

    ref = Sim.from_case(CASE, f64=sim._f64)
    (ref.set_state_native if native else ref.set_state)(*state)
    ref.step(steps).sync()
    sim.step(steps).sync()
    a, b = sim.fields(FIELDS), ref.fields(FIELDS)
    for k in FIELDS:
        assert np.array_equal(a[k], b[k]), k
    assert sim.heat_flux()["q_now"] == ref.heat_flux()["q_now"]
    ref.close()


@pytest.mark.parametrize("f64", [False, True])
def test_non_finite_population_is_reported_unstable(f64):
    from paper_1912_02018_gb300 import Sim
    from paper_1912_02018_gb300._native import LBM_EUNSTABLE, LbmError

    sim = Sim.from_case(CASE, f64=f64).step(5)
    f, T, side, n = sim.get_state()
    bad = f.copy()
    bad[3, 40, 100] = np.nan  # one population of one fluid node far from the cylinder
    sim.set_state(bad, T, side, n)
    sim.step(1)
    with pytest.raises(LbmError) as e:
        sim.sync()
    assert e.value.status == LBM_EUNSTABLE
    assert "non-finite" in str(e.value) or "radicand" in str(e.value)
    with pytest.raises(LbmError):  # latched until a state is restored
        sim.sync()
    sim.set_state(f, T, side, n)
    _same_as_fresh(sim, (f, T, side, n), 3, native=False)
    sim.close()


@pytest.mark.parametrize("kind,name", [("collide", "collision tile"), ("energy", "energy tile")])
def test_starved_tile_copies_time_out_and_the_context_recovers(kind, name):
    from paper_1912_02018_gb300 import Sim
    from paper_1912_02018_gb300._native import LBM_ETIMEOUT, LbmError

    sim = Sim.from_case(CASE, f64=False).step(5)
    state = sim.get_state_native()
    sim.inject_fault(kind)
    sim.step(1)
    with pytest.raises(LbmError) as e:
        sim.sync()
    assert e.value.status == LBM_ETIMEOUT and name in str(e.value), str(e.value)
    sim.set_state_native(*state)
    sim.sync()
    _same_as_fresh(sim, state, 4, native=True)
    # the hook covers one step only
    sim.step(2).sync()
    sim.close()


def test_inject_fault_rejects_an_unknown_kind():
    import ctypes as C

    from paper_1912_02018_gb300 import Sim
    from paper_1912_02018_gb300 import _native as N

    sim = Sim.from_case(CASE, f64=False)
    assert N.lib().lbm_inject_fault(sim.h, C.c_int32(7)) == N.LBM_EINVAL
    sim.step(1).sync()
    sim.close()
