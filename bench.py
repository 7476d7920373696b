#!/usr/bin/env python
"""Throughput of the boiling-LBM time step on GB300, printed as one JSON line.

A step is one full lattice update of the workload (pull-streaming with boundary
substitutions, rho/psi, interaction force, CM collision, wall heat flux, two Runge-Kutta
stages of the temperature equation).  Default workload: the largest single domain of the
measurement plan, 2048 x 1024 lattice, cylinder D = 128 at (512, 512), Re = 30000, film-boiling
superheat 0.20 Tc, FP32 (the 1536 x 768 paper-shaped domain is --workload paper_shaped).

  value      MLUPS over the K timed steps, inputs resident in HBM, L2 flushed (a 256 MB
             write) before every timed step; CUDA events on the library's stream.
  e2e        the same metric through the C ABI with host buffers: each step takes its state
             from pinned host memory (the context's own formats; staged on the context's copy
             stream while the step before runs, lbm_stage_state_native / lbm_take_staged),
             steps once and reads T back in its own format (lbm_get_state_native) plus the heat
             flux; sync_restore_value: the same with the synchronous lbm_set_state_native.
  roofline   the dominant kernel's algorithmic bytes per launch / its mean event-timed
             duration, against the measured HBM copy bandwidth (the kernels' durations come
             from a second pass of the K steps with an event pair around every kernel).
  adjoint    cost of the checkpointed adjoint window (512 x 256, D = 32, 500 steps,
             checkpoint every 50) relative to the forward window, FP32 (adjoint) and FP64
             (adjoint_f64) builds.
  probe      the 8192 x 4096 roofline probe (step MLUPS and HBM fraction).
  batch      the 64-domain boiling-curve sweep, batched against sequential contexts.
  cpu_baseline  the FP64 CPU oracle on a bounded number of steps of the same workload.

--impl reference times that oracle alone (the reference arm for this method: the
paper ships no code).  Under torchrun (N > 1) every rank runs its own replica
(replicas only: the method has no data-path exchange between independent domains).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synthetic_inputs as si  # noqa: E402

METRIC = "MLUPS and % HBM roofline per boiling step; adjoint/forward cost ratio"
UNIT = "MLUPS"
WORKLOADS = {
    "paper_shaped": si.PAPER_SHAPED.replace(warmup=0, name="1536x768_D96_Re300_dT0.10Tc_fp32"),
    "precision": si.PRECISION.replace(warmup=0, name="2048x1024_D128_Re30000_dT0.20Tc_fp32"),
    "small": si.SMALL.replace(name="128x64_D16_Re30_dT0.05Tc_fp32"),
    "probe": si.cylinder_case(8192, 4096, 512.0, Re=300.0, superheat_Tc=0.1, name="8192x4096_D512_probe_fp32"),
    # the double shear layer of Sec. III.B (single phase, collision pass only) with each operator
    "shear512_cm": si.shear_layer_case(512, 0.3, collision=0).replace(name="shear_layer_L512_Ma0.3_Re3e4_cm_fp32"),
    "shear512_bgk": si.shear_layer_case(512, 0.3, collision=1).replace(name="shear_layer_L512_Ma0.3_Re3e4_bgk_fp32"),
}


def workload_init(case):
    """Initial fields of a workload (None: the library's default state with the seeded noise)."""
    if case.name.startswith("shear_layer"):
        ux, uy = si.shear_layer_velocity(case.nx, 0.3)
        return {"rho": np.ones((case.ny, case.nx)), "ux": ux, "uy": uy}
    return {"drho": case.drho()}
# Algorithmic bytes per lattice update of each kernel (FP32 compute; POP bytes per stored
# population): the values a kernel must read and write by its contract, each once.
POP = {"f32": 4, "f64": 8, "f16s": 2}[next((a.split("=", 1)[1] for a in sys.argv if a.startswith("--storage=")),
                                           sys.argv[sys.argv.index("--storage") + 1] if "--storage" in sys.argv else "f32")]
ALG_BYTES = {
    "k_rho_psi": 9 * POP + 4 + 4,           # f, T in; psi out
    "k_collide": 9 * POP + 4 + 9 * POP + 12,  # f, psi in; f*, rho, ux, uy out (no psi when single phase)
    # T, rho, ux, uy in; T out; and psi of the next step: the new populations in, psi out
    "k_energy": 4 * 4 + 4 + 9 * POP + 4,
}
STEP_ALG_BYTES = 9 * POP * 2 + 4 * 2      # the whole step: populations and T in and out
KERNEL_SRCS = [os.path.join(ROOT, "paper_1912_02018_gb300", "csrc", n) for n in ("lbm_kernels.cuh", "lbm_tma.cuh")]


def kernel_hash() -> str:
    """Hash of the step kernels' sources (the TMA staging included)."""
    h = hashlib.sha256()
    for p in KERNEL_SRCS:
        h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_traffic(kernel: str, workload: str):
    """Per-launch DRAM bytes from a committed ncu summary, if its kernel hash is current."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not h or not t or h.group(1) != kernel_hash():
        return None
    return float(t.group(1))


class Clocks:
    """nvidia-smi sampler (every 50 ms) for SM clock and throttle reasons."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.rows = []
        self.mark = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.p = None

    def _read(self):
        for line in self.p.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.rows.append((time.time(), parts))

    def window(self, t0, t1):
        if self.p:
            time.sleep(0.5)
            self.p.terminate()
        rows = [r for t, r in self.rows if t0 <= t <= t1] or [r for _, r in self.rows]
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[0]) for r in rows if num(r[0]) is not None]
        mx = [num(r[1]) for r in rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[3 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_sample(case, budget_s: float, max_steps: int):
    """Time the FP64 oracle on the full workload for as many steps as fit in budget_s."""
    from oracle import Oracle

    o = Oracle(case, **workload_init(case))
    t = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter() - t
    n = max(1, min(max_steps - 1, int(budget_s / max(t1, 1e-6)) - 1))
    t = time.perf_counter()
    o.step(n)
    dt = time.perf_counter() - t
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    if os.environ.get("OMP_NUM_THREADS"):
        cores = min(cores, int(os.environ["OMP_NUM_THREADS"]))
    mlups = case.nx * case.ny * n / dt / 1e6
    return {"value": mlups, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} FP64 oracle steps of the full {case.nx}x{case.ny} workload after 1 untimed step "
                      f"({dt:.2f} s)"}, dt / n * 1e3, n


def workload_config(case, args) -> dict:
    """The `config` of a bench line: the same keys for the GPU arm and the oracle (reference) arm."""
    return {"workload": case.name, "nx": case.nx, "ny": case.ny, "D": case.D, "Re": case.Re,
            "superheat_Tc": case.superheat_Tc, "G": case.G, "sigma": case.sigma, "storage": args.storage,
            "psi": ["double-float (FP32 pairs)", "IEEE f64", "f32"][args.psi_mode],
            "l2": "flushed (256 MB write) before every timed step", "parallelism": "replicas"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    case = WORKLOADS[args.workload]
    cpu, ms_per_step, n = oracle_sample(case, budget_s=min(120.0, 6.0 * max(args.steps, 1)), max_steps=args.steps + 1)
    line = {"impl": "reference", "metric": METRIC, "value": cpu["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": n, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(case, args),
            "cpu_baseline": cpu,
            "e2e": {"value": cpu["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def batch_sweep_record(steps: int, warmup: int) -> dict:
    """The 64-domain boiling-curve sweep batched (tuned tiles, CUDA graph) against the same
    domains stepped one after another through their own contexts (MLUPS of each, CUDA events)."""
    import torch

    from paper_1912_02018_gb300 import Batch, Sim

    cases = si.batch_sweep(64, seed=1)
    nodes = sum(c.nx * c.ny for c in cases)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b = Batch(cases)
    variant = b.tune(2)
    b.step(warmup)
    torch.cuda.synchronize()
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1)
    b.sync()
    b.close()
    sims = [Sim.from_case(c) for c in cases]
    for _ in range(warmup):
        for s in sims:
            s.step(1)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        for s in sims:
            s.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1)
    for s in sims:
        s.sync()
        s.close()
    return {"workload": "sweep64_12Dx6D_D40-128_Re300_fp32", "domains": len(cases), "nodes": nodes,
            "steps": steps, "warmup": warmup, "tile_variant": variant,
            "batched_mlups": nodes * steps / (ms_b / 1e3) / 1e6, "batched_ms_per_step": ms_b / steps,
            "sequential_mlups": nodes * steps / (ms_s / 1e3) / 1e6, "sequential_ms_per_step": ms_s / steps,
            "speedup_vs_sequential": ms_s / ms_b}


def run_batch(args):
    """Boiling-curve sweep: 64 independent domains, batched (tuned tiles, CUDA graph) against the
    same 64 domains stepped one after another through their own contexts."""
    import torch

    from paper_1912_02018_gb300 import Batch, Sim

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    cases = si.batch_sweep(64, seed=1)
    nodes = sum(c.nx * c.ny for c in cases)
    stream = torch.cuda.current_stream()
    b = Batch(cases)
    variant = b.tune(2)
    b.step(args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1)
    b.close()
    sims = [Sim.from_case(c) for c in cases]
    for _ in range(args.warmup):
        for s in sims:
            s.step(1)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        for s in sims:
            s.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1)
    line = {"metric": METRIC, "value": nodes * args.steps / (ms_b / 1e3) / 1e6, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "sweep64_12Dx6D_D40-128_Re300", "domains": len(cases), "nodes": nodes,
                       "l2": "inputs larger than L2", "tile_variant": variant},
            "sequential": {"value": nodes * args.steps / (ms_s / 1e3) / 1e6, "ms_per_step": ms_s / args.steps},
            "speedup_vs_sequential": ms_s / ms_b}
    print(json.dumps(line), flush=True)
    return 0


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest of the ranks' values (replica timing: the job is as slow as its slowest rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(nodes: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job throughput of `world` replicas that each updated `nodes` nodes `steps` times."""
    return nodes * steps * world / seconds / 1e6


def probe_record(args, steps: int = 10, warmup: int = 3) -> dict:
    """The 8192 x 4096 roofline probe (D = 512, 33.5 M nodes, far larger than L2): step MLUPS and
    the HBM fraction of the step's algorithmic bytes, per-kernel mean event times."""
    import torch

    from paper_1912_02018_gb300 import Sim

    case = WORKLOADS["probe"]
    nodes = case.nx * case.ny
    sim = Sim.from_case(case, f64=False, storage=args.storage, psi_mode=args.psi_mode)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        sim.step(1)
    sim.sync()
    ms = {}
    for per_kernel in (False, True):  # the timed steps, then the same steps with per-kernel events
        sim.profile(per_kernel)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        sim.sync()
        ms[per_kernel] = e0.elapsed_time(e1)
    prof = sim.profile_read()
    ms = ms[False]
    sim.close()
    peak, kind = measured_peaks()
    gbs = STEP_ALG_BYTES * nodes * steps / (ms / 1e3) / 1e9
    return {"workload": case.name, "nodes": nodes, "steps": steps, "warmup": warmup,
            "mlups": nodes * steps / (ms / 1e3) / 1e6, "ms_per_step": ms / steps,
            "step_alg_bytes_per_lup": STEP_ALG_BYTES, "achieved_gbs": gbs, "frac": gbs / peak,
            "peak_kind": f"{kind} copy bandwidth",
            "kernels_us": {k: v[1] / v[0] * 1e3 for k, v in prof.items() if v[0]},
            "l2": "inputs (3.7 GB) far larger than L2; no flush"}


def adjoint_cost(window=500, ckpt_every=50, spin_up=2000, f64=False):
    """Cost of the adjoint window against the forward steps it differentiates, on the
    512 x 256 lattice, D = 32, Re = 300 (FP32 or, with f64, FP64 forward and adjoint fields;
    FP64 parameter sums): forward = lbm_step over the window; adjoint = lbm_adjoint_window (its
    own checkpointed forward pass, then segment recompute and reverse steps)."""
    import ctypes as C

    import torch

    from paper_1912_02018_gb300 import Sim
    from paper_1912_02018_gb300 import _native as N

    case = si.ADJOINT
    sim = Sim.from_case(case, f64=f64).step(spin_up)
    state = sim.get_state()
    stream = torch.cuda.current_stream()
    L = N.lib()
    res = {}
    for rep in range(2):  # the first pass allocates the adjoint buffers
        sim.set_state(*state)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        torch.cuda.synchronize()
        e[0].record(stream)
        sim.step(window)
        e[1].record(stream)
        sim.set_state(*state)
        g = N.WindowGrad()
        torch.cuda.synchronize()
        e[2].record(stream)
        N.check(L.lbm_adjoint_window(sim.h, window, ckpt_every, C.byref(g)), sim.h)
        e[3].record(stream)
        torch.cuda.synchronize()
        fwd, adj = e[0].elapsed_time(e[1]), e[2].elapsed_time(e[3])
        res = {"workload": case.name, "precision": "f64" if f64 else "f32", "window": window,
               "ckpt_every": ckpt_every, "spin_up": spin_up,
               "forward_ms": fwd, "adjoint_window_ms": adj, "reverse_ms": adj - fwd,
               "ratio": (adj - fwd) / fwd, "ratio_incl_forward": adj / fwd, "J": g.J,
               "dJ_dsuperheat": g.dJ_dsuperheat, "dJ_du_in": g.dJ_du_in,
               "note": "ratio = (adjoint window - forward window) / forward window; L2-resident lattice"}
    sim.close()
    return res


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1912_02018_gb300 import Sim

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    case = WORKLOADS[args.workload]
    nodes = case.nx * case.ny
    init = workload_init(case) if case.name.startswith("shear_layer") else None  # else made on the device
    sim = Sim.from_case(case, f64=False, storage=args.storage, psi_mode=args.psi_mode, init=init)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    clocks = Clocks(local) if rank == 0 else None
    for _ in range(args.warmup):
        flush.zero_()
        sim.step(1)
    sim.sync()

    def timed_steps(per_kernel):
        # K steps, each after the L2 flush, one event pair per step on the library's stream;
        # with per_kernel the library also brackets every kernel with an event pair
        sim.profile(per_kernel)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        w0 = time.time()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            sim.step(1)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        w1 = time.time()
        if world > 1:
            dist.barrier()
        sim.sync()
        return sum(a.elapsed_time(b) for a, b in ev), w0, w1

    # the timed region carries no per-kernel events: an event between the step's two passes
    # costs time and stops the energy pass from starting while the collision ends
    launches0 = sim.info()["kernel_launches"]
    ms, t_wall0, t_wall1 = timed_steps(False)
    launches = sim.info()["kernel_launches"] - launches0
    # per-kernel durations: the same K steps once more, every kernel between its own events
    ms_k, _, _ = timed_steps(True)
    prof = sim.profile_read()
    sim.profile(False)
    ms = max_over_ranks(ms, world)
    ms_k = max_over_ranks(ms_k, world)
    value = aggregate_mlups(nodes, args.steps, world, ms / 1e3)

    # end to end through the C ABI with pinned host buffers: every step takes its state from
    # host memory in the context's own formats and reads the new T back in its own format too,
    # plus the heat flux.  The state of step i + 1 is staged (copied on the context's copy
    # stream, lbm_stage_state_native) while step i runs, then swapped in (lbm_take_staged);
    # e2e_sync repeats the loop with the synchronous restore (lbm_set_state_native)
    f0, T0, side0, n0 = sim.get_state_native()
    f_h = torch.from_numpy(f0).pin_memory()
    T_h = torch.from_numpy(T0).pin_memory()
    out_h = torch.empty_like(T_h).pin_memory()
    from paper_1912_02018_gb300 import _native as N

    L = N.lib()
    e2e_steps = max(1, min(args.steps, 50))

    def e2e_run(staged):
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t = time.perf_counter()
        if staged:
            N.check(L.lbm_stage_state_native(sim.h, f_h.data_ptr(), T_h.data_ptr(), None, -1), sim.h)
        for i in range(e2e_steps):
            if staged:
                N.check(L.lbm_take_staged(sim.h), sim.h)
            else:
                N.check(L.lbm_set_state_native(sim.h, f_h.data_ptr(), T_h.data_ptr(), None, -1), sim.h)
            N.check(L.lbm_step(sim.h, 1), sim.h)
            if staged and i + 1 < e2e_steps:
                N.check(L.lbm_stage_state_native(sim.h, f_h.data_ptr(), T_h.data_ptr(), None, -1), sim.h)
            N.check(L.lbm_get_state_native(sim.h, None, out_h.data_ptr(), None, None), sim.h)
            sim.heat_flux()
        return max_over_ranks(time.perf_counter() - t, world)

    e2e_run(True)  # the first staging allocates the staging buffers
    e2e_s = e2e_run(True)
    e2e_sync_s = e2e_run(False)
    e2e = {"value": aggregate_mlups(nodes, e2e_steps, world, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": int(f_h.numel() * f_h.element_size() + T_h.numel() * T_h.element_size()),
           "d2h_bytes_per_step": int(out_h.numel() * out_h.element_size() + 5 * 8), "steps": e2e_steps,
           "restore": "staged: step i + 1's state is copied on the context's copy stream while step i runs",
           "sync_restore_value": aggregate_mlups(nodes, e2e_steps, world, e2e_sync_s)}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    clk = clocks.window(t_wall0, t_wall1) if clocks else None
    peak, peak_kind = measured_peaks()
    ours = {k: v for k, v in prof.items() if v[0] > 0}
    dom = max(ours, key=lambda k: ours[k][1])
    per_launch_ms = ours[dom][1] / ours[dom][0]
    alg_lup = ALG_BYTES.get(dom, 0) - (4 if (dom == "k_collide" and case.G == 0) else 0)
    alg = alg_lup * nodes
    achieved = alg / (per_launch_ms / 1e3) / 1e9
    traffic = ncu_traffic(dom, args.workload)
    kernels = {k: {"launches": v[0], "ms_total": round(v[1], 4), "share": round(v[1] / sum(x[1] for x in ours.values()), 4),
                   "alg_bytes_per_lup": (alg_lup if k == dom else ALG_BYTES.get(k))} for k, v in ours.items()}
    step_bytes = STEP_ALG_BYTES if case.energy else 9 * POP * 2  # populations (and T when it evolves) in and out
    step_gbs = step_bytes * nodes * args.steps / (ms / 1e3) / 1e9 / world
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(case, args),
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": f"{peak_kind} copy bandwidth",
                     "alg_bytes_per_launch": alg},
        "step_roofline": {"alg_bytes_per_lup": step_bytes, "achieved_gbs": step_gbs, "frac": step_gbs / peak},
        "kernels": kernels, "gpu_launches": launches, "e2e": e2e, "clocks": clk,
        "kernel_timing": {"steps": args.steps, "ms_per_step": ms_k / args.steps,
                          "note": "kernels' event-timed durations come from a second pass of the same K flushed "
                                  "steps with an event pair around every kernel (its per-step time here); the "
                                  "timed region above has one event pair per step"},
    }
    if world == 1 and not args.no_adjoint:
        line["adjoint"] = adjoint_cost()
        line["adjoint_f64"] = adjoint_cost(f64=True)
    if world == 1 and args.workload == "precision" and not args.no_probe:
        line["probe"] = probe_record(args)
    if world == 1 and not args.no_batch:
        line["batch"] = batch_sweep_record(steps=60, warmup=6)
    if world == 1 and not args.no_cpu_baseline:
        cpu, _, _ = oracle_sample(case, budget_s=args.cpu_seconds, max_steps=10 ** 6)
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["sweep64"], default="precision")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint-window cost measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-domain batched-sweep record")
    ap.add_argument("--no-probe", action="store_true", help="skip the 8192 x 4096 roofline-probe record")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--storage", default="f32", choices=("f32", "f64", "f16s"),
                    help="population storage of the FP32 build (shifted FP16: f - w rho_l)")
    ap.add_argument("--psi-mode", type=int, default=0, choices=(0, 1, 2),
                    help="psi evaluation of the FP32 build: 0 double-float (default), 1 IEEE FP64, 2 FP32")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "sweep64":
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
