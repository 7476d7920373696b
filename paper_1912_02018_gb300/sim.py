"""Python face of the C ABI: one simulation handle (argument marshalling only).

Every step of the boiling update runs in the CUDA kernels behind liblbm.so; this
module converts arguments, hands PyTorch's allocator and current stream to the
library, and copies results into numpy / torch arrays.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _native as N

_PARAM_DEFAULTS = dict(a=2.0 / 49.0, b=2.0 / 21.0, R=1.0, acentric=0.344, G=-2.0, sigma=0.38, Tr_sat=0.86,
                       Re=30.0, u_in=0.05, nu_l=0.0, nu_ratio=1.0, Pr_l=0.862, Pr_v=1.5, c_v=11.0, g=-1.0,
                       outlet_U=-1.0, warmup=0, energy=1, seed=0, noise_amp=1e-4, psi_mode=0, wall_dT=(),
                       body_fx=0.0, collision=0)


def _structs(nx, ny, D, xc, yc, periodic_x, superheat_Tc, rho_s, f64, storage, params, walls=0):
    kw = dict(_PARAM_DEFAULTS)
    unknown = set(params) - set(kw)
    if unknown:
        raise TypeError(f"unknown parameters {sorted(unknown)}")
    kw.update(params)
    dom = N.Domain(int(nx), int(ny), int(periodic_x), int(walls))
    cyl = N.Cylinder(float(xc), float(yc), float(D), float(superheat_Tc), float(rho_s))
    knots = np.ascontiguousarray(kw.pop("wall_dT", ()) or (), dtype=np.float64)
    if knots.size:
        cyl.wall_dT = knots.ctypes.data_as(C.POINTER(C.c_double))
        cyl.n_wall = knots.size
        cyl._keep = knots  # copied by the library at creation
    prm = N.Params(a=kw["a"], b=kw["b"], R=kw["R"], acentric=kw["acentric"], G=kw["G"], sigma=kw["sigma"],
                   Tr_sat=kw["Tr_sat"], Re=kw["Re"], u_in=kw["u_in"], nu_l=kw["nu_l"],
                   nu_ratio=kw["nu_ratio"], Pr_l=kw["Pr_l"], Pr_v=kw["Pr_v"], c_v=kw["c_v"], g=kw["g"],
                   outlet_U=kw["outlet_U"], warmup_steps=int(kw["warmup"]), energy=int(kw["energy"]),
                   storage=N.LBM_STORE_F64 if f64 else N.STORAGE[storage], compute_f64=1 if f64 else 0,
                   psi_mode=int(kw["psi_mode"]), seed=int(kw["seed"]), noise_amp=kw["noise_amp"],
                   body_fx=float(kw["body_fx"]), collision=int(kw["collision"]))
    return dom, cyl, prm, kw


def _torch_allocator(torch, device, enabled):
    """Device memory for the library from PyTorch's caching allocator (or None: cudaMalloc)."""
    blocks = {}
    if not enabled:
        return blocks, None, None, None
    dev = torch.device("cuda", device)

    def _alloc(nbytes, user):
        t = torch.empty(int(nbytes), dtype=torch.uint8, device=dev)
        blocks[t.data_ptr()] = t
        return t.data_ptr()

    def _free(ptr, user):
        blocks.pop(ptr, None)

    cb = (N.ALLOC_FN(_alloc), N.FREE_FN(_free))
    allocator = N.Allocator(cb[0], cb[1], None)
    return blocks, cb, allocator, C.byref(allocator)


def _case_kwargs(case):
    if getattr(case, "wall_q", 0.5) != 0.5:
        raise ValueError("the CUDA library places flat walls halfway between the last fluid node and the wall "
                         "(link fraction 1/2)")
    names = [k for k in _PARAM_DEFAULTS if hasattr(case, k)]
    params = {k: getattr(case, k) for k in names}
    if hasattr(case, "U_out"):
        params["outlet_U"] = case.U_out
    return dict(nx=case.nx, ny=case.ny, D=case.D, xc=case.xc, yc=case.yc, periodic_x=case.periodic_x,
                superheat_Tc=case.superheat_Tc, rho_s=getattr(case, "rho_s", 0.0), walls=getattr(case, "walls", 0),
                params=params)


def _dense(a, n):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    if a.size != n:
        raise ValueError(f"initial field has {a.size} values, expected {n}")
    return a


class Sim:
    """One boiling-on-a-cylinder simulation on the current CUDA device.

    nx, ny, periodic_x             lattice (flow along +x; periodic in y)
    D, xc, yc, superheat_Tc, rho_s  cylinder (D <= 0: none)
    f64                            FP64 arithmetic and storage (else FP32 arithmetic)
    storage                        FP32 arithmetic only: populations stored as "f32" (default), "f64" or
                                   "f16s" (shifted FP16)
    init                           optional dict of [ny][nx] arrays: rho, drho, ux, uy, T
    other keywords                 fields of lbm_params (see include/lbm.h)
    torch_alloc                    device memory from PyTorch's caching allocator
    """

    def __init__(self, nx, ny, D=0.0, xc=0.0, yc=0.0, periodic_x=0, superheat_Tc=0.05, rho_s=0.0, f64=False,
                 storage="f32", init=None, stream=None, torch_alloc=True, walls=0, **params):
        import torch

        self._torch = torch
        L = N.lib()
        self.nx, self.ny, self.D = int(nx), int(ny), float(D)
        dom, cyl, prm, self.params = _structs(nx, ny, D, xc, yc, periodic_x, superheat_Tc, rho_s, f64, storage, params,
                                              walls)
        self._f64, self._storage = bool(f64), prm.storage
        n = self.nx * self.ny
        init = init or {}
        keep = {k: _dense(init.get(k), n) for k in ("rho", "drho", "ux", "uy", "T")}
        ini = N.Init(*[keep[k].ctypes.data if keep[k] is not None else None
                       for k in ("rho", "drho", "ux", "uy", "T")])
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._owner = None
        self._blocks, self._alloc_cb, self._allocator, alloc_p = _torch_allocator(torch, self.device, torch_alloc)
        h = C.c_void_p()
        N.check(L.lbm_create(C.byref(dom), C.byref(cyl), C.byref(prm), C.byref(ini), alloc_p,
                             C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h
        self.n_wall = len(params.get("wall_dT", ()) or ())

    @classmethod
    def from_case(cls, case, f64=False, **kw):
        """Build from an object with the attributes of a workload description (nx, ny, D, ...)."""
        k = _case_kwargs(case)
        params = {p: v for p, v in k.pop("params").items() if p not in kw}
        return cls(k["nx"], k["ny"], D=k["D"], xc=k["xc"], yc=k["yc"], periodic_x=k["periodic_x"],
                   superheat_Tc=k["superheat_Tc"], rho_s=k["rho_s"], f64=f64, walls=k["walls"], **params, **kw)

    # ------------------------------------------------------------------ lifecycle
    @classmethod
    def _borrowed(cls, handle, nx, ny, D, owner):
        """A view of a domain owned by a Batch (no ownership of the handle)."""
        import torch

        self = cls.__new__(cls)
        self._torch = torch
        self.h = handle
        self.nx, self.ny, self.D = nx, ny, D
        self._owner = owner
        self._blocks = {}
        self.n_wall = 0
        self._f64 = owner._f64
        self._storage = N.LBM_STORE_F64 if owner._f64 else N.LBM_STORE_F32
        self.device = torch.cuda.current_device()
        return self

    def close(self):
        if getattr(self, "_owner", None) is not None:
            self.h = None
            return
        if getattr(self, "h", None) is not None and self.h.value:
            N.lib().lbm_destroy(self.h)
            self.h = None
            self._blocks.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st):
        N.check(st, self.h)

    # ------------------------------------------------------------------ stepping
    def step(self, n: int = 1):
        self._chk(N.lib().lbm_step(self.h, int(n)))
        return self

    def sync(self):
        self._chk(N.lib().lbm_sync(self.h))
        return self

    # ------------------------------------------------------------------ outputs
    def heat_flux(self) -> dict:
        v = [C.c_double() for _ in range(4)]
        cnt = C.c_int64()
        self._chk(N.lib().lbm_wall_heat_flux(self.h, *[C.byref(x) for x in v], C.byref(cnt)))
        return {"q_now": v[0].value, "q_mean": v[1].value, "q_std": v[2].value, "nu_mean": v[3].value,
                "count": cnt.value}

    def reset_heat_flux(self):
        self._chk(N.lib().lbm_reset_heat_flux(self.h))

    def fields(self, names=("rho", "ux", "uy", "T", "psi")) -> dict:
        mask = 0
        for k in names:
            mask |= N.FIELD_BITS[k]
        order = [k for k in N.FIELD_BITS if mask & N.FIELD_BITS[k]]
        out = np.empty((len(order), self.ny, self.nx))
        self._chk(N.lib().lbm_fields(self.h, mask, out.ctypes.data, out.nbytes, 0))
        return {k: out[i] for i, k in enumerate(order)}

    def fields_device(self, names=("rho", "T")):
        """Fields as a CUDA float64 tensor [len(names), ny, nx] (device-to-device copy)."""
        torch = self._torch
        mask = 0
        for k in names:
            mask |= N.FIELD_BITS[k]
        order = [k for k in N.FIELD_BITS if mask & N.FIELD_BITS[k]]
        out = torch.empty((len(order), self.ny, self.nx), dtype=torch.float64, device=f"cuda:{self.device}")
        self._chk(N.lib().lbm_fields(self.h, mask, out.data_ptr(), out.numel() * 8, 1))
        return out, order

    def get_state(self):
        n = self.nx * self.ny
        f = np.empty((9, self.ny, self.nx))
        T = np.empty((self.ny, self.nx))
        side = np.empty((3, self.ny))
        steps = C.c_int64()
        self._chk(N.lib().lbm_get_state(self.h, f.ctypes.data, T.ctypes.data, side.ctypes.data, C.byref(steps)))
        assert f.size == 9 * n
        return f, T, side, steps.value

    def set_state(self, f=None, T=None, side=None, steps=-1):
        n = self.nx * self.ny
        keep = [_dense(f, 9 * n), _dense(T, n), _dense(side, 3 * self.ny)]
        ptrs = [a.ctypes.data if a is not None else None for a in keep]
        self._chk(N.lib().lbm_set_state(self.h, *ptrs, int(steps)))

    def native_dtypes(self):
        """numpy dtypes of a native checkpoint: (populations, T and outlet rows)."""
        pop = {N.LBM_STORE_F64: np.float64, N.LBM_STORE_F32: np.float32, N.LBM_STORE_F16S: np.float16}
        return pop[self._storage], (np.float64 if self._f64 else np.float32)

    def get_state_native(self):
        """Checkpoint in the context's own formats (lbm_get_state_native)."""
        fdt, tdt = self.native_dtypes()
        f = np.empty((9, self.ny, self.nx), dtype=fdt)
        T = np.empty((self.ny, self.nx), dtype=tdt)
        side = np.empty((3, self.ny), dtype=tdt)
        steps = C.c_int64()
        self._chk(N.lib().lbm_get_state_native(self.h, f.ctypes.data, T.ctypes.data, side.ctypes.data,
                                               C.byref(steps)))
        return f, T, side, steps.value

    def set_state_native(self, f=None, T=None, side=None, steps=-1):
        fdt, tdt = self.native_dtypes()
        keep = [None if a is None else np.ascontiguousarray(a, dtype=dt)
                for a, dt in ((f, fdt), (T, tdt), (side, tdt))]
        self._chk(N.lib().lbm_set_state_native(self.h, *[a.ctypes.data if a is not None else None for a in keep],
                                               int(steps)))

    def stage_state_native(self, f, T, side=None, steps=-1):
        """Start copying a native-format state into the staging buffers (lbm_stage_state_native);
        returns at once.  The arrays (numpy, or pinned CPU torch tensors for an asynchronous
        copy) are kept referenced here until the next staging."""
        fdt, tdt = self.native_dtypes()

        def ptr(a, dt):
            if a is None:
                return None, None
            if hasattr(a, "data_ptr"):  # a CPU torch tensor (pinned for an asynchronous copy)
                if a.device.type != "cpu" or not a.is_contiguous() or a.element_size() != np.dtype(dt).itemsize:
                    raise ValueError("expected a contiguous CPU tensor of the native type")
                return a, a.data_ptr()
            a = np.ascontiguousarray(a, dtype=dt)
            return a, a.ctypes.data

        kf, pf = ptr(f, fdt)
        kT, pT = ptr(T, tdt)
        ks, ps = ptr(side, tdt)
        self._staged_keep = (kf, kT, ks)
        self._chk(N.lib().lbm_stage_state_native(self.h, pf, pT, ps, int(steps)))
        return self

    def take_staged(self):
        """Make the staged state the current one (lbm_take_staged; no host wait)."""
        self._chk(N.lib().lbm_take_staged(self.h))
        return self

    def info(self) -> dict:
        inf = N.Info()
        self._chk(N.lib().lbm_info(self.h, C.byref(inf)))
        return {k: getattr(inf, k) for k, _ in N.Info._fields_}

    # ------------------------------------------------------------------ adjoint
    def adjoint_window(self, n: int, ckpt_every: int = 50, per_node: bool = False) -> dict:
        """Run n steps and return J (the window's mean wall heat flux) with its gradient with
        respect to superheat_Tc, u_in (inlet condition only), the wall_dT knots and, with
        per_node, T_w at every solid node ([ny][nx])."""
        knots = np.zeros(max(self.n_wall, 1))
        dTw = np.zeros((self.ny, self.nx)) if per_node else None
        g = N.WindowGrad()
        if self.n_wall:
            g.dJ_dwall_dT = knots.ctypes.data_as(C.POINTER(C.c_double))
        if dTw is not None:
            g.dJ_dTw = dTw.ctypes.data_as(C.POINTER(C.c_double))
        self._chk(N.lib().lbm_adjoint_window(self.h, int(n), int(ckpt_every), C.byref(g)))
        out = {"J": g.J, "superheat": g.dJ_dsuperheat, "u_in": g.dJ_du_in,
               "wall_dT": knots[:self.n_wall].copy()}
        if dTw is not None:
            out["Tw"] = dTw
        return out

    def adjoint_step(self, fb=None, Tb=None, sb=None, q_weight: float = 0.0) -> dict:
        """Vector-Jacobian product of one step at the current state (lbm_adjoint_step)."""
        n = self.nx * self.ny
        keep = [_dense(fb, 9 * n), _dense(Tb, n), _dense(sb, 3 * self.ny)]
        fo = np.empty((9, self.ny, self.nx))
        To = np.empty((self.ny, self.nx))
        so = np.empty((3, self.ny))
        dTw = np.empty((self.ny, self.nx))
        du = C.c_double()
        self._chk(N.lib().lbm_adjoint_step(self.h, *[a.ctypes.data if a is not None else None for a in keep],
                                           float(q_weight), fo.ctypes.data, To.ctypes.data, so.ctypes.data,
                                           dTw.ctypes.data, C.byref(du)))
        return {"f": fo, "T": To, "side": so, "Tw": dTw, "u_in": du.value}

    # ------------------------------------------------------------------ timing
    def inject_fault(self, kind: str):
        """Test hook of the bounded device waits: the next step starves the TMA-staged tiles of
        one pass ("collide" or "energy"), whose short bounded waits then run out (LBM_ETIMEOUT at
        the next synchronising call; set_state restores a state to continue from)."""
        k = {"collide": N.LBM_FAULT_STARVE_COLLIDE, "energy": N.LBM_FAULT_STARVE_ENERGY}[kind]
        self._chk(N.lib().lbm_inject_fault(self.h, k))
        return self

    def profile(self, enable=True):
        self._chk(N.lib().lbm_profile(self.h, 1 if enable else 0))

    def profile_read(self) -> dict:
        k = 16
        names = (C.c_char_p * k)()
        launches = (C.c_int64 * k)()
        ms = (C.c_double * k)()
        nk = C.c_int32()
        self._chk(N.lib().lbm_profile_read(self.h, names, launches, ms, k, C.byref(nk)))
        return {names[i].decode(): (launches[i], ms[i]) for i in range(nk.value) if names[i]}


class Batch:
    """Independent domains stepped together (lbm_batch_*): one launch per pass over all
    domains' tiles, pairs of steps replayed from a CUDA graph once every domain is past its
    warm-up.  domain(i) gives a Sim view of domain i for fields and heat flux."""

    def __init__(self, cases, f64=False, stream=None, torch_alloc=True):
        import torch

        self._torch = torch
        L = N.lib()
        kws = [_case_kwargs(c) for c in cases]
        n = len(kws)
        doms, cyls, prms = (N.Domain * n)(), (N.Cylinder * n)(), (N.Params * n)()
        for i, k in enumerate(kws):
            doms[i], cyls[i], prms[i], _ = _structs(k["nx"], k["ny"], k["D"], k["xc"], k["yc"], k["periodic_x"],
                                                    k["superheat_Tc"], k["rho_s"], f64, "f32", k["params"], k["walls"])
        self.shapes = [(k["nx"], k["ny"], k["D"]) for k in kws]
        self._f64 = bool(f64)
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._blocks, self._alloc_cb, self._allocator, alloc_p = _torch_allocator(torch, self.device, torch_alloc)
        h = C.c_void_p()
        N.check(L.lbm_batch_create(n, doms, cyls, prms, alloc_p, C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h

    def __len__(self):
        return len(self.shapes)

    def step(self, n: int = 1):
        N.check(N.lib().lbm_batch_step(self.h, int(n)))
        return self

    def tune(self, steps_per_variant: int = 2) -> int:
        v = C.c_int32()
        N.check(N.lib().lbm_batch_tune(self.h, int(steps_per_variant), C.byref(v)))
        return v.value

    def graph(self, enable: bool = True):
        N.check(N.lib().lbm_batch_graph(self.h, 1 if enable else 0))

    def domain(self, i: int) -> Sim:
        hd = C.c_void_p()
        N.check(N.lib().lbm_batch_domain(self.h, int(i), C.byref(hd)))
        nx, ny, D = self.shapes[i]
        return Sim._borrowed(hd, nx, ny, D, self)

    def sync(self):
        self._torch.cuda.current_stream().synchronize()
        for i in range(len(self)):
            self.domain(i).sync()
        return self

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            N.lib().lbm_batch_destroy(self.h)
            self.h = None
            self._blocks.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
