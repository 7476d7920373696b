"""Gradient of the time-averaged wall heat flux by reverse-mode automatic differentiation of
a plain FP64 PyTorch restatement of the time step.

TEST INFRASTRUCTURE ONLY (part of the oracle; only tests, the smoke check and the
benchmark's CPU leg may import it).  Nothing here is differentiated by hand: the step is
written forward, once, and torch.autograd supplies the derivative.

Objective (Sec. IV.B): J = (1/n) sum_{s<n} q_s, where q_s is the wall heat-flux sample of
step s (mean over the fluid nodes next to the cylinder of -lambda dT/dn, from the
temperature entering the step and the density of that step's collision), over a window of
n steps that starts from a given state (post-collision f*, T, outlet side values).
Parameters theta:
  superheat  (T_w - T_sat)/T_c of the heated cylinder (Sec. IV.A);
  u_in       speed of the Zou-He inlet (Sec. IV.A).  nu_l, g and the outlet speed U are
             inputs of the window held at the values derived for the base case, so this is
             the partial derivative with respect to the inlet boundary condition alone;
  wall_dT    knots of the angular wall-superheat profile (fractions of T_c); a solid node
             at angle phi from +x gets the periodic-linear interpolation of the knots.
The temperature of solid nodes is T_w(theta) throughout the window (also in the state it
starts from).

The step follows the C oracle's order: pull-streaming with the cylinder (linear
interpolated bounce-back), Zou-He inlet and convective-outlet substitutions; rho and psi of
Eq. (potential) with the Peng-Robinson EOS of Eq. (eos); the interaction force of
Eq. (interForce) and gravity; the CM collision of Sec. II.A-B with the consistency terms of
Eq. (postColl2), written with the raw-moment matrix M and the shift matrix N(u) of App. A;
the heat-flux sample; the Heun update of Eq. (energy) with third-order upwind convection
and the isotropic gradient and Laplacian of Sec. II.C.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .stepper import derive

CS2 = 1.0 / 3.0
CX = (0, 1, -1, 0, 0, 1, -1, 1, -1)
CY = (0, 0, 0, 1, -1, 1, -1, -1, 1)
OPP = (0, 2, 1, 4, 3, 6, 5, 8, 7)
# Eq. (interForce) stencil as 12 +/- pairs and the weights w(|e|^2) of Sec. II.B
EX = (1, 2, -2, -1, 0, 1, 2, -2, -1, 0, 1, 2)
EY = (0, 0, 1, 1, 1, 1, 1, 2, 2, 2, 2, 2)
WISO = {1: 4.0 / 21.0, 2: 4.0 / 45.0, 4: 1.0 / 60.0, 5: 2.0 / 315.0, 8: 1.0 / 5040.0}

_T = torch.float64


def _M_matrix() -> np.ndarray:
    """Raw moments: rows 1, cx, cy, cx^2+cy^2, cx^2-cy^2, cxcy, cx^2cy, cxcy^2, cx^2cy^2 (App. A)."""
    cx = np.array(CX, dtype=np.float64)
    cy = np.array(CY, dtype=np.float64)
    return np.stack([np.ones(9), cx, cy, cx * cx + cy * cy, cx * cx - cy * cy, cx * cy, cx * cx * cy,
                     cx * cy * cy, cx * cx * cy * cy])


def _N_matrix(ux: torch.Tensor, uy: torch.Tensor) -> torch.Tensor:
    """Shift matrix N(u) of App. A (central moments k = N(u) m), one per node: (n, 9, 9)."""
    n = ux.shape[0]
    z = torch.zeros(n, dtype=_T)
    o = torch.ones(n, dtype=_T)
    u, v = ux, uy
    rows = [
        [o, z, z, z, z, z, z, z, z],
        [-u, o, z, z, z, z, z, z, z],
        [-v, z, o, z, z, z, z, z, z],
        [u * u + v * v, -2.0 * u, -2.0 * v, o, z, z, z, z, z],
        [u * u - v * v, -2.0 * u, 2.0 * v, z, o, z, z, z, z],
        [u * v, -v, -u, z, z, o, z, z, z],
        [-u * u * v, 2.0 * u * v, u * u, -v / 2.0, -v / 2.0, -2.0 * u, o, z, z],
        [-u * v * v, v * v, 2.0 * u * v, -u / 2.0, u / 2.0, -2.0 * v, z, o, z],
        [u * u * v * v, -2.0 * u * v * v, -2.0 * u * u * v, (u * u + v * v) / 2.0, -(u * u - v * v) / 2.0,
         4.0 * u * v, -2.0 * v, -2.0 * u, o],
    ]
    return torch.stack([torch.stack(r, dim=-1) for r in rows], dim=-2)


class GradientOracle:
    """Differentiable FP64 step for one case (nx, ny small: every node is a tensor entry).
    Every step of a window applies the force and the energy equation (step >= warm-up)."""

    def __init__(self, case):
        p, d = derive(case)
        self.case, self.d = case, d
        self.nx, self.ny = nx, ny = case.nx, case.ny
        self.N = N = nx * ny
        self.periodic = bool(case.periodic_x)
        self.G, self.sigma = p.G, p.sigma
        self.a, self.b, self.R, self.kappa, self.Tc = p.a, p.b, p.R, p.kappa, p.Tc
        self.T_sat = p.T_sat
        self.rho_l, self.rho_v, self.rho_s = p.rho_l, p.rho_v, p.rho_s
        self.nu_l, self.nu_v, self.alpha_l, self.alpha_v, self.c_v = p.nu_l, p.nu_v, p.alpha_l, p.alpha_v, p.c_v
        self.g, self.U = p.g, p.U_out
        self.u_in0, self.superheat0 = case.u_in, case.superheat_Tc
        self.n_wall = len(case.wall_dT) if case.wall_dT else 0

        ys, xs = np.divmod(np.arange(N), nx)
        r = 0.5 * case.D
        solid = ((xs - case.xc) ** 2 + (ys - case.yc) ** 2 <= r * r) if case.D > 0 else np.zeros(N, bool)
        self.solid_np = solid
        self.solid = torch.from_numpy(solid)
        self.fluid_idx = torch.from_numpy(np.nonzero(~solid)[0])
        inlet = (xs == 0) & (not self.periodic)
        self.inlet = torch.from_numpy(inlet)
        self.dirichlet = torch.from_numpy(solid | inlet)

        # stencil positions as the oracle reads them: periodic in y, clamped (zero-gradient) in x
        def at(dx, dy):
            yy = (ys + dy) % ny
            xx = xs + dx
            xx = xx % nx if self.periodic else np.clip(xx, 0, nx - 1)
            return torch.from_numpy(yy * nx + xx)

        self.at = {(dx, dy): at(dx, dy) for dx in range(-2, 3) for dy in range(-2, 3)}

        # pull tables: fp_i(node) = ca * fs[pa, ia] + cb * fs[pb, ib]
        pa = np.zeros((9, N), np.int64)
        ia = np.zeros((9, N), np.int64)
        ca = np.zeros((9, N))
        pb = np.zeros((9, N), np.int64)
        ib = np.zeros((9, N), np.int64)
        cb = np.zeros((9, N))
        bnodes, bnx, bny = [], [], []
        for nid in range(N):
            if solid[nid]:
                continue
            x, y = xs[nid], ys[nid]
            touches = False
            for i in range(9):
                sx, sy = x - CX[i], (y - CY[i]) % ny
                if self.periodic:
                    sx %= nx
                pa[i, nid], ia[i, nid] = i, nid
                if sx < 0 or sx >= nx:
                    continue  # inlet / outlet unknown, set below
                if solid[sy * nx + sx]:
                    touches = True
                    q = self._link_fraction(x, y, -CX[i], -CY[i])
                    io = OPP[i]
                    if q < 0.5:
                        xp, yp = x + CX[i], (y + CY[i]) % ny
                        if self.periodic:
                            xp %= nx
                        ok = 0 <= xp < nx and not solid[yp * nx + xp]
                        pa[i, nid], ia[i, nid], ca[i, nid] = io, nid, (2.0 * q if ok else 1.0)
                        if ok:
                            pb[i, nid], ib[i, nid], cb[i, nid] = io, yp * nx + xp, 1.0 - 2.0 * q
                    else:
                        pa[i, nid], ia[i, nid], ca[i, nid] = io, nid, 1.0 / (2.0 * q)
                        pb[i, nid], ib[i, nid], cb[i, nid] = i, nid, (2.0 * q - 1.0) / (2.0 * q)
                else:
                    pa[i, nid], ia[i, nid], ca[i, nid] = i, sy * nx + sx, 1.0
            if touches:
                rr = math.hypot(x - case.xc, y - case.yc)
                bnodes.append(nid)
                bnx.append((x - case.xc) / rr)
                bny.append((y - case.yc) / rr)
        self.pull_a = torch.from_numpy(pa * N + ia)
        self.pull_ca = torch.from_numpy(ca)
        self.pull_b = torch.from_numpy(pb * N + ib)
        self.pull_cb = torch.from_numpy(cb)
        self.bnode = torch.tensor(bnodes, dtype=torch.int64)
        self.bn = (torch.tensor(bnx, dtype=_T), torch.tensor(bny, dtype=_T))

        # wall profile: solid node -> interpolation weights over the knots
        Wk = np.zeros((N, max(self.n_wall, 1)))
        if self.n_wall:
            for nid in np.nonzero(solid)[0]:
                s = math.atan2(ys[nid] - case.yc, xs[nid] - case.xc) / (2.0 * math.pi)
                s = s + 1.0 if s < 0.0 else s
                pos = s * self.n_wall
                fl = math.floor(pos)
                k0 = int(fl) % self.n_wall
                k1 = (k0 + 1) % self.n_wall
                t = pos - fl
                Wk[nid, k0] += 1.0 - t
                Wk[nid, k1] += t
        self.Wk = torch.from_numpy(Wk)
        self.Minv = torch.from_numpy(np.linalg.inv(_M_matrix()))
        self.M = torch.from_numpy(_M_matrix())

    def _link_fraction(self, x, y, cx, cy):
        c = self.case
        dx, dy, r = x - c.xc, y - c.yc, 0.5 * c.D
        A = float(cx * cx + cy * cy)
        B = dx * cx + dy * cy
        C0 = dx * dx + dy * dy - r * r
        return (-B - math.sqrt(B * B - A * C0)) / A

    # ------------------------------------------------------------ thermodynamics
    def p_eos(self, rho, T):
        """Peng-Robinson pressure, Eq. (eos)."""
        s = 1.0 + self.kappa * (1.0 - torch.sqrt(T / self.Tc))
        rep = rho * self.R * T / (1.0 - self.b * rho)
        att = self.a * (s * s) * rho * rho / (1.0 + 2.0 * self.b * rho - self.b * self.b * rho * rho)
        return rep - att

    def dpdT(self, rho, T):
        """(dp/dT) at fixed rho of Eq. (eos), with phi'(T) by the chain rule."""
        s = 1.0 + self.kappa * (1.0 - torch.sqrt(T / self.Tc))
        dphi = -self.kappa * s / torch.sqrt(T * self.Tc)
        rep = rho * self.R / (1.0 - self.b * rho)
        att = self.a * dphi * rho * rho / (1.0 + 2.0 * self.b * rho - self.b * self.b * rho * rho)
        return rep - att

    def psi(self, rho, T):
        """Eq. (potential): psi = sqrt(2 (p_EOS - rho cs^2) / (G cs^2))."""
        return torch.sqrt(2.0 * (self.p_eos(rho, T) - rho * CS2) / (self.G * CS2))

    def phase(self, rho):
        if not self.rho_l > self.rho_v:
            return torch.ones_like(rho)
        return torch.clamp((rho - self.rho_v) / (self.rho_l - self.rho_v), 0.0, 1.0)

    def nu(self, rho):
        return self.nu_v + self.phase(rho) * (self.nu_l - self.nu_v)

    def lam(self, rho):
        return rho * self.c_v * (self.alpha_v + self.phase(rho) * (self.alpha_l - self.alpha_v))

    # ------------------------------------------------------------ stencils (Sec. II.C)
    def grad(self, f):
        sx = torch.zeros_like(f)
        sy = torch.zeros_like(f)
        for ex, ey in zip(EX, EY):
            w = WISO[ex * ex + ey * ey]
            d = f[self.at[(ex, ey)]] - f[self.at[(-ex, -ey)]]
            sx = sx + w * d * ex
            sy = sy + w * d * ey
        return sx, sy

    def lap(self, f):
        acc = torch.zeros_like(f)
        for ex, ey in zip(EX, EY):
            w = WISO[ex * ex + ey * ey]
            acc = acc + w * ((f[self.at[(ex, ey)]] + f[self.at[(-ex, -ey)]]) - 2.0 * f)
        return 2.0 * acc

    def upwind(self, f, v, ax):
        """Third-order upwind derivative along axis ax, biased against the sign of v."""
        def sh(k):
            return f[self.at[(k, 0) if ax == 0 else (0, k)]] - f

        plus = (sh(-2) - 6.0 * sh(-1) + 2.0 * sh(1)) / 6.0
        minus = (-2.0 * sh(-1) + 6.0 * sh(1) - sh(2)) / 6.0
        return torch.where(v >= 0.0, plus, minus)

    def energy_rhs(self, T, rho, ux, uy, lam):
        conv = ux * self.upwind(T, ux, 0) + uy * self.upwind(T, uy, 1)
        gx, gy = self.grad(T)
        lp = self.lap(T)
        lx, ly = self.grad(lam)
        dxux, _ = self.grad(ux)
        _, dyuy = self.grad(uy)
        divu = dxux + dyuy
        diff = lam * lp + (lx * gx + ly * gy)
        work = T * self.dpdT(rho, T) * divu
        return -conv + diff / (rho * self.c_v) - work / (rho * self.c_v)

    # ------------------------------------------------------------ one step
    def wall_T(self, superheat, knots):
        T_wall = self.T_sat + superheat * self.Tc
        if self.n_wall:
            return T_wall + (self.Wk @ knots) * self.Tc
        return T_wall + torch.zeros(self.N, dtype=_T)

    def step(self, fs, T, side, u_in, Tw):
        """One step. fs: (9, N) post-collision populations; T: (N,); side: (3, ny).
        Returns (fs', T', side', q)."""
        N, nx, ny = self.N, self.nx, self.ny
        flat = fs.reshape(-1)
        fp = self.pull_ca * flat[self.pull_a] + self.pull_cb * flat[self.pull_b]
        fp = list(fp.unbind(0))
        side_new = side
        if not self.periodic:
            rows = torch.arange(ny) * nx
            fl = ~self.solid[rows]
            r_in = rows[fl]
            f0, f2, f3, f4, f6, f8 = (fp[i][r_in] for i in (0, 2, 3, 4, 6, 8))
            rho_in = (f0 + f3 + f4 + 2.0 * (f2 + f6 + f8)) / (1.0 - u_in)
            fp[1] = fp[1].index_put((r_in,), f2 + 2.0 / 3.0 * rho_in * u_in)
            fp[5] = fp[5].index_put((r_in,), f6 - 0.5 * (f3 - f4) + rho_in * u_in / 6.0)
            fp[7] = fp[7].index_put((r_in,), f8 + 0.5 * (f3 - f4) + rho_in * u_in / 6.0)
            out = rows + nx - 1
            fo = ~self.solid[out]
            r_out = out[fo]
            new_side = []
            for j, i in enumerate((2, 6, 8)):
                v = (side[j][fo] + self.U * fp[i][r_out - 1]) / (1.0 + self.U)
                fp[i] = fp[i].index_put((r_out,), v)
                new_side.append(side[j].index_put((fo.nonzero()[:, 0],), v))
            side_new = torch.stack(new_side)
        fp = torch.stack(fp)
        fi = self.fluid_idx
        rho = torch.full((N,), self.rho_s, dtype=_T).index_put((fi,), self._sum9(fp[:, fi]))
        psi = self.psi(rho, T) if self.G != 0.0 else torch.zeros(N, dtype=_T)
        # force at fluid nodes
        if self.G != 0.0:
            sx, sy = self.grad(psi)
            Fmx = -self.G * CS2 * psi * sx
            Fmy = -self.G * CS2 * psi * sy
        else:
            Fmx = Fmy = torch.zeros(N, dtype=_T)
        Fx = Fmx - (rho - self.rho_l) * self.g
        Fy = Fmy
        r = rho[fi]
        fs_f, ux_f, uy_f = self.collide(fp[:, fi], r, Fx[fi], Fy[fi], Fmx[fi], Fmy[fi], psi[fi],
                                        1.0 / (self.nu(r) / CS2 + 0.5),
                                        self.sigma if self.G != 0.0 else 0.0)
        fs_new = self._put_cols(fs, fi, fs_f)
        ux = torch.zeros(N, dtype=_T).index_put((fi,), ux_f)
        uy = torch.zeros(N, dtype=_T).index_put((fi,), uy_f)
        lam = self.lam(rho)
        # heat-flux sample from the temperature entering the step
        if len(self.bnode):
            gx, gy = self.grad(T)
            b = self.bnode
            q = (-lam[b] * (gx[b] * self.bn[0] + gy[b] * self.bn[1])).sum() / len(b)
        else:
            q = torch.zeros((), dtype=_T)
        # Heun: T1 = T + L(T); T' = (T + T1 + L(T1)) / 2; Dirichlet at the wall and the inlet
        L0 = self.energy_rhs(T, rho, ux, uy, lam)
        T1 = torch.where(self.solid, Tw, torch.where(self.inlet, torch.full_like(T, self.T_sat), T + L0))
        L1 = self.energy_rhs(T1, rho, ux, uy, lam)
        Tn = torch.where(self.solid, Tw,
                         torch.where(self.inlet, torch.full_like(T, self.T_sat), (T + T1 + L1) * 0.5))
        return fs_new, Tn, side_new, q

    @staticmethod
    def _sum9(f):
        r = f[0]
        for i in range(1, 9):
            r = r + f[i]
        return r

    @staticmethod
    def _put_cols(fs, idx, vals):
        out = fs.clone()
        out[:, idx] = vals
        return out

    def collide(self, f, rho, Fx, Fy, Fmx, Fmy, psi, omega, sigma):
        """CM collision, Sec. II.A-B: k = N(u) M f, k* of Eq. (postColl2), N(u) m* = k*, f* = M^-1 m*."""
        m = self.M @ f
        ux = (m[1] + 0.5 * Fx) / rho
        uy = (m[2] + 0.5 * Fy) / rho
        Nu = _N_matrix(ux, uy)
        k = torch.einsum("nij,jn->in", Nu, m)
        alpha = sigma / (psi * psi) if sigma != 0.0 else torch.zeros_like(psi)
        Fm2 = Fmx * Fmx + Fmy * Fmy
        zero = torch.zeros_like(rho)
        keq = [rho, zero, zero, 2.0 * rho / 3.0, zero, zero, zero, zero, rho / 9.0]
        Rp = [zero, Fx, Fy, 4.0 * alpha * Fm2, zero, zero, Fy / 3.0, Fx / 3.0, 4.0 / 3.0 * alpha * Fm2]
        ks = []
        for j in range(9):
            K = omega if j in (4, 5) else 1.0
            ks.append((1.0 - K) * k[j] + K * keq[j] + (1.0 - K / 2.0) * Rp[j])
        ks = torch.stack(ks, dim=1).unsqueeze(-1)  # (n, 9, 1)
        ms = torch.linalg.solve_triangular(Nu, ks, upper=False, unitriangular=True).squeeze(-1)
        return (self.Minv @ ms.T), ux, uy

    # ------------------------------------------------------------ window objective
    def objective(self, fs0, T0, side0, n, superheat, u_in, knots):
        """J = mean of the n heat-flux samples of a window from state (fs0, T0, side0)."""
        Tw = self.wall_T(superheat, knots)
        fs = torch.as_tensor(np.asarray(fs0).reshape(9, self.N), dtype=_T)
        T = torch.where(self.solid, Tw, torch.as_tensor(np.asarray(T0).reshape(-1), dtype=_T))
        side = torch.as_tensor(np.asarray(side0).reshape(3, self.ny), dtype=_T)
        J = torch.zeros((), dtype=_T)
        for _ in range(n):
            fs, T, side, q = self.step(fs, T, side, u_in, Tw)
            J = J + q
        return J / n, (fs, T, side)

    def gradient(self, fs0, T0, side0, n, superheat=None, u_in=None, knots=None):
        """J and dJ/d(superheat, u_in, knots) by reverse-mode differentiation (FP64)."""
        sh = torch.tensor(self.superheat0 if superheat is None else superheat, dtype=_T, requires_grad=True)
        ui = torch.tensor(self.u_in0 if u_in is None else u_in, dtype=_T, requires_grad=True)
        kn0 = self.case.wall_dT if knots is None else knots
        kn = torch.tensor(list(kn0) if self.n_wall else [0.0], dtype=_T, requires_grad=True)
        J, _ = self.objective(fs0, T0, side0, n, sh, ui, kn)
        J.backward()
        return {"J": float(J.detach()), "superheat": float(sh.grad), "u_in": float(ui.grad),
                "wall_dT": kn.grad.numpy().copy() if self.n_wall else np.zeros(0)}
