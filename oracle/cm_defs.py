"""Definition-level statement of the CM collision, in plain FP64 numpy.

TEST INFRASTRUCTURE ONLY (part of the oracle; only tests, the smoke check and the
benchmark's CPU-baseline leg may import it).

This is the collision written straight from Eq. (collision) of Saito et al.
(arXiv:1912.02018), with no moment shortcuts:
    f* = f + Lambda (f^eq - f) + (I - Lambda/2) F_i,  Lambda = T^{-1} K T,
where T(u) is the central-moment basis of Eq. (matrix), f^eq the fourth-order
Hermite equilibrium of Eq. (equi), and F_i the Huang forcing of Eq. (forcingTerm)
with the standard Hermite normalisation (coefficient 1/(n! cs^{2n}) on order n).
The thermodynamic-consistency modification of Eq. (force2) replaces R_3 and R_8 by
R'_3 = 4 alpha |F_m|^2 and R'_8 = (4/3) alpha |F_m|^2, alpha = sigma / psi^2, so it
adds T^{-1} (I - K/2) (R'_3 e_3 + R'_8 e_8) to the result.
The C stepper computes the same collision by a different route (printed k^eq, R
and the M, N matrices), so agreement between the two is a real check.
"""
from __future__ import annotations

import numpy as np

CS2 = 1.0 / 3.0
CX = np.array([0, 1, -1, 0, 0, 1, -1, 1, -1], dtype=np.float64)
CY = np.array([0, 0, 0, 1, -1, 1, -1, -1, 1], dtype=np.float64)
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=np.float64)


def T_matrix(ux: float, uy: float) -> np.ndarray:
    """Central-moment basis of Eq. (matrix), rows in the paper's order."""
    cx = CX - ux
    cy = CY - uy
    return np.stack([
        np.ones(9), cx, cy, cx * cx + cy * cy, cx * cx - cy * cy, cx * cy,
        cx * cx * cy, cx * cy * cy, cx * cx * cy * cy,
    ])


def M_matrix() -> np.ndarray:
    """Raw-moment matrix M of App. A (T at u = 0)."""
    return T_matrix(0.0, 0.0)


def hermite(ux, uy):
    """D2Q9 Hermite polynomials used by Eq. (equi) and Eq. (forcingTerm)."""
    H = {
        "x": CX, "y": CY,
        "xx": CX * CX - CS2, "yy": CY * CY - CS2, "xy": CX * CY,
        "xxy": CX * CX * CY - CS2 * CY, "xyy": CX * CY * CY - CS2 * CX,
        "xxyy": CX * CX * CY * CY - CS2 * (CX * CX + CY * CY) + CS2 * CS2,
    }
    return H


def feq(rho: float, ux: float, uy: float) -> np.ndarray:
    """Fourth-order Hermite equilibrium, Eq. (equi)."""
    H = hermite(ux, uy)
    t1 = (H["x"] * ux + H["y"] * uy) / CS2
    t2 = (H["xx"] * ux * ux + 2 * H["xy"] * ux * uy + H["yy"] * uy * uy) / (2 * CS2 ** 2)
    t3 = (H["xxy"] * ux * ux * uy + H["xyy"] * ux * uy * uy) / (2 * CS2 ** 3)
    t4 = H["xxyy"] * ux * ux * uy * uy / (4 * CS2 ** 4)
    return W * rho * (1 + t1 + t2 + t3 + t4)


def huang_force(Fx: float, Fy: float, ux: float, uy: float) -> np.ndarray:
    """Discrete forcing term of Eq. (forcingTerm) (Huang et al. 2018).

    Coefficients of the Hermite expansion of the force: a1 = F, a2 = [Fu],
    a3 = [Fuu] (xxy, xyy components), a4 = [Fuuu] (xxyy component); the full
    contraction with the symmetric Hermite tensors counts each distinct index
    set by its multiplicity (2 for xy, 3 for xxy/xyy, 6 for xxyy).
    """
    H = hermite(ux, uy)
    a2xx = 2 * Fx * ux
    a2yy = 2 * Fy * uy
    a2xy = Fx * uy + Fy * ux
    a3xxy = 2 * Fx * ux * uy + Fy * ux * ux
    a3xyy = 2 * Fy * ux * uy + Fx * uy * uy
    a4xxyy = 2 * Fx * ux * uy * uy + 2 * Fy * ux * ux * uy
    o1 = (Fx * H["x"] + Fy * H["y"]) / CS2
    o2 = (a2xx * H["xx"] + 2 * a2xy * H["xy"] + a2yy * H["yy"]) / (2 * CS2 ** 2)
    o3 = 3 * (a3xxy * H["xxy"] + a3xyy * H["xyy"]) / (6 * CS2 ** 3)
    o4 = 6 * a4xxyy * H["xxyy"] / (24 * CS2 ** 4)
    return W * (o1 + o2 + o3 + o4)


def velocity(f: np.ndarray, Fx: float, Fy: float):
    rho = f.sum()
    return rho, (f @ CX + 0.5 * Fx) / rho, (f @ CY + 0.5 * Fy) / rho


def collide_direct(f, Fx, Fy, Fmx, Fmy, psi, omega, sigma):
    """One-node collision straight from Eq. (collision) plus Eq. (force2)."""
    f = np.asarray(f, dtype=np.float64)
    rho, ux, uy = velocity(f, Fx, Fy)
    T = T_matrix(ux, uy)
    Ti = np.linalg.inv(T)
    K = np.diag([1, 1, 1, 1, omega, omega, 1, 1, 1]).astype(np.float64)
    Lam = Ti @ K @ T
    I = np.eye(9)
    Fi = huang_force(Fx, Fy, ux, uy)
    out = f + Lam @ (feq(rho, ux, uy) - f) + (I - Lam / 2) @ Fi
    if sigma != 0.0:
        alpha = sigma / (psi * psi)
        Fm2 = Fmx * Fmx + Fmy * Fmy
        extra = np.zeros(9)
        extra[3] = 4 * alpha * Fm2
        extra[8] = 4.0 / 3.0 * alpha * Fm2
        out = out + Ti @ ((I - K / 2) @ extra)
    return out, rho, ux, uy


def collide_bgk_direct(f, Fx, Fy, omega):
    """The comparison operator of Sec. III.B: single-rate BGK on the same fourth-order Hermite
    equilibrium and forcing, in population space, f* = f + omega (f^eq - f) + (1 - omega/2) F_i."""
    f = np.asarray(f, dtype=np.float64)
    rho, ux, uy = velocity(f, Fx, Fy)
    out = f + omega * (feq(rho, ux, uy) - f) + (1.0 - omega / 2.0) * huang_force(Fx, Fy, ux, uy)
    return out, rho, ux, uy
