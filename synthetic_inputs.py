"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds only input data: workload descriptions (raw configuration
numbers) and a counter-based random generator.  It contains none of the
method's arithmetic; each implementation derives its own constants (critical
point, coexistence densities, viscosities, gravity) from these numbers.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014).  Value k of stream `seed` is the SplitMix64
finaliser applied to seed + (k + 1) * 0x9E3779B97F4A7C15 (mod 2^64); a uniform
number in [-1, 1) is 2 * (z >> 11) * 2^-53 - 1.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, index: np.ndarray) -> np.ndarray:
    """SplitMix64 output for counter values `index` of stream `seed` (uint64 array)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (index.astype(np.uint64) + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, n: int) -> np.ndarray:
    """n uniform numbers in [-1, 1) from stream `seed`, counter 0..n-1."""
    z = splitmix64(seed, np.arange(n, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


def density_perturbation(nx: int, ny: int, seed: int, amp: float) -> np.ndarray:
    """Seeded perturbation added to the initial liquid density, shape (ny, nx), node id = y*nx + x."""
    return (amp * uniform_pm1(seed, nx * ny)).reshape(ny, nx)


@dataclass
class Case:
    """Raw description of one boiling-on-a-cylinder run (lattice units).

    superheat_Tc: wall superheat as a fraction of the critical temperature; wall_dT adds a
    periodic-linear angular profile over len(wall_dT) equally spaced knots (angle from +x).
    g < 0 means "derive from u_in/sqrt(g D) = 4"; U_out < 0 means "use u_in";
    nu_l == 0 means "derive from Re"; rho_s == 0 means "use the liquid density".
    """
    nx: int
    ny: int
    D: float
    xc: float
    yc: float
    periodic_x: int = 0
    walls: int = 0  # flat walls: bit 0 the column x = 0 (heated, instead of the inlet), bit 1 the rows y = 0, ny-1
    wall_q: float = 0.5  # flat walls' surface: this fraction of a link from the last fluid node
    body_fx: float = 0.0  # uniform body force along +x
    collision: int = 0  # 0: the central-moment collision; 1: single-rate BGK (the comparison operator)
    a: float = 2.0 / 49.0
    b: float = 2.0 / 21.0
    R: float = 1.0
    acentric: float = 0.344
    G: float = -2.0
    sigma: float = 0.38
    Tr_sat: float = 0.86
    superheat_Tc: float = 0.05
    Re: float = 30.0
    u_in: float = 0.05
    nu_l: float = 0.0
    nu_ratio: float = 1.0
    Pr_l: float = 0.862
    Pr_v: float = 1.5
    c_v: float = 11.0
    g: float = -1.0
    U_out: float = -1.0
    warmup: int = 0
    energy: int = 1
    rho_s: float = 0.0
    seed: int = 0
    noise_amp: float = 1e-4
    wall_dT: tuple = ()  # optional angular profile of extra wall superheat (fractions of Tc), equal knots
    name: str = ""

    def replace(self, **kw) -> "Case":
        return dataclasses.replace(self, **kw)

    def drho(self) -> np.ndarray:
        return density_perturbation(self.nx, self.ny, self.seed, self.noise_amp)


def cylinder_case(nx: int, ny: int, D: float, **kw) -> Case:
    """Cylinder of diameter D centred at (nx/4, ny/2)."""
    return Case(nx=nx, ny=ny, D=D, xc=nx / 4.0, yc=ny / 2.0, **kw)


# Plain method, FP64 parity case: 128x64, D=16 at (32,32), superheat 0.05 Tc, Re=30, no warm-up.
SMALL = cylinder_case(128, 64, 16.0, Re=30.0, superheat_Tc=0.05, name="128x64_D16_Re30")

# Paper-shaped single domain: 1536x768, D=96, FP32; Re sweep 30..30000, superheat 0.02..0.20 Tc.
PAPER_SHAPED = cylinder_case(1536, 768, 96.0, Re=300.0, superheat_Tc=0.10, warmup=9600,
                             name="1536x768_D96_Re300")
PAPER_SHAPED_RE = (30.0, 300.0, 3000.0, 30000.0)
PAPER_SHAPED_SUPERHEAT = (0.02, 0.05, 0.10, 0.20)

# Precision-study domain: 2048x1024, D=128, Re=30000, film boiling at 0.2 Tc.
PRECISION = cylinder_case(2048, 1024, 128.0, Re=30000.0, superheat_Tc=0.20, warmup=12800,
                          name="2048x1024_D128_Re30000")

# Adjoint domain: 512x256, D=32, Re=300.
ADJOINT = cylinder_case(512, 256, 32.0, Re=300.0, superheat_Tc=0.05, name="512x256_D32_Re300")


def batch_sweep(n: int = 64, seed: int = 1) -> list[Case]:
    """Boiling-curve sweep: D from {40,64,96,128} by SplitMix64(seed, k) mod 4 on 12D x 6D
    lattices, superheat log-spaced 0.01..0.25 Tc, Re = 300."""
    ds = (40, 64, 96, 128)
    pick = splitmix64(seed, np.arange(n, dtype=np.uint64)) % np.uint64(4)
    sh = np.geomspace(0.01, 0.25, n)
    out = []
    for k in range(n):
        D = ds[int(pick[k])]
        out.append(Case(nx=12 * D, ny=6 * D, D=float(D), xc=3.0 * D, yc=3.0 * D, Re=300.0,
                        superheat_Tc=float(sh[k]), seed=seed + k, name=f"sweep{k}_D{D}"))
    return out


def poiseuille_case(L: int, U0: float = 0.01, nu: float = 1.0 / 6.0, nx: int = 8) -> Case:
    """Poiseuille flow (Sec. III.C): a single-phase channel of width L between the no-slip planes
    (flat walls on the rows y = 0 and y = L + 1, halfway bounce-back: surfaces at y = 1/2 and
    L + 1/2), periodic in x, driven by the uniform force F_x = 8 nu U0 / L^2 (rho_0 = 1), whose
    steady profile is u_x = 4 U0 y' (L - y') / L^2 with y' the distance from the lower surface."""
    return Case(nx=nx, ny=L + 2, D=0.0, xc=0.0, yc=0.0, periodic_x=1, walls=2, G=0.0, energy=0, u_in=0.0,
                nu_l=nu, nu_ratio=1.0, g=0.0, body_fx=8.0 * nu * U0 / (L * L), noise_amp=0.0,
                name=f"poiseuille_L{L}")


def poiseuille_profile(L: int, U0: float = 0.01) -> np.ndarray:
    """The closed-form steady u_x at the fluid rows y = 1 .. L of poiseuille_case(L)."""
    yp = np.arange(1, L + 1) - 0.5
    return 4.0 * U0 * yp * (L - yp) / (L * L)


def shear_layer_case(L: int = 512, Ma: float = 0.1, Re: float = 3.0e4, collision: int = 0) -> Case:
    """Double shear layer (Sec. III.B): a periodic L x L single-phase fluid (G = 0, T fixed), with
    u0 = Ma c_s (c_s^2 = 1/3) and nu = u0 L / Re; the initial velocity is shear_layer_velocity and
    the initial density 1."""
    u0 = Ma / np.sqrt(3.0)
    return Case(nx=L, ny=L, D=0.0, xc=0.0, yc=0.0, periodic_x=1, G=0.0, sigma=0.0, energy=0, u_in=0.0,
                nu_l=u0 * L / Re, nu_ratio=1.0, g=0.0, noise_amp=0.0, collision=collision,
                name=f"shear_layer_L{L}_Ma{Ma:g}_{'bgk' if collision else 'cm'}")


def shear_layer_velocity(L: int, Ma: float, kappa: float = 80.0, delta: float = 0.05):
    """Initial (u_x, u_y) of the double shear layer (Sec. III.B) at the nodes (x, y), 0 <= x, y < L,
    shape (L, L): two tanh shear layers of width 1/kappa at y/L = 1/4 and 3/4 and a transverse
    sine perturbation of relative amplitude delta."""
    u0 = Ma / np.sqrt(3.0)
    y, x = np.mgrid[0:L, 0:L].astype(np.float64) / L
    ux = np.where(y <= 0.5, u0 * np.tanh(kappa * (y - 0.25)), u0 * np.tanh(kappa * (0.75 - y)))
    uy = u0 * delta * np.sin(2.0 * np.pi * (x + 0.25))
    return ux, uy

