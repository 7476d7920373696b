// Kernels of one time step of the CM pseudopotential boiling LBM (arXiv:1912.02018),
// templated on the compute type C (double or float) and population storage type S.
//
// Layout: structure of arrays, every field [ny][pitch] with x fastest; populations are
// 9 such planes.  One thread per node, 32x8 thread blocks.  Each kernel is a single
// pass over HBM:
//   k_rho_psi   pull f (with boundary substitutions) -> rho -> psi(rho, T) in FP64
//   k_collide   pull f again, interaction force from the psi stencil, CM collision,
//               store f* (the other buffer), rho, u
//   k_heat_flux wall heat flux over the boundary-node list (FP64 accumulation)
//   k_T_stage   one Heun stage of the temperature equation
// The operation order inside each node follows the paper's equations term by term so
// that the FP64 build (compiled without FMA contraction) rounds like a plain reference.
#pragma once

#include <cstdint>

#include "lbm_internal.h"

namespace lbm {
namespace kern {

constexpr int kBX = 32;
constexpr int kBY = 8;

// ---------------------------------------------------------------- lattice tables
// D2Q9 velocities, Eq. (velVec).
__device__ __forceinline__ constexpr int cxv(int i) {
  return i == 1 || i == 5 || i == 7 ? 1 : (i == 2 || i == 6 || i == 8 ? -1 : 0);
}
__device__ __forceinline__ constexpr int cyv(int i) {
  return i == 3 || i == 5 || i == 8 ? 1 : (i == 4 || i == 6 || i == 7 ? -1 : 0);
}
__device__ __forceinline__ constexpr int oppv(int i) {
  return i == 0 ? 0 : (i % 2 == 1 ? i + 1 : i - 1);
}
// The 24-neighbour stencil of Eq. (interForce) as 12 pairs (e, -e), with w(|e|^2).
__device__ __forceinline__ constexpr int exv(int k) {
  return k == 0 ? 1 : k == 1 ? 2 : k == 2 ? -2 : k == 3 ? -1 : k == 4 ? 0 : k == 5 ? 1 : k == 6 ? 2
       : k == 7 ? -2 : k == 8 ? -1 : k == 9 ? 0 : k == 10 ? 1 : 2;
}
__device__ __forceinline__ constexpr int eyv(int k) { return k < 2 ? 0 : (k < 7 ? 1 : 2); }
__device__ __forceinline__ constexpr double wiso(int k) {
  // |e|^2 = 1: 4/21, 2: 4/45, 4: 1/60, 5: 2/315, 8: 1/5040
  return (exv(k) * exv(k) + eyv(k) * eyv(k)) == 1 ? 4.0 / 21.0
       : (exv(k) * exv(k) + eyv(k) * eyv(k)) == 2 ? 4.0 / 45.0
       : (exv(k) * exv(k) + eyv(k) * eyv(k)) == 4 ? 1.0 / 60.0
       : (exv(k) * exv(k) + eyv(k) * eyv(k)) == 5 ? 2.0 / 315.0
       : 1.0 / 5040.0;
}

// ---------------------------------------------------------------- addressing
__device__ __forceinline__ int wrap_y(const Geo& g, int y) {  // offsets |dy| <= 2 < ny
  return y < 0 ? y + g.ny : (y >= g.ny ? y - g.ny : y);
}
// x for a stencil read: periodic, or the nearest boundary column (zero-gradient ghost).
__device__ __forceinline__ int stencil_x(const Geo& g, int x) {
  if (g.periodic_x) return x < 0 ? x + g.nx : (x >= g.nx ? x - g.nx : x);
  return x < 0 ? 0 : (x >= g.nx ? g.nx - 1 : x);
}
template <typename C>
__device__ __forceinline__ C at(const Geo& g, const C* __restrict__ fld, int x, int y) {
  return fld[(long long)wrap_y(g, y) * g.pitch + stencil_x(g, x)];
}
template <typename C, typename S>
__device__ __forceinline__ C ldf(const Geo& g, const S* __restrict__ f, int i, int y, int x) {
  return static_cast<C>(f[i * g.plane + (long long)y * g.pitch + x]);
}

// ---------------------------------------------------------------- thermodynamics
// Peng-Robinson EOS, Eq. (eos), and psi of Eq. (potential); FP64 in every build.
__device__ __forceinline__ double psi_eos(const Phys& ph, double rho, double T, double& rad) {
  const double cs2 = 1.0 / 3.0;
  double s = 1.0 + ph.kappa * (1.0 - sqrt(T / ph.Tc));
  double phi = s * s;
  double rep = rho * ph.R * T / (1.0 - ph.b * rho);
  double att = ph.a * phi * rho * rho / (1.0 + 2.0 * ph.b * rho - ph.b * ph.b * rho * rho);
  double p = rep - att;
  rad = 2.0 * (p - rho * cs2) / (ph.G * cs2);
  return sqrt(rad);
}
// (dp/dT) at fixed rho, the derivative of Eq. (eos).
template <typename C>
__device__ __forceinline__ C dpdT_eos(const Phys& ph, C rho, C T) {
  C s = C(1) + C(ph.kappa) * (C(1) - sqrt(T / C(ph.Tc)));
  C dphi = -C(ph.kappa) * s / sqrt(T * C(ph.Tc));
  C rep = rho * C(ph.R) / (C(1) - C(ph.b) * rho);
  C att = C(ph.a) * dphi * rho * rho / (C(1) + C(2) * C(ph.b) * rho - C(ph.b) * C(ph.b) * rho * rho);
  return rep - att;
}
// Phase fraction for the transport properties, and nu(rho), lambda(rho).
template <typename C>
__device__ __forceinline__ C phase_frac(const Phys& ph, C rho) {
  if (!(ph.rho_l > ph.rho_v)) return C(1);
  C f = (rho - C(ph.rho_v)) / (C(ph.rho_l) - C(ph.rho_v));
  f = f < C(0) ? C(0) : f;
  return f > C(1) ? C(1) : f;
}
template <typename C>
__device__ __forceinline__ C nu_of(const Phys& ph, C rho) {
  return C(ph.nu_v) + phase_frac(ph, rho) * (C(ph.nu_l) - C(ph.nu_v));
}
template <typename C>
__device__ __forceinline__ C lam_of(const Phys& ph, C rho) {
  C alpha = C(ph.alpha_v) + phase_frac(ph, rho) * (C(ph.alpha_l) - C(ph.alpha_v));
  return rho * C(ph.c_v) * alpha;
}

// ---------------------------------------------------------------- stencils (Sec. II.C)
// Isotropic gradient sum_k w_k phi(x+e_k) e_k over +/- pairs.
template <typename C, bool kX = true, bool kY = true>
__device__ __forceinline__ void iso_grad(const Geo& g, const C* __restrict__ fld, int x, int y, C& gx, C& gy) {
  C sx = C(0), sy = C(0);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const int ex = exv(k), ey = eyv(k);
    const C w = C(wiso(k));
    if ((kX && ex != 0) || (kY && ey != 0)) {
      C d = at(g, fld, x + ex, y + ey) - at(g, fld, x - ex, y - ey);
      if (kX && ex != 0) sx = sx + w * d * C(ex);
      if (kY && ey != 0) sy = sy + w * d * C(ey);
    }
  }
  gx = sx;
  gy = sy;
}
// Isotropic Laplacian 2 sum_k w_k (phi(x+e_k) - phi(x)) over +/- pairs.
template <typename C>
__device__ __forceinline__ C iso_lap(const Geo& g, const C* __restrict__ fld, int x, int y) {
  C c = at(g, fld, x, y), s = C(0);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const int ex = exv(k), ey = eyv(k);
    C d = (at(g, fld, x + ex, y + ey) + at(g, fld, x - ex, y - ey)) - C(2) * c;
    s = s + C(wiso(k)) * d;
  }
  return C(2) * s;
}
// Isotropic gradient of lambda(rho), lambda evaluated at each stencil point.
template <typename C>
__device__ __forceinline__ void iso_grad_lambda(const Geo& g, const Phys& ph, const C* __restrict__ rho, int x, int y,
                                                C& gx, C& gy) {
  C sx = C(0), sy = C(0);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const int ex = exv(k), ey = eyv(k);
    const C w = C(wiso(k));
    C d = lam_of(ph, at(g, rho, x + ex, y + ey)) - lam_of(ph, at(g, rho, x - ex, y - ey));
    if (ex != 0) sx = sx + w * d * C(ex);
    if (ey != 0) sy = sy + w * d * C(ey);
  }
  gx = sx;
  gy = sy;
}
// Third-order upwind derivative along (dx, dy), biased against the sign of v.
template <typename C>
__device__ __forceinline__ C upwind3(const Geo& g, const C* __restrict__ fld, int x, int y, int dx, int dy, C v) {
  C c = at(g, fld, x, y);
  if (v >= C(0)) {
    C m2 = at(g, fld, x - 2 * dx, y - 2 * dy) - c;
    C m1 = at(g, fld, x - dx, y - dy) - c;
    C p1 = at(g, fld, x + dx, y + dy) - c;
    return (m2 - C(6) * m1 + C(2) * p1) / C(6);
  } else {
    C m1 = at(g, fld, x - dx, y - dy) - c;
    C p1 = at(g, fld, x + dx, y + dy) - c;
    C p2 = at(g, fld, x + 2 * dx, y + 2 * dy) - c;
    return (-C(2) * m1 + C(6) * p1 - p2) / C(6);
  }
}

// Right-hand side of Eq. (energy) with rho and u frozen.
template <typename C>
__device__ C energy_rhs(const Geo& g, const Phys& ph, const C* __restrict__ T, const C* __restrict__ rho,
                        const C* __restrict__ ux, const C* __restrict__ uy, int x, int y) {
  const long long id = (long long)y * g.pitch + x;
  const C r = rho[id], u = ux[id], v = uy[id], Tc = T[id];
  C conv = u * upwind3(g, T, x, y, 1, 0, u) + v * upwind3(g, T, x, y, 0, 1, v);
  C gx, gy, lx, ly, dxux, dyuy, unused;
  iso_grad(g, T, x, y, gx, gy);
  C lap = iso_lap(g, T, x, y);
  iso_grad_lambda(g, ph, rho, x, y, lx, ly);
  iso_grad<C, true, false>(g, ux, x, y, dxux, unused);
  iso_grad<C, false, true>(g, uy, x, y, unused, dyuy);
  C divu = dxux + dyuy;
  C diff = lam_of(ph, r) * lap + (lx * gx + ly * gy);
  C work = Tc * dpdT_eos(ph, r, Tc) * divu;
  return -conv + diff / (r * C(ph.c_v)) - work / (r * C(ph.c_v));
}

// ---------------------------------------------------------------- streaming (Sec. IV.A BCs)
// Fraction q of the link from fluid node (x, y) along (cx, cy) that lies in the fluid.
__device__ __forceinline__ double link_fraction(const Geo& g, int x, int y, int cx, int cy) {
  double dx = x - g.xc, dy = y - g.yc, r = g.r;
  double A = (double)(cx * cx + cy * cy);
  double B = dx * cx + dy * cy;
  double C0 = dx * dx + dy * dy - r * r;
  return (-B - sqrt(B * B - A * C0)) / A;
}

// Pull with substitutions for nodes next to the wall, the inlet or the outlet.
template <typename C, typename S, bool kWriteSide>
__device__ __noinline__ void pull_slow(const Geo g, const Phys ph, const S* __restrict__ f,
                                       const uint8_t* __restrict__ mask, C* side, int x, int y, C* fo) {
  for (int i = 0; i < 9; ++i) {
    const int cx = cxv(i), cy = cyv(i);
    int sx = x - cx;
    const int sy = wrap_y(g, y - cy);
    if (g.periodic_x) sx = sx < 0 ? sx + g.nx : (sx >= g.nx ? sx - g.nx : sx);
    C v;
    if (sx < 0 || sx >= g.nx) {
      v = C(0);  // unknown at the inlet or outlet; replaced below
    } else if (mask[(long long)sy * g.pitch + sx] & kSolid) {
      // linear interpolated bounce-back; the wall lies along c_opp(i)
      const int io = oppv(i);
      const C q = C(link_fraction(g, x, y, -cx, -cy));
      const C a = ldf<C>(g, f, io, y, x);
      if (q < C(0.5)) {
        int nxp = x + cx;
        const int nyp = wrap_y(g, y + cy);
        if (g.periodic_x) nxp = nxp < 0 ? nxp + g.nx : (nxp >= g.nx ? nxp - g.nx : nxp);
        const bool ok = nxp >= 0 && nxp < g.nx && !(mask[(long long)nyp * g.pitch + nxp] & kSolid);
        v = ok ? C(2) * q * a + (C(1) - C(2) * q) * ldf<C>(g, f, io, nyp, nxp) : a;
      } else {
        v = a / (C(2) * q) + (C(2) * q - C(1)) / (C(2) * q) * ldf<C>(g, f, i, y, x);
      }
    } else {
      v = ldf<C>(g, f, i, sy, sx);
    }
    fo[i] = v;
  }
  if (g.periodic_x) return;
  if (x == 0) {
    // Zou-He velocity inlet, u = (u_in, 0): unknowns f1, f5, f7
    const C u = C(ph.u_in);
    const C rho = (fo[0] + fo[3] + fo[4] + C(2) * (fo[2] + fo[6] + fo[8])) / (C(1) - u);
    fo[1] = fo[2] + C(2.0 / 3.0) * rho * u;
    fo[5] = fo[6] - C(0.5) * (fo[3] - fo[4]) + rho * u / C(6);
    fo[7] = fo[8] + C(0.5) * (fo[3] - fo[4]) + rho * u / C(6);
  }
  if (x == g.nx - 1) {
    // convective outlet: f(t+1) = (f(t) + U f_{nx-2}(t+1)) / (1 + U) for f2, f6, f8
    const C U = C(ph.U_out);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int i = j == 0 ? 2 : (j == 1 ? 6 : 8);
      const C inner = ldf<C>(g, f, i, wrap_y(g, y - cyv(i)), g.nx - 1);
      const C v = (side[j * g.ny + y] + U * inner) / (C(1) + U);
      fo[i] = v;
      if (kWriteSide) side[j * g.ny + y] = v;
    }
  }
}

template <typename C, typename S, bool kWriteSide>
__device__ __forceinline__ void pull_node(const Geo& g, const Phys& ph, const S* __restrict__ f,
                                          const uint8_t* __restrict__ mask, C* side, int x, int y, uint8_t m,
                                          C fo[9]) {
  const bool edge = !g.periodic_x && (x == 0 || x == g.nx - 1);
  if ((m & kNearWall) || edge) {
    pull_slow<C, S, kWriteSide>(g, ph, f, mask, side, x, y, fo);
    return;
  }
  const int ym = y == 0 ? g.ny - 1 : y - 1;
  const int yp = y == g.ny - 1 ? 0 : y + 1;
  int xm = x - 1, xp = x + 1;
  if (g.periodic_x) {
    xm = xm < 0 ? g.nx - 1 : xm;
    xp = xp >= g.nx ? 0 : xp;
  }
  fo[0] = ldf<C>(g, f, 0, y, x);
  fo[1] = ldf<C>(g, f, 1, y, xm);
  fo[2] = ldf<C>(g, f, 2, y, xp);
  fo[3] = ldf<C>(g, f, 3, ym, x);
  fo[4] = ldf<C>(g, f, 4, yp, x);
  fo[5] = ldf<C>(g, f, 5, ym, xm);
  fo[6] = ldf<C>(g, f, 6, yp, xp);
  fo[7] = ldf<C>(g, f, 7, yp, xm);
  fo[8] = ldf<C>(g, f, 8, ym, xp);
}

// ---------------------------------------------------------------- CM collision (Sec. II.A-B)
// Raw moments -> central moments k4, k5 (T = N M), post-collision CMs of Eq. (postColl2),
// m* = N(u)^{-1} k* by forward substitution, f* = M^{-1} m*.  Closed form of the 9x9
// algebra, term order as in the matrix products.
template <typename C>
__device__ __forceinline__ void collide(const C f[9], C rho, C Fx, C Fy, C Fmx, C Fmy, C psi, C omega, C sigma,
                                        C fs[9], C& ux, C& uy) {
  const C m1 = ((((f[1] - f[2]) + f[5]) - f[6]) + f[7]) - f[8];
  const C m2 = ((((f[3] - f[4]) + f[5]) - f[6]) - f[7]) + f[8];
  const C m4 = ((f[1] + f[2]) - f[3]) - f[4];
  const C m5 = ((f[5] + f[6]) - f[7]) - f[8];
  ux = (m1 + C(0.5) * Fx) / rho;
  uy = (m2 + C(0.5) * Fy) / rho;
  const C u = ux, v = uy;
  // shift matrix N(u), App. A
  const C N10 = -u, N20 = -v;
  const C N30 = u * u + v * v, N31 = C(-2) * u, N32 = C(-2) * v;
  const C N40 = u * u - v * v, N41 = C(-2) * u, N42 = C(2) * v;
  const C N50 = u * v, N51 = -v, N52 = -u;
  const C N60 = -u * u * v, N61 = C(2) * u * v, N62 = u * u, N63 = -v / C(2), N64 = -v / C(2), N65 = C(-2) * u;
  const C N70 = -u * v * v, N71 = v * v, N72 = C(2) * u * v, N73 = -u / C(2), N74 = u / C(2), N75 = C(-2) * v;
  const C N80 = u * u * v * v, N81 = C(-2) * u * v * v, N82 = C(-2) * u * u * v, N83 = (u * u + v * v) / C(2),
          N84 = -(u * u - v * v) / C(2), N85 = C(4) * u * v, N86 = C(-2) * v, N87 = C(-2) * u;
  const C k4 = ((N40 * rho + N41 * m1) + N42 * m2) + m4;
  const C k5 = ((N50 * rho + N51 * m1) + N52 * m2) + m5;
  // post-collision central moments
  const C alpha = sigma != C(0) ? sigma / (psi * psi) : C(0);
  const C Fm2 = Fmx * Fmx + Fmy * Fmy;
  const C ks0 = rho;
  const C ks1 = C(0.5) * Fx;
  const C ks2 = C(0.5) * Fy;
  const C ks3 = C(2) * rho / C(3) + C(0.5) * (C(4) * alpha * Fm2);
  const C ks4 = (C(1) - omega) * k4;
  const C ks5 = (C(1) - omega) * k5;
  const C ks6 = C(0.5) * (Fy / C(3));
  const C ks7 = C(0.5) * (Fx / C(3));
  const C ks8 = rho / C(9) + C(0.5) * (C(4.0 / 3.0) * alpha * Fm2);
  // forward substitution N m* = k*
  const C ms0 = ks0;
  const C ms1 = ks1 - N10 * ms0;
  const C ms2 = ks2 - N20 * ms0;
  const C ms3 = ((ks3 - N30 * ms0) - N31 * ms1) - N32 * ms2;
  const C ms4 = ((ks4 - N40 * ms0) - N41 * ms1) - N42 * ms2;
  const C ms5 = ((ks5 - N50 * ms0) - N51 * ms1) - N52 * ms2;
  const C ms6 = (((((ks6 - N60 * ms0) - N61 * ms1) - N62 * ms2) - N63 * ms3) - N64 * ms4) - N65 * ms5;
  const C ms7 = (((((ks7 - N70 * ms0) - N71 * ms1) - N72 * ms2) - N73 * ms3) - N74 * ms4) - N75 * ms5;
  const C ms8 =
      (((((((ks8 - N80 * ms0) - N81 * ms1) - N82 * ms2) - N83 * ms3) - N84 * ms4) - N85 * ms5) - N86 * ms6) - N87 * ms7;
  // f* = M^{-1} m*
  const C h = C(0.5), q = C(0.25);
  fs[0] = (ms0 - ms3) + ms8;
  fs[1] = (((h * ms1 + q * ms3) + q * ms4) - h * ms7) - h * ms8;
  fs[2] = (((-h * ms1 + q * ms3) + q * ms4) + h * ms7) - h * ms8;
  fs[3] = (((h * ms2 + q * ms3) - q * ms4) - h * ms6) - h * ms8;
  fs[4] = (((-h * ms2 + q * ms3) - q * ms4) + h * ms6) - h * ms8;
  fs[5] = ((q * ms5 + q * ms6) + q * ms7) + q * ms8;
  fs[6] = ((q * ms5 - q * ms6) - q * ms7) + q * ms8;
  fs[7] = ((-q * ms5 - q * ms6) + q * ms7) + q * ms8;
  fs[8] = ((-q * ms5 + q * ms6) - q * ms7) + q * ms8;
}

// ---------------------------------------------------------------- kernels
template <typename C, typename S>
__global__ void __launch_bounds__(kBX* kBY) k_rho_psi(Geo g, Phys ph, const S* __restrict__ f,
                                                      const C* __restrict__ T, const uint8_t* __restrict__ mask,
                                                      C* side, C* __restrict__ psi, int* status) {
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const long long id = (long long)y * g.pitch + x;
  const uint8_t m = mask[id];
  double r;
  if (m & kSolid) {
    r = ph.rho_s;
  } else {
    C fo[9];
    pull_node<C, S, false>(g, ph, f, mask, side, x, y, m, fo);
    C s = fo[0];
#pragma unroll
    for (int i = 1; i < 9; ++i) s = s + fo[i];
    r = (double)s;
  }
  double rad;
  const double p = psi_eos(ph, r, (double)T[id], rad);
  if (!(rad > 0.0)) atomicOr(status, 2);
  psi[id] = (C)p;
}

template <typename C, typename S>
__global__ void __launch_bounds__(kBX* kBY) k_collide(Geo g, Phys ph, const S* __restrict__ f, S* __restrict__ fn,
                                                      const C* __restrict__ psi, const uint8_t* __restrict__ mask,
                                                      C* side, C* __restrict__ rho_o, C* __restrict__ ux_o,
                                                      C* __restrict__ uy_o, int forcing, int* status) {
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const long long id = (long long)y * g.pitch + x;
  const uint8_t m = mask[id];
  if (m & kSolid) {
    rho_o[id] = C(ph.rho_s);
    ux_o[id] = C(0);
    uy_o[id] = C(0);
    return;
  }
  C fo[9];
  pull_node<C, S, true>(g, ph, f, mask, side, x, y, m, fo);
  C rho = fo[0];
#pragma unroll
  for (int i = 1; i < 9; ++i) rho = rho + fo[i];
  const bool multiphase = ph.G != 0.0;
  const C cs2 = C(1.0 / 3.0);
  C Fmx = C(0), Fmy = C(0), Fx = C(0), Fy = C(0), p0 = C(0);
  if (multiphase) p0 = psi[id];
  if (forcing && multiphase) {
    C sx, sy;
    iso_grad(g, psi, x, y, sx, sy);
    Fmx = -C(ph.G) * cs2 * p0 * sx;
    Fmy = -C(ph.G) * cs2 * p0 * sy;
  }
  if (forcing) {
    Fx = Fmx - (rho - C(ph.rho_l)) * C(ph.g);
    Fy = Fmy;
  }
  const C omega = C(1) / (nu_of(ph, rho) / cs2 + C(0.5));
  const C sig = (forcing && multiphase) ? C(ph.sigma) : C(0);
  C fs[9], ux, uy;
  collide(fo, rho, Fx, Fy, Fmx, Fmy, p0, omega, sig, fs, ux, uy);
#pragma unroll
  for (int i = 0; i < 9; ++i) fn[i * g.plane + id] = static_cast<S>(fs[i]);
  rho_o[id] = rho;
  ux_o[id] = ux;
  uy_o[id] = uy;
  if (!(rho > C(0)) || !(ux == ux) || !(uy == uy)) atomicOr(status, 1);
}

template <typename C>
__global__ void __launch_bounds__(256) k_heat_flux(Geo g, Phys ph, const C* __restrict__ T, const C* __restrict__ rho,
                                                    const int* __restrict__ bnode, const double* __restrict__ bn,
                                                    int nb, double* hf) {
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const int id = bnode[b];
    const int y = id / g.pitch, x = id - y * g.pitch;
    C gx, gy;
    iso_grad(g, T, x, y, gx, gy);
    const double lam = (double)lam_of(ph, rho[id]);
    acc += -lam * ((double)gx * bn[b] + (double)gy * bn[nb + b]);
  }
  // fixed-shape tree: warp shuffles, then warp 0 over the 8 warp sums
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ double ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) {
      const double q = nb > 0 ? v / nb : 0.0;
      hf[0] = q;
      hf[1] += q;
      hf[2] += q * q;
      hf[3] += 1.0;
    }
  }
}

template <typename C>
__global__ void __launch_bounds__(kBX* kBY) k_T_stage(Geo g, Phys ph, const C* __restrict__ Tin, const C* Tbase,
                                                      C* Tout, const C* __restrict__ rho, const C* __restrict__ ux,
                                                      const C* __restrict__ uy, const uint8_t* __restrict__ mask,
                                                      int stage) {
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const long long id = (long long)y * g.pitch + x;
  C out;
  if (mask[id] & kSolid) {
    out = C(ph.T_wall);
  } else if (!g.periodic_x && x == 0) {
    out = C(ph.T_sat);
  } else {
    const C L = energy_rhs(g, ph, Tin, rho, ux, uy, x, y);
    out = stage == 1 ? Tin[id] + L : ((Tbase[id] + Tin[id]) + L) * C(0.5);
  }
  Tout[id] = out;
}

// ---------------------------------------------------------------- init / export / import
// Fourth-order Hermite equilibrium, Eq. (equi).
__device__ __forceinline__ void feq_hermite(double rho, double ux, double uy, double fe[9]) {
  const double cs2 = 1.0 / 3.0;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const double w = i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    const double cx = cxv(i), cy = cyv(i);
    const double Hxx = cx * cx - cs2, Hyy = cy * cy - cs2, Hxy = cx * cy;
    const double Hxxy = cx * cx * cy - cs2 * cy;
    const double Hxyy = cx * cy * cy - cs2 * cx;
    const double Hxxyy = cx * cx * cy * cy - cs2 * (cx * cx + cy * cy) + cs2 * cs2;
    const double t1 = (cx * ux + cy * uy) / cs2;
    const double t2 = (Hxx * ux * ux + 2.0 * Hxy * ux * uy + Hyy * uy * uy) / (2.0 * cs2 * cs2);
    const double t3 = (Hxxy * ux * ux * uy + Hxyy * ux * uy * uy) / (2.0 * cs2 * cs2 * cs2);
    const double t4 = Hxxyy * ux * ux * uy * uy / (4.0 * cs2 * cs2 * cs2 * cs2);
    fe[i] = w * rho * (1.0 + t1 + t2 + t3 + t4);
  }
}

// SplitMix64 (Steele, Lea, Flood 2014): value k of stream `seed`, mapped to [-1, 1).
__device__ __forceinline__ double splitmix_pm1(unsigned long long seed, unsigned long long k) {
  unsigned long long z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * 0x1.0p-53 * 2.0 - 1.0;
}

// in: optional dense [ny][nx] double arrays (rho, drho, ux, uy, T), any NULL.
template <typename C, typename S>
__global__ void __launch_bounds__(kBX* kBY) k_init(Geo g, Phys ph, const double* rho0, const double* drho,
                                                   const double* ux0, const double* uy0, const double* T0,
                                                   unsigned long long seed, double noise_amp, S* f, C* T, C* rho_o,
                                                   C* ux_o, C* uy_o, C* side, const uint8_t* __restrict__ mask) {
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const long long id = (long long)y * g.pitch + x;
  const long long k = (long long)y * g.nx + x;
  double r = rho0 ? rho0[k] : ph.rho_l;
  r = r + (drho ? drho[k] : noise_amp * splitmix_pm1(seed, (unsigned long long)k));
  double u = ux0 ? ux0[k] : ph.u_in, v = uy0 ? uy0[k] : 0.0;
  double t = T0 ? T0[k] : ph.T_sat;
  if (mask[id] & kSolid) {
    r = ph.rho_s;
    u = 0.0;
    v = 0.0;
    t = ph.T_wall;
  }
  double fe[9];
  feq_hermite(r, u, v, fe);
#pragma unroll
  for (int i = 0; i < 9; ++i) f[i * g.plane + id] = static_cast<S>(fe[i]);
  T[id] = (C)t;
  rho_o[id] = (C)r;
  ux_o[id] = (C)u;
  uy_o[id] = (C)v;
  if (!g.periodic_x && x == g.nx - 1) {
    side[0 * g.ny + y] = (C)fe[2];
    side[1 * g.ny + y] = (C)fe[6];
    side[2 * g.ny + y] = (C)fe[8];
  }
}

template <typename E>
__global__ void k_export(Geo g, const E* __restrict__ src, long long src_pitch, int rows, double* __restrict__ dst,
                         int ncols) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= ncols || y >= rows) return;
  dst[(long long)y * ncols + x] = (double)src[(long long)y * src_pitch + x];
}

static __global__ void k_export_solid(Geo g, const uint8_t* __restrict__ mask, double* __restrict__ dst) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  dst[(long long)y * g.nx + x] = (mask[(long long)y * g.pitch + x] & kSolid) ? 1.0 : 0.0;
}

template <typename E>
__global__ void k_import(Geo g, E* __restrict__ dst, long long dst_pitch, int rows, const double* __restrict__ src,
                         int ncols) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= ncols || y >= rows) return;
  dst[(long long)y * dst_pitch + x] = static_cast<E>(src[(long long)y * ncols + x]);
}

}  // namespace kern

// ---------------------------------------------------------------- launchers
template <typename C, typename S>
int step_impl(const Geo& g, const Phys& ph, const Dev& d, int cur, int forcing, int energy, cudaStream_t s,
              const LaunchHook* hook) {
  using namespace kern;
  const dim3 blk(kBX, kBY), grd((g.nx + kBX - 1) / kBX, (g.ny + kBY - 1) / kBY);
  const S* f = static_cast<const S*>(d.f[cur]);
  S* fn = static_cast<S*>(d.f[cur ^ 1]);
  C* T = static_cast<C*>(d.T);
  C* T1 = static_cast<C*>(d.T1);
  C* psi = static_cast<C*>(d.psi);
  C* rho = static_cast<C*>(d.rho);
  C* ux = static_cast<C*>(d.ux);
  C* uy = static_cast<C*>(d.uy);
  C* side = static_cast<C*>(d.side);
  int n = 0;
  auto pre = [&](int k) { if (hook) hook->before(hook->self, k); };
  auto post = [&](int k) { if (hook) hook->after(hook->self, k); ++n; };
  if (ph.G != 0.0) {
    pre(kKRhoPsi);
    k_rho_psi<C, S><<<grd, blk, 0, s>>>(g, ph, f, T, d.mask, side, psi, d.status);
    post(kKRhoPsi);
  }
  pre(kKCollide);
  k_collide<C, S><<<grd, blk, 0, s>>>(g, ph, f, fn, psi, d.mask, side, rho, ux, uy, forcing, d.status);
  post(kKCollide);
  if (energy && forcing) {
    if (d.nb > 0) {
      pre(kKHeatFlux);
      k_heat_flux<C><<<1, 256, 0, s>>>(g, ph, T, rho, d.bnode, d.bn, d.nb, d.hf);
      post(kKHeatFlux);
    }
    pre(kKTStage1);
    k_T_stage<C><<<grd, blk, 0, s>>>(g, ph, T, T, T1, rho, ux, uy, d.mask, 1);
    post(kKTStage1);
    pre(kKTStage2);
    k_T_stage<C><<<grd, blk, 0, s>>>(g, ph, T1, T, T, rho, ux, uy, d.mask, 2);
    post(kKTStage2);
  }
  return cudaPeekAtLastError() == cudaSuccess ? n : -1;
}

template <typename C, typename S>
int export_impl(const Geo& g, const Dev& d, int cur, int which, double* dst, cudaStream_t s) {
  using namespace kern;
  const dim3 blk(256);
  if (which >= 20 && which < 23) {
    const C* src = static_cast<const C*>(d.side) + (which - 20) * g.ny;
    k_export<C><<<dim3((g.ny + 255) / 256, 1), blk, 0, s>>>(g, src, g.ny, 1, dst, g.ny);
  } else if (which >= 10 && which < 19) {
    const S* src = static_cast<const S*>(d.f[cur]) + (which - 10) * g.plane;
    k_export<S><<<dim3((g.nx + 255) / 256, g.ny), blk, 0, s>>>(g, src, g.pitch, g.ny, dst, g.nx);
  } else if (which == 5) {
    k_export_solid<<<dim3((g.nx + 255) / 256, g.ny), blk, 0, s>>>(g, d.mask, dst);
  } else {
    const void* p = which == 0 ? d.rho : which == 1 ? d.ux : which == 2 ? d.uy : which == 3 ? d.T : d.psi;
    k_export<C><<<dim3((g.nx + 255) / 256, g.ny), blk, 0, s>>>(g, static_cast<const C*>(p), g.pitch, g.ny, dst, g.nx);
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

template <typename C, typename S>
int import_impl(const Geo& g, const Dev& d, int cur, int which, const double* src, cudaStream_t s) {
  using namespace kern;
  const dim3 blk(256);
  if (which >= 20 && which < 23) {
    C* dst = static_cast<C*>(d.side) + (which - 20) * g.ny;
    k_import<C><<<dim3((g.ny + 255) / 256, 1), blk, 0, s>>>(g, dst, g.ny, 1, src, g.ny);
  } else if (which >= 10 && which < 19) {
    S* dst = static_cast<S*>(d.f[cur]) + (which - 10) * g.plane;
    k_import<S><<<dim3((g.nx + 255) / 256, g.ny), blk, 0, s>>>(g, dst, g.pitch, g.ny, src, g.nx);
  } else if (which == 3) {
    k_import<C><<<dim3((g.nx + 255) / 256, g.ny), blk, 0, s>>>(g, static_cast<C*>(d.T), g.pitch, g.ny, src, g.nx);
  } else {
    return -1;
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

template <typename C, typename S>
int init_impl(const Geo& g, const Phys& ph, const Dev& d, const double* rho0, const double* drho, const double* ux0,
              const double* uy0, const double* T0, unsigned long long seed, double amp, cudaStream_t s) {
  using namespace kern;
  const dim3 blk(kBX, kBY), grd((g.nx + kBX - 1) / kBX, (g.ny + kBY - 1) / kBY);
  k_init<C, S><<<grd, blk, 0, s>>>(g, ph, rho0, drho, ux0, uy0, T0, seed, amp, static_cast<S*>(d.f[0]),
                                   static_cast<C*>(d.T), static_cast<C*>(d.rho), static_cast<C*>(d.ux),
                                   static_cast<C*>(d.uy), static_cast<C*>(d.side), d.mask);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace lbm
