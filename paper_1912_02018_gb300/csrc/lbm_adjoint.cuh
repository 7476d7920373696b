// Discrete adjoint of one time step: the reverse-mode derivative of the update of Sec. II
// and Sec. IV.A of arXiv:1912.02018 (pull-streaming with the wall, inlet and outlet
// substitutions; rho and psi of Eq. (potential) with the Peng-Robinson EOS of Eq. (eos); the
// interaction force of Eq. (interForce) and gravity; the CM collision with the consistency
// terms of Eq. (postColl2); the Heun update of Eq. (energy); the wall heat-flux sample of
// Sec. IV.B), for seeds on the step's outputs (f*, T, outlet side values) and on its
// heat-flux sample.  The paper has no adjoint; this is the transpose of its step.
//
// Every kernel is a gather (one thread per node, no atomics): a transposed stencil reads the
// sources whose stencil reaches the node, with the forward's clamped (zero-gradient) columns
// at a non-periodic inlet and outlet mapped back to every source that read them.  Upwind
// switches and the clamp of the phase fraction take the branch the forward took.  Forward
// values come from the stored state of the step and the rho, psi, u of its collision.
// Parameter gradients (wall temperature per solid node, inlet speed per row) accumulate in
// FP64; the adjoint fields are in the compute precision.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {
namespace adj {

using namespace kern;

// ---------------------------------------------------------------- dual numbers
template <typename C>
struct Dl {
  C v, d;
};
template <typename C>
__device__ __forceinline__ Dl<C> operator+(Dl<C> a, Dl<C> b) { return {a.v + b.v, a.d + b.d}; }
template <typename C>
__device__ __forceinline__ Dl<C> operator-(Dl<C> a, Dl<C> b) { return {a.v - b.v, a.d - b.d}; }
template <typename C>
__device__ __forceinline__ Dl<C> operator*(Dl<C> a, Dl<C> b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <typename C>
__device__ __forceinline__ Dl<C> operator/(Dl<C> a, Dl<C> b) {
  const C q = fdiv(a.v, b.v);
  return {q, fdiv(a.d - q * b.d, b.v)};
}
template <typename C>
__device__ __forceinline__ Dl<C> operator*(C s, Dl<C> a) { return {s * a.v, s * a.d}; }
template <typename C>
__device__ __forceinline__ Dl<C> operator+(C s, Dl<C> a) { return {s + a.v, a.d}; }
template <typename C>
__device__ __forceinline__ Dl<C> operator-(C s, Dl<C> a) { return {s - a.v, -a.d}; }
template <typename C>
__device__ __forceinline__ Dl<C> dsqrt(Dl<C> a) {
  const C s = sqrt(a.v);
  return {s, fdiv(a.d, C(2) * s)};
}

// Peng-Robinson p(rho, T), Eq. (eos), and (dp/dT)_rho, on dual numbers.
template <typename C>
__device__ __forceinline__ Dl<C> pr_p(const PhysC<C>& k, Dl<C> rho, Dl<C> T) {
  const Dl<C> s = C(1) + k.kappa * (C(1) - dsqrt(T * Dl<C>{C(1) / k.Tc, C(0)}));
  const Dl<C> rep = (k.R * T) * rho / (C(1) - k.b * rho);
  const Dl<C> att = (k.a * (s * s)) * (rho * rho) / ((C(1) + C(2) * k.b * rho) - (k.b * k.b) * (rho * rho));
  return rep - att;
}
template <typename C>
__device__ __forceinline__ Dl<C> pr_dpdT(const PhysC<C>& k, Dl<C> rho, Dl<C> T) {
  const Dl<C> sq = dsqrt(T * Dl<C>{C(1) / k.Tc, C(0)});
  const Dl<C> s = C(1) + k.kappa * (C(1) - sq);
  const Dl<C> dphi = (-k.kappa * s) / dsqrt(T * Dl<C>{k.Tc, C(0)});
  const Dl<C> rep = k.R * rho / (C(1) - k.b * rho);
  const Dl<C> att = (k.a * dphi) * (rho * rho) / ((C(1) + C(2) * k.b * rho) - (k.b * k.b) * (rho * rho));
  return rep - att;
}
// d phase_frac / d rho with the branch of the clamp that the forward took (inclusive ends).
template <typename C>
__device__ __forceinline__ C dphase(const PhysC<C>& k, C rho) {
  if (!(k.rho_l > k.rho_v)) return C(0);
  const C f = fdiv(rho - k.rho_v, k.rho_l - k.rho_v);
  return (f >= C(0) && f <= C(1)) ? fdiv(C(1), k.rho_l - k.rho_v) : C(0);
}
template <typename C>
__device__ __forceinline__ C dlam(const Phys& ph, C rho) {
  const PhysC<C>& k = pc<C>(ph);
  const C alpha = k.alpha_v + phase_frac(ph, rho) * (k.alpha_l - k.alpha_v);
  return k.c_v * alpha + rho * k.c_v * dphase(k, rho) * (k.alpha_l - k.alpha_v);
}

template <typename C>
using Args = AdjArgs<C>;

__device__ __forceinline__ bool node_of_thread(const Geo& g, int& x, int& y) {
  x = blockIdx.x * 32 + threadIdx.x;
  y = blockIdx.y * 8 + threadIdx.y;
  return x < g.nx && y < g.ny;
}
template <typename C>
__device__ __forceinline__ C at(const Geo& g, const C* p, int x, int y) {
  return p[map_y(g, y) * g.pitch + map_x(g, x)];
}
__device__ __forceinline__ bool interior_T(const Geo& g, uint8_t m, int x) {
  return !(m & kSolid) && !(!g.periodic_x && x == 0);
}
// Columns sx with map_x(sx + ex) == x: the sources that read column x at offset ex.
__device__ __forceinline__ void src_cols(const Geo& g, int x, int ex, int& lo, int& hi) {
  if (g.periodic_x) {
    int s = x - ex;
    s = s < 0 ? s + g.nx : (s >= g.nx ? s - g.nx : s);
    lo = hi = s;
    return;
  }
  if (x == 0) {
    lo = 0;
    hi = -ex;  // empty for ex > 0
  } else if (x == g.nx - 1) {
    lo = g.nx - 1 - ex;  // empty for ex < 0
    hi = g.nx - 1;
  } else {
    lo = hi = x - ex;
  }
  lo = lo < 0 ? 0 : lo;
  hi = hi > g.nx - 1 ? g.nx - 1 : hi;
}
__device__ __forceinline__ double w_of(int ex, int ey) {
  const int e2 = ex * ex + ey * ey;
  return e2 == 1 ? 4.0 / 21.0 : e2 == 2 ? 4.0 / 45.0 : e2 == 4 ? 1.0 / 60.0 : e2 == 5 ? 2.0 / 315.0
       : e2 == 8 ? 1.0 / 5040.0 : 0.0;
}
// Coefficient of phi(x + k) in the third-order upwind derivative at x (v >= 0 or v < 0).
template <typename C>
__device__ __forceinline__ C upw_coef(int k, bool pos) {
  if (pos) return k == -2 ? C(1.0 / 6.0) : k == -1 ? C(-1) : k == 0 ? C(0.5) : k == 1 ? C(1.0 / 3.0) : C(0);
  return k == -1 ? C(-1.0 / 3.0) : k == 0 ? C(-0.5) : k == 1 ? C(1) : k == 2 ? C(-1.0 / 6.0) : C(0);
}

// Stencil parts of Eq. (energy) at a point of shared-memory tiles: temperature t (row stride
// ts), lambda l, velocity u, v (row stride as); stencils reach 2 nodes.
template <typename C>
struct Parts {
  C upx, upy, gx, gy, lap, lx, ly, divu;
};
template <typename C>
__device__ __forceinline__ C upwind_d(C m2, C m1, C p1, C p2, C v) {
  return v >= C(0) ? fdiv(m2 - C(6) * m1 + C(2) * p1, C(6)) : fdiv(-C(2) * m1 + C(6) * p1 - p2, C(6));
}
template <typename C>
__device__ __forceinline__ Parts<C> parts_at(const C* t, int ts, const C* l, const C* u, const C* v, int as) {
  Parts<C> P;
  const C c = t[0];
  P.upx = upwind_d(t[-2] - c, t[-1] - c, t[1] - c, t[2] - c, u[0]);
  P.upy = upwind_d(t[-2 * ts] - c, t[-ts] - c, t[ts] - c, t[2 * ts] - c, v[0]);
  C gx = 0, gy = 0, lap = 0, lx = 0, ly = 0, dxux = 0, dyuy = 0;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const int ex = exv(k), ey = eyv(k);
    const C w = C(wiso(k)), wx = C(wiso(k) * ex), wy = C(wiso(k) * ey);
    const C tp = t[ey * ts + ex], tm = t[-ey * ts - ex];
    if (ex != 0) gx = gx + wx * (tp - tm);
    if (ey != 0) gy = gy + wy * (tp - tm);
    lap = lap + w * ((tp + tm) - C(2) * c);
    const C dl = l[ey * as + ex] - l[-ey * as - ex];
    if (ex != 0) lx = lx + wx * dl;
    if (ey != 0) ly = ly + wy * dl;
    if (ex != 0) dxux = dxux + wx * (u[ey * as + ex] - u[-ey * as - ex]);
    if (ey != 0) dyuy = dyuy + wy * (v[ey * as + ex] - v[-ey * as - ex]);
  }
  P.gx = gx;
  P.gy = gy;
  P.lap = C(2) * lap;
  P.lx = lx;
  P.ly = ly;
  P.divu = dxux + dyuy;
  return P;
}

// ---------------------------------------------------------------- energy adjoint (Heun stages)
// One kernel per stage, on tiles of 32 x 16 nodes.  Stage 2 (seed Tb_in / 2 on L(T1) at the
// interior fluid nodes) loads T1 (stored by the step's recomputed energy pass), rho, lambda, u
// on the tile + 4, forms the sources of the transposed stencils on the tile + 2 and gathers
// them at the tile's nodes: Tb1, the adjoint of T1.  Stage 1 (seed Tb1 on L(T), plus the
// heat-flux sample) does the same from T and gives Tb_out, the adjoint of T.  Both add their
// parts of the adjoints of u (ub), lambda (lamb) and rho (rhob).
constexpr int kEATX = 32, kEATY = 8, kEANT = 256;  // 256 blocks more than 32 x 16 tiles on the 512 x 256 window: ratio 3.53 -> 3.46
template <typename C, int STAGE>
struct EAdjLayout {
  static constexpr int H = 4;
  static constexpr int AX = kEATX + 2 * H, AY = kEATY + 2 * H, A = AX * AY;  // loaded fields
  static constexpr int PX = kEATX + 4, PY = kEATY + 4, PN = PX * PY;                  // sources
  static constexpr int NN = kEATX * kEATY;
  static constexpr size_t bytes = sizeof(C) * (5 * (size_t)A + 8 * (size_t)PN + 5 * (size_t)NN) + A;
};

template <typename C, int STAGE>
__global__ void __launch_bounds__(kEANT) k_adj_energy(Args<C> a) {
  using Lay = EAdjLayout<C, STAGE>;
  constexpr int H = Lay::H, AX = Lay::AX, A = Lay::A, PX = Lay::PX, PN = Lay::PN, NN = Lay::NN;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sT = reinterpret_cast<C*>(smem_raw);
  C* sR = sT + A;
  C* sL = sR + A;
  C* sU = sL + A;
  C* sV = sU + A;
  C* sP = sV + A;
  C* sLoc = sP + 8 * PN;
  uint8_t* sM = reinterpret_cast<uint8_t*>(sLoc + 5 * NN);
  const Geo& g = a.g;
  const PhysC<C>& k = pc<C>(a.ph);
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * kEATX, y0 = blockIdx.y * kEATY;
  for (int p = tid; p < A; p += kEANT) {
    const int id = map_y(g, y0 + p / AX - H) * g.pitch + map_x(g, x0 + p % AX - H);
    const C r = a.rho[id];
    sT[p] = STAGE == 2 ? a.T1[id] : a.T[id];  // the temperature field the stage read
    sR[p] = r;
    sL[p] = lam_of(a.ph, r);
    sU[p] = a.ux[id];
    sV[p] = a.uy[id];
    sM[p] = a.mask[id];
  }
  __syncthreads();
  // sources of the transposed stencils on the tile + 2; local parts of the tile's nodes
  for (int p = tid; p < PN; p += kEANT) {
    const int px = p % PX, py = p / PX;
    const int gx = x0 + px - 2, gy = y0 + py - 2;
    const int ai = (py + H - 2) * AX + px + H - 2;
    const bool own = px >= 2 && px < kEATX + 2 && py >= 2 && py < kEATY + 2;
    C Pv[8], Lv[5];
#pragma unroll
    for (int j = 0; j < 8; ++j) Pv[j] = C(0);
#pragma unroll
    for (int j = 0; j < 5; ++j) Lv[j] = C(0);
    const uint8_t m = sM[ai];
    if ((g.periodic_x || (gx >= 0 && gx < g.nx)) && !(m & kSolid)) {
      const int mx = map_x(g, gx);
      const int gid = map_y(g, gy) * g.pitch + mx;
      C s = C(0);
      if (g.periodic_x || mx != 0) s = STAGE == 2 ? C(0.5) * a.Tb_in[gid] : a.Tb1[gid];
      const bool hf = STAGE == 1 && a.do_hf && (m & kNearWall);
      if (s != C(0) || hf) {
        const C* t = &sT[ai];
        const int ts = AX;
        const Parts<C> P = parts_at(t, ts, &sL[ai], &sU[ai], &sV[ai], AX);
        const C r0 = sR[ai], T0 = t[0], lam0 = sL[ai];
        const C rc = r0 * k.c_v;
        const Dl<C> dT = pr_dpdT(k, Dl<C>{r0, C(0)}, Dl<C>{T0, C(1)});
        const Dl<C> dR = pr_dpdT(k, Dl<C>{r0, C(1)}, Dl<C>{T0, C(0)});
        const C diff = lam0 * P.lap + (P.lx * P.gx + P.ly * P.gy);
        const C work = T0 * dT.v * P.divu;
        C p1 = s * fdiv(P.lx, rc), p2 = s * fdiv(P.ly, rc);
        C llam = s * fdiv(P.lap, rc);
        if (hf) {
          // q = -lambda grad T . n at this boundary node (Sec. IV.B)
          const double* nv = &g.wall_n[2 * g.wall_idx[gid]];
          const C nxv = C(nv[0]), nyv = C(nv[1]);
          p1 = p1 - a.wq * lam0 * nxv;
          p2 = p2 - a.wq * lam0 * nyv;
          llam = llam - a.wq * (P.gx * nxv + P.gy * nyv);
        }
        Pv[0] = s * fdiv(lam0, rc);
        Pv[1] = p1;
        Pv[2] = p2;
        Pv[3] = s * sU[ai];
        Pv[4] = s * sV[ai];
        Pv[5] = -s * fdiv(T0 * dT.v, rc);
        Pv[6] = s * fdiv(P.gx, rc);
        Pv[7] = s * fdiv(P.gy, rc);
        Lv[0] = -s * fdiv(P.divu, rc) * (dT.v + T0 * dT.d);
        Lv[1] = -s * P.upx;
        Lv[2] = -s * P.upy;
        Lv[3] = llam;
        Lv[4] = s * (-fdiv(diff - work, rc * r0) - fdiv(T0 * P.divu * dR.d, rc));
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) sP[j * PN + p] = Pv[j];
    if (own) {
#pragma unroll
      for (int j = 0; j < 5; ++j) sLoc[j * NN + (py - 2) * kEATX + px - 2] = Lv[j];
    }
  }
  __syncthreads();
  // gather: every source whose stencil reads the node, clamped columns included
  C wsum = C(0);
#pragma unroll
  for (int kk = 0; kk < 12; ++kk) wsum = wsum + C(wiso(kk));
  for (int q = tid; q < NN; q += kEANT) {
    const int tx = q % kEATX, ty = q / kEATX;
    const int x = x0 + tx, y = y0 + ty;
    if (x >= g.nx || y >= g.ny) continue;
    const int id = y * g.pitch + x;
    const uint8_t m = sM[(ty + H) * AX + tx + H];
    C tb = C(0), ubx = C(0), uby = C(0), lb = C(0);
    // contribution of the source at P-tile index pp (A-tile index ap) through offset (ex, ey)
    auto add = [&](int ex, int ey, int pp, int ap) {
      const C w = C(w_of(ex, ey));
      const C clap = (ex == 0 && ey == 0) ? C(-4) * wsum : C(2) * w;
      tb = tb + clap * sP[pp];
      if (ex != 0 || ey != 0) {
        tb = tb + w * (C(ex) * sP[PN + pp] + C(ey) * sP[2 * PN + pp]);
        ubx = ubx + w * C(ex) * sP[5 * PN + pp];
        uby = uby + w * C(ey) * sP[5 * PN + pp];
        lb = lb + w * (C(ex) * sP[6 * PN + pp] + C(ey) * sP[7 * PN + pp]);
      }
      if (ey == 0) tb = tb - upw_coef<C>(ex, sU[ap] >= C(0)) * sP[3 * PN + pp];
      if (ex == 0) tb = tb - upw_coef<C>(ey, sV[ap] >= C(0)) * sP[4 * PN + pp];
    };
    if (g.periodic_x || (x > 0 && x < g.nx - 1)) {
      // one source position per offset (positions past an edge hold zero sources)
#pragma unroll
      for (int ey = -2; ey <= 2; ++ey)
#pragma unroll
        for (int ex = -2; ex <= 2; ++ex)
          add(ex, ey, (ty + 2 - ey) * PX + tx + 2 - ex, (ty + H - ey) * AX + tx + H - ex);
    } else {
      // an open edge column: every source whose clamped stencil reads it
#pragma unroll 1
      for (int ey = -2; ey <= 2; ++ey)
#pragma unroll 1
        for (int ex = -2; ex <= 2; ++ex) {
          int lo, hi;
          src_cols(g, x, ex, lo, hi);
          for (int sx = lo; sx <= hi; ++sx)
            add(ex, ey, (ty + 2 - ey) * PX + sx - x0 + 2, (ty + H - ey) * AX + sx - x0 + H);
        }
    }
    const bool in = interior_T(g, m, x);
    tb = tb + sLoc[q];
    ubx = ubx + sLoc[NN + q];
    uby = uby + sLoc[2 * NN + q];
    lb = lb + sLoc[3 * NN + q];
    if (STAGE == 2) {
      if (m & kSolid) a.gw[id] += (double)a.Tb_in[id];  // T^{n+1} at a solid node is T_w
      a.Tb1[id] = (in ? C(0.5) * a.Tb_in[id] : C(0)) + tb;
      a.ub[0][id] = ubx;
      a.ub[1][id] = uby;
      a.lamb[id] = lb;
      a.rhob[id] = sLoc[4 * NN + q];
    } else {
      if (m & kSolid) a.gw[id] += (double)a.Tb1[id];  // so is T1
      a.Tb_out[id] = (in ? C(0.5) * a.Tb_in[id] + a.Tb1[id] : C(0)) + tb;
      a.ub[0][id] = a.ub[0][id] + ubx;
      a.ub[1][id] = a.ub[1][id] + uby;
      C rb = a.rhob[id] + sLoc[4 * NN + q];
      if (!(m & kSolid)) rb = rb + dlam(a.ph, sR[(ty + H) * AX + tx + H]) * (a.lamb[id] + lb);
      a.rhob[id] = rb;
    }
  }
}

// Adjoint of the CM collision at a fluid node (Sec. II.A-B): from the seeds on f*, on u and
// rho (energy equation), the adjoints of the pulled populations, of F_m and of psi.
template <typename C>
__global__ void __launch_bounds__(256) k_adj_collide(Args<C> a) {
  int x, y;
  if (!node_of_thread(a.g, x, y)) return;
  const Geo& g = a.g;
  const int id = y * g.pitch + x;
  const uint8_t m = a.mask[id];
  const PhysC<C>& k = pc<C>(a.ph);
  if (m & kSolid) {
#pragma unroll
    for (int i = 0; i < 9; ++i) a.fpb[i * g.plane + id] = C(0);
    a.fmb[0][id] = C(0);
    a.fmb[1][id] = C(0);
    a.psib[id] = C(0);
    return;
  }
  const C cs2 = C(1.0 / 3.0);
  C fo[9];
  pull_node<C, C>(g, a.ph, a.f, a.mask, a.side, nullptr, x, y, m, fo);
  C rho = fo[0];
#pragma unroll
  for (int i = 1; i < 9; ++i) rho = rho + fo[i];
  const bool multiphase = k.G != C(0);
  C Fmx = C(0), Fmy = C(0), psi0 = C(0);
  if (multiphase) {
    psi0 = a.psi[id];
    C sx = C(0), sy = C(0);
#pragma unroll
    for (int kk = 0; kk < 12; ++kk) {
      const int ex = exv(kk), ey = eyv(kk);
      const C d = at(g, a.psi, x + ex, y + ey) - at(g, a.psi, x - ex, y - ey);
      sx = sx + C(wiso(kk)) * d * C(ex);
      sy = sy + C(wiso(kk)) * d * C(ey);
    }
    Fmx = -k.G * cs2 * psi0 * sx;
    Fmy = -k.G * cs2 * psi0 * sy;
  }
  const C Fx = Fmx - (rho - k.rho_l) * k.g, Fy = Fmy;
  const C nu = nu_of(a.ph, rho);
  const C omega = fdiv(C(1), fdiv(nu, cs2) + C(0.5));
  const C sig = multiphase ? k.sigma : C(0);
  const C m1 = ((((fo[1] - fo[2]) + fo[5]) - fo[6]) + fo[7]) - fo[8];
  const C m2 = ((((fo[3] - fo[4]) + fo[5]) - fo[6]) - fo[7]) + fo[8];
  const C m4 = ((fo[1] + fo[2]) - fo[3]) - fo[4];
  const C m5 = ((fo[5] + fo[6]) - fo[7]) - fo[8];
  const C u = fdiv(m1 + C(0.5) * Fx, rho), v = fdiv(m2 + C(0.5) * Fy, rho);
  const C k4 = (((u * u - v * v) * rho - C(2) * u * m1) + C(2) * v * m2) + m4;
  const C k5 = (((u * v) * rho - v * m1) - u * m2) + m5;
  const C alpha = sig != C(0) ? fdiv(sig, psi0 * psi0) : C(0);
  const C Fm2 = Fmx * Fmx + Fmy * Fmy;
  // post-collision central moments k*
  const C K0 = rho, K1 = C(0.5) * Fx, K2 = C(0.5) * Fy;
  const C K3 = fdiv(C(2) * rho, C(3)) + C(2) * alpha * Fm2;
  const C K4 = (C(1) - omega) * k4, K5 = (C(1) - omega) * k5;
  const C K6 = fdiv(Fy, C(6)), K7 = fdiv(Fx, C(6));
  // seeds on f*; m*-bar = M^{-T} f*-bar (closed form of M^{-1})
  C fb[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) fb[i] = a.fb_in[i * g.plane + id];
  const C h = C(0.5), q = C(0.25);
  const C s14 = (fb[1] + fb[2]) + (fb[3] + fb[4]);
  const C s58 = (fb[5] + fb[6]) + (fb[7] + fb[8]);
  const C b0 = fb[0];
  const C b1 = h * (fb[1] - fb[2]);
  const C b2 = h * (fb[3] - fb[4]);
  const C b3 = q * s14 - fb[0];
  const C b4 = q * ((fb[1] + fb[2]) - (fb[3] + fb[4]));
  const C b5 = q * ((fb[5] + fb[6]) - (fb[7] + fb[8]));
  const C b6 = h * (fb[4] - fb[3]) + q * ((fb[5] - fb[6]) - (fb[7] - fb[8]));
  const C b7 = h * (fb[2] - fb[1]) + q * ((fb[5] - fb[6]) + (fb[7] - fb[8]));
  const C b8 = (fb[0] - h * s14) + q * s58;
  // m* = N(-u) k*: k*-bar = N(-u)^T m*-bar and the u-derivative of N(-u) k*
  const C uu = u * u, vv = v * v, uv = u * v;
  const C kb0 = b0 + u * b1 + v * b2 + (uu + vv) * b3 + (uu - vv) * b4 + uv * b5 + uu * v * b6 + u * vv * b7 +
                uu * vv * b8;
  const C kb1 = b1 + C(2) * u * b3 + C(2) * u * b4 + v * b5 + C(2) * uv * b6 + vv * b7 + C(2) * u * vv * b8;
  const C kb2 = b2 + C(2) * v * b3 - C(2) * v * b4 + u * b5 + uu * b6 + C(2) * uv * b7 + C(2) * uu * v * b8;
  const C kb3 = b3 + h * v * b6 + h * u * b7 + h * (uu + vv) * b8;
  const C kb4 = b4 + h * v * b6 - h * u * b7 - h * (uu - vv) * b8;
  const C kb5 = b5 + C(2) * u * b6 + C(2) * v * b7 + C(4) * uv * b8;
  const C kb6 = b6 + C(2) * v * b8;
  const C kb7 = b7 + C(2) * u * b8;
  const C kb8 = b8;
  C ubar = b1 * K0 + b3 * (C(2) * u * K0 + C(2) * K1) + b4 * (C(2) * u * K0 + C(2) * K1) + b5 * (v * K0 + K2) +
           b6 * (C(2) * uv * K0 + C(2) * v * K1 + C(2) * u * K2 + C(2) * K5) +
           b7 * (vv * K0 + C(2) * v * K2 + h * K3 - h * K4) +
           b8 * (C(2) * u * vv * K0 + C(2) * vv * K1 + C(4) * uv * K2 + u * K3 - u * K4 + C(4) * v * K5 +
                 C(2) * K7);
  C vbar = b2 * K0 + b3 * (C(2) * v * K0 + C(2) * K2) - b4 * (C(2) * v * K0 + C(2) * K2) + b5 * (u * K0 + K1) +
           b6 * (uu * K0 + C(2) * u * K1 + h * K3 + h * K4) +
           b7 * (C(2) * uv * K0 + C(2) * v * K1 + C(2) * u * K2 + C(2) * K5) +
           b8 * (C(2) * uu * v * K0 + C(4) * uv * K1 + C(2) * uu * K2 + v * K3 + v * K4 + C(4) * u * K5 +
                 C(2) * K6);
  // k* -> rho, F, alpha |F_m|^2, k4, k5, omega
  C rb = kb0 + fdiv(C(2) * kb3, C(3)) + fdiv(kb8, C(9));
  C Fbx = h * kb1 + fdiv(kb7, C(6)), Fby = h * kb2 + fdiv(kb6, C(6));
  const C Abar = C(2) * kb3 + fdiv(C(2) * kb8, C(3));
  C Fmbx = Abar * alpha * C(2) * Fmx, Fmby = Abar * alpha * C(2) * Fmy;
  const C psib = sig != C(0) ? Abar * Fm2 * fdiv(C(-2) * sig, psi0 * psi0 * psi0) : C(0);
  const C k4b = (C(1) - omega) * kb4, k5b = (C(1) - omega) * kb5;
  const C omb = -(k4 * kb4 + k5 * kb5);
  C mb0 = (uu - vv) * k4b + uv * k5b;
  C mb1 = C(-2) * u * k4b - v * k5b;
  C mb2 = C(2) * v * k4b - u * k5b;
  const C mb4 = k4b, mb5 = k5b;
  ubar = ubar + (C(2) * u * rho - C(2) * m1) * k4b + (v * rho - m2) * k5b;
  vbar = vbar + (C(2) * m2 - C(2) * v * rho) * k4b + (u * rho - m1) * k5b;
  // energy-equation seeds on u and rho
  ubar = ubar + a.ub[0][id];
  vbar = vbar + a.ub[1][id];
  // u = (m1 + F/2) / rho
  mb1 = mb1 + fdiv(ubar, rho);
  mb2 = mb2 + fdiv(vbar, rho);
  Fbx = Fbx + fdiv(ubar, C(2) * rho);
  Fby = Fby + fdiv(vbar, C(2) * rho);
  rb = rb - fdiv(u * ubar + v * vbar, rho);
  // omega = 1 / (nu(rho)/cs^2 + 1/2)
  rb = rb - omb * omega * omega * fdiv(dphase(k, rho) * (k.nu_l - k.nu_v), cs2);
  // F = F_m + gravity
  Fmbx = Fmbx + Fbx;
  Fmby = Fmby + Fby;
  rb = rb - k.g * Fbx;
  rb = rb + a.rhob[id];
  mb0 = mb0 + rb;
  // f-bar = M^T m-bar (m3, m6, m7, m8 do not reach k4, k5 or u)
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int cx = cxv(i), cy = cyv(i);
    a.fpb[i * g.plane + id] = mb0 + C(cx) * mb1 + C(cy) * mb2 + C(cx * cx - cy * cy) * mb4 + C(cx * cy) * mb5;
  }
  a.fmb[0][id] = Fmbx;
  a.fmb[1][id] = Fmby;
  a.psib[id] = psib;
}

// Adjoint of the interaction force (transposed psi stencil) and of psi(rho, T): the psi part of
// the rho adjoint goes into the node's pulled-population adjoints (rho = sum of them), the
// psi part of the T adjoint into Tb_out.  Then, at the Zou-He inlet, the adjoints of the
// unknowns f1, f5, f7 are folded into their knowns (and d/du_in is accumulated), so that fpb
// holds the adjoint of every value the pull read.
template <typename C>
__global__ void __launch_bounds__(256) k_adj_force(Args<C> a) {
  constexpr int HX = 36, HY = 12;  // 32 x 8 tile + 2 nodes
  __shared__ C sPsi[HX * HY], sFx[HX * HY], sFy[HX * HY];
  const Geo& g = a.g;
  const PhysC<C>& k = pc<C>(a.ph);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 8;
  const bool multiphase = k.G != C(0);
  if (multiphase) {
    for (int p = ty * 32 + tx; p < HX * HY; p += 256) {
      const int gx = x0 + p % HX - 2;
      const int id = map_y(g, y0 + p / HX - 2) * g.pitch + map_x(g, gx);
      const bool real = g.periodic_x || (gx >= 0 && gx < g.nx);  // a ghost column is no source
      sPsi[p] = a.psi[id];
      sFx[p] = real ? a.fmb[0][id] : C(0);
      sFy[p] = real ? a.fmb[1][id] : C(0);
    }
    __syncthreads();
  }
  const int x = x0 + tx, y = y0 + ty;
  if (x >= g.nx || y >= g.ny) return;
  const int id = y * g.pitch + x;
  const uint8_t m = a.mask[id];
  const C cs2 = C(1.0 / 3.0), gc = -k.G * cs2;
  C rp = C(0);
  if (multiphase) {
    const int c = (ty + 2) * HX + tx + 2;
    C pb = a.psib[id];
    if (!(m & kSolid)) {
      C sx, sy;
      grad_t(&sPsi[c], HX, sx, sy);
      pb = pb + gc * (sFx[c] * sx + sFy[c] * sy);
    }
    auto add = [&](int ex, int ey, int s) {
      pb = pb + gc * sPsi[s] * C(w_of(ex, ey)) * (C(ex) * sFx[s] + C(ey) * sFy[s]);
    };
    if (g.periodic_x || (x > 0 && x < g.nx - 1)) {
      // one source position per offset (ghost positions carry no F_m adjoint)
#pragma unroll
      for (int ey = -2; ey <= 2; ++ey)
#pragma unroll
        for (int ex = -2; ex <= 2; ++ex)
          if (ex != 0 || ey != 0) add(ex, ey, (ty + 2 - ey) * HX + tx + 2 - ex);
    } else {
#pragma unroll 1
      for (int ey = -2; ey <= 2; ++ey)
#pragma unroll 1
        for (int ex = -2; ex <= 2; ++ex) {
          if (ex == 0 && ey == 0) continue;
          int lo, hi;
          src_cols(g, x, ex, lo, hi);
          for (int sx = lo; sx <= hi; ++sx) add(ex, ey, (ty + 2 - ey) * HX + sx - x0 + 2);
        }
    }
    // psi = sqrt(rad), rad = k2 (p - rho cs^2), k2 = 2 / (G cs^2)
    const C r0 = a.rho[id], T0 = a.T[id], psi0 = sPsi[c];
    const C k2 = fdiv(C(2), k.G * cs2);
    const C dpr = pr_p(k, Dl<C>{r0, C(1)}, Dl<C>{T0, C(0)}).d;
    const C dpt = dpdT_eos(a.ph, r0, T0);
    const C inv2psi = fdiv(C(1), C(2) * psi0);
    if (!(m & kSolid)) rp = pb * k2 * (dpr - cs2) * inv2psi;
    a.Tb_out[id] = a.Tb_out[id] + pb * k2 * dpt * inv2psi;
  }
  if (m & kSolid) return;
  C fb[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) fb[i] = a.fpb[i * g.plane + id] + rp;
  if (!g.periodic_x && x == 0) {
    // Zou-He: f1 = f2 + (2/3) rho_in u, f5 = f6 - (f3 - f4)/2 + rho_in u / 6, f7 = f8 + (f3 - f4)/2
    // + rho_in u / 6, rho_in = (f0 + f3 + f4 + 2 (f2 + f6 + f8)) / (1 - u)
    const C u = k.u_in;
    const C bsum = fdiv(C(2) * fb[1], C(3)) + fdiv(fb[5] + fb[7], C(6));
    const C r1 = fdiv(u * bsum, C(1) - u);
    C fo[9];
    pull_node<C, C>(g, a.ph, a.f, a.mask, a.side, nullptr, x, y, m, fo);
    const C rho_in = fdiv(fo[0] + fo[3] + fo[4] + C(2) * (fo[2] + fo[6] + fo[8]), C(1) - u);
    a.uin[y] += (double)bsum * (double)rho_in / (1.0 - (double)u);
    fb[0] = fb[0] + r1;
    fb[3] = fb[3] + r1 - C(0.5) * fb[5] + C(0.5) * fb[7];
    fb[4] = fb[4] + r1 + C(0.5) * fb[5] - C(0.5) * fb[7];
    fb[2] = fb[2] + C(2) * r1 + fb[1];
    fb[6] = fb[6] + C(2) * r1 + fb[5];
    fb[8] = fb[8] + C(2) * r1 + fb[7];
    fb[1] = fb[5] = fb[7] = C(0);
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) a.fpb[i * g.plane + id] = fb[i];
}

// Transposed pull-streaming (a push written as a gather): the adjoint of f* entering the
// step and of the outlet's side values, from the adjoints of the pulled values (fpb).
template <typename C>
__global__ void __launch_bounds__(256) k_adj_pull(Args<C> a) {
  int x, y;
  if (!node_of_thread(a.g, x, y)) return;
  const Geo& g = a.g;
  const int id = y * g.pitch + x;
  const uint8_t m = a.mask[id];
  const PhysC<C>& k = pc<C>(a.ph);
  if (!g.periodic_x && x == g.nx - 1) {
    // convective outlet: v = (side + U inner) / (1 + U), also the next side value
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int i = j == 0 ? 2 : (j == 1 ? 6 : 8);
      const C sb = a.sb_in[j * g.ny + y];
      a.sb_out[j * g.ny + y] = (m & kSolid) ? sb : fdiv(a.fpb[i * g.plane + id] + sb, C(1) + k.U_out);
    }
  }
  if (m & kSolid) {
#pragma unroll
    for (int i = 0; i < 9; ++i) a.fb_out[i * g.plane + id] = C(0);
    return;
  }
  if (!(m & kNear2) && (g.periodic_x || (x >= 1 && x <= g.nx - 2))) {
    // no solid node within two nodes and no open boundary next door: plain pulls only
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      int zx = x + cxv(i);
      if (g.periodic_x) zx = zx < 0 ? zx + g.nx : (zx >= g.nx ? zx - g.nx : zx);
      a.fb_out[i * g.plane + id] = a.fpb[i * g.plane + wrap_y(g, y + cyv(i)) * g.pitch + zx];
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int cx = cxv(i), cy = cyv(i);
    C acc = C(0);
    // z = x + c_i pulls direction i from x (a fluid source: a plain pull), and, when the
    // wall cuts z's link along -c_i with q < 1/2, its Bouzidi value of direction opp(i)
    int zx = x + cx;
    const int zy = wrap_y(g, y + cy);
    if (g.periodic_x) zx = zx < 0 ? zx + g.nx : (zx >= g.nx ? zx - g.nx : zx);
    if (zx >= 0 && zx < g.nx && !(a.mask[zy * g.pitch + zx] & kSolid)) {
      acc = acc + a.fpb[i * g.plane + zy * g.pitch + zx];
      int wx = zx + cx;
      const int wy = wrap_y(g, zy + cy);
      if (g.periodic_x) wx = wx < 0 ? wx + g.nx : (wx >= g.nx ? wx - g.nx : wx);
      if (i != 0 && wx >= 0 && wx < g.nx && (a.mask[wy * g.pitch + wx] & kSolid)) {
        const C qz = link_q<C>(g, zx, zy, oppv(i));
        if (qz < C(0.5)) acc = acc + (C(1) - C(2) * qz) * a.fpb[oppv(i) * g.plane + zy * g.pitch + zx];
      }
    }
    if (i != 0) {
      // Bouzidi at x itself: direction j = opp(i) reads f*(x, i); direction i reads f*(x, i)
      // when q >= 1/2
      const int j = oppv(i);
      int sx = x - cxv(j);
      const int sy = wrap_y(g, y - cyv(j));
      if (g.periodic_x) sx = sx < 0 ? sx + g.nx : (sx >= g.nx ? sx - g.nx : sx);
      if (sx >= 0 && sx < g.nx && (a.mask[sy * g.pitch + sx] & kSolid)) {
        const C qj = link_q<C>(g, x, y, j);
        C ca;
        if (qj < C(0.5)) {
          int nxp = x + cxv(j);
          const int nyp = wrap_y(g, y + cyv(j));
          if (g.periodic_x) nxp = nxp < 0 ? nxp + g.nx : (nxp >= g.nx ? nxp - g.nx : nxp);
          const bool ok = nxp >= 0 && nxp < g.nx && !(a.mask[nyp * g.pitch + nxp] & kSolid);
          ca = ok ? C(2) * qj : C(1);
        } else {
          ca = fdiv(C(1), C(2) * qj);
        }
        acc = acc + ca * a.fpb[j * g.plane + id];
      }
      int tx = x - cx;
      const int ty = wrap_y(g, y - cy);
      if (g.periodic_x) tx = tx < 0 ? tx + g.nx : (tx >= g.nx ? tx - g.nx : tx);
      if (tx >= 0 && tx < g.nx && (a.mask[ty * g.pitch + tx] & kSolid)) {
        const C qi = link_q<C>(g, x, y, i);
        if (!(qi < C(0.5))) acc = acc + fdiv(C(2) * qi - C(1), C(2) * qi) * a.fpb[i * g.plane + id];
      }
    }
    if (!g.periodic_x && x == g.nx - 1 && (i == 2 || i == 6 || i == 8)) {
      // the outlet value of row y + c_y(i) reads f*(x, i) as its inner value
      const int jo = i == 2 ? 0 : (i == 6 ? 1 : 2);
      const int yo = wrap_y(g, y + cy);
      const int oid = yo * g.pitch + x;
      if (!(a.mask[oid] & kSolid)) {
        const C vb = a.fpb[i * g.plane + oid] + a.sb_in[jo * g.ny + yo];
        acc = acc + fdiv(k.U_out * vb, C(1) + k.U_out);
      }
    }
    a.fb_out[i * g.plane + id] = acc;
  }
}

// The window starts with the solid nodes at their wall temperature.
template <typename C>
__global__ void __launch_bounds__(256) k_adj_wall_seed(Geo g, const uint8_t* mask, const C* Tb, double* gw) {
  int x, y;
  if (!node_of_thread(g, x, y)) return;
  const int id = y * g.pitch + x;
  if (mask[id] & kSolid) gw[id] += (double)Tb[id];
}
template <typename C>
__global__ void __launch_bounds__(256) k_impose_wall(Geo g, const uint8_t* mask, const C* wallT, C* T) {
  int x, y;
  if (!node_of_thread(g, x, y)) return;
  const int id = y * g.pitch + x;
  if (mask[id] & kSolid) T[id] = wallT[id];
}
// Dense [ny][nx] doubles <-> typed [ny][pitch] planes.
template <typename C>
__global__ void __launch_bounds__(256) k_dense_to_plane(Geo g, const double* src, C* dst) {
  int x, y;
  if (!node_of_thread(g, x, y)) return;
  dst[y * g.pitch + x] = (C)src[y * g.nx + x];
}
template <typename C>
__global__ void __launch_bounds__(256) k_plane_to_dense(Geo g, const C* src, double* dst) {
  int x, y;
  if (!node_of_thread(g, x, y)) return;
  dst[y * g.nx + x] = (double)src[y * g.pitch + x];
}

// One reverse step (5 launches).  Returns the number of launches or -1.
// Shared-memory opt-in of the energy stages on the current device (before any launch or capture).
template <typename C>
int adjoint_setup_impl() {
  cudaFuncSetAttribute(k_adj_energy<C, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)EAdjLayout<C, 2>::bytes);
  cudaFuncSetAttribute(k_adj_energy<C, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)EAdjLayout<C, 1>::bytes);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}
template <typename C, int STAGE>
void launch_energy_adj(const Args<C>& a, cudaStream_t s) {
  using Lay = EAdjLayout<C, STAGE>;
  const dim3 grd((a.g.nx + kEATX - 1) / kEATX, (a.g.ny + kEATY - 1) / kEATY);
  k_adj_energy<C, STAGE><<<grd, kEANT, Lay::bytes, s>>>(a);
}
template <typename C>
int adjoint_step_impl(const Args<C>& a, cudaStream_t s) {
  const dim3 blk(32, 8), grd((a.g.nx + 31) / 32, (a.g.ny + 7) / 8);
  launch_energy_adj<C, 2>(a, s);
  launch_energy_adj<C, 1>(a, s);
  k_adj_collide<C><<<grd, blk, 0, s>>>(a);
  k_adj_force<C><<<grd, blk, 0, s>>>(a);
  k_adj_pull<C><<<grd, blk, 0, s>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? 5 : -1;
}

}  // namespace adj
}  // namespace lbm
