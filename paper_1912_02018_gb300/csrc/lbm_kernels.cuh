// Kernels of one time step of the CM pseudopotential boiling LBM (arXiv:1912.02018),
// templated on the compute type C (double or float) and population storage type S.
//
// Layout: structure of arrays, every field [ny][pitch] with x fastest; populations are
// 9 such planes, ping-ponged between two buffers.  The kernels:
//   k_rho_psi pull f with boundary substitutions, rho, psi(rho, T); writes psi.  Runs only
//             when no energy pass made psi (first step, after a restore, warm-up).
//   k_collide per 32x8 tile: the pull window of the 9 planes (1-node halo) and the psi tile
//             (2-node halo) staged in shared memory by TMA (edge tiles: plain loads);
//             interaction force, gravity, CM collision; writes f*, rho, u.
//   k_energy  per 32x16 tile: T, rho, u staged by TMA with a 4-node halo, lambda(rho);
//             Heun stage 1 on a 2-node halo, stage 2 on the tile, two nodes per thread;
//             writes T^{n+1} and, from the pull of the new populations, psi of the next
//             step; blocks holding wall nodes sum the wall heat flux in FP64 and the last
//             block to finish adds the per-block partials in block order.
//   kb_*      the same passes over the tiles of many domains in one launch per pass.
// The operation order inside each node follows the paper's equations term by term so
// that the FP64 build (compiled without FMA contraction) rounds like a plain reference;
// the FP32 build writes its roundings out (packed FP32x2 stencils, explicit fma) so that
// every kernel that inlines the same code gives the same bits.
#pragma once

#include <cuda_fp16.h>

#include <cstdint>

#include "lbm_internal.h"
#include "lbm_tma.cuh"

namespace lbm {
namespace kern {

// ---------------------------------------------------------------- programmatic dependent launch
// A pass launched with the programmatic-stream-serialization attribute may start while the
// kernel before it in the stream is still running (sm_90+).  wait(): the calling thread blocks
// until that kernel has completed and its writes are visible; trigger(): once every block of
// this pass has called it (or exited), the next such pass may start.  Both are no-ops in a
// pass launched without the attribute.  A pass reads nothing the previous kernel writes, and
// writes nothing at all, before wait().
namespace pdl {
__device__ __forceinline__ void wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
}  // namespace pdl

// ---------------------------------------------------------------- lattice tables
// D2Q9 velocities, Eq. (velVec).
__device__ __forceinline__ constexpr int cxv(int i) {
  return i == 1 || i == 5 || i == 7 ? 1 : (i == 2 || i == 6 || i == 8 ? -1 : 0);
}
__device__ __forceinline__ constexpr int cyv(int i) {
  return i == 3 || i == 5 || i == 8 ? 1 : (i == 4 || i == 6 || i == 7 ? -1 : 0);
}
__device__ __forceinline__ constexpr int oppv(int i) { return i == 0 ? 0 : (i % 2 == 1 ? i + 1 : i - 1); }
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

// Constants in the compute precision.
template <typename C>
__device__ __forceinline__ const PhysC<C>& pc(const Phys& ph);
template <>
__device__ __forceinline__ const PhysC<double>& pc<double>(const Phys& ph) {
  return ph.d;
}
template <>
__device__ __forceinline__ const PhysC<float>& pc<float>(const Phys& ph) {
  return ph.f;
}

// Division in the compute precision: IEEE in the FP64 build (which must round like the
// reference), the 2-ulp hardware approximation in the FP32 build.
template <typename C>
__device__ __forceinline__ C fdiv(C a, C b) {
  return a / b;
}
template <>
__device__ __forceinline__ float fdiv<float>(float a, float b) {
  return __fdividef(a, b);
}

// Sums and products whose rounding the source fixes, whatever kernel they are inlined into:
// FP32 fuses a b + c into one fma; FP64 rounds the product and the sum separately, as the
// FP64 build (compiled without contraction) does for every expression.
template <typename C>
__device__ __forceinline__ C mad(C a, C b, C c);
template <>
__device__ __forceinline__ float mad<float>(float a, float b, float c) {
  return __fmaf_rn(a, b, c);
}
template <>
__device__ __forceinline__ double mad<double>(double a, double b, double c) {
  return __dadd_rn(__dmul_rn(a, b), c);
}
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }

// ---------------------------------------------------------------- addressing
// Node coordinate of an arbitrary lattice position for stencil reads: periodic in y; in x
// periodic, or the nearest boundary column (zero-gradient ghost) at the inlet and outlet.
__device__ __forceinline__ int map_y(const Geo& g, int y) {
  if (y >= 0 && y < g.ny) return y;
  if (y < 0 && y + g.ny >= 0) return y + g.ny;
  if (y >= g.ny && y - g.ny < g.ny) return y - g.ny;
  y %= g.ny;  // only for lattices smaller than a tile
  return y < 0 ? y + g.ny : y;
}
__device__ __forceinline__ int map_x(const Geo& g, int x) {
  if (x >= 0 && x < g.nx) return x;
  if (g.periodic_x) {
    if (x < 0 && x + g.nx >= 0) return x + g.nx;
    if (x >= g.nx && x - g.nx < g.nx) return x - g.nx;
    x %= g.nx;
    return x < 0 ? x + g.nx : x;
  }
  return x < 0 ? 0 : g.nx - 1;
}
__device__ __forceinline__ int wrap_y(const Geo& g, int y) {  // offsets |dy| <= 2 < ny
  return y < 0 ? y + g.ny : (y >= g.ny ? y - g.ny : y);
}
// Population storage: FP64 or FP32 values as they are, or shifted FP16 h_i = f_i - w_i rho_l
// (the shift keeps liquid populations near zero, where FP16 is finest).
template <typename C, typename S>
struct PopIO {
  static __device__ __forceinline__ C ld(S v, int, const Phys&) { return static_cast<C>(v); }
  static __device__ __forceinline__ S st(C v, int, const Phys&) { return static_cast<S>(v); }
  static __device__ __forceinline__ double ld_d(S v, int, const Phys&) { return static_cast<double>(v); }
  static __device__ __forceinline__ S st_d(double v, int, const Phys&) { return static_cast<S>(v); }
};
template <typename C>
struct PopIO<C, __half> {
  static __device__ __forceinline__ C ld(__half v, int i, const Phys& ph) {
    return static_cast<C>(__half2float(v) + ph.pop_shift[i]);
  }
  static __device__ __forceinline__ __half st(C v, int i, const Phys& ph) {
    return __float2half_rn(static_cast<float>(v) - ph.pop_shift[i]);
  }
  static __device__ __forceinline__ double ld_d(__half v, int i, const Phys& ph) {
    return static_cast<double>(__half2float(v) + ph.pop_shift[i]);
  }
  static __device__ __forceinline__ __half st_d(double v, int i, const Phys& ph) {
    return __float2half_rn(static_cast<float>(v) - ph.pop_shift[i]);
  }
};
template <typename C, typename S>
__device__ __forceinline__ C ldf(const Geo& g, const Phys& ph, const S* __restrict__ f, int i, int y, int x) {
  return PopIO<C, S>::ld(f[i * g.plane + y * g.pitch + x], i, ph);
}

// ---------------------------------------------------------------- double-float arithmetic
// A double-float value is a pair (hi, lo) of FP32 words standing for the real number hi + lo.
// Building blocks: Knuth's TwoSum and Dekker's FastTwoSum (error-free sums), the FMA-based
// exact product, and products, sums and a quotient of pairs after Joldes, Muller and Popescu,
// "Tight and rigorous error bounds for basic building blocks of double-word arithmetic" (ACM
// TOMS 2017), here in their cheapest forms: results are left unnormalised (|lo| a few ulps of
// hi, never renormalised by a FastTwoSum), the lo * lo term of a product is dropped, and a
// difference uses FastTwoSum of the high words where the order of the operands is known.
// Square roots and the quotient start from the FP32 approximations (rsqrt.approx, rcp.approx)
// and take one correction from an exact residual (Karp and Markstein, "High-precision division
// and square root", ACM TOMS 1997).  Each result carries about 2^-44 relative error.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF df_of(F2 v) { return {v.hi, v.lo}; }
__device__ __forceinline__ DF df_neg(DF a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// a * f for an FP32 f
__device__ __forceinline__ DF df_mulf(DF a, float f) {
  const float p = __fmul_rn(a.hi, f);
  return {p, __fmaf_rn(a.lo, f, __fmaf_rn(a.hi, f, -p))};
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  return {p, __fmaf_rn(a.lo, b.hi, e)};
}
__device__ __forceinline__ DF df_sqr(DF a) {
  const float p = __fmul_rn(a.hi, a.hi);
  return {p, __fmaf_rn(__fadd_rn(a.hi, a.hi), a.lo, __fmaf_rn(a.hi, a.hi, -p))};
}
// c - a where |c.hi| >= |a.hi| (FastTwoSum of the high words)
__device__ __forceinline__ DF df_csub(DF c, DF a) {
  const float s = __fsub_rn(c.hi, a.hi);
  const float t = __fsub_rn(__fsub_rn(c.hi, s), a.hi);
  return {s, __fadd_rn(t, __fsub_rn(c.lo, a.lo))};
}
// c - a for an FP32 c with |c| >= |a.hi|
__device__ __forceinline__ DF df_fsub(float c, DF a) {
  const float s = __fsub_rn(c, a.hi);
  const float t = __fsub_rn(__fsub_rn(c, s), a.hi);
  return {s, __fsub_rn(t, a.lo)};
}
// a + b for any magnitudes (TwoSum of the high words)
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float t = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return {s, __fadd_rn(t, __fadd_rn(a.lo, b.lo))};
}
// a / b: q1 = a.hi / b.hi from the approximate reciprocal, then the exact remainder
// a - b q1 (a.hi - b.hi q1 is exact by Sterbenz's lemma) divided once more
__device__ __forceinline__ DF df_div(DF a, DF b) {
  const float r = rcp_approx(b.hi);
  const float q1 = __fmul_rn(a.hi, r);
  const float p = __fmul_rn(b.hi, q1);
  const float e = __fmaf_rn(b.lo, q1, __fmaf_rn(b.hi, q1, -p));
  const float d = __fadd_rn(__fsub_rn(a.hi, p), __fsub_rn(a.lo, e));
  return {q1, __fmul_rn(d, r)};
}
// sqrt(a): s = a.hi rsqrt(a.hi), corrected by (a - s^2) / (2 s) with the residual from one fma
__device__ __forceinline__ DF df_sqrt(DF a) {
  const float r = rsqrt_approx(a.hi);
  const float s = __fmul_rn(a.hi, r);
  const float res = __fadd_rn(__fmaf_rn(-s, s, a.hi), a.lo);
  return {s, __fmul_rn(res, __fmul_rn(0.5f, r))};
}

// ---------------------------------------------------------------- thermodynamics
// Peng-Robinson EOS, Eq. (eos), and psi of Eq. (potential) in IEEE FP64.
__device__ __forceinline__ double psi_eos(const Phys& ph, double rho, double T, double& rad) {
  const double cs2 = 1.0 / 3.0;
  const PhysC<double>& k = ph.d;
  double s = 1.0 + k.kappa * (1.0 - sqrt(T / k.Tc));
  double phi = s * s;
  double rep = rho * k.R * T / (1.0 - k.b * rho);
  double att = k.a * phi * rho * rho / (1.0 + 2.0 * k.b * rho - k.b * k.b * rho * rho);
  double p = rep - att;
  rad = 2.0 * (p - rho * cs2) / (k.G * cs2);
  return sqrt(rad);
}
// The same in double-float arithmetic (inputs and result FP32), over one denominator: with
// x = b rho and D = 1 + 2x - x^2 = 2 - (1 - x)^2,
//   rad = rho [kR T D - ka phi rho (1 - x) - (k/3)(1 - x) D] / ((1 - x) D),  k = 2/(G cs^2),
//   phi = (K1 - kappa sqrt(T/Tc))^2,  K1 = 1 + kappa
// (kR, ka, k/3, K1 folded on the host).  The numerator has condition number ~2 over the
// liquid-vapour range, so the cheap sums above keep the radicand within ~2^-42 of exact; psi
// is then the correctly rounded FP32 value (checked on 20,000 sampled (rho, T) against a
// 120-bit evaluation in a CPU emulation of these operations).  The FastTwoSum differences need
// kappa sqrt(T/Tc) <= 1 + kappa (T <= 3.5 Tc) and b rho <= 1, which hold wherever Eq. (eos) is
// defined on the lattice.
__device__ __forceinline__ float psi_eos_df(const Phys& ph, float rho, float T, float& rad_hi) {
  const DF sq = df_sqrt(df_mulf(df_of(ph.invTc2), T));
  const DF phi = df_sqr(df_csub(df_of(ph.K12), df_mul(df_of(ph.kappa2), sq)));
  const DF omx = df_fsub(1.0f, df_mulf(df_of(ph.b2), rho));
  const DF D = df_fsub(2.0f, df_sqr(omx));
  const DF den = df_mul(omx, D);
  const DF A = df_mul(df_mulf(df_of(ph.kR2), T), D);
  const DF B = df_mul(df_mulf(df_mul(df_of(ph.ka2), phi), rho), omx);
  const DF num = df_add(df_add(A, df_neg(B)), df_neg(df_mul(df_of(ph.k32), den)));
  const DF rad = df_div(df_mulf(num, rho), den);
  rad_hi = rad.hi;
  const DF r = df_sqrt(rad);
  return __fadd_rn(r.hi, r.lo);
}
// The same in plain FP32.
__device__ __forceinline__ float psi_eos_f32(const Phys& ph, float rho, float T, float& rad) {
  float s = 1.0f + ph.kappa2.hi * (1.0f - sqrtf(T * ph.invTc2.hi));
  float phi = s * s;
  float b = ph.b2.hi;
  float rep = rho * ph.R2.hi * T / (1.0f - b * rho);
  float att = ph.a2.hi * phi * rho * rho / (1.0f + 2.0f * b * rho - b * b * rho * rho);
  rad = (rep - att - rho * ph.cs22.hi) * ph.k2.hi;
  return sqrtf(rad);
}
template <typename C, int PSI>
__device__ __forceinline__ C psi_of(const Phys& ph, C rho, C T, int* status) {
  if constexpr (PSI == kPsiDF) {
    float rad;
    float p = psi_eos_df(ph, (float)rho, (float)T, rad);
    if (!(rad > 0.0f)) atomicOr(status, 2);
    return (C)p;
  } else if constexpr (PSI == kPsiF32) {
    float rad;
    float p = psi_eos_f32(ph, (float)rho, (float)T, rad);
    if (!(rad > 0.0f)) atomicOr(status, 2);
    return (C)p;
  } else {
    double rad;
    double p = psi_eos(ph, (double)rho, (double)T, rad);
    if (!(rad > 0.0)) atomicOr(status, 2);
    return (C)p;
  }
}
// (dp/dT) at fixed rho, the derivative of Eq. (eos).
template <typename C>
__device__ __forceinline__ C dpdT_eos(const Phys& ph, C rho, C T) {
  C s = C(1) + pc<C>(ph).kappa * (C(1) - sqrt(fdiv(T, pc<C>(ph).Tc)));
  C dphi = fdiv(-pc<C>(ph).kappa * s, sqrt(T * pc<C>(ph).Tc));
  C rep = fdiv(rho * pc<C>(ph).R, C(1) - pc<C>(ph).b * rho);
  C att = fdiv(pc<C>(ph).a * dphi * rho * rho,
               C(1) + C(2) * pc<C>(ph).b * rho - pc<C>(ph).b * pc<C>(ph).b * rho * rho);
  return rep - att;
}
// Phase fraction for the transport properties, and nu(rho), lambda(rho).
template <typename C>
__device__ __forceinline__ C phase_frac(const Phys& ph, C rho) {
  if (!(pc<C>(ph).rho_l > pc<C>(ph).rho_v)) return C(1);
  C f = fdiv(sub(rho, pc<C>(ph).rho_v), sub(pc<C>(ph).rho_l, pc<C>(ph).rho_v));
  f = f < C(0) ? C(0) : f;
  return f > C(1) ? C(1) : f;
}
template <typename C>
__device__ __forceinline__ C nu_of(const Phys& ph, C rho) {
  return mad(phase_frac(ph, rho), sub(pc<C>(ph).nu_l, pc<C>(ph).nu_v), pc<C>(ph).nu_v);
}
template <typename C>
__device__ __forceinline__ C lam_of(const Phys& ph, C rho) {
  C alpha = mad(phase_frac(ph, rho), sub(pc<C>(ph).alpha_l, pc<C>(ph).alpha_v), pc<C>(ph).alpha_v);
  return mul(mul(rho, pc<C>(ph).c_v), alpha);
}

// ---------------------------------------------------------------- stencils on tiles (Sec. II.C)
// p points at the stencil centre of a row-major tile with row stride s.
// Isotropic gradient sum_k w_k phi(x+e_k) e_k over +/- pairs.
template <typename C, bool kX = true, bool kY = true>
__device__ __forceinline__ void grad_t(const C* p, int s, C& gx, C& gy) {
  C sx = C(0), sy = C(0);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const int ex = exv(k), ey = eyv(k);
    if ((kX && ex != 0) || (kY && ey != 0)) {
      // w e is w scaled by a power of two: (w e) d rounds exactly like (w d) e
      C d = sub(p[ey * s + ex], p[-ey * s - ex]);
      if (kX && ex != 0) sx = mad(C(wiso(k) * ex), d, sx);
      if (kY && ey != 0) sy = mad(C(wiso(k) * ey), d, sy);
    }
  }
  gx = sx;
  gy = sy;
}
// ---------------------------------------------------------------- streaming (Sec. IV.A BCs)
// Link fraction q of direction i at a near-wall node: the fraction of the link from the node
// along -c_i that lies in the fluid (smallest root of |d + t c|^2 = r^2, tabulated at creation).
template <typename C>
__device__ __forceinline__ C link_q(const Geo& g, int x, int y, int i) {
  return static_cast<const C*>(g.wall_q)[g.wall_idx[y * g.pitch + x] * 8 + i - 1];
}

// Pull with substitutions for nodes next to the wall, the inlet or the outlet: linear
// interpolated bounce-back on the cylinder, Zou-He inlet, convective outlet.
// side_out != nullptr: store the outlet's new streamed values there.
template <typename C, typename S>
__device__ __forceinline__ void pull_slow(const Geo& g, const Phys& ph, const S* __restrict__ f,
                                          const uint8_t* __restrict__ mask, const C* __restrict__ side_in,
                                          C* __restrict__ side_out, int x, int y, C fo[9]) {
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int cx = cxv(i), cy = cyv(i);
    int sx = x - cx;
    const int sy = wrap_y(g, y - cy);
    if (g.periodic_x) sx = sx < 0 ? sx + g.nx : (sx >= g.nx ? sx - g.nx : sx);
    C v;
    if (sx < 0 || sx >= g.nx) {
      v = C(0);  // unknown at the inlet or outlet; replaced below
    } else if (mask[sy * g.pitch + sx] & kSolid) {
      // linear interpolated bounce-back; the wall lies along c_opp(i)
      const int io = oppv(i);
      const C q = link_q<C>(g, x, y, i);
      const C a = ldf<C>(g, ph, f, io, y, x);
      if (q < C(0.5)) {
        int nxp = x + cx;
        const int nyp = wrap_y(g, y + cy);
        if (g.periodic_x) nxp = nxp < 0 ? nxp + g.nx : (nxp >= g.nx ? nxp - g.nx : nxp);
        const bool ok = nxp >= 0 && nxp < g.nx && !(mask[nyp * g.pitch + nxp] & kSolid);
        const C q2 = mul(C(2), q);
        v = ok ? add(mul(q2, a), mul(sub(C(1), q2), ldf<C>(g, ph, f, io, nyp, nxp))) : a;
      } else {
        const C q2 = mul(C(2), q);
        v = add(fdiv(a, q2), mul(fdiv(sub(q2, C(1)), q2), ldf<C>(g, ph, f, i, y, x)));
      }
    } else {
      v = ldf<C>(g, ph, f, i, sy, sx);
    }
    fo[i] = v;
  }
  if (g.periodic_x) return;
  if (x == 0) {
    // Zou-He velocity inlet, u = (u_in, 0): unknowns f1, f5, f7
    const C u = pc<C>(ph).u_in;
    const C rho = fdiv(add(add(add(fo[0], fo[3]), fo[4]), mul(C(2), add(add(fo[2], fo[6]), fo[8]))), sub(C(1), u));
    fo[1] = add(fo[2], mul(mul(C(2.0 / 3.0), rho), u));
    fo[5] = add(sub(fo[6], mul(C(0.5), sub(fo[3], fo[4]))), fdiv(mul(rho, u), C(6)));
    fo[7] = add(add(fo[8], mul(C(0.5), sub(fo[3], fo[4]))), fdiv(mul(rho, u), C(6)));
  }
  if (x == g.nx - 1) {
    // convective outlet: f(t+1) = (f(t) + U f_{nx-2}(t+1)) / (1 + U) for f2, f6, f8.  FP32 takes
    // the same update as f(t) + k (f_{nx-2}(t+1) - f(t)), k = U / (1 + U) rounded once from FP64:
    // the quotient with 1 + U rounded to FP32 has its fixed point about 1e-6 above the interior
    // value, a steady mass source at the outlet that shifts the open domain's pressure level over
    // long runs (the FP64 build keeps the quotient, term for term as written)
    const C U = pc<C>(ph).U_out;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int i = j == 0 ? 2 : (j == 1 ? 6 : 8);
      const C inner = ldf<C>(g, ph, f, i, wrap_y(g, y - cyv(i)), g.nx - 1);
      const C s0 = side_in[j * g.ny + y];
      C v;
      if constexpr (sizeof(C) == 4) v = mad(pc<C>(ph).U_k, sub(inner, s0), s0);
      else v = fdiv(add(s0, mul(U, inner)), add(C(1), U));
      fo[i] = v;
      if (side_out) side_out[j * g.ny + y] = v;
    }
  }
}

template <typename C, typename S>
__device__ __forceinline__ void pull_node(const Geo& g, const Phys& ph, const S* __restrict__ f,
                                          const uint8_t* __restrict__ mask, const C* __restrict__ side_in,
                                          C* __restrict__ side_out, int x, int y, uint8_t m, C fo[9]) {
  // the plain pulls are issued before the node type is tested (columns clamped at an open
  // edge), so they overlap the mask read; wall and edge nodes then redo the pull
  const int ym = y == 0 ? g.ny - 1 : y - 1;
  const int yp = y == g.ny - 1 ? 0 : y + 1;
  int xm = x - 1, xp = x + 1;
  if (g.periodic_x) {
    xm = xm < 0 ? g.nx - 1 : xm;
    xp = xp >= g.nx ? 0 : xp;
  } else {
    xm = xm < 0 ? 0 : xm;
    xp = xp >= g.nx ? g.nx - 1 : xp;
  }
  fo[0] = ldf<C>(g, ph, f, 0, y, x);
  fo[1] = ldf<C>(g, ph, f, 1, y, xm);
  fo[2] = ldf<C>(g, ph, f, 2, y, xp);
  fo[3] = ldf<C>(g, ph, f, 3, ym, x);
  fo[4] = ldf<C>(g, ph, f, 4, yp, x);
  fo[5] = ldf<C>(g, ph, f, 5, ym, xm);
  fo[6] = ldf<C>(g, ph, f, 6, yp, xp);
  fo[7] = ldf<C>(g, ph, f, 7, yp, xm);
  fo[8] = ldf<C>(g, ph, f, 8, ym, xp);
  const bool edge = !g.periodic_x && (x == 0 || x == g.nx - 1);
  if ((m & kNearWall) || edge) pull_slow<C, S>(g, ph, f, mask, side_in, side_out, x, y, fo);
}

// psi at node (x, y): pull, rho = sum f, Eq. (potential); solid nodes use rho_s.
template <typename C, typename S, int PSI>
__device__ __forceinline__ C psi_node(const Geo& g, const Phys& ph, const S* __restrict__ f,
                                      const C* __restrict__ T, const uint8_t* __restrict__ mask,
                                      const C* __restrict__ side_in, int x, int y, int* status) {
  const int id = y * g.pitch + x;
  const uint8_t m = mask[id];
  const C t = T[id];
  C fo[9];
  pull_node<C, S>(g, ph, f, mask, side_in, nullptr, x, y, m, fo);
  C rho = fo[0];
#pragma unroll
  for (int i = 1; i < 9; ++i) rho = rho + fo[i];
  if (m & kSolid) rho = pc<C>(ph).rho_s;
  return psi_of<C, PSI>(ph, rho, t, status);
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
  ux = fdiv(m1 + C(0.5) * Fx, rho);
  uy = fdiv(m2 + C(0.5) * Fy, rho);
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
  const C alpha = sigma != C(0) ? fdiv(sigma, psi * psi) : C(0);
  const C Fm2 = Fmx * Fmx + Fmy * Fmy;
  const C ks0 = rho;
  const C ks1 = C(0.5) * Fx;
  const C ks2 = C(0.5) * Fy;
  const C ks3 = fdiv(C(2) * rho, C(3)) + C(0.5) * (C(4) * alpha * Fm2);
  const C ks4 = (C(1) - omega) * k4;
  const C ks5 = (C(1) - omega) * k5;
  const C ks6 = C(0.5) * fdiv(Fy, C(3));
  const C ks7 = C(0.5) * fdiv(Fx, C(3));
  const C ks8 = fdiv(rho, C(9)) + C(0.5) * (C(4.0 / 3.0) * alpha * Fm2);
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
// The same for FP32 with every rounding written out (explicit fma, mul, add), so that the
// result does not depend on which kernel inlines it.  Forward substitution of N(u) m* = k*
// in closed form; m*_1 = k*_1 + u rho = m1 + Fx and m*_2 = m2 + Fy hold exactly since
// u rho = m1 + Fx / 2.
template <>
__device__ __forceinline__ void collide<float>(const float f[9], float rho, float Fx, float Fy, float Fmx, float Fmy,
                                               float psi, float omega, float sigma, float fs[9], float& ux,
                                               float& uy) {
  const float a56 = __fsub_rn(f[5], f[6]), a78 = __fsub_rn(f[7], f[8]);
  const float m1 = __fadd_rn(__fadd_rn(__fsub_rn(f[1], f[2]), a56), a78);
  const float m2 = __fsub_rn(__fadd_rn(__fsub_rn(f[3], f[4]), a56), a78);
  const float m4 = __fsub_rn(__fadd_rn(f[1], f[2]), __fadd_rn(f[3], f[4]));
  const float m5 = __fsub_rn(__fadd_rn(f[5], f[6]), __fadd_rn(f[7], f[8]));
  const float u = __fdividef(__fmaf_rn(0.5f, Fx, m1), rho), v = __fdividef(__fmaf_rn(0.5f, Fy, m2), rho);
  ux = u;
  uy = v;
  const float uu = __fmul_rn(u, u), vv = __fmul_rn(v, v), uv = __fmul_rn(u, v);
  const float s2 = __fadd_rn(uu, vv), d2 = __fsub_rn(uu, vv), u2 = __fmul_rn(2.0f, u), v2 = __fmul_rn(2.0f, v);
  // central moments k4, k5 of the pre-collision populations (Eq. (postColl2) shift)
  const float k4 = __fmaf_rn(d2, rho, __fmaf_rn(v2, m2, __fmaf_rn(-u2, m1, m4)));
  const float k5 = __fmaf_rn(uv, rho, __fmaf_rn(-v, m1, __fmaf_rn(-u, m2, m5)));
  // post-collision central moments with the consistency terms alpha |Fm|^2
  const float alpha = sigma != 0.0f ? __fdividef(sigma, __fmul_rn(psi, psi)) : 0.0f;
  const float aF = __fmul_rn(alpha, __fmaf_rn(Fmx, Fmx, __fmul_rn(Fmy, Fmy)));
  const float om = __fsub_rn(1.0f, omega);
  const float ks3 = __fmaf_rn(2.0f, aF, __fmul_rn(2.0f / 3.0f, rho));
  const float ks4 = __fmul_rn(om, k4), ks5 = __fmul_rn(om, k5);
  const float ks6 = __fmul_rn(1.0f / 6.0f, Fy), ks7 = __fmul_rn(1.0f / 6.0f, Fx);
  const float ks8 = __fmaf_rn(2.0f / 3.0f, aF, __fmul_rn(1.0f / 9.0f, rho));
  // raw moments m* = N(u)^{-1} k*
  const float ms1 = __fadd_rn(m1, Fx), ms2 = __fadd_rn(m2, Fy);
  const float ms3 = __fmaf_rn(u2, ms1, __fmaf_rn(v2, ms2, __fmaf_rn(-s2, rho, ks3)));
  const float ms4 = __fmaf_rn(u2, ms1, __fmaf_rn(-v2, ms2, __fmaf_rn(-d2, rho, ks4)));
  const float ms5 = __fmaf_rn(v, ms1, __fmaf_rn(u, ms2, __fmaf_rn(-uv, rho, ks5)));
  const float uv2 = __fmul_rn(2.0f, uv);
  const float ms6 = __fmaf_rn(u2, ms5, __fmaf_rn(__fmul_rn(0.5f, v), __fadd_rn(ms3, ms4),
                              __fmaf_rn(-uu, ms2, __fmaf_rn(-uv2, ms1, __fmaf_rn(__fmul_rn(uu, v), rho, ks6)))));
  const float ms7 = __fmaf_rn(v2, ms5, __fmaf_rn(__fmul_rn(0.5f, u), __fsub_rn(ms3, ms4),
                              __fmaf_rn(-uv2, ms2, __fmaf_rn(-vv, ms1, __fmaf_rn(__fmul_rn(u, vv), rho, ks7)))));
  const float ms8 = __fmaf_rn(
      u2, ms7,
      __fmaf_rn(v2, ms6,
                __fmaf_rn(__fmul_rn(-2.0f, uv2), ms5,
                          __fmaf_rn(__fmul_rn(0.5f, d2), ms4,
                                    __fmaf_rn(__fmul_rn(-0.5f, s2), ms3,
                                              __fmaf_rn(__fmul_rn(uv2, u), ms2,
                                                        __fmaf_rn(__fmul_rn(uv2, v), ms1,
                                                                  __fmaf_rn(-__fmul_rn(uu, vv), rho, ks8))))))));
  // f* = M^{-1} m*
  const float A = __fmul_rn(0.25f, __fadd_rn(ms3, ms4)), B = __fmul_rn(0.25f, __fsub_rn(ms3, ms4));
  const float c = __fmaf_rn(-0.5f, ms8, A), e = __fmaf_rn(-0.5f, ms8, B);
  const float d = __fmul_rn(0.5f, __fsub_rn(ms1, ms7)), gy = __fmul_rn(0.5f, __fsub_rn(ms2, ms6));
  fs[0] = __fadd_rn(__fsub_rn(rho, ms3), ms8);
  fs[1] = __fadd_rn(c, d);
  fs[2] = __fsub_rn(c, d);
  fs[3] = __fadd_rn(e, gy);
  fs[4] = __fsub_rn(e, gy);
  const float sp = __fadd_rn(ms5, ms8), tp = __fadd_rn(ms6, ms7), wm = __fsub_rn(ms8, ms5), zm = __fsub_rn(ms6, ms7);
  fs[5] = __fmul_rn(0.25f, __fadd_rn(sp, tp));
  fs[6] = __fmul_rn(0.25f, __fsub_rn(sp, tp));
  fs[7] = __fmul_rn(0.25f, __fsub_rn(wm, zm));
  fs[8] = __fmul_rn(0.25f, __fadd_rn(wm, zm));
}

// Single-rate BGK on the same equilibrium and forcing, the operator the paper compares the CM
// collision with (Sec. III.B): f* = f + omega (f^eq - f) + (1 - omega/2) F_i, u as above.  T(u) =
// N(u) M is linear and maps f^eq and F_i to k^eq = (rho, 0, 0, 2 rho/3, 0, 0, 0, 0, rho/9) and
// R = (0, F_x, F_y, 0, 0, 0, F_y/3, F_x/3, 0), so f* = (1 - omega) f + M^{-1} N(u)^{-1} k' with
// k' = omega k^eq + (1 - omega/2) R: the forward substitution and reconstruction of the CM
// collision on k'.  No consistency term (it belongs to the CM forcing of Eq. (force2)).
template <typename C>
__device__ __forceinline__ void collide_bgk(const C f[9], C rho, C Fx, C Fy, C omega, C fs[9], C& ux, C& uy) {
  const C m1 = ((((f[1] - f[2]) + f[5]) - f[6]) + f[7]) - f[8];
  const C m2 = ((((f[3] - f[4]) + f[5]) - f[6]) - f[7]) + f[8];
  ux = fdiv(m1 + C(0.5) * Fx, rho);
  uy = fdiv(m2 + C(0.5) * Fy, rho);
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
  const C cf = C(1) - C(0.5) * omega;
  const C ks0 = omega * rho;
  const C ks1 = cf * Fx;
  const C ks2 = cf * Fy;
  const C ks3 = omega * fdiv(C(2) * rho, C(3));
  const C ks6 = cf * fdiv(Fy, C(3));
  const C ks7 = cf * fdiv(Fx, C(3));
  const C ks8 = omega * fdiv(rho, C(9));
  // forward substitution N m' = k' (k'_4 = k'_5 = 0)
  const C ms0 = ks0;
  const C ms1 = ks1 - N10 * ms0;
  const C ms2 = ks2 - N20 * ms0;
  const C ms3 = ((ks3 - N30 * ms0) - N31 * ms1) - N32 * ms2;
  const C ms4 = ((-N40 * ms0) - N41 * ms1) - N42 * ms2;
  const C ms5 = ((-N50 * ms0) - N51 * ms1) - N52 * ms2;
  const C ms6 = (((((ks6 - N60 * ms0) - N61 * ms1) - N62 * ms2) - N63 * ms3) - N64 * ms4) - N65 * ms5;
  const C ms7 = (((((ks7 - N70 * ms0) - N71 * ms1) - N72 * ms2) - N73 * ms3) - N74 * ms4) - N75 * ms5;
  const C ms8 =
      (((((((ks8 - N80 * ms0) - N81 * ms1) - N82 * ms2) - N83 * ms3) - N84 * ms4) - N85 * ms5) - N86 * ms6) - N87 * ms7;
  // f* = (1 - omega) f + M^{-1} m'
  const C h = C(0.5), q = C(0.25), r = C(1) - omega;
  fs[0] = r * f[0] + ((ms0 - ms3) + ms8);
  fs[1] = r * f[1] + ((((h * ms1 + q * ms3) + q * ms4) - h * ms7) - h * ms8);
  fs[2] = r * f[2] + ((((-h * ms1 + q * ms3) + q * ms4) + h * ms7) - h * ms8);
  fs[3] = r * f[3] + ((((h * ms2 + q * ms3) - q * ms4) - h * ms6) - h * ms8);
  fs[4] = r * f[4] + ((((-h * ms2 + q * ms3) - q * ms4) + h * ms6) - h * ms8);
  fs[5] = r * f[5] + (((q * ms5 + q * ms6) + q * ms7) + q * ms8);
  fs[6] = r * f[6] + (((q * ms5 - q * ms6) - q * ms7) + q * ms8);
  fs[7] = r * f[7] + (((-q * ms5 - q * ms6) + q * ms7) + q * ms8);
  fs[8] = r * f[8] + (((-q * ms5 + q * ms6) - q * ms7) + q * ms8);
}

// ---------------------------------------------------------------- k_rho_psi, k_collide
constexpr int kCollTX = 32, kCollTY = 8;

// psi(rho, T) at every node of tile (bx, by) of 32 x 8 nodes (rho from the pulled
// populations, rho_s in the solid).
template <typename C, typename S, int PSI>
__device__ __forceinline__ void rho_psi_tile(const Geo& g, const Phys& ph, const S* __restrict__ f,
                                             const C* __restrict__ T, const uint8_t* __restrict__ mask,
                                             const C* __restrict__ side_in, C* __restrict__ psi_o, int* status, int bx,
                                             int by) {
  const int x = bx * kCollTX + threadIdx.x, y = by * 8 + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  psi_o[y * g.pitch + x] = psi_node<C, S, PSI>(g, ph, f, T, mask, side_in, x, y, status);
}
template <typename C, typename S, int PSI>
__global__ void __launch_bounds__(256) k_rho_psi(Geo g, Phys ph, const S* __restrict__ f, const C* __restrict__ T,
                                                const uint8_t* __restrict__ mask, const C* __restrict__ side_in,
                                                C* __restrict__ psi_o, int* status) {
  rho_psi_tile<C, S, PSI>(g, ph, f, T, mask, side_in, psi_o, status, blockIdx.x, blockIdx.y);
}

// Shared-memory staging of a collision tile.  Populations: the tile's rows with a 1-row halo,
// columns from x0 - XA (XA elements = 16 bytes, the alignment of a TMA copy's first column);
// psi: a 2-row and PA-column halo.  Tiles whose staged boxes lie inside the lattice (no wrap,
// no open edge) are copied by TMA; the others load psi and pull with plain loads.
template <typename C, typename S, int CTY>
struct CollStage {
  static constexpr int XA = 16 / (int)sizeof(S), FW = kCollTX + 2 * XA, FH = CTY + 2;
  static constexpr int PA = 16 / (int)sizeof(C) < 2 ? 2 : 16 / (int)sizeof(C), PW = kCollTX + 2 * PA, PH = CTY + 4;
  static constexpr int MARGIN = XA > PA ? XA : PA;  // columns a staged tile needs left and right of it
};
template <typename C, typename S, int CTY>
__device__ __forceinline__ bool coll_staged(const Geo& g, int x0, int y0) {
  constexpr int M = CollStage<C, S, CTY>::MARGIN;
  return x0 >= M && x0 + kCollTX + M <= g.nx && y0 >= 2 && y0 + CTY + 2 <= g.ny;
}

// One fluid-or-solid node (x, y) = (x0 + tx, y0 + ty) of a collision tile, mask m: pull (from
// the staged populations s_f of a staged tile, else from global memory with the boundary
// substitutions), interaction force from the psi tile s_psi with its 2-node halo, gravity,
// CM collision (or, with OP = kCollBGK, the BGK comparison operator); writes f* (other
// buffer), rho, u and the outlet's streamed values.
template <typename C, typename S, int CTY, int OP = kCollCM>
__device__ __forceinline__ void collide_node(const Geo& g, const Phys& ph, const S* __restrict__ f,
                                             S* __restrict__ fn, const C* __restrict__ psi,
                                             const uint8_t* __restrict__ mask, const C* __restrict__ side_in,
                                             C* __restrict__ side_out, C* __restrict__ rho_o, C* __restrict__ ux_o,
                                             C* __restrict__ uy_o, int forcing, int* status, int tx, int ty, int x,
                                             int y, uint8_t m, bool staged, const S* s_f, const C* s_psi) {
  using CS = CollStage<C, S, CTY>;
  constexpr int HX = CS::PW;
  const PhysC<C>& k = pc<C>(ph);
  const int id = y * g.pitch + x;
  if (m & kSolid) {
    rho_o[id] = k.rho_s;
    ux_o[id] = C(0);
    uy_o[id] = C(0);
    return;
  }
  const bool multiphase = k.G != C(0);
  const bool need_psi = multiphase && forcing;
  C fo[9];
  if (staged) {
    // a staged tile holds no inlet or outlet column; wall nodes redo the pull with substitutions
#pragma unroll
    for (int i = 0; i < 9; ++i)
      fo[i] = PopIO<C, S>::ld(s_f[(i * CS::FH + ty + 1 - cyv(i)) * CS::FW + tx + CS::XA - cxv(i)], i, ph);
    if (m & kNearWall) pull_slow<C, S>(g, ph, f, mask, side_in, side_out, x, y, fo);
  } else {
    pull_node<C, S>(g, ph, f, mask, side_in, side_out, x, y, m, fo);
  }
  C rho = fo[0];
#pragma unroll
  for (int i = 1; i < 9; ++i) rho = rho + fo[i];
  const C cs2 = C(1.0 / 3.0);
  C Fmx = C(0), Fmy = C(0), Fx = C(0), Fy = C(0), psi0 = C(0);
  const int pc0 = (ty + 2) * HX + tx + CS::PA;  // this node in the psi tile
  if (multiphase) psi0 = need_psi ? s_psi[pc0] : psi[id];
  if (need_psi) {
    C sx, sy;
    grad_t(&s_psi[pc0], HX, sx, sy);
    Fmx = -k.G * cs2 * psi0 * sx;
    Fmy = -k.G * cs2 * psi0 * sy;
  }
  if (forcing) {
    Fx = sub(Fmx, mul(sub(rho, k.rho_l), k.g));
    if (k.body_fx != C(0)) Fx = add(Fx, k.body_fx);
    Fy = Fmy;
  }
  const C omega = fdiv(C(1), add(fdiv(nu_of(ph, rho), cs2), C(0.5)));
  const C sig = need_psi ? k.sigma : C(0);
  C fs[9], ux, uy;
  if constexpr (OP == kCollBGK) collide_bgk(fo, rho, Fx, Fy, omega, fs, ux, uy);
  else collide(fo, rho, Fx, Fy, Fmx, Fmy, psi0, omega, sig, fs, ux, uy);
#pragma unroll
  for (int i = 0; i < 9; ++i) fn[i * g.plane + id] = PopIO<C, S>::st(fs[i], i, ph);
  rho_o[id] = rho;
  ux_o[id] = ux;
  uy_o[id] = uy;
  if (!(rho > C(0)) || !(ux == ux) || !(uy == uy)) atomicOr(status, 1);
}

// The psi tile of tile (x0, y0) with plain loads (periodic in y, clamped or periodic in x).
template <typename C, typename S, int CTY>
__device__ __forceinline__ void psi_tile_plain(const Geo& g, const C* __restrict__ psi, int x0, int y0, C* s_psi) {
  using CS = CollStage<C, S, CTY>;
  for (int p = threadIdx.y * kCollTX + threadIdx.x; p < CS::PW * CS::PH; p += kCollTX * CTY) {
    const int hx = p % CS::PW, hy = p / CS::PW;
    s_psi[p] = psi[map_y(g, y0 + hy - 2) * g.pitch + map_x(g, x0 + hx - CS::PA)];
  }
}

// Collision tile (bx, by) of 32 x CTY nodes.  tm_f, tm_psi: tensor maps of f and psi for TMA
// staging, or null.
template <typename C, typename S, int CTY, int OP = kCollCM>
__device__ __forceinline__ void collide_tile(const Geo& g, const Phys& ph, const S* __restrict__ f,
                                             S* __restrict__ fn, const C* __restrict__ psi,
                                             const uint8_t* __restrict__ mask, const C* __restrict__ side_in,
                                             C* __restrict__ side_out, C* __restrict__ rho_o, C* __restrict__ ux_o,
                                             C* __restrict__ uy_o, int forcing, int* status, int bx, int by,
                                             const CUtensorMap* tm_f = nullptr, const CUtensorMap* tm_psi = nullptr,
                                             bool starve = false, bool early_f = false) {
  using CS = CollStage<C, S, CTY>;
  constexpr int HX = CS::PW, HY = CS::PH;
  __shared__ __align__(128) S s_f[9 * CS::FH * CS::FW];
  __shared__ __align__(128) C s_psi[HY * HX];
  __shared__ uint64_t s_bar;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kCollTX + tx;
  const int x0 = bx * kCollTX, y0 = by * CTY;
  const int x = x0 + tx, y = y0 + ty;
  const bool need_psi = pc<C>(ph).G != C(0) && forcing;
  const bool staged = tm_f && (!need_psi || tm_psi) && coll_staged<C, S, CTY>(g, x0, y0);
  if (staged) {
    if (tid == 0) tma::bar_init(&s_bar, 1);
    __syncthreads();
    if (tid == 0) {
      const uint32_t bytes = sizeof(S) * 9 * CS::FH * CS::FW + (need_psi ? sizeof(C) * HX * HY : 0);
      tma::bar_expect_tx(&s_bar, bytes);
      // (the test hook leaves the barrier armed with no copy issued)
      if (!starve && early_f) tma::load_3d(s_f, tm_f, &s_bar, x0 - CS::XA, y0 - 1, 0);
    }
    pdl::wait();  // psi is the previous kernel's output
    pdl::trigger();
    if (tid == 0 && !starve) {
      if (!early_f) tma::load_3d(s_f, tm_f, &s_bar, x0 - CS::XA, y0 - 1, 0);
      if (need_psi) tma::load_2d(s_psi, tm_psi, &s_bar, x0 - CS::PA, y0 - 2);
    }
  } else {
    pdl::wait();
    pdl::trigger();
    if (need_psi) {
      psi_tile_plain<C, S, CTY>(g, psi, x0, y0, s_psi);
      __syncthreads();
    }
  }
  const bool inside = x < g.nx && y < g.ny;
  const uint8_t m = inside ? mask[y * g.pitch + x] : kSolid;
  const int tries = starve ? tma::kStarveTries : tma::kWaitTries;
  if (staged && !tma::bar_wait(&s_bar, 0, tries)) {
    // the copies did not land in time: report it, give them a second bound to land before the
    // block's shared memory is released, and produce nothing
    if (tid == 0) atomicOr(status, kStatusTimeoutCollide);
    tma::bar_wait(&s_bar, 0, tries);
    return;
  }
  if (!inside) return;
  collide_node<C, S, CTY, OP>(g, ph, f, fn, psi, mask, side_in, side_out, rho_o, ux_o, uy_o, forcing, status, tx, ty,
                              x, y, m, staged, s_f, s_psi);
}

template <typename C, typename S, int OP = kCollCM>
// FP32: at most 36 registers, so 7 blocks share an SM and more pulls are in flight (the pass
// waits on DRAM: +10% over the default register budget; with FP16 storage 7 blocks and a few
// spilled registers still beat 6 blocks without spills, 30.8 vs 32.6 us at 1536 x 768)
__global__ void __launch_bounds__(kCollTX* kCollTY, sizeof(C) == 4 ? 7 : 1)
    k_collide(Geo g, Phys ph, const S* __restrict__ f, S* __restrict__ fn, const C* __restrict__ psi,
              const uint8_t* __restrict__ mask, const C* __restrict__ side_in, C* __restrict__ side_out,
              C* __restrict__ rho_o, C* __restrict__ ux_o, C* __restrict__ uy_o, int forcing, int* status,
              const __grid_constant__ CUtensorMap tm_f, const __grid_constant__ CUtensorMap tm_psi, int flags) {
  const bool staged = flags & kLaunchStaged;
  collide_tile<C, S, kCollTY, OP>(g, ph, f, fn, psi, mask, side_in, side_out, rho_o, ux_o, uy_o, forcing, status,
                                  blockIdx.x, blockIdx.y, staged ? &tm_f : nullptr, staged ? &tm_psi : nullptr,
                                  (flags & kLaunchStarve) != 0, (flags & kLaunchEarlyF) != 0);
}

// ---------------------------------------------------------------- k_energy
// Fixed-shape block sum (warp shuffles, then the first warp over the warp sums).
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (tid < 32) {
    s = tid < NT / 32 ? red[tid] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

// Two x-adjacent nodes per thread: a 5x6 window (rows -2..2, columns -2..3 around the
// left node) is read from a shared tile with three aligned 2-vector loads per row; both
// nodes' stencils are then evaluated from registers in the same term order as above.
template <typename C>
struct Vec2;
template <>
struct Vec2<float> {
  using T = float2;
};
template <>
struct Vec2<double> {
  using T = double2;
};
template <typename C>
__device__ __forceinline__ void load_window(const C* p, int s, C w[5][6]) {
  using T2 = typename Vec2<C>::T;
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const T2* q = reinterpret_cast<const T2*>(p + (r - 2) * s - 2);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T2 v = q[c];
      w[r][2 * c] = v.x;
      w[r][2 * c + 1] = v.y;
    }
  }
}
template <typename C, bool kX = true, bool kY = true>
__device__ __forceinline__ void grad_w(const C w[5][6], int c0, C& gx, C& gy) {
  C sx = C(0), sy = C(0);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const int ex = exv(k), ey = eyv(k);
    if ((kX && ex != 0) || (kY && ey != 0)) {
      C d = w[2 + ey][c0 + ex] - w[2 - ey][c0 - ex];
      if (kX && ex != 0) sx = sx + C(wiso(k) * ex) * d;
      if (kY && ey != 0) sy = sy + C(wiso(k) * ey) * d;
    }
  }
  gx = sx;
  gy = sy;
}
template <typename C>
__device__ __forceinline__ C lap_w(const C w[5][6], int c0) {
  const C c = w[2][c0];
  C acc = C(0);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const int ex = exv(k), ey = eyv(k);
    C d = (w[2 + ey][c0 + ex] + w[2 - ey][c0 - ex]) - C(2) * c;
    acc = acc + C(wiso(k)) * d;
  }
  return C(2) * acc;
}
template <typename C>
__device__ __forceinline__ C upwind3_w(const C w[5][6], int c0, bool along_x, C v) {
  const C c = w[2][c0];
  auto at = [&](int o) { return along_x ? w[2][c0 + o] : w[2 + o][c0]; };
  if (v >= C(0)) {
    C m2 = at(-2) - c, m1 = at(-1) - c, p1 = at(1) - c;
    return fdiv(m2 - C(6) * m1 + C(2) * p1, C(6));
  }
  C m1 = at(-1) - c, p1 = at(1) - c, p2 = at(2) - c;
  return fdiv(-C(2) * m1 + C(6) * p1 - p2, C(6));
}
// Eq. (energy) splits into parts that depend on rho and u only, frozen during the step
// (lambda, grad lambda, div u), and parts that depend on the temperature being advanced.
template <typename C>
struct Frozen {
  C lam0, lx, ly, divu;
};
// Frozen parts at the two nodes whose left one is at lam[0], u[0], v[0] (row stride as;
// left node index even).
template <typename C>
__device__ __forceinline__ void frozen_pair(const C* lam, const C* u, const C* v, int as, Frozen<C> fz[2]) {
  C w[5][6], unused, dxux[2], dyuy[2];
  load_window(lam, as, w);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    fz[k].lam0 = w[2][2 + k];
    grad_w(w, 2 + k, fz[k].lx, fz[k].ly);
  }
  load_window(u, as, w);
#pragma unroll
  for (int k = 0; k < 2; ++k) grad_w<C, true, false>(w, 2 + k, dxux[k], unused);
  load_window(v, as, w);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    grad_w<C, false, true>(w, 2 + k, unused, dyuy[k]);
    fz[k].divu = dxux[k] + dyuy[k];
  }
}
// Right-hand side at the same two nodes for the temperature tile t (row stride ts):
// -u.grad T + (lambda lap T + grad lambda.grad T)/(rho c_v) - T (dp/dT)_rho div u / (rho c_v).
template <typename C>
__device__ __forceinline__ void energy_rhs_pair(const Phys& ph, const C* t, int ts, const C* u, const C* v,
                                                const C* r, const Frozen<C> fz[2], C L[2]) {
  C w[5][6];
  load_window(t, ts, w);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const C u0 = u[k], v0 = v[k], T0 = w[2][2 + k], r0 = r[k];
    C conv = u0 * upwind3_w(w, 2 + k, true, u0) + v0 * upwind3_w(w, 2 + k, false, v0);
    C gx, gy;
    grad_w(w, 2 + k, gx, gy);
    C lap = lap_w(w, 2 + k);
    C diff = fz[k].lam0 * lap + (fz[k].lx * gx + fz[k].ly * gy);
    C work = T0 * dpdT_eos(ph, r0, T0) * fz[k].divu;
    L[k] = -conv + fdiv(diff, r0 * pc<C>(ph).c_v) - fdiv(work, r0 * pc<C>(ph).c_v);
  }
}

// FP32: the two nodes of a pair are one packed float2 throughout the stencil sums (sm_100+
// FFMA2/FADD2/FMUL2), halving the FP32 instructions of the energy pass.  The window of a pair
// is kept as aligned column pairs A[r][j] = (c_2j, c_2j+1) and shifted pairs B[r][j] =
// (c_2j+1, c_2j+2); the value pair at offset ex is A[r][1 + ex/2] for even ex, B[r][(1 + ex)/2]
// for odd ex.  Each packed operation rounds like the scalar one it replaces.
struct Win2 {
  float2 A[5][3], B[5][2];
};
__device__ __forceinline__ void load_win2(const float* p, int s, Win2& W) {
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const float2* q = reinterpret_cast<const float2*>(p + (r - 2) * s - 2);
#pragma unroll
    for (int c = 0; c < 3; ++c) W.A[r][c] = q[c];
    W.B[r][0] = make_float2(W.A[r][0].y, W.A[r][1].x);
    W.B[r][1] = make_float2(W.A[r][1].y, W.A[r][2].x);
  }
}
__device__ __forceinline__ float2 win_at(const Win2& W, int r, int ex) {
  return (ex & 1) ? W.B[r][(1 + ex) / 2] : W.A[r][1 + ex / 2];
}
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
template <bool kX = true, bool kY = true>
__device__ __forceinline__ void grad_w2(const Win2& W, float2& gx, float2& gy) {
  float2 sx = f2(0.f), sy = f2(0.f);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const int ex = exv(k), ey = eyv(k);
    if ((kX && ex != 0) || (kY && ey != 0)) {
      const float2 d = sub2(win_at(W, 2 + ey, ex), win_at(W, 2 - ey, -ex));
      if (kX && ex != 0) sx = __ffma2_rn(f2(float(wiso(k) * ex)), d, sx);
      if (kY && ey != 0) sy = __ffma2_rn(f2(float(wiso(k) * ey)), d, sy);
    }
  }
  gx = sx;
  gy = sy;
}
__device__ __forceinline__ float2 lap_w2(const Win2& W) {
  const float2 c = W.A[2][1];
  float2 acc = f2(0.f);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const int ex = exv(k), ey = eyv(k);
    const float2 d = __ffma2_rn(c, f2(-2.f), __fadd2_rn(win_at(W, 2 + ey, ex), win_at(W, 2 - ey, -ex)));
    acc = __ffma2_rn(f2(float(wiso(k))), d, acc);
  }
  return __fmul2_rn(f2(2.f), acc);
}
// Six times the third-order upwind derivative of the pair along x (row 2) or y (column pair
// 1), each node biased against the sign of its own velocity v.
__device__ __forceinline__ float2 upwind6_w2(const Win2& W, bool along_x, float2 v) {
  float2 q[5];
#pragma unroll
  for (int o = -2; o <= 2; ++o) q[o + 2] = along_x ? win_at(W, 2, o) : W.A[2 + o][1];
  const float2 c = q[2];
  const float2 m2 = sub2(q[0], c), m1 = sub2(q[1], c), p1 = sub2(q[3], c), p2 = sub2(q[4], c);
  const float2 pos = __ffma2_rn(f2(2.f), p1, __ffma2_rn(f2(-6.f), m1, m2));
  const float2 neg = sub2(__ffma2_rn(f2(6.f), p1, __fmul2_rn(f2(-2.f), m1)), p2);
  return make_float2(v.x >= 0.f ? pos.x : neg.x, v.y >= 0.f ? pos.y : neg.y);
}
template <>
__device__ __forceinline__ void frozen_pair<float>(const float* lam, const float* u, const float* v, int as,
                                                   Frozen<float> fz[2]) {
  Win2 W;
  float2 lx, ly, dxux, dyuy, unused;
  load_win2(lam, as, W);
  fz[0].lam0 = W.A[2][1].x;
  fz[1].lam0 = W.A[2][1].y;
  grad_w2(W, lx, ly);
  load_win2(u, as, W);
  grad_w2<true, false>(W, dxux, unused);
  load_win2(v, as, W);
  grad_w2<false, true>(W, unused, dyuy);
  const float2 dv = __fadd2_rn(dxux, dyuy);
  fz[0].lx = lx.x, fz[0].ly = ly.x, fz[0].divu = dv.x;
  fz[1].lx = lx.y, fz[1].ly = ly.y, fz[1].divu = dv.y;
}
__device__ __forceinline__ float2 pk_div(float2 a, float2 b) {
  return make_float2(__fdividef(a.x, b.x), __fdividef(a.y, b.y));
}
template <>
__device__ __forceinline__ void energy_rhs_pair<float>(const Phys& ph, const float* t, int ts, const float* u,
                                                       const float* v, const float* r, const Frozen<float> fz[2],
                                                       float L[2]) {
  Win2 W;
  load_win2(t, ts, W);
  const float2 u2 = make_float2(u[0], u[1]), v2 = make_float2(v[0], v[1]);
  const float2 conv6 = __ffma2_rn(u2, upwind6_w2(W, true, u2), __fmul2_rn(v2, upwind6_w2(W, false, v2)));
  float2 gx, gy;
  grad_w2(W, gx, gy);
  const float2 lap = lap_w2(W);
  const float2 diff = __ffma2_rn(make_float2(fz[0].lam0, fz[1].lam0), lap,
                                 __ffma2_rn(make_float2(fz[0].lx, fz[1].lx), gx,
                                            __fmul2_rn(make_float2(fz[0].ly, fz[1].ly), gy)));
  // (dp/dT)_rho of Eq. (eos) with phi = (1 + kappa (1 - sqrt(T/Tc)))^2, dphi/dT = -kappa
  // sqrt(phi) / sqrt(T Tc):  rep + att (kappa (1 + kappa) / sqrt(T Tc) - kappa^2 / Tc), with
  // rep = rho R / (1 - b rho) and att = a rho^2 / (1 + 2 b rho - b^2 rho^2)
  const PhysC<float>& k = ph.f;
  const float2 rho = make_float2(r[0], r[1]), T0 = W.A[2][1];
  const float2 rep = pk_div(__fmul2_rn(f2(k.R), rho), __ffma2_rn(f2(-k.b), rho, f2(1.0f)));
  const float2 att = pk_div(__fmul2_rn(__fmul2_rn(f2(k.a), rho), rho),
                            __ffma2_rn(rho, __ffma2_rn(f2(-k.b * k.b), rho, f2(2.0f * k.b)), f2(1.0f)));
  const float2 rs = make_float2(rsqrtf(T0.x * k.Tc), rsqrtf(T0.y * k.Tc));
  const float2 dpdT = __ffma2_rn(att, __ffma2_rn(f2(ph.dpdT_c1), rs, f2(-ph.dpdT_c2)), rep);
  const float2 work = __fmul2_rn(__fmul2_rn(T0, dpdT), make_float2(fz[0].divu, fz[1].divu));
  const float2 Lp = __ffma2_rn(sub2(diff, work), pk_div(f2(1.0f), __fmul2_rn(f2(k.c_v), rho)),
                               __fmul2_rn(f2(-1.0f / 6.0f), conv6));
  L[0] = Lp.x;
  L[1] = Lp.y;
}

// Density of the pulled populations, rho = sum_i f*_i(x - c_i), at the nodes (x0, y) and
// (x0 + 1, y), x0 even, for a pair none of whose pulls crosses the lattice edge or meets the
// wall (1 <= x0, x0 + 2 <= nx - 1, 1 <= y <= ny - 2, no near-wall node): the planes with c_x = 0
// are read as aligned vectors, the others as scalars, all from one base address; the sum runs
// in the order i = 0..8, as in the general pull, so both give the same bits.
template <typename S>
struct PairLoad;
template <>
struct PairLoad<float> {
  static __device__ __forceinline__ void ld(const float* q, float& a, float& b) {
    const float2 v = *reinterpret_cast<const float2*>(q);
    a = v.x, b = v.y;
  }
};
template <>
struct PairLoad<double> {
  static __device__ __forceinline__ void ld(const double* q, double& a, double& b) {
    const double2 v = *reinterpret_cast<const double2*>(q);
    a = v.x, b = v.y;
  }
};
template <>
struct PairLoad<__half> {
  static __device__ __forceinline__ void ld(const __half* q, __half& a, __half& b) {
    const __half2 v = *reinterpret_cast<const __half2*>(q);
    a = __low2half(v), b = __high2half(v);
  }
};
template <typename C, typename S>
__device__ __forceinline__ void pair_rho(const Geo& g, const Phys& ph, const S* __restrict__ f, int x0, int y,
                                         C r[2]) {
  const S* p = f + y * g.pitch + x0;
  C v[9][2];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const S* q = p + i * g.plane - cyv(i) * g.pitch - cxv(i);
    S a, b;
    if (cxv(i) == 0) {
      PairLoad<S>::ld(q, a, b);
    } else {
      a = q[0];
      b = q[1];
    }
    v[i][0] = PopIO<C, S>::ld(a, i, ph);
    v[i][1] = PopIO<C, S>::ld(b, i, ph);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    C t = v[0][k];
#pragma unroll
    for (int i = 1; i < 9; ++i) t = t + v[i][k];
    r[k] = t;
  }
}

// Heun stage 2 at the pair whose left node is (x, y), T^{n+1} = (T + T1 + L(T1)) / 2, from
// shared tiles: inputs sT, sL, sU, sV, sR, sM (row stride ax, pair at index a) and the stage-1
// temperature sT1 (row stride bx, pair at index b); fz: the pair's frozen parts.  Nodes with
// x >= nx or y >= ylim are skipped.  Writes T^{n+1}, T1 (t1_out) and, with FUSE and psi_out,
// psi of the next step from the pull of the new populations fnew, side_new (Eq. potential);
// adds the pair's wall heat flux -lambda grad T^n . n (Sec. IV.B) to q and sets mine when
// the pair holds a near-wall node.
template <typename C, typename S, int PSI, bool FUSE>
__device__ __forceinline__ void stage2_pair(const Geo& g, const Phys& ph, const C* sT, const C* sL, const C* sU,
                                            const C* sV, const C* sR, const uint8_t* sM, int ax, int a, const C* sT1,
                                            int bx, int b, const Frozen<C>* fz_in, int x0, int y, int ylim,
                                            C* __restrict__ Tout, C* __restrict__ t1_out, int do_hf,
                                            const S* __restrict__ fnew, const uint8_t* __restrict__ mask,
                                            const C* __restrict__ side_new, C* __restrict__ psi_out, int* status,
                                            double& q, int& mine) {
  const Frozen<C> fz[2] = {fz_in[0], fz_in[1]};
  C L[2];
  energy_rhs_pair(ph, &sT1[b], bx, &sU[a], &sV[a], &sR[a], fz, L);
  C tnew[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int x = x0 + k;
    if (x < g.nx && y < ylim) {
      C out;
      if (sM[a + k] & kSolid) out = sT[a + k];
      else if (!g.periodic_x && x == 0) out = pc<C>(ph).T_sat;
      else out = ((sT[a + k] + sT1[b + k]) + L[k]) * C(0.5);
      Tout[y * g.pitch + x] = out;
      tnew[k] = out;
      if (t1_out) t1_out[y * g.pitch + x] = sT1[b + k];  // the stage-1 temperature, for the adjoint
      if (do_hf && (sM[a + k] & kNearWall)) {
        C gx, gy;
        grad_t(&sT[a + k], ax, gx, gy);
        const double* nv = &g.wall_n[2 * g.wall_idx[y * g.pitch + x]];
        q += -(double)sL[a + k] * ((double)gx * nv[0] + (double)gy * nv[1]);
        mine = 1;
      }
    }
  }
  if constexpr (FUSE) {
    if (psi_out) {
      const uint8_t m0 = sM[a], m1 = sM[a + 1];
      C r[2];
      // a pair away from the wall, the open edges and the periodic seams pulls from one base
      // address; the others take the general pull with its boundary substitutions
      if (!((m0 | m1) & kNearWall) && y >= 1 && y + 1 < g.ny && x0 >= 1 && x0 + 3 <= g.nx) {
        pair_rho<C, S>(g, ph, fnew, x0, y, r);
      } else {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          r[k] = C(0);
          if (x0 + k < g.nx && y < ylim) {
            C fo[9];
            pull_node<C, S>(g, ph, fnew, mask, side_new, nullptr, x0 + k, y, k ? m1 : m0, fo);
            C t = fo[0];
#pragma unroll
            for (int i = 1; i < 9; ++i) t = t + fo[i];
            r[k] = t;
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int x = x0 + k;
        if (x < g.nx && y < ylim) {
          const C rho = ((k ? m1 : m0) & kSolid) ? pc<C>(ph).rho_s : r[k];
          psi_out[y * g.pitch + x] = psi_of<C, PSI>(ph, rho, tnew[k], status);
        }
      }
    }
  }
}

// Block-level end of the wall heat flux: FP64 block sums only in the blocks that hold wall
// nodes (the others skip the fence and the counter); the last of those n_wall blocks to
// finish adds all nblocks partials in block order (zero elsewhere), updates the running
// statistics hf and clears the partials for the next launch.  Every thread of the block calls it.
template <int NT>
__device__ __forceinline__ void heat_flux_blocks(double q, int mine, double* partial, unsigned* counter, int n_wall,
                                                 int bid, int nblocks, double* hf, int nb, double* red,
                                                 int* done_last) {
  const int tid = threadIdx.x;
  if (__syncthreads_or(mine)) {
    const double s = block_sum<NT>(q, red);
    if (tid == 0) {
      partial[bid] = s;
      __threadfence();
      *done_last = atomicInc(counter, n_wall - 1) == (unsigned)(n_wall - 1);
    }
    __syncthreads();
    if (*done_last) {
      __threadfence();
      double acc = 0.0;
      for (int i = tid; i < nblocks; i += NT) acc += __ldcg(&partial[i]);
      acc = block_sum<NT>(acc, red);  // its barrier also ends every thread's reads above
      for (int i = tid; i < nblocks; i += NT) partial[i] = 0.0;
      if (tid == 0) {
        const double qv = acc / nb;
        hf[0] = qv;
        hf[1] += qv;
        hf[2] += qv * qv;
        hf[3] += 1.0;
      }
    }
  }
}

template <typename C, int TY_ = (sizeof(C) == 8 ? 8 : kEnergyTY)>
struct EnergyTile {
  static constexpr int TX = kEnergyTX;
  static constexpr int TY = TY_;          // FP64 defaults to 8 rows to keep shared memory under 48 KB
  static constexpr int NT = TX * TY / 2;  // two nodes per thread
};

// Both Heun stages on tile (bx, by); bid, nblocks: this tile's index among the domain's
// nblocks tiles (for the heat-flux partials and the last-block reduction).
// With FUSE, and psi_out set, the tile also evaluates psi of the next step at its nodes: the
// pull of the populations this step's collision wrote (fnew, side_new), rho their sum (rho_s
// in the solid), T the new temperature (Eq. potential) -- the next step then needs no psi pass.
// maps: tensor maps of the inputs, with which an interior tile stages them by TMA (else null:
// plain loads); t1_out: where to store the stage-1 temperature (the adjoint's recompute).
template <typename C, int ETY, typename S = C, int PSI = kPsiF64, bool FUSE = false>
__device__ __forceinline__ void energy_tile(const Geo& g, const Phys& ph, const C* __restrict__ Tin,
                                            C* __restrict__ Tout, const C* __restrict__ rho, const C* __restrict__ ux,
                                            const C* __restrict__ uy, const uint8_t* __restrict__ mask,
                                            double* partial, unsigned* counter, double* hf, int nb, int do_hf,
                                            int n_wall_tiles, int bx, int by, int bid, int nblocks,
                                            const S* __restrict__ fnew = nullptr, const C* __restrict__ side_new = nullptr,
                                            C* __restrict__ psi_out = nullptr, int* status = nullptr,
                                            C* __restrict__ t1_out = nullptr, const EnergyMaps* maps = nullptr,
                                            bool starve = false) {
  constexpr int TX = EnergyTile<C, ETY>::TX, TY = EnergyTile<C, ETY>::TY, NT = EnergyTile<C, ETY>::NT;
  constexpr int H = 4, AX = TX + 2 * H, AY = TY + 2 * H;  // inputs: tile + 4
  constexpr int BX = TX + 4, BY = TY + 4;                 // stage 1: tile + 2
  static_assert(AX * AY * sizeof(C) % 128 == 0 && AX * sizeof(C) % 16 == 0, "TMA boxes of the input tile");
  static_assert(AX % 4 == 0 && (AX * AY) % 4 == 0, "word-wise mask and float4 lambda staging");
  __shared__ __align__(128) C sT[AY * AX];
  __shared__ __align__(128) C sL[AY * AX];
  __shared__ __align__(128) C sRUV[3 * AY * AX];  // rho, u_x, u_y: the planes of one TMA box
  C* const sR = sRUV;
  C* const sU = sRUV + AY * AX;
  C* const sV = sRUV + 2 * AY * AX;
  __shared__ uint64_t s_bar;
  __shared__ __align__(16) C sT1[BY * BX];
  __shared__ Frozen<C> sF[TX * TY];
  __shared__ __align__(16) uint8_t sM[AY * AX];
  __shared__ double red[NT / 32];
  __shared__ int done_last;
  const int tid = threadIdx.x;
  const int x0 = bx * TX, y0 = by * TY;
  const bool interior = x0 >= H && y0 >= H && x0 + TX + H <= g.nx && y0 + TY + H <= g.ny;
  if (maps && interior) {
    // the input boxes by TMA (T; rho, u_x, u_y in one 3-plane box; first column x0 - 4:
    // 16-byte aligned); the mask with plain
    // loads while they fly; lambda(rho) once rho has landed
    if (tid == 0) tma::bar_init(&s_bar, 1);
    __syncthreads();
    if (tid == 0) {
      tma::bar_expect_tx(&s_bar, 4 * AX * AY * sizeof(C));
      // T comes from the energy pass before the previous kernel (the collision, which does not
      // write it): its copy starts before that kernel ends; the test hook leaves the barrier
      // armed with no copy issued
      if (!starve) tma::load_2d(sT, &maps->T, &s_bar, x0 - H, y0 - H);
    }
    // the mask as 32-bit words (x0 - 4 and the row pitch are multiples of 4 bytes)
    for (int p = tid; p < (AX / 4) * AY; p += NT) {
      const int r = p / (AX / 4), c = p - r * (AX / 4);
      reinterpret_cast<uint32_t*>(sM)[p] =
          *reinterpret_cast<const uint32_t*>(mask + (y0 + r - H) * g.pitch + x0 - H + 4 * c);
    }
    pdl::wait();  // rho, u and the new populations are the collision's output
    pdl::trigger();
    if (tid == 0 && !starve) tma::load_3d(sRUV, &maps->ruv, &s_bar, x0 - H, y0 - H, 0);
    const int tries = starve ? tma::kStarveTries : tma::kWaitTries;
    const bool landed = tma::bar_wait(&s_bar, 0, tries);
    if (__syncthreads_or(!landed)) {
      // a copy did not land in time: report it, let the copies land (bounded) and stop the tile
      // (a tile that holds wall nodes then misses its heat-flux partial; restoring a state with
      // lbm_set_state resets that bookkeeping)
      if (tid == 0) atomicOr(status, kStatusTimeoutEnergy);
      tma::bar_wait(&s_bar, 0, tries);
      return;
    }
    if constexpr (sizeof(C) == 4) {
      for (int p = tid; p < AX * AY / 4; p += NT) {  // four nodes per thread
        const float4 r4 = reinterpret_cast<const float4*>(sR)[p];
        reinterpret_cast<float4*>(sL)[p] =
            make_float4(lam_of(ph, r4.x), lam_of(ph, r4.y), lam_of(ph, r4.z), lam_of(ph, r4.w));
      }
    } else {
      for (int p = tid; p < AX * AY; p += NT) sL[p] = lam_of(ph, sR[p]);
    }
  } else {
    pdl::wait();
    pdl::trigger();
    for (int p = tid; p < AX * AY; p += NT) {
      const int gx = x0 + p % AX - H, gy = y0 + p / AX - H;
      const int nid = interior ? gy * g.pitch + gx : map_y(g, gy) * g.pitch + map_x(g, gx);
      const C r = rho[nid];
      sT[p] = Tin[nid];
      sR[p] = r;
      sL[p] = lam_of(ph, r);
      sU[p] = ux[nid];
      sV[p] = uy[nid];
      sM[p] = mask[nid];
    }
  }
  __syncthreads();
  // stage 1: T1 = T + L(T) on the tile and a 2-node halo, two nodes per thread; the frozen
  // parts of the tile's own nodes are kept for stage 2
  for (int p = tid; p < (BX / 2) * BY; p += NT) {
    const int by = p / (BX / 2), bx = (p % (BX / 2)) * 2;
    const int a = (by + 2) * AX + bx + 2;
    Frozen<C> fz[2];
    frozen_pair(&sL[a], &sU[a], &sV[a], AX, fz);
    C L[2];
    energy_rhs_pair(ph, &sT[a], AX, &sU[a], &sV[a], &sR[a], fz, L);
    const int tx = bx - 2, ty = by - 2;
    if (tx >= 0 && tx < TX && ty >= 0 && ty < TY) {
      sF[ty * TX + tx] = fz[0];
      sF[ty * TX + tx + 1] = fz[1];
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int gx = x0 + bx + k - 2;
      C t1;
      if (sM[a + k] & kSolid) t1 = sT[a + k];  // solid nodes keep their wall temperature
      else if (!g.periodic_x && gx == 0) t1 = pc<C>(ph).T_sat;
      else t1 = sT[a + k] + L[k];
      sT1[by * BX + bx + k] = t1;  // positions past a non-periodic edge are replaced below
    }
  }
  __syncthreads();
  if (!g.periodic_x && (x0 < 2 || x0 + TX + 2 > g.nx)) {
    for (int p = tid; p < BX * BY; p += NT) {
      const int bx = p % BX, by = p / BX;
      const int gx = x0 + bx - 2;
      if (gx < 0 || gx >= g.nx) sT1[p] = sT1[by * BX + (map_x(g, gx) - x0 + 2)];
    }
    __syncthreads();
  }
  // stage 2 on the tile: T^{n+1} = (T + T1 + L(T1)) / 2
  const int tx = (tid % (TX / 2)) * 2, ty = tid / (TX / 2);
  double q = 0.0;
  int mine = 0;
  stage2_pair<C, S, PSI, FUSE>(g, ph, sT, sL, sU, sV, sR, sM, AX, (ty + H) * AX + tx + H, sT1, BX,
                               (ty + 2) * BX + tx + 2, &sF[ty * TX + tx], x0 + tx, y0 + ty, g.ny, Tout, t1_out, do_hf,
                               fnew, mask, side_new, psi_out, status, q, mine);
  if (do_hf) heat_flux_blocks<NT>(q, mine, partial, counter, n_wall_tiles, bid, nblocks, hf, nb, red, &done_last);
}
template <typename C, typename S, int PSI>
// FP32: at most 51 registers, 5 blocks per SM (+2.5%); with FP16 storage 64 registers and
// 4 blocks (the conversions of the fused psi pull need them: no spills)
__global__ void __launch_bounds__(EnergyTile<C>::NT, sizeof(C) == 4 ? (sizeof(S) == 2 ? 4 : 5) : 1)
    k_energy(Geo g, Phys ph, const C* __restrict__ Tin, C* __restrict__ Tout, const C* __restrict__ rho,
             const C* __restrict__ ux, const C* __restrict__ uy, const uint8_t* __restrict__ mask,
             double* partial, unsigned* counter, double* hf, int nb, int do_hf, int n_wall_tiles,
             const S* __restrict__ fnew, const C* __restrict__ side_new, C* __restrict__ psi_out, int* status,
             C* __restrict__ t1_out, const __grid_constant__ EnergyMaps maps, int flags) {
  energy_tile<C, EnergyTile<C>::TY, S, PSI, true>(g, ph, Tin, Tout, rho, ux, uy, mask, partial, counter, hf, nb,
                                                   do_hf, n_wall_tiles, blockIdx.x, blockIdx.y,
                                                   blockIdx.y * gridDim.x + blockIdx.x, gridDim.x * gridDim.y, fnew,
                                                   side_new, psi_out, status, t1_out,
                                                   (flags & kLaunchStaged) ? &maps : nullptr,
                                                   (flags & kLaunchStarve) != 0);
}

// ---------------------------------------------------------------- batched passes
// Every block of a batched pass finds its domain through the block -> domain map and its
// tile from its index within that domain; the tile bodies are the single-domain ones.
// psi of the state with population parity p sits in domain buffer p (psi, psi_next): the
// energy pass of a step with parity cur writes psi of the next state into buffer cur ^ 1,
// so the psi pass runs only when the host no longer knows psi (creation, a state change).
template <typename C>
__device__ __forceinline__ C* psi_buf(const BatchDomain& D, int p) {
  return static_cast<C*>(p ? D.d.psi_next : D.d.psi);
}
template <typename C, typename S, int PSI>
__global__ void __launch_bounds__(256) kb_rho_psi(const BatchDomain* __restrict__ doms, const int* __restrict__ map,
                                                 int cur, int tcur) {
  const BatchDomain& D = doms[map[blockIdx.x]];
  if (pc<C>(D.ph).G == C(0)) return;
  const int local = blockIdx.x - D.psi_first;
  rho_psi_tile<C, S, PSI>(D.g, D.ph, static_cast<const S*>(D.d.f[cur]), static_cast<const C*>(D.d.T[tcur]),
                          D.d.mask, static_cast<const C*>(D.d.side[cur]), psi_buf<C>(D, cur), D.d.status,
                          local % D.psi_ntx, local / D.psi_ntx);
}
// A batched launch covers the blocks [block0, block0 + gridDim.x) of a pass, which belong to
// the domains dom0 ..; their tensor maps come as kernel parameters (index k - dom0).
template <typename C, typename S, int CTY>
__global__ void __launch_bounds__(kCollTX* CTY, (sizeof(C) == 4 && CTY == 8) ? 7 : 1)
    kb_collide(const BatchDomain* __restrict__ doms, const int* __restrict__ map, int cur, long long step,
               int block0, int dom0, const __grid_constant__ CollLaunchMaps maps) {
  const int blk = block0 + blockIdx.x, k = map[blk];
  const BatchDomain& D = doms[k];
  const int local = blk - D.coll_first;
  collide_tile<C, S, CTY>(D.g, D.ph, static_cast<const S*>(D.d.f[cur]), static_cast<S*>(D.d.f[cur ^ 1]),
                          psi_buf<C>(D, cur), D.d.mask, static_cast<const C*>(D.d.side[cur]),
                          static_cast<C*>(D.d.side[cur ^ 1]), static_cast<C*>(D.d.rho), static_cast<C*>(D.d.ux),
                          static_cast<C*>(D.d.uy), step >= D.warmup, D.d.status, local % D.coll_ntx,
                          local / D.coll_ntx, D.tma ? &maps.f[k - dom0] : nullptr,
                          D.tma ? &maps.psi[k - dom0] : nullptr);
}
template <typename C, int ETY, int PSI>
// FP32: a register budget for 1280 threads per SM, as the single-domain energy pass
__global__ void __launch_bounds__(EnergyTile<C, ETY>::NT, sizeof(C) == 4 ? 1280 / EnergyTile<C, ETY>::NT : 1) kb_energy(const BatchDomain* __restrict__ doms,
                                                                   const int* __restrict__ map, int cur, int tcur,
                                                                   long long step, int block0, int dom0,
                                                                   const __grid_constant__ EnLaunchMaps maps) {
  const int blk = block0 + blockIdx.x, k = map[blk];
  const BatchDomain& D = doms[k];
  const int local = blk - D.en_first, bx = local % D.en_ntx, by = local / D.en_ntx;
  const C* Tin = static_cast<const C*>(D.d.T[tcur]);
  C* Tout = static_cast<C*>(D.d.T[tcur ^ 1]);
  const C* fnew = static_cast<const C*>(D.d.f[cur ^ 1]);
  const C* side_new = static_cast<const C*>(D.d.side[cur ^ 1]);
  C* psi_next = pc<C>(D.ph).G != C(0) ? psi_buf<C>(D, cur ^ 1) : nullptr;
  if (!D.energy || step < D.warmup) {
    // no energy update for this domain this step: carry T over so all domains flip together,
    // and make psi of the next state from the new populations and the unchanged T
    constexpr int TX = EnergyTile<C, ETY>::TX, TY = EnergyTile<C, ETY>::TY;
    for (int p = threadIdx.x; p < TX * TY; p += EnergyTile<C, ETY>::NT) {
      const int x = bx * TX + p % TX, y = by * TY + p / TX;
      if (x < D.g.nx && y < D.g.ny) {
        Tout[y * D.g.pitch + x] = Tin[y * D.g.pitch + x];
        if (psi_next)
          psi_next[y * D.g.pitch + x] =
              psi_node<C, C, PSI>(D.g, D.ph, fnew, Tin, D.d.mask, side_new, x, y, D.d.status);
      }
    }
    return;
  }
  const EnergyMaps* em = D.tma ? &maps.e[k - dom0] : nullptr;
  energy_tile<C, ETY, C, PSI, true>(D.g, D.ph, Tin, Tout, static_cast<const C*>(D.d.rho),
                                    static_cast<const C*>(D.d.ux), static_cast<const C*>(D.d.uy), D.d.mask,
                                    D.d.partial, D.d.counter, D.d.hf, D.d.nb, D.d.nb > 0,
                                    D.d.wall_tiles[ETY == 16 ? 1 : 0], bx, by, local, D.en_nblocks, fnew, side_new,
                                    psi_next, D.d.status, nullptr, em);
}

template <typename C, typename S, int PSI, int CTY, int ETY>
int batch_step_impl(const BatchDomain* doms, const int* map_psi, int nb_psi, const int* map_coll, int nb_coll,
                    const int* map_en, int nb_en, int cur, int tcur, long long step, int need_psi,
                    const BatchDomain* hdoms, const DomainMaps* hmaps, int ndom, cudaStream_t s) {
  int n = 0;
  if (need_psi) {
    kb_rho_psi<C, S, PSI><<<nb_psi, dim3(kCollTX, 8), 0, s>>>(doms, map_psi, cur, tcur);
    ++n;
  }
  for (int d0 = 0; d0 < ndom; d0 += kBatchCollDomains) {
    const int d1 = d0 + kBatchCollDomains < ndom ? d0 + kBatchCollDomains : ndom;
    CollLaunchMaps m;
    for (int k = d0; k < d1; ++k) {
      m.f[k - d0] = hmaps[k].f[cur];
      m.psi[k - d0] = hmaps[k].psi[cur];
    }
    const int b0 = hdoms[d0].coll_first, b1 = d1 < ndom ? hdoms[d1].coll_first : nb_coll;
    kb_collide<C, S, CTY><<<b1 - b0, dim3(kCollTX, CTY), 0, s>>>(doms, map_coll, cur, step, b0, d0, m);
    ++n;
  }
  for (int d0 = 0; d0 < ndom; d0 += kBatchEnDomains) {
    const int d1 = d0 + kBatchEnDomains < ndom ? d0 + kBatchEnDomains : ndom;
    EnLaunchMaps m;
    for (int k = d0; k < d1; ++k) m.e[k - d0] = hmaps[k].em[tcur];
    const int b0 = hdoms[d0].en_first, b1 = d1 < ndom ? hdoms[d1].en_first : nb_en;
    kb_energy<C, ETY, PSI><<<b1 - b0, EnergyTile<C, ETY>::NT, 0, s>>>(doms, map_en, cur, tcur, step, b0, d0, m);
    ++n;
  }
  return cudaPeekAtLastError() == cudaSuccess ? n : -1;
}

// Tensor maps of one batched domain for tile heights (cty, ety), as the single-domain step
// encodes them per launch (here once per layout: the buffers of a domain do not move).
template <typename C, typename S>
bool batch_maps_impl(BatchDomain& D, DomainMaps& m, int cty, int ety) {
  const Geo& g = D.g;
  const int XA = 16 / (int)sizeof(S), PA = 16 / (int)sizeof(C) < 2 ? 2 : 16 / (int)sizeof(C);
  bool ok = D.d.tma != 0;
  for (int p = 0; p < 2 && ok; ++p) {
    ok = tma::encode<S>(&m.f[p], D.d.f[p], g.nx, g.ny, g.pitch, g.plane, 9, kCollTX + 2 * XA, cty + 2) &&
         tma::encode<C>(&m.psi[p], p ? D.d.psi_next : D.d.psi, g.nx, g.ny, g.pitch, g.plane, 1,
                        kCollTX + 2 * PA, cty + 4) &&
         tma::encode<C>(&m.em[p].T, D.d.T[p], g.nx, g.ny, g.pitch, g.plane, 1, kEnergyTX + 8, ety + 8) &&
         static_cast<const C*>(D.d.ux) == static_cast<const C*>(D.d.rho) + g.plane &&
         static_cast<const C*>(D.d.uy) == static_cast<const C*>(D.d.rho) + 2 * (size_t)g.plane &&
         tma::encode<C>(&m.em[p].ruv, D.d.rho, g.nx, g.ny, g.pitch, g.plane, 3, kEnergyTX + 8, ety + 8);
  }
  D.tma = ok ? 1 : 0;
  return ok;
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
__global__ void __launch_bounds__(256) k_init(Geo g, Phys ph, const double* rho0, const double* drho,
                                             const double* ux0, const double* uy0, const double* T0,
                                             const double* Tw, unsigned long long seed, double noise_amp, S* f,
                                             C* T, C* rho_o,
                                             C* ux_o, C* uy_o, C* side, const uint8_t* __restrict__ mask) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 8 + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int id = y * g.pitch + x;
  const int k = y * g.nx + x;
  double r = rho0 ? rho0[k] : ph.d.rho_l;
  r = r + (drho ? drho[k] : noise_amp * splitmix_pm1(seed, (unsigned long long)k));
  double u = ux0 ? ux0[k] : ph.d.u_in, v = uy0 ? uy0[k] : 0.0;
  double t = T0 ? T0[k] : ph.d.T_sat;
  if (mask[id] & kSolid) {
    r = ph.d.rho_s;
    u = 0.0;
    v = 0.0;
    t = Tw ? Tw[k] : ph.d.T_wall;
  }
  double fe[9];
  feq_hermite(r, u, v, fe);
#pragma unroll
  for (int i = 0; i < 9; ++i) f[i * g.plane + id] = PopIO<C, S>::st_d(fe[i], i, ph);
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
__global__ void k_export(Geo g, const E* __restrict__ src, int src_pitch, int rows, double* __restrict__ dst,
                         int ncols) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= ncols || y >= rows) return;
  dst[y * ncols + x] = (double)src[y * src_pitch + x];
}

static __global__ void k_export_solid(Geo g, const uint8_t* __restrict__ mask, double* __restrict__ dst) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  dst[y * g.nx + x] = (mask[y * g.pitch + x] & kSolid) ? 1.0 : 0.0;
}

// Component comp (0: x, 1: y) of the force F = F_m + F_g (+ the body force) that the collision
// applied at every node (Eq. interForce with gravity along -x, Sec. IV.A), recomputed from the
// psi and rho that collision used with the same stencil code and roundings; zero on solid nodes
// and when the step ran without forcing (warm-up).
template <typename C>
__global__ void k_export_force(Geo g, Phys ph, const C* __restrict__ psi, const C* __restrict__ rho,
                               const uint8_t* __restrict__ mask, int forcing, int comp, double* __restrict__ dst) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int id = y * g.pitch + x;
  double out = 0.0;
  if (forcing && !(mask[id] & kSolid)) {
    const PhysC<C>& k = pc<C>(ph);
    const C cs2 = C(1.0 / 3.0);
    C Fmx = C(0), Fmy = C(0);
    if (k.G != C(0)) {
      C w[25];
#pragma unroll
      for (int r = 0; r < 5; ++r)
#pragma unroll
        for (int c = 0; c < 5; ++c) w[r * 5 + c] = psi[map_y(g, y + r - 2) * g.pitch + map_x(g, x + c - 2)];
      C sx, sy;
      grad_t(&w[12], 5, sx, sy);
      Fmx = -k.G * cs2 * w[12] * sx;
      Fmy = -k.G * cs2 * w[12] * sy;
    }
    C Fx = sub(Fmx, mul(sub(rho[id], k.rho_l), k.g));
    if (k.body_fx != C(0)) Fx = add(Fx, k.body_fx);
    out = comp == 0 ? (double)Fx : (double)Fmy;
  }
  dst[y * g.nx + x] = out;
}

template <typename C, typename S>
__global__ void k_export_pop(Geo g, Phys ph, const S* __restrict__ src, int i, double* __restrict__ dst) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  dst[y * g.nx + x] = PopIO<C, S>::ld_d(src[y * g.pitch + x], i, ph);
}
template <typename C, typename S>
__global__ void k_import_pop(Geo g, Phys ph, S* __restrict__ dst, int i, const double* __restrict__ src) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  dst[y * g.pitch + x] = PopIO<C, S>::st_d(src[y * g.nx + x], i, ph);
}

template <typename E>
__global__ void k_import(Geo g, E* __restrict__ dst, int dst_pitch, int rows, const double* __restrict__ src,
                         int ncols) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= ncols || y >= rows) return;
  dst[y * dst_pitch + x] = static_cast<E>(src[y * ncols + x]);
}

}  // namespace kern

// ---------------------------------------------------------------- launchers
// Launch kernel k (smem bytes of dynamic shared memory) on stream s, as a programmatic dependent
// of the kernel before it when pdl is set.
template <typename... KArgs, typename... Args>
cudaError_t launch_dep(bool pdl, dim3 grd, dim3 blk, size_t smem, cudaStream_t s, void (*k)(KArgs...),
                       Args&&... args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grd;
  cfg.blockDim = blk;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, static_cast<Args&&>(args)...);
}

template <typename C, typename S, int PSI>
int step_impl(const Geo& g, const Phys& ph, const Dev& d, int cur, int tcur, int forcing, int energy, cudaStream_t s,
              const LaunchHook* hook, int* t_flipped, PsiChain* chain) {
  using namespace kern;
  const S* f = static_cast<const S*>(d.f[cur]);
  S* fn = static_cast<S*>(d.f[cur ^ 1]);
  const C* T = static_cast<const C*>(d.T[tcur]);
  C* Tn = static_cast<C*>(d.T[tcur ^ 1]);
  C* rho = static_cast<C*>(d.rho);
  C* ux = static_cast<C*>(d.ux);
  C* uy = static_cast<C*>(d.uy);
  C* psi = static_cast<C*>(d.psi);
  const C* side_in = static_cast<const C*>(d.side[cur]);
  C* side_out = static_cast<C*>(d.side[cur ^ 1]);
  int n = 0;
  auto pre = [&](int k) {
    if (hook) hook->before(hook->self, k);
  };
  auto post = [&](int k) {
    if (hook) hook->after(hook->self, k);
    ++n;
  };
  const dim3 blk(kCollTX, kCollTY), grd((g.nx + kCollTX - 1) / kCollTX, (g.ny + kCollTY - 1) / kCollTY);
  if (ph.d.G != 0.0 && !(chain && chain->have)) {
    pre(kKRhoPsi);
    k_rho_psi<C, S, PSI><<<grd, blk, 0, s>>>(g, ph, f, T, d.mask, side_in, psi, d.status);
    post(kKRhoPsi);
  }
  // tensor maps of this step's populations and psi for the TMA-staged tiles (plain loads
  // everywhere when a map cannot be made)
  using CS = CollStage<C, S, kCollTY>;
  CUtensorMap tm_f, tm_psi;
  const bool staged = d.tma && tma::encode<S>(&tm_f, f, g.nx, g.ny, g.pitch, g.plane, 9, CS::FW, CS::FH) &&
                      tma::encode<C>(&tm_psi, psi, g.nx, g.ny, g.pitch, g.plane, 1, CS::PW, CS::PH);
  pre(kKCollide);
  const int cflags = staged ? (kLaunchStaged | ((d.starve & kStarveCollide) ? kLaunchStarve : 0) |
                               ((d.pdl && d.f_ready) ? kLaunchEarlyF : 0))
                            : 0;
  if (d.collision == kCollBGK)
    launch_dep(d.pdl, grd, blk, 0, s, k_collide<C, S, kCollBGK>, g, ph, f, fn, psi, d.mask, side_in, side_out, rho, ux,
               uy, forcing, d.status, tm_f, tm_psi, cflags);
  else
    launch_dep(d.pdl, grd, blk, 0, s, k_collide<C, S, kCollCM>, g, ph, f, fn, psi, d.mask, side_in, side_out, rho, ux, uy,
               forcing, d.status, tm_f, tm_psi, cflags);
  post(kKCollide);
  *t_flipped = 0;
  if (energy && forcing) {
    const int do_hf = d.nb > 0;
    const bool fuse = chain && chain->want && ph.d.G != 0.0;
    pre(kKEnergy);
    using ET = EnergyTile<C>;
    const dim3 blk(ET::NT), grd((g.nx + ET::TX - 1) / ET::TX, (g.ny + ET::TY - 1) / ET::TY);
    constexpr int AX = ET::TX + 8, AY = ET::TY + 8;
    EnergyMaps em;
    const bool ruv = ux == rho + g.plane && uy == rho + 2 * (size_t)g.plane;  // consecutive planes
    const bool e_staged = d.tma && ruv && tma::encode<C>(&em.T, T, g.nx, g.ny, g.pitch, g.plane, 1, AX, AY) &&
                          tma::encode<C>(&em.ruv, rho, g.nx, g.ny, g.pitch, g.plane, 3, AX, AY);
    launch_dep(d.pdl, grd, blk, 0, s, k_energy<C, S, PSI>, g, ph, T, Tn, rho, ux, uy, d.mask, d.partial, d.counter,
               d.hf, d.nb, do_hf, d.wall_tiles[ET::TY == 16 ? 1 : 0], fuse ? static_cast<const S*>(fn) : nullptr,
               static_cast<const C*>(side_out), fuse ? static_cast<C*>(d.psi_next) : nullptr, d.status,
               static_cast<C*>(d.t1_out), em,
               e_staged ? (kLaunchStaged | ((d.starve & kStarveEnergy) ? kLaunchStarve : 0)) : 0);
    post(kKEnergy);
    *t_flipped = 1;
    if (chain) chain->made = fuse ? 1 : 0;
  } else if (chain) {
    chain->made = 0;
  }
  return cudaPeekAtLastError() == cudaSuccess ? n : -1;
}

template <typename C, typename S>
int export_impl(const Geo& g, const Phys& ph, const Dev& d, int cur, int tcur, int which, double* dst, cudaStream_t s) {
  using namespace kern;
  const dim3 blk(256);
  if (which >= 20 && which < 23) {
    const C* src = static_cast<const C*>(d.side[cur]) + (which - 20) * g.ny;
    k_export<C><<<dim3((g.ny + 255) / 256, 1), blk, 0, s>>>(g, src, g.ny, 1, dst, g.ny);
  } else if (which >= 10 && which < 19) {
    const S* src = static_cast<const S*>(d.f[cur]) + (which - 10) * g.plane;
    k_export_pop<C, S><<<dim3((g.nx + 255) / 256, g.ny), blk, 0, s>>>(g, ph, src, which - 10, dst);
  } else if (which == 5) {
    k_export_solid<<<dim3((g.nx + 255) / 256, g.ny), blk, 0, s>>>(g, d.mask, dst);
  } else if (which >= 30 && which < 34) {  // 30 + comp + 2 forcing: the force of the last collision
    k_export_force<C><<<dim3((g.nx + 255) / 256, g.ny), blk, 0, s>>>(
        g, ph, static_cast<const C*>(d.psi), static_cast<const C*>(d.rho), d.mask, (which - 30) >> 1, (which - 30) & 1,
        dst);
  } else {
    const void* p = which == 0 ? d.rho : which == 1 ? d.ux : which == 2 ? d.uy : which == 3 ? d.T[tcur] : d.psi;
    k_export<C><<<dim3((g.nx + 255) / 256, g.ny), blk, 0, s>>>(g, static_cast<const C*>(p), g.pitch, g.ny, dst, g.nx);
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

template <typename C, typename S>
int import_impl(const Geo& g, const Phys& ph, const Dev& d, int cur, int tcur, int which, const double* src,
                cudaStream_t s) {
  using namespace kern;
  const dim3 blk(256);
  if (which >= 20 && which < 23) {
    C* dst = static_cast<C*>(d.side[cur]) + (which - 20) * g.ny;
    k_import<C><<<dim3((g.ny + 255) / 256, 1), blk, 0, s>>>(g, dst, g.ny, 1, src, g.ny);
  } else if (which >= 10 && which < 19) {
    S* dst = static_cast<S*>(d.f[cur]) + (which - 10) * g.plane;
    k_import_pop<C, S><<<dim3((g.nx + 255) / 256, g.ny), blk, 0, s>>>(g, ph, dst, which - 10, src);
  } else if (which == 3) {
    k_import<C><<<dim3((g.nx + 255) / 256, g.ny), blk, 0, s>>>(g, static_cast<C*>(d.T[tcur]), g.pitch, g.ny, src,
                                                                 g.nx);
  } else {
    return -1;
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

template <typename C, typename S>
int init_impl(const Geo& g, const Phys& ph, const Dev& d, const double* rho0, const double* drho, const double* ux0,
              const double* uy0, const double* T0, const double* Tw, unsigned long long seed, double amp,
              cudaStream_t s) {
  using namespace kern;
  const dim3 blk(32, 8), grd((g.nx + 31) / 32, (g.ny + 7) / 8);
  k_init<C, S><<<grd, blk, 0, s>>>(g, ph, rho0, drho, ux0, uy0, T0, Tw, seed, amp, static_cast<S*>(d.f[0]),
                                   static_cast<C*>(d.T[0]), static_cast<C*>(d.rho), static_cast<C*>(d.ux),
                                   static_cast<C*>(d.uy), static_cast<C*>(d.side[0]), d.mask);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace lbm
