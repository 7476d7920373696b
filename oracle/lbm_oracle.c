/*
 * Plain FP64 CPU oracle for one time step of the central-moment (CM)
 * pseudopotential lattice Boltzmann boiling model of Saito, De Rosis, Fei, Luo,
 * Ebihara, Kaneko and Abe, "Lattice Boltzmann modeling and simulation of
 * forced-convection boiling on a cylinder" (arXiv:1912.02018).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct statement
 * of the method that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
 * no code, header, table or constant with the CUDA library.
 *
 * Everything is double precision, evaluated in the order written (build with
 * -ffp-contract=off so the compiler does not fuse multiply-adds).  The CM
 * collision is done with explicit 9x9 matrices: raw moments m = M f, central
 * moments k = N(u) m, post-collision k* by Eq. (posColl0) with the modified
 * forcing of Eq. (force2), m* from N(u) m* = k* by forward substitution (N is
 * unit lower triangular, App. A), and f* = M^{-1} m* with M^{-1} obtained once by
 * Gauss-Jordan elimination ("two-step reconstruction", Sec. II.A).
 *
 * Per step (order fixed; the paper gives none):
 *   1. pull-streaming, Eq. (streaming), with boundary substitutions: Zou-He
 *      velocity inlet at x=0, convective outlet at x=nx-1, linear interpolated
 *      bounce-back on the cylinder (Sec. IV.A); periodic in y;
 *   2. rho = sum f_i; psi(rho, T) from Eq. (potential) with the Peng-Robinson
 *      EOS, Eq. (eos);
 *   3. interaction force, Eq. (interForce), on the 24-neighbour stencil, plus
 *      gravity (rho - rho_l) g along -x;
 *   4. u from Sec. II.A (rho u = sum f c + F/2) and CM collision with the
 *      consistency terms, Eq. (postColl2);
 *   5. wall heat flux sample q(t) = mean over boundary nodes of -lambda dT/dn
 *      (Sec. IV.B) from the temperature entering this step;
 *   6. temperature, Eq. (energy): two-stage Runge-Kutta (Heun), third-order
 *      upwind convection, isotropic 24-neighbour gradient and Laplacian (Sec. II.C).
 * For n < warmup the force and steps 5-6 are skipped (Sec. IV.A).
 *
 * Also here: flat walls and a uniform body force (the Poiseuille and Stefan
 * set-ups of Sec. III.C and III.E) and, with collision = 1, the single-rate BGK
 * operator that Sec. III.B compares the CM collision with (K = omega I on the
 * same equilibrium and forcing central moments, no consistency terms).
 */
#define _USE_MATH_DEFINES
#include <math.h>
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 9

/* D2Q9 velocities, Eq. (velVec). */
static const int CX[Q] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
static const int CY[Q] = {0, 0, 0, 1, -1, 1, -1, -1, 1};

/* The 24-neighbour stencil of Eq. (interForce), as 12 +/- pairs e and -e. */
static const int EX[12] = {1, 2, -2, -1, 0, 1, 2, -2, -1, 0, 1, 2};
static const int EY[12] = {0, 0, 1, 1, 1, 1, 1, 2, 2, 2, 2, 2};

/* Weights w(|e|^2) listed in Sec. II.B. */
static double w_iso(int e2)
{
    switch (e2) {
    case 1: return 4.0 / 21.0;
    case 2: return 4.0 / 45.0;
    case 4: return 1.0 / 60.0;
    case 5: return 2.0 / 315.0;
    case 8: return 1.0 / 5040.0;
    default: return 0.0;
    }
}

typedef struct {
    int32_t nx, ny, periodic_x, energy;
    int64_t warmup;
    double xc, yc, D;           /* cylinder; D <= 0 means no cylinder */
    double a, b, R, kappa, Tc;  /* Peng-Robinson EOS, Eq. (eos) */
    double G, sigma;            /* interaction strength; consistency constant */
    double T_sat, T_wall;
    double rho_l, rho_v, rho_s; /* coexistence densities; virtual solid density */
    double nu_l, nu_v, alpha_l, alpha_v, c_v;
    double g, u_in, U_out;      /* gravity; inlet speed; convective-outlet speed */
    int32_t n_wall;             /* optional angular wall-superheat profile (knots, fractions of Tc) */
    int32_t walls;              /* flat solid walls: bit 0 the column x = 0 (at T_wall, instead of the
                                   inlet), bit 1 the rows y = 0 and y = ny - 1 */
    const double *wall_dT;
    double body_fx;             /* uniform body force along +x (0: none) */
    int32_t collision;          /* 0: CM collision (Sec. II.A); 1: single-rate BGK on the same equilibrium
                                   and forcing, the comparison operator of Sec. III.B */
    int32_t reserved;
    double wall_q;              /* link fraction of the links into a flat wall: the wall surface lies
                                   wall_q of a link from the last fluid node (<= 0: 1/2, halfway) */
} orc_params;

typedef struct {
    orc_params p;
    int64_t n;
    int N;
    uint8_t *solid;
    double *qlink;  /* [N*9]: link fraction where the pull source is solid, else -1 */
    double *fs;     /* post-collision populations, [9][N] */
    double *fp;     /* pulled populations of the current step, [9][N] */
    double *side;   /* [3][ny] last streamed values of f_2, f_6, f_8 at x = nx-1 */
    double *T, *T1, *L;
    double *rho, *ux, *uy, *psi, *lam;
    double *Tw;     /* wall temperature of each solid node */
    int nb;
    int *bnode;
    double *bnx, *bny;
    double q_now, q_sum, q_sumsq;
    int64_t q_count;
    double Minv[Q * Q];
} orc_t;

/* ---------- small helpers ---------- */

static int wrap(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

/* Field value at (x, y) for a stencil: periodic in y; in x periodic or
 * zero-gradient (the value of the nearest boundary column). */
static double at(const orc_t *o, const double *fld, int x, int y)
{
    const orc_params *p = &o->p;
    y = wrap(y, p->ny);
    if (p->periodic_x) x = wrap(x, p->nx);
    else if (x < 0) x = 0;
    else if (x >= p->nx) x = p->nx - 1;
    return fld[y * p->nx + x];
}

/* ---------- thermodynamics, Eq. (eos) and Eq. (potential) ---------- */

static double pr_phi(const orc_params *p, double T)
{
    double s = 1.0 + p->kappa * (1.0 - sqrt(T / p->Tc));
    return s * s;
}

double orc_p_eos(const orc_params *p, double rho, double T)
{
    double rep = rho * p->R * T / (1.0 - p->b * rho);
    double att = p->a * pr_phi(p, T) * rho * rho / (1.0 + 2.0 * p->b * rho - p->b * p->b * rho * rho);
    return rep - att;
}

/* (dp/dT) at constant rho: derivative of Eq. (eos); phi'(T) by the chain rule. */
double orc_dpdT(const orc_params *p, double rho, double T)
{
    double s = 1.0 + p->kappa * (1.0 - sqrt(T / p->Tc));
    double dphi = -p->kappa * s / sqrt(T * p->Tc);
    double rep = rho * p->R / (1.0 - p->b * rho);
    double att = p->a * dphi * rho * rho / (1.0 + 2.0 * p->b * rho - p->b * p->b * rho * rho);
    return rep - att;
}

/* psi = sqrt(2 (p_EOS - rho cs^2) / (G cs^2)), Eq. (potential). */
double orc_psi(const orc_params *p, double rho, double T)
{
    const double cs2 = 1.0 / 3.0;
    double rad = 2.0 * (orc_p_eos(p, rho, T) - rho * cs2) / (p->G * cs2);
    return sqrt(rad);
}

/* Phase fraction used to interpolate transport properties between phases. */
static double phase_frac(const orc_params *p, double rho)
{
    if (!(p->rho_l > p->rho_v)) return 1.0;
    double ph = (rho - p->rho_v) / (p->rho_l - p->rho_v);
    if (ph < 0.0) ph = 0.0;
    if (ph > 1.0) ph = 1.0;
    return ph;
}

double orc_nu(const orc_params *p, double rho)
{
    return p->nu_v + phase_frac(p, rho) * (p->nu_l - p->nu_v);
}

double orc_lambda(const orc_params *p, double rho)
{
    double alpha = p->alpha_v + phase_frac(p, rho) * (p->alpha_l - p->alpha_v);
    return rho * p->c_v * alpha;
}

/* ---------- equilibrium, Eq. (equi) ---------- */

void orc_feq(double rho, double ux, double uy, double feq[Q])
{
    static const double W[Q] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                                1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
    const double cs2 = 1.0 / 3.0;
    for (int i = 0; i < Q; ++i) {
        double cx = CX[i], cy = CY[i];
        double Hxx = cx * cx - cs2, Hyy = cy * cy - cs2, Hxy = cx * cy;
        double Hxxy = cx * cx * cy - cs2 * cy;
        double Hxyy = cx * cy * cy - cs2 * cx;
        double Hxxyy = cx * cx * cy * cy - cs2 * (cx * cx + cy * cy) + cs2 * cs2;
        double t1 = (cx * ux + cy * uy) / cs2;
        double t2 = (Hxx * ux * ux + 2.0 * Hxy * ux * uy + Hyy * uy * uy) / (2.0 * cs2 * cs2);
        double t3 = (Hxxy * ux * ux * uy + Hxyy * ux * uy * uy) / (2.0 * cs2 * cs2 * cs2);
        double t4 = Hxxyy * ux * ux * uy * uy / (4.0 * cs2 * cs2 * cs2 * cs2);
        feq[i] = W[i] * rho * (1.0 + t1 + t2 + t3 + t4);
    }
}

/* ---------- CM matrices, Eq. (matrix), Eq. (transD2Q9), Eq. (shiftD2Q9) ---------- */

/* Raw-moment matrix M: rows 1, cx, cy, cx^2+cy^2, cx^2-cy^2, cxcy, cx^2cy, cxcy^2, cx^2cy^2. */
void orc_matrix_M(double M[Q * Q])
{
    for (int i = 0; i < Q; ++i) {
        double cx = CX[i], cy = CY[i];
        M[0 * Q + i] = 1.0;
        M[1 * Q + i] = cx;
        M[2 * Q + i] = cy;
        M[3 * Q + i] = cx * cx + cy * cy;
        M[4 * Q + i] = cx * cx - cy * cy;
        M[5 * Q + i] = cx * cy;
        M[6 * Q + i] = cx * cx * cy;
        M[7 * Q + i] = cx * cy * cy;
        M[8 * Q + i] = cx * cx * cy * cy;
    }
}

/* Shift matrix N(u) exactly as printed in App. A (T = N M). */
void orc_matrix_N(double ux, double uy, double N[Q * Q])
{
    memset(N, 0, sizeof(double) * Q * Q);
    for (int j = 0; j < Q; ++j) N[j * Q + j] = 1.0;
    N[1 * Q + 0] = -ux;
    N[2 * Q + 0] = -uy;
    N[3 * Q + 0] = ux * ux + uy * uy; N[3 * Q + 1] = -2.0 * ux; N[3 * Q + 2] = -2.0 * uy;
    N[4 * Q + 0] = ux * ux - uy * uy; N[4 * Q + 1] = -2.0 * ux; N[4 * Q + 2] = 2.0 * uy;
    N[5 * Q + 0] = ux * uy; N[5 * Q + 1] = -uy; N[5 * Q + 2] = -ux;
    N[6 * Q + 0] = -ux * ux * uy; N[6 * Q + 1] = 2.0 * ux * uy; N[6 * Q + 2] = ux * ux;
    N[6 * Q + 3] = -uy / 2.0; N[6 * Q + 4] = -uy / 2.0; N[6 * Q + 5] = -2.0 * ux;
    N[7 * Q + 0] = -ux * uy * uy; N[7 * Q + 1] = uy * uy; N[7 * Q + 2] = 2.0 * ux * uy;
    N[7 * Q + 3] = -ux / 2.0; N[7 * Q + 4] = ux / 2.0; N[7 * Q + 5] = -2.0 * uy;
    N[8 * Q + 0] = ux * ux * uy * uy; N[8 * Q + 1] = -2.0 * ux * uy * uy; N[8 * Q + 2] = -2.0 * ux * ux * uy;
    N[8 * Q + 3] = (ux * ux + uy * uy) / 2.0; N[8 * Q + 4] = -(ux * ux - uy * uy) / 2.0;
    N[8 * Q + 5] = 4.0 * ux * uy; N[8 * Q + 6] = -2.0 * uy; N[8 * Q + 7] = -2.0 * ux;
}

/* Inverse of a 9x9 matrix by Gauss-Jordan elimination with partial pivoting. */
int orc_invert9(const double A[Q * Q], double Ainv[Q * Q])
{
    double a[Q][2 * Q];
    for (int r = 0; r < Q; ++r)
        for (int c = 0; c < 2 * Q; ++c)
            a[r][c] = c < Q ? A[r * Q + c] : (c - Q == r ? 1.0 : 0.0);
    for (int c = 0; c < Q; ++c) {
        int piv = c;
        for (int r = c + 1; r < Q; ++r)
            if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
        if (a[piv][c] == 0.0) return -1;
        if (piv != c)
            for (int k = 0; k < 2 * Q; ++k) { double t = a[c][k]; a[c][k] = a[piv][k]; a[piv][k] = t; }
        double d = a[c][c];
        for (int k = 0; k < 2 * Q; ++k) a[c][k] /= d;
        for (int r = 0; r < Q; ++r) {
            if (r == c || a[r][c] == 0.0) continue;
            double m = a[r][c];
            for (int k = 0; k < 2 * Q; ++k) a[r][k] -= m * a[c][k];
        }
    }
    for (int r = 0; r < Q; ++r)
        for (int c = 0; c < Q; ++c) Ainv[r * Q + c] = a[r][Q + c];
    return 0;
}

/*
 * CM collision of one node, Sec. II.A-B.
 *   f      : pulled (pre-collision) populations
 *   Fx, Fy : total body force F = F_m + F_g
 *   Fmx,Fmy: interaction force F_m alone (enters the consistency terms)
 *   psi    : pseudopotential at the node (used only when sigma != 0)
 *   omega  : relaxation rate of k_4, k_5
 *   bgk    : 0 for the CM collision, K = diag(1, 1, 1, 1, omega, omega, 1, 1, 1); 1 for the
 *            single-rate BGK operator of the Sec. III.B comparison, K = omega I on the same
 *            equilibrium and forcing central moments (in population space f* = f + omega (f^eq - f)
 *            + (1 - omega/2) F_i, as T(u) is linear); the consistency terms are CM-only
 * Outputs f* (post-collision), rho and u (rho u = sum f c + F/2).
 */
void orc_collide_node(const double f[Q], double Fx, double Fy, double Fmx, double Fmy, double psi,
                      double omega, double sigma, int bgk, const double Minv[Q * Q], double fstar[Q],
                      double *rho_out, double *ux_out, double *uy_out)
{
    double M[Q * Q], N[Q * Q];
    orc_matrix_M(M);
    double m[Q];
    for (int j = 0; j < Q; ++j) {
        double s = 0.0;
        for (int i = 0; i < Q; ++i) s += M[j * Q + i] * f[i];
        m[j] = s;
    }
    double rho = m[0];
    double ux = (m[1] + 0.5 * Fx) / rho;
    double uy = (m[2] + 0.5 * Fy) / rho;
    orc_matrix_N(ux, uy, N);
    double k[Q];
    for (int j = 0; j < Q; ++j) {
        double s = 0.0;
        for (int l = 0; l < Q; ++l) s += N[j * Q + l] * m[l];
        k[j] = s;
    }
    /* equilibrium CMs (Sec. II.A) and forcing CMs with the consistency terms, Eq. (force2) */
    double keq[Q] = {rho, 0.0, 0.0, 2.0 * rho / 3.0, 0.0, 0.0, 0.0, 0.0, rho / 9.0};
    double alpha = (sigma != 0.0 && !bgk) ? sigma / (psi * psi) : 0.0;
    double Fm2 = Fmx * Fmx + Fmy * Fmy;
    double Rp[Q] = {0.0, Fx, Fy, 4.0 * alpha * Fm2, 0.0, 0.0, Fy / 3.0, Fx / 3.0, 4.0 / 3.0 * alpha * Fm2};
    double K[Q] = {1.0, 1.0, 1.0, 1.0, omega, omega, 1.0, 1.0, 1.0};
    if (bgk)
        for (int j = 0; j < Q; ++j) K[j] = omega;
    double ks[Q];
    for (int j = 0; j < Q; ++j)
        ks[j] = (1.0 - K[j]) * k[j] + K[j] * keq[j] + (1.0 - K[j] / 2.0) * Rp[j];
    /* two-step reconstruction: N(u) m* = k* (unit lower triangular), f* = M^{-1} m* */
    double ms[Q];
    for (int j = 0; j < Q; ++j) {
        double s = ks[j];
        for (int l = 0; l < j; ++l) s -= N[j * Q + l] * ms[l];
        ms[j] = s;
    }
    for (int i = 0; i < Q; ++i) {
        double s = 0.0;
        for (int j = 0; j < Q; ++j) s += Minv[i * Q + j] * ms[j];
        fstar[i] = s;
    }
    *rho_out = rho;
    *ux_out = ux;
    *uy_out = uy;
}

/* ---------- isotropic finite differences (Sec. II.C, same stencil as Eq. interForce) ---------- */

/* Gradient: sum_k w_k phi(x+e_k) e_k, accumulated over +/- pairs. */
static void iso_grad(const orc_t *o, const double *fld, int x, int y, double *gx, double *gy)
{
    double sx = 0.0, sy = 0.0;
    for (int k = 0; k < 12; ++k) {
        double w = w_iso(EX[k] * EX[k] + EY[k] * EY[k]);
        double d = at(o, fld, x + EX[k], y + EY[k]) - at(o, fld, x - EX[k], y - EY[k]);
        sx += w * d * EX[k];
        sy += w * d * EY[k];
    }
    *gx = sx;
    *gy = sy;
}

/* Laplacian: 2 sum_k w_k (phi(x+e_k) - phi(x)), accumulated over +/- pairs. */
static double iso_lap(const orc_t *o, const double *fld, int x, int y)
{
    double c = at(o, fld, x, y), s = 0.0;
    for (int k = 0; k < 12; ++k) {
        double w = w_iso(EX[k] * EX[k] + EY[k] * EY[k]);
        double d = (at(o, fld, x + EX[k], y + EY[k]) + at(o, fld, x - EX[k], y - EY[k])) - 2.0 * c;
        s += w * d;
    }
    return 2.0 * s;
}

/* Third-order upwind first derivative along (dx, dy), biased against the sign of v:
 * v >= 0: (phi_{-2} - 6 phi_{-1} + 3 phi_0 + 2 phi_{+1}) / 6, mirrored for v < 0,
 * written as differences from phi_0. */
static double upwind3(const orc_t *o, const double *fld, int x, int y, int dx, int dy, double v)
{
    double c = at(o, fld, x, y);
    if (v >= 0.0) {
        double m2 = at(o, fld, x - 2 * dx, y - 2 * dy) - c;
        double m1 = at(o, fld, x - dx, y - dy) - c;
        double p1 = at(o, fld, x + dx, y + dy) - c;
        return (m2 - 6.0 * m1 + 2.0 * p1) / 6.0;
    } else {
        double m1 = at(o, fld, x - dx, y - dy) - c;
        double p1 = at(o, fld, x + dx, y + dy) - c;
        double p2 = at(o, fld, x + 2 * dx, y + 2 * dy) - c;
        return (-2.0 * m1 + 6.0 * p1 - p2) / 6.0;
    }
}

/* Right-hand side of Eq. (energy) at one node, with rho and u frozen:
 * -u.grad T + (lambda lap T + grad lambda . grad T)/(rho c_v) - T (dp/dT)_rho div u/(rho c_v). */
static double energy_rhs(const orc_t *o, const double *T, int x, int y)
{
    const orc_params *p = &o->p;
    int id = y * p->nx + x;
    double rho = o->rho[id], ux = o->ux[id], uy = o->uy[id], Tc = T[id];
    double conv = ux * upwind3(o, T, x, y, 1, 0, ux) + uy * upwind3(o, T, x, y, 0, 1, uy);
    double gx, gy, lx, ly, dxux, dyux, dxuy, dyuy;
    iso_grad(o, T, x, y, &gx, &gy);
    double lap = iso_lap(o, T, x, y);
    iso_grad(o, o->lam, x, y, &lx, &ly);
    iso_grad(o, o->ux, x, y, &dxux, &dyux);
    iso_grad(o, o->uy, x, y, &dxuy, &dyuy);
    double divu = dxux + dyuy;
    double diff = o->lam[id] * lap + (lx * gx + ly * gy);
    double work = Tc * orc_dpdT(p, rho, Tc) * divu;
    return -conv + diff / (rho * p->c_v) - work / (rho * p->c_v);
}

/* ---------- geometry ---------- */

static int is_cylinder_xy(const orc_params *p, int x, int y)
{
    if (!(p->D > 0.0)) return 0;
    double dx = x - p->xc, dy = y - p->yc, r = 0.5 * p->D;
    return dx * dx + dy * dy <= r * r;
}

/* Solid nodes: the cylinder, and the flat walls: the column x = 0 (the heated wall of the
 * Stefan problem, Sec. III.E, turned so that its normal is +x) and the rows y = 0, ny - 1
 * (the no-slip planes of the Poiseuille flow, Sec. III.C). */
static int is_solid_xy(const orc_params *p, int x, int y)
{
    return ((p->walls & 1) && x == 0) || ((p->walls & 2) && (y == 0 || y == p->ny - 1)) || is_cylinder_xy(p, x, y);
}

/* Fraction q of the link from fluid node (x, y) along (cx, cy) that lies in the fluid:
 * smallest root t in (0, 1] of |d + t c|^2 = r^2, d = node - centre. */
static double link_fraction(const orc_params *p, int x, int y, int cx, int cy)
{
    double dx = x - p->xc, dy = y - p->yc, r = 0.5 * p->D;
    double A = (double)(cx * cx + cy * cy);
    double B = dx * cx + dy * cy;
    double C = dx * dx + dy * dy - r * r;
    return (-B - sqrt(B * B - A * C)) / A;
}

/* ---------- public API ---------- */

orc_t *orc_create(const orc_params *p, const double *rho0, const double *ux0, const double *uy0,
                  const double *T0)
{
    orc_t *o = (orc_t *)calloc(1, sizeof(orc_t));
    o->p = *p;
    int nx = p->nx, ny = p->ny, N = nx * ny;
    o->N = N;
    o->solid = (uint8_t *)calloc(N, 1);
    o->qlink = (double *)malloc(sizeof(double) * N * Q);
    o->fs = (double *)malloc(sizeof(double) * N * Q);
    o->fp = (double *)malloc(sizeof(double) * N * Q);
    o->side = (double *)malloc(sizeof(double) * 3 * ny);
    double **fields[] = {&o->T, &o->T1, &o->L, &o->rho, &o->ux, &o->uy, &o->psi, &o->lam, &o->Tw};
    for (unsigned k = 0; k < sizeof(fields) / sizeof(fields[0]); ++k)
        *fields[k] = (double *)calloc(N, sizeof(double));
    double M[Q * Q];
    orc_matrix_M(M);
    orc_invert9(M, o->Minv);

    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) o->solid[y * nx + x] = (uint8_t)is_solid_xy(p, x, y);

    /* link fractions and boundary-node list */
    o->bnode = (int *)malloc(sizeof(int) * N);
    o->bnx = (double *)malloc(sizeof(double) * N);
    o->bny = (double *)malloc(sizeof(double) * N);
    o->nb = 0;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int id = y * nx + x, touches = 0, touches_cyl = 0;
            for (int i = 0; i < Q; ++i) o->qlink[id * Q + i] = -1.0;
            if (o->solid[id]) continue;
            for (int i = 1; i < Q; ++i) {
                int sx = x - CX[i], sy = wrap(y - CY[i], ny);
                if (p->periodic_x) sx = wrap(sx, nx);
                if (sx < 0 || sx >= nx) continue;
                if (o->solid[sy * nx + sx]) {
                    /* a flat wall's surface lies wall_q of a link from the fluid node (halfway by
                     * default); a wall parallel to the lattice cuts every link into it at the same
                     * fraction, diagonal links included */
                    int cyl = is_cylinder_xy(p, sx, sy);
                    double qw = p->wall_q > 0.0 ? p->wall_q : 0.5;
                    o->qlink[id * Q + i] = cyl ? link_fraction(p, x, y, -CX[i], -CY[i]) : qw;
                    touches = 1;
                    touches_cyl |= cyl;
                }
            }
            if (touches) {
                /* outward normal: from the cylinder centre, else that of the flat wall */
                double nxv = 1.0, nyv = 0.0;
                if ((p->walls & 2) && y == 1) { nxv = 0.0; nyv = 1.0; }
                if ((p->walls & 2) && y == ny - 2) { nxv = 0.0; nyv = -1.0; }
                if (touches_cyl) {
                    double dx = x - p->xc, dy = y - p->yc, r = sqrt(dx * dx + dy * dy);
                    nxv = dx / r;
                    nyv = dy / r;
                }
                o->bnode[o->nb] = id;
                o->bnx[o->nb] = nxv;
                o->bny[o->nb] = nyv;
                o->nb++;
            }
        }

    /* wall temperature: T_w = T_sat + superheat, plus an optional angular profile interpolated
     * periodically-linearly between n_wall equally spaced knots (angle from the +x axis) */
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int id = y * nx + x;
            if (!o->solid[id]) continue;
            double tw = p->T_wall;
            if (p->n_wall > 0 && p->wall_dT && is_cylinder_xy(p, x, y)) {
                double th = atan2(y - p->yc, x - p->xc);
                double s = th / (2.0 * M_PI);
                if (s < 0.0) s += 1.0;
                double pos = s * p->n_wall;
                double fl = floor(pos);
                int k0 = ((int)fl) % p->n_wall, k1 = (k0 + 1) % p->n_wall;
                double t = pos - fl;
                double d = (1.0 - t) * p->wall_dT[k0] + t * p->wall_dT[k1];
                tw = p->T_wall + d * p->Tc;
            }
            o->Tw[id] = tw;
        }

    /* initial state (Sec. IV.A): f* = f^eq(rho0, u0) in the fluid */
    for (int id = 0; id < N; ++id) {
        double feq[Q];
        double r = rho0 ? rho0[id] : p->rho_l;
        double u = ux0 ? ux0[id] : p->u_in, v = uy0 ? uy0[id] : 0.0;
        if (o->solid[id]) { r = p->rho_s; u = 0.0; v = 0.0; }
        orc_feq(r, u, v, feq);
        for (int i = 0; i < Q; ++i) o->fs[i * N + id] = feq[i];
        o->rho[id] = r;
        o->ux[id] = u;
        o->uy[id] = v;
        o->T[id] = o->solid[id] ? o->Tw[id] : (T0 ? T0[id] : p->T_sat);
    }
    if (!p->periodic_x)
        for (int y = 0; y < ny; ++y) {
            int id = y * nx + nx - 1;
            o->side[0 * ny + y] = o->fs[2 * N + id];
            o->side[1 * ny + y] = o->fs[6 * N + id];
            o->side[2 * ny + y] = o->fs[8 * N + id];
        }
    return o;
}

void orc_destroy(orc_t *o)
{
    if (!o) return;
    free(o->solid); free(o->qlink); free(o->fs); free(o->fp); free(o->side);
    free(o->T); free(o->T1); free(o->L); free(o->rho); free(o->ux); free(o->uy);
    free(o->psi); free(o->lam); free(o->Tw); free(o->bnode); free(o->bnx); free(o->bny);
    free(o);
}

/* Streaming (pull) with boundary substitutions, for every fluid node. */
static void pull_all(orc_t *o)
{
    const orc_params *p = &o->p;
    int nx = p->nx, ny = p->ny, N = o->N;
    static const int OPP[Q] = {0, 2, 1, 4, 3, 6, 5, 8, 7};
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int id = y * nx + x;
            if (o->solid[id]) continue;
            for (int i = 0; i < Q; ++i) {
                int sx = x - CX[i], sy = wrap(y - CY[i], ny);
                if (p->periodic_x) sx = wrap(sx, nx);
                double v;
                if (sx < 0 || sx >= nx) {
                    v = 0.0; /* filled below by the inlet / outlet conditions */
                } else if (o->solid[sy * nx + sx]) {
                    /* linear interpolated bounce-back (Bouzidi 2001); the wall lies along c_opp */
                    double q = o->qlink[id * Q + i];
                    int io = OPP[i];
                    if (q < 0.5) {
                        int nxp = x + CX[i], nyp = wrap(y + CY[i], ny);
                        if (p->periodic_x) nxp = wrap(nxp, nx);
                        int ok = nxp >= 0 && nxp < nx && !o->solid[nyp * nx + nxp];
                        if (ok)
                            v = 2.0 * q * o->fs[io * N + id] + (1.0 - 2.0 * q) * o->fs[io * N + nyp * nx + nxp];
                        else
                            v = o->fs[io * N + id];
                    } else {
                        v = o->fs[io * N + id] / (2.0 * q) + (2.0 * q - 1.0) / (2.0 * q) * o->fs[i * N + id];
                    }
                } else {
                    v = o->fs[i * N + sy * nx + sx];
                }
                o->fp[i * N + id] = v;
            }
        }
    if (p->periodic_x) return;
    /* Zou-He velocity inlet at x = 0: unknowns f1, f5, f7 for u = (u_in, 0). */
    for (int y = 0; y < ny; ++y) {
        int id = y * nx;
        if (o->solid[id]) continue;
        double f0 = o->fp[0 * N + id], f2 = o->fp[2 * N + id], f3 = o->fp[3 * N + id];
        double f4 = o->fp[4 * N + id], f6 = o->fp[6 * N + id], f8 = o->fp[8 * N + id];
        double u = p->u_in;
        double rho = (f0 + f3 + f4 + 2.0 * (f2 + f6 + f8)) / (1.0 - u);
        o->fp[1 * N + id] = f2 + 2.0 / 3.0 * rho * u;
        o->fp[5 * N + id] = f6 - 0.5 * (f3 - f4) + rho * u / 6.0;
        o->fp[7 * N + id] = f8 + 0.5 * (f3 - f4) + rho * u / 6.0;
    }
    /* Convective outlet at x = nx-1 (Lou 2013): f(t+1) = (f(t) + U f_{nx-2}(t+1)) / (1 + U)
     * for the unknowns f2, f6, f8; f(t) is the previous step's streamed value. */
    static const int OUTD[3] = {2, 6, 8};
    for (int y = 0; y < ny; ++y) {
        int id = y * nx + nx - 1, inner = y * nx + nx - 2;
        if (o->solid[id]) continue;
        for (int j = 0; j < 3; ++j) {
            int i = OUTD[j];
            double v = (o->side[j * ny + y] + p->U_out * o->fp[i * N + inner]) / (1.0 + p->U_out);
            o->fp[i * N + id] = v;
            o->side[j * ny + y] = v;
        }
    }
}

static void heat_flux_sample(orc_t *o)
{
    if (o->nb == 0) return; /* no cylinder surface, no sample (Sec. IV.B) */
    double s = 0.0;
    for (int b = 0; b < o->nb; ++b) {
        int id = o->bnode[b], x = id % o->p.nx, y = id / o->p.nx;
        double gx, gy;
        iso_grad(o, o->T, x, y, &gx, &gy);
        s += -o->lam[id] * (gx * o->bnx[b] + gy * o->bny[b]);
    }
    double q = s / o->nb;
    o->q_now = q;
    o->q_sum += q;
    o->q_sumsq += q * q;
    o->q_count++;
}

static int is_dirichlet_T(const orc_t *o, int x, int id)
{
    return o->solid[id] || (!o->p.periodic_x && x == 0);
}

void orc_step(orc_t *o, int64_t nsteps)
{
    orc_params *p = &o->p;
    int nx = p->nx, ny = p->ny, N = o->N;
    const double cs2 = 1.0 / 3.0;
    for (int64_t s = 0; s < nsteps; ++s) {
        int forcing = o->n >= p->warmup;
        pull_all(o);
        /* density and pseudopotential */
#pragma omp parallel for schedule(static)
        for (int id = 0; id < N; ++id) {
            double r = p->rho_s;
            if (!o->solid[id]) {
                r = 0.0;
                for (int i = 0; i < Q; ++i) r += o->fp[i * N + id];
            }
            o->rho[id] = r;
            o->psi[id] = p->G != 0.0 ? orc_psi(p, r, o->T[id]) : 0.0;
        }
        /* interaction force, gravity, collision */
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int id = y * nx + x;
                if (o->solid[id]) { o->ux[id] = 0.0; o->uy[id] = 0.0; continue; }
                double Fmx = 0.0, Fmy = 0.0, Fx = 0.0, Fy = 0.0;
                if (forcing && p->G != 0.0) {
                    double sx, sy;
                    iso_grad(o, o->psi, x, y, &sx, &sy);
                    Fmx = -p->G * cs2 * o->psi[id] * sx;
                    Fmy = -p->G * cs2 * o->psi[id] * sy;
                }
                if (forcing) {
                    Fx = Fmx - (o->rho[id] - p->rho_l) * p->g;
                    if (p->body_fx != 0.0) Fx = Fx + p->body_fx;
                    Fy = Fmy;
                }
                double f[Q], fst[Q], r, u, v;
                for (int i = 0; i < Q; ++i) f[i] = o->fp[i * N + id];
                double omega = 1.0 / (orc_nu(p, o->rho[id]) / cs2 + 0.5);
                double sig = (forcing && p->G != 0.0) ? p->sigma : 0.0;
                orc_collide_node(f, Fx, Fy, Fmx, Fmy, o->psi[id], omega, sig, p->collision, o->Minv, fst, &r, &u, &v);
                for (int i = 0; i < Q; ++i) o->fs[i * N + id] = fst[i];
                o->ux[id] = u;
                o->uy[id] = v;
            }
        if (p->energy && forcing) {
            for (int id = 0; id < N; ++id) o->lam[id] = orc_lambda(p, o->rho[id]);
            heat_flux_sample(o);
            /* Heun: T1 = T + L(T);  T^{n+1} = (T + T1 + L(T1)) / 2 */
#pragma omp parallel for schedule(static)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    int id = y * nx + x;
                    if (o->solid[id]) o->T1[id] = o->Tw[id];
                    else if (is_dirichlet_T(o, x, id)) o->T1[id] = p->T_sat;
                    else o->T1[id] = o->T[id] + energy_rhs(o, o->T, x, y);
                }
#pragma omp parallel for schedule(static)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    int id = y * nx + x;
                    o->L[id] = is_dirichlet_T(o, x, id) ? 0.0 : energy_rhs(o, o->T1, x, y);
                }
            for (int id = 0; id < N; ++id) {
                int x = id % nx;
                if (o->solid[id]) o->T[id] = o->Tw[id];
                else if (is_dirichlet_T(o, x, id)) o->T[id] = p->T_sat;
                else o->T[id] = (o->T[id] + o->T1[id] + o->L[id]) * 0.5;
            }
        }
        o->n++;
    }
}

/* Field access. which: 0 rho, 1 ux, 2 uy, 3 T, 4 psi, 5 solid mask */
void orc_get_field(const orc_t *o, int which, double *out)
{
    const double *src = NULL;
    switch (which) {
    case 0: src = o->rho; break;
    case 1: src = o->ux; break;
    case 2: src = o->uy; break;
    case 3: src = o->T; break;
    case 4: src = o->psi; break;
    case 5:
        for (int id = 0; id < o->N; ++id) out[id] = o->solid[id];
        return;
    default: return;
    }
    memcpy(out, src, sizeof(double) * o->N);
}

void orc_get_f(const orc_t *o, double *out) { memcpy(out, o->fs, sizeof(double) * Q * o->N); }
void orc_get_side(const orc_t *o, double *out) { memcpy(out, o->side, sizeof(double) * 3 * o->p.ny); }

void orc_set_state(orc_t *o, const double *f, const double *T, const double *side, int64_t n)
{
    if (f) memcpy(o->fs, f, sizeof(double) * Q * o->N);
    if (T) memcpy(o->T, T, sizeof(double) * o->N);
    if (side) memcpy(o->side, side, sizeof(double) * 3 * o->p.ny);
    o->n = n;
}

int64_t orc_steps(const orc_t *o) { return o->n; }
int orc_n_boundary(const orc_t *o) { return o->nb; }

void orc_boundary(const orc_t *o, int *node, double *nxv, double *nyv)
{
    memcpy(node, o->bnode, sizeof(int) * o->nb);
    memcpy(nxv, o->bnx, sizeof(double) * o->nb);
    memcpy(nyv, o->bny, sizeof(double) * o->nb);
}

void orc_link_fractions(const orc_t *o, double *out) { memcpy(out, o->qlink, sizeof(double) * Q * o->N); }

void orc_heat_flux(const orc_t *o, double *out4)
{
    out4[0] = o->q_now;
    out4[1] = o->q_sum;
    out4[2] = o->q_sumsq;
    out4[3] = (double)o->q_count;
}

/*
 * Energy right-hand side L(T) on given fields (for tests of Eq. energy alone).
 * rho, ux, uy, T are [ny][nx]; out receives L(T) at every node (0 at Dirichlet nodes).
 */
void orc_energy_rhs_fields(const orc_params *p, const double *rho, const double *ux, const double *uy,
                           const double *T, double *out)
{
    orc_t *o = orc_create(p, rho, ux, uy, T);
    memcpy(o->rho, rho, sizeof(double) * o->N);
    memcpy(o->ux, ux, sizeof(double) * o->N);
    memcpy(o->uy, uy, sizeof(double) * o->N);
    memcpy(o->T, T, sizeof(double) * o->N);
    for (int id = 0; id < o->N; ++id) o->lam[id] = orc_lambda(p, o->rho[id]);
    for (int id = 0; id < o->N; ++id) {
        int x = id % p->nx, y = id / p->nx;
        out[id] = is_dirichlet_T(o, x, id) ? 0.0 : energy_rhs(o, o->T, x, y);
    }
    orc_destroy(o);
}

/* Interaction force F_m at every node for a given psi field (tests of Eq. interForce). */
void orc_interaction_force(const orc_params *p, const double *psi, double *Fx, double *Fy)
{
    orc_t *o = orc_create(p, NULL, NULL, NULL, NULL);
    memcpy(o->psi, psi, sizeof(double) * o->N);
    const double cs2 = 1.0 / 3.0;
    for (int id = 0; id < o->N; ++id) {
        int x = id % p->nx, y = id / p->nx;
        double sx, sy;
        iso_grad(o, o->psi, x, y, &sx, &sy);
        Fx[id] = -p->G * cs2 * o->psi[id] * sx;
        Fy[id] = -p->G * cs2 * o->psi[id] * sy;
    }
    orc_destroy(o);
}
