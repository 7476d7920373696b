"""Pins of the oracle's full time step against closed forms, invariants and the paper's claims.

Saito et al. (arXiv:1912.02018): Sec. II (collision, force, energy equation), Sec. III.D
(static interfaces), Sec. IV.A (boundary conditions, warm-up) and App. A (pressure tensor).
"""
import numpy as np
import pytest
from scipy import integrate, optimize

import synthetic_inputs as si
from oracle import Oracle, stepper


def periodic_case(n, m=None, **kw):
    base = dict(nx=n, ny=m or n, D=0.0, xc=0.0, yc=0.0, periodic_x=1, g=0.0, u_in=0.0, noise_amp=0.0)
    base.update(kw)
    return si.Case(**base)


def zeros(c):
    return np.zeros((c.ny, c.nx))


# ---------------------------------------------------------------- invariants

def test_uniform_fluid_at_rest_stays_exactly_at_rest():
    c = periodic_case(24, G=-1.0, sigma=0.38, energy=1, nu_l=0.05)
    o = Oracle(c, ux=zeros(c), uy=zeros(c))
    _, d = stepper.derive(c)
    o.step(2)  # the reconstruction reaches its rounding fixed point within two steps
    first = o.fields()
    o.step(40)
    last = o.fields()
    assert np.all(last["ux"] == 0.0) and np.all(last["uy"] == 0.0)
    assert np.all(last["T"] == d.T_sat)
    for k in ("rho", "psi"):
        assert np.array_equal(first[k], last[k])
    assert np.abs(last["rho"] - d.rho_l).max() <= 8 * np.spacing(d.rho_l)


def test_mass_conserved_to_roundoff_with_periodic_boundaries():
    c = periodic_case(32, G=-1.0, sigma=0.38, energy=1, nu_l=0.1, g=2e-5, superheat_Tc=0.0)
    _, d = stepper.derive(c)
    rng = np.random.default_rng(7)
    rho0 = 0.5 * (d.rho_l + d.rho_v) + rng.uniform(-0.5, 0.5, (32, 32))
    o = Oracle(c, rho=rho0, ux=zeros(c), uy=zeros(c))
    m0 = rho0.sum()
    for _ in range(5):
        o.step(60)
        assert abs(o.field("rho").sum() - m0) / m0 < 1e-13
    assert np.ptp(o.field("rho")) > 1.0  # it did phase-separate


def test_uniform_flow_through_inlet_and_outlet_stays_uniform():
    c = si.Case(nx=64, ny=12, D=0.0, xc=0.0, yc=0.0, G=-1.0, sigma=0.38, energy=1, u_in=0.05,
                Re=100.0, nu_l=0.04, noise_amp=0.0)
    o = Oracle(c)
    _, d = stepper.derive(c)
    o.step(150)
    f = o.fields()
    assert np.abs(f["ux"] - 0.05).max() < 1e-13
    assert np.abs(f["uy"]).max() < 1e-14
    assert np.abs(f["rho"] - d.rho_l).max() < 1e-12
    assert np.abs(f["T"] - d.T_sat).max() < 1e-15


def test_zou_he_inlet_imposes_the_inlet_velocity():
    c = si.SMALL.replace(G=0.0, g=0.0, energy=0, noise_amp=1e-2)
    o = Oracle(c, drho=c.drho())
    o.step(3)
    f = o.fields()
    fluid = o.field("solid")[:, 0] == 0
    assert np.abs(f["ux"][fluid, 0] - c.u_in).max() < 1e-15
    assert np.abs(f["uy"][fluid, 0]).max() < 1e-15


def test_fluid_at_rest_around_cylinder_stays_at_rest():
    c = periodic_case(48, D=12.0, xc=24.3, yc=23.7, G=0.0, sigma=0.0, energy=0, nu_l=0.1)
    o = Oracle(c, rho=np.ones((48, 48)), ux=zeros(c), uy=zeros(c))
    o.step(100)
    f = o.fields()
    fluid = o.field("solid") == 0
    assert np.abs(f["ux"][fluid]).max() < 1e-15 and np.abs(f["uy"][fluid]).max() < 1e-15
    assert np.abs(f["rho"][fluid] - 1.0).max() < 1e-14


def test_link_fractions_put_the_wall_on_the_circle():
    c = si.SMALL.replace(xc=32.3, yc=31.8)
    o = Oracle(c)
    q = o.link_fractions()
    solid = o.field("solid").astype(bool)
    cx = np.array([0, 1, -1, 0, 0, 1, -1, 1, -1])
    cy = np.array([0, 0, 0, 1, -1, 1, -1, -1, 1])
    r = c.D / 2
    count = 0
    for y in range(c.ny):
        for x in range(c.nx):
            for i in range(1, 9):
                src_solid = solid[(y - cy[i]) % c.ny, x - cx[i]] if 0 <= x - cx[i] < c.nx else False
                if solid[y, x] or not src_solid:
                    assert q[y, x, i] == -1.0
                    continue
                count += 1
                assert 0.0 < q[y, x, i] <= 1.0
                px, py = x - q[y, x, i] * cx[i], y - q[y, x, i] * cy[i]
                assert abs(np.hypot(px - c.xc, py - c.yc) - r) < 1e-12
    assert count > 0


def test_heat_flux_of_a_linear_temperature_field():
    # grad T is exact on the isotropic stencil for a linear field, so q_b = -lambda (a n_x + b n_y)
    c = periodic_case(48, D=12.0, xc=24.3, yc=23.6, G=0.0, sigma=0.0, energy=1, nu_l=0.1)
    _, d = stepper.derive(c)
    o = Oracle(c, ux=zeros(c), uy=zeros(c))
    y, x = np.mgrid[0:48, 0:48].astype(float)
    a, b = 3e-4, -1.7e-4
    o.set_state(T=d.T_sat + a * (x - c.xc) + b * (y - c.yc), n=0)
    o.step(1)
    solid = o.field("solid").astype(bool)
    near = np.zeros_like(solid)
    for sx, sy in [(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1), (1, -1), (-1, 1)]:
        near |= np.roll(np.roll(solid, sy, 0), sx, 1)
    bnd = near & ~solid
    rx, ry = x[bnd] - c.xc, y[bnd] - c.yc
    rr = np.hypot(rx, ry)
    lam = d.rho_l * c.c_v * d.alpha_l
    expect = np.mean(-lam * (a * rx / rr + b * ry / rr))
    hf = o.heat_flux()
    assert hf["count"] == 1
    assert abs(hf["q_now"] - expect) < 1e-9 * abs(expect)
    assert len(o.boundary()[0]) == bnd.sum()


def test_warmup_skips_force_and_energy():
    c = si.SMALL.replace(warmup=4)
    o = Oracle(c, drho=c.drho())
    _, d = stepper.derive(c)
    o.step(4)
    solid = o.field("solid").astype(bool)
    assert np.all(o.field("T")[~solid] == d.T_sat)
    assert o.heat_flux()["count"] == 0
    o.step(3)
    assert o.heat_flux()["count"] == 3
    assert np.any(o.field("T")[~solid] != d.T_sat)


def test_sigma_enters_through_sigma_over_psi_squared():
    # F_m is unchanged by G -> 2G (psi^2 halves), so (G, sigma) and (2G, sigma/2) are the same model
    c1 = si.SMALL.replace(G=-1.0, sigma=0.38)
    c2 = si.SMALL.replace(G=-2.0, sigma=0.19)
    o1 = Oracle(c1, drho=c1.drho()).step(20)
    o2 = Oracle(c2, drho=c2.drho()).step(20)
    for k in ("rho", "ux", "uy", "T"):
        a, b = o1.field(k), o2.field(k)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_wall_profile_interpolates_knots_periodically_in_the_angle():
    # knots at angles 0, pi/2, pi, 3pi/2 measured from +x; solid nodes on the axes take a knot,
    # nodes on the diagonals the mean of the two neighbouring knots (the last pair wraps around)
    knots = (0.01, 0.03, -0.02, 0.04)
    c = si.SMALL.replace(wall_dT=knots)  # cylinder of radius 8 at (32, 32)
    o = Oracle(c, drho=c.drho()).step(3)
    _, d = stepper.derive(c)
    T = o.field("T")
    expect = {(35, 32): knots[0], (32, 35): knots[1], (29, 32): knots[2], (32, 29): knots[3],
              (34, 34): 0.5 * (knots[0] + knots[1]), (34, 30): 0.5 * (knots[3] + knots[0]),
              (30, 30): 0.5 * (knots[2] + knots[3])}
    for (x, y), k in expect.items():
        assert o.field("solid")[y, x] == 1
        assert abs(T[y, x] - (d.T_wall + k * d.Tc)) < 1e-14 * d.T_wall, (x, y)


def test_uniform_wall_profile_equals_a_larger_superheat():
    a = si.SMALL.replace(superheat_Tc=0.05, wall_dT=(0.02, 0.02, 0.02))
    b = si.SMALL.replace(superheat_Tc=0.07)
    oa = Oracle(a, drho=a.drho()).step(30)
    ob = Oracle(b, drho=b.drho()).step(30)
    for k in ("rho", "ux", "uy", "T"):
        x, y = oa.field(k), ob.field(k)
        assert np.abs(x - y).max() <= 1e-12 * np.abs(y).max(), k


# ---------------------------------------------------------------- closed forms

def test_taylor_green_decay_matches_closed_form():
    n, nu, u0 = 64, 0.02, 1e-3
    k = 2 * np.pi / n
    c = periodic_case(n, G=0.0, sigma=0.0, energy=0, nu_l=nu)
    y, x = np.mgrid[0:n, 0:n].astype(float)
    ux = u0 * np.sin(k * x) * np.cos(k * y)
    uy = -u0 * np.cos(k * x) * np.sin(k * y)
    o = Oracle(c, rho=np.ones((n, n)), ux=ux, uy=uy).step(1000)
    amp = (o.field("ux") * ux).sum() / (ux * ux).sum()
    assert abs(amp / np.exp(-2 * nu * k * k * 1000) - 1) < 5e-3


def test_heat_conduction_decay_matches_closed_form():
    n, t = 64, 300
    k = 2 * np.pi / n
    c = periodic_case(n, 6, G=0.0, sigma=0.0, energy=1, nu_l=0.1)
    _, d = stepper.derive(c)
    x = np.tile(np.arange(n, dtype=float), (6, 1))
    A = 1e-3
    o = Oracle(c, rho=np.full((6, n), d.rho_l), ux=np.zeros((6, n)), uy=np.zeros((6, n)),
               T=d.T_sat + A * np.sin(k * x)).step(t)
    amp = ((o.field("T") - d.T_sat) * np.sin(k * x)).sum() / (np.sin(k * x) ** 2).sum()
    assert abs(amp / (A * np.exp(-d.alpha_l * k * k * t)) - 1) < 5e-3


def test_heat_advection_by_uniform_flow_matches_closed_form():
    n, t, u = 64, 320, 0.05
    k = 2 * np.pi / n
    c = periodic_case(n, 6, G=0.0, sigma=0.0, energy=1, nu_l=0.01, u_in=u)
    _, d = stepper.derive(c)
    x = np.tile(np.arange(n, dtype=float), (6, 1))
    A = 1e-3
    o = Oracle(c, rho=np.full((6, n), d.rho_l), T=d.T_sat + A * np.sin(k * x)).step(t)
    expect = d.T_sat + A * np.exp(-d.alpha_l * k * k * t) * np.sin(k * (x - u * t))
    assert np.abs(o.field("T") - expect).max() < 0.02 * A
    # the opposite direction is wrong by a full amplitude: the upwinding sign matters
    wrong = d.T_sat + A * np.exp(-d.alpha_l * k * k * t) * np.sin(k * (x + u * t))
    assert np.abs(o.field("T") - wrong).max() > 0.5 * A


def test_pressure_work_term_matches_eos_derivative():
    n = 64
    k = 2 * np.pi / n
    c = periodic_case(n, 4, G=-1.0, energy=1, nu_l=0.1)
    _, d = stepper.derive(c)
    x = np.tile(np.arange(n, dtype=float), (4, 1))
    eps = 1e-3
    rho = np.full((4, n), 5.0)
    T = np.full((4, n), d.T_sat)
    L = stepper.energy_rhs(c, rho, eps * np.sin(k * x), np.zeros((4, n)), T)
    dpdT = d.eos.dp_dT(5.0, d.T_sat)
    expect = -d.T_sat * dpdT * eps * k * np.cos(k * x) / (5.0 * c.c_v)
    assert np.abs(L - expect).max() < 5e-3 * np.abs(expect).max()


def test_interaction_force_is_minus_gradient_of_eos_excess_pressure():
    # F_m = -G cs^2 psi grad psi = -grad(p_EOS - rho cs^2) in the continuum limit (Eq. interForce, Eq. potential)
    n = 128
    c = periodic_case(n, 4, G=-1.0)
    _, d = stepper.derive(c)
    x = np.tile(np.arange(n, dtype=float), (4, 1))
    rho = 4.0 + 0.5 * np.sin(2 * np.pi * x / n)
    psi = np.vectorize(lambda r: np.sqrt(2 * (d.eos.p(r, d.T_sat) - r / 3) / (-1 / 3)))(rho)
    fx, fy = stepper.interaction_force(c, psi)
    excess = np.vectorize(lambda r: d.eos.p(r, d.T_sat) - r / 3)(rho)[0]
    grad = (np.roll(excess, -1) - np.roll(excess, 1)) / 2
    assert np.abs(fx[0] + grad).max() < 2e-3 * np.abs(grad).max()
    assert np.abs(fy).max() < 1e-14


# ---------------------------------------------------------------- static interfaces (Sec. III.D, App. A)

def flat_interface(sigma, G=-1.0, nx=200, steps=8000):
    c = periodic_case(nx, 4, G=G, sigma=sigma, energy=0, nu_l=0.1)
    _, d = stepper.derive(c)
    x = np.arange(nx)
    prof = d.rho_v + (d.rho_l - d.rho_v) * 0.5 * (np.tanh((x - nx / 4) / 3) - np.tanh((x - 3 * nx / 4) / 3))
    rho = np.tile(prof, (4, 1))
    o = Oracle(c, rho=rho, ux=np.zeros_like(rho), uy=np.zeros_like(rho)).step(steps)
    r = o.field("rho")[0]
    return r[nx // 2], r[0], d


def mechanical_stability_coexistence(d, G, sigma):
    """Coexistence from the 1-D pressure tensor of App. A: P = p_EOS + g k psi psi'' + (sigma g^2 - g k/2) psi'^2,
    g = G cs^2, k = 2/7 (fourth moment of the 24-neighbour weights); it gives
    int (p0 - p_EOS) psi'/psi^(1+eps) drho = 0 with eps = 1 - 2 sigma g / k."""
    e, T = d.eos, d.T_sat
    g, kap = G / 3.0, 2.0 / 7.0
    eps = 1.0 - 2.0 * sigma * g / kap

    def psi(r):
        return np.sqrt(2 * (e.p(r, T) - r / 3) / g)

    def dpsi(r, h=1e-7):
        return (psi(r + h) - psi(r - h)) / (2 * h)

    ra, rb = e.spinodals(T)

    def branches(p0):
        return (optimize.brentq(lambda r: e.p(r, T) - p0, 1e-9, ra),
                optimize.brentq(lambda r: e.p(r, T) - p0, rb, 0.999 / e.b))

    def cond(p0):
        rv, rl = branches(p0)
        return integrate.quad(lambda r: (p0 - e.p(r, T)) * dpsi(r) / psi(r) ** (1 + eps), rv, rl, limit=400)[0]

    p0 = optimize.brentq(cond, max(e.p(rb, T), 1e-9) + 1e-12, e.p(ra, T) - 1e-12)
    return branches(p0)


@pytest.mark.slow
def test_flat_interface_consistency_term():
    rl38, rv38, d = flat_interface(0.38)
    rl0, rv0, _ = flat_interface(0.0)
    # Sec. III.D: sigma = 0.38 brings the coexistence densities towards Maxwell's rule
    assert abs(rv38 - d.rho_v) < abs(rv0 - d.rho_v)
    assert abs(rl38 - d.rho_l) < abs(rl0 - d.rho_l)
    assert abs(rl38 - d.rho_l) < 0.01 * d.rho_l
    # the shift caused by sigma agrees with the pressure tensor of App. A
    th38 = mechanical_stability_coexistence(d, -1.0, 0.38)[0]
    th0 = mechanical_stability_coexistence(d, -1.0, 0.0)[0]
    assert abs((rv38 - rv0) / (th38 - th0) - 1) < 0.2


@pytest.mark.slow
def test_flat_interface_near_maxwell_with_the_default_interaction_strength():
    # Sec. III.D: with sigma = 0.38 the coexistence densities lie close to Maxwell's rule.  F_m does not
    # depend on G, but the consistency term does (alpha = sigma / psi^2, psi^2 ~ 1/G); the workloads' G
    # (synthetic_inputs.Case) is the value at which this statement holds (G = -1 leaves rho_v 28% low)
    G = si.Case(nx=1, ny=1, D=0.0, xc=0.0, yc=0.0).G
    rl, rv, d = flat_interface(0.38, G=G)
    assert abs(rl / d.rho_l - 1) < 0.01
    assert abs(rv / d.rho_v - 1) < 0.05


@pytest.mark.slow
def test_laplace_law_pressure_jump_is_linear_in_inverse_radius():
    # Sec. III.D: static vapour bubbles of several radii in a periodic box; the pressure jump between
    # the bulk inside and outside, p_EOS(rho_in) - p_EOS(rho_out), is proportional to 1/R.  Four radii
    # (equimolar radius of the settled bubble); acceptance: a straight-line fit of dp against 1/R with
    # R^2 >= 0.99 and an intercept within 5% of the largest dp.  Measured at the default G = -2:
    # R^2 = 0.9998, intercept -3.8% (bubbles from R = 14 add a Tolman-like 1/R^2 part: -5.4%).
    n, steps = 128, 16000

    def bubble(R):
        c = periodic_case(n, sigma=0.38, energy=0, nu_l=1.0 / 6.0)
        _, d = stepper.derive(c)
        y, x = np.mgrid[0:n, 0:n]
        r = np.hypot(x - n / 2 + 0.5, y - n / 2 + 0.5)
        rho = d.rho_l + (d.rho_v - d.rho_l) * 0.5 * (1 - np.tanh((r - R) / 2))
        o = Oracle(c, rho=rho, ux=np.zeros_like(rho), uy=np.zeros_like(rho)).step(steps)
        f = o.field("rho")
        rin, rout = f[n // 2, n // 2], f[0, 0]
        Reff = np.sqrt(((rout - f) / (rout - rin)).sum() / np.pi)
        return d.eos.p(rin, d.T_sat) - d.eos.p(rout, d.T_sat), Reff

    res = np.array([bubble(R) for R in (20, 28, 36, 44)])
    dp, Reff = res[:, 0], res[:, 1]
    assert np.all(np.diff(dp) < 0) and np.all(dp > 0)
    A = np.vstack([1.0 / Reff, np.ones_like(Reff)]).T
    (slope, icpt), *_ = np.linalg.lstsq(A, dp, rcond=None)
    pred = A @ np.array([slope, icpt])
    r2 = 1.0 - ((dp - pred) ** 2).sum() / ((dp - dp.mean()) ** 2).sum()
    assert r2 >= 0.99, (dp, Reff, r2)
    assert abs(icpt) <= 0.05 * dp.max(), (dp, Reff, icpt)
