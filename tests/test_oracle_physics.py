"""Physics pins of the FP64 oracle: invariants, closed forms and textbook
reductions of the method (see the docstring of each test for the passage it
follows).  Sizes are chosen so each test runs in seconds on a few CPU cores.
"""
import math

import numpy as np
import pytest

from oracle import closed_forms as CF
from oracle import oracle as O
from paper_2311_05097_gb300 import analysis as A
from paper_2311_05097_gb300 import workloads as W


def make(case, **over):
    prm = dict(case["params"])
    prm.update(over)
    s = O.OracleSim(case["shape"], O.make_params(**prm))
    s.init(case["phi0"], case["phi"], case.get("u"))
    return s


def rel_mass_drift(m1, m0, phi_init):
    """|sum phi(t) - sum phi(0)| / sum |phi(0)| (normalisation that stays
    meaningful when sum phi is near zero)."""
    return abs(m1 - m0) / np.abs(phi_init).sum()


# ---- invariants ---------------------------------------------------------------------

@pytest.mark.parametrize("solid", [False, True])
def test_mass_conserved_2d(solid):
    """sum phi is conserved: the equilibrium and the source of Eq. (30) have the
    exact zeroth moments phi and 0, and streaming only moves populations."""
    c = W.small_case((40, 52), seed=3, solid=solid, theta_deg=60.0, u_amp=0.01)
    s = make(c)
    m0 = s.diagnostics()["mass"]
    s.step(300)
    assert rel_mass_drift(s.diagnostics()["mass"], m0, c["phi"]) < 1e-13


def test_mass_conserved_3d():
    c = W.small_case((12, 14, 18), seed=4, solid=True, theta_deg=120.0, u_amp=0.01)
    s = make(c)
    m0 = s.diagnostics()["mass"]
    s.step(40)
    assert rel_mass_drift(s.diagnostics()["mass"], m0, c["phi"]) < 1e-13


def test_mass_conserved_with_moving_particle():
    c = W.small_case((48, 40), seed=5, solid=False)
    s = O.OracleSim(c["shape"], O.make_params(**c["params"]))
    s.set_particle(0, O.Particle(x=(15.0, 20.0), u=(0.01, -0.005), w=(0, 0, 0.001), R=6.0,
                                 rho_p=2.0))
    # phi vanishes inside solids initially (the pattern of Eq. 39)
    phi = (1.0 - W.disc(c["shape"], (15.0, 20.0), 6.0, 4.0)) * c["phi"]
    s.init(c["phi0"], phi)
    m0 = s.diagnostics()["mass"]
    s.step(100)
    assert rel_mass_drift(s.diagnostics()["mass"], m0, phi) < 1e-13


def energy_series(s, n_samples, every):
    E, EK = [], []
    for _ in range(n_samples):
        d = s.diagnostics()
        E.append(d["E_total"])
        EK.append(d["E_K"])
        s.step(every)
    d = s.diagnostics()
    E.append(d["E_total"])
    EK.append(d["E_K"])
    return np.array(E), np.array(EK)


@pytest.mark.parametrize("case", ["drop", "wall"])
def test_total_energy_decays(case):
    """Theorem 1 (Sec. 2.3): with stationary geometry and no body force the total
    energy E_F + E_K does not increase.  The lattice scheme is weakly
    compressible, so energy also sits in pressure waves that E_total does not
    count; sampled every 50 steps E_total must fall overall, each rise must stay
    below the kinetic-energy scale, and rises may add up to at most 2 % of the
    total decrease."""
    if case == "drop":
        c = W.static_drop(n=64, R=16.0)
    else:
        c = W.flat_wall_drop(64, 60.0, 10.0, r0=16, mu1=0.1, mu2=0.01, sigma=0.01, M=0.02)
    s = make(c)
    E, EK = energy_series(s, 30, 50)
    dE = np.diff(E)
    drop = E[0] - E[-1]
    assert drop > 0
    assert dE.max() <= EK.max()
    assert dE[dE > 0].sum() <= 0.02 * drop


# ---- closed forms -------------------------------------------------------------------

def test_flat_interface_keeps_tanh_profile():
    """phi = tanh(2 x/D) is the equilibrium of Eq. (1) (mu of Eq. (9) vanishes in
    the continuum): a flat interface stays put, the profile changing only by the
    O(1/D^2) discretisation error."""
    ny, nx = 64, 4
    y = np.arange(ny, dtype=float)[:, None] * np.ones((1, nx))
    D = 4.0
    phi = np.tanh(2.0 * (16.0 - np.abs(y - 31.5)) / D)
    case = dict(shape=(ny, nx), phi0=np.zeros((ny, nx)), phi=phi,
                params=W.params(sigma=0.01, D=D, M=0.02, rho1=1.0, rho2=0.1, mu1=0.1, mu2=0.01))
    s = make(case)
    s.step(500)
    m = s.macros()
    assert np.abs(m["phi"] - phi).max() < 2e-2
    assert np.abs(m["u"]).max() < 2e-5
    # the interface does not move: phi = 0 crossings stay within 0.01 cells
    col = m["phi"][:, 1]
    j = np.nonzero(col[:-1] * col[1:] < 0)[0]
    xs = j + col[j] / (col[j] - col[j + 1])
    np.testing.assert_allclose(xs, [15.5, 47.5], atol=1e-2)


def test_laplace_law_2d():
    """Pressure jump of a static drop: P_in - P_out = sigma/R in 2D (potential
    form of the surface force in Eq. 16b with sigma from Eq. 1); averaged over
    the capillary oscillation after 600 steps."""
    R = 16.0
    c = W.static_drop(n=64, R=R)
    s = make(c)
    s.step(600)
    dps = []
    for _ in range(24):
        s.step(100)
        dps.append(A.laplace_jump(s.macros()["P"], (31.5, 31.5), R, 4.0))
    dp = float(np.mean(dps))
    assert abs(dp / (0.01 / R) - 1.0) < 0.08


@pytest.mark.parametrize("d0", [1.0 / 3.0, 0.4])
def test_taylor_green_decay(d0):
    """Single-phase reduction (sigma = 0, rho1 = rho2, phi0 = 0): the velocity of
    a Taylor-Green vortex decays at 2 nu k^2 with nu from Eq. (35)."""
    n, mu = 32, 0.05
    k = 2 * math.pi / n
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    U = 1e-3
    u = np.stack([U * np.sin(k * x) * np.cos(k * y), -U * np.cos(k * x) * np.sin(k * y)])
    P = -0.25 * U * U * (np.cos(2 * k * x) + np.cos(2 * k * y))
    s = O.OracleSim((n, n), O.make_params(sigma=0.0, rho1=1.0, rho2=1.0, mu1=mu, mu2=mu, d0=d0))
    s.init(np.zeros((n, n)), np.ones((n, n)), u, P)
    s.step(20)
    a0 = np.abs(s.macros()["u"][0]).max()
    s.step(400)
    a1 = np.abs(s.macros()["u"][0]).max()
    rate = -math.log(a1 / a0) / 400
    assert abs(rate / CF.taylor_green_rate(mu, k) - 1) < 0.01


def poiseuille(D, wall=8, width=32, mu=0.5, Fb=1e-6, steps=12000):
    ny, nx = width + 2 * wall, 4
    phi0 = W.slab_walls((ny, nx), wall, D, axis=1)
    case = dict(shape=(ny, nx), phi0=phi0, phi=1.0 - phi0,
                params=W.params(sigma=0.0, D=D, rho1=1.0, rho2=1.0, mu1=mu, mu2=mu,
                                Fb=(Fb, 0.0, 0.0)))
    s = make(case)
    s.step(steps)
    u = s.macros()["u"][0][:, 1]
    return u, phi0[:, 1]


def test_poiseuille_in_indicator_channel():
    """Channel between smooth-indicator walls driven by F_b (Eq. 16b with the
    viscosity mu/(1 - phi0)): in the fluid core the profile is the parabola
    u'' = -F_b/mu; the no-slip line sits inside the diffuse wall layer and moves
    to the phi0 = 1/2 level as D shrinks."""
    mu, Fb = 0.5, 1e-6
    errs = []
    for D in (4.0, 2.0):
        u, p0 = poiseuille(D, mu=mu, Fb=Fb)
        core = p0 < 1e-4
        y = np.arange(len(u), dtype=float)
        coef = np.polyfit(y[core], u[core], 2)
        assert abs(2 * coef[0] / (-Fb / mu) - 1) < 0.01
        # parabola through the phi0 = 1/2 levels (walls at 7.5 and 7.5 + 32)
        h = 16.0
        ua = Fb / (2 * mu) * (h * h - (y - 23.5) ** 2)
        errs.append(np.linalg.norm((u - ua)[core]) / np.linalg.norm(ua[core]))
    assert errs[1] < 0.75 * errs[0]


def test_particle_force_and_torque_closed_form():
    """Eq. (27) with f = phi0 (u_s - u*)/dt: a particle translating at u_p and
    spinning at w in a fluid at rest (phi = 0, theta = 90 deg, so no capillary
    force) feels F_f = -rho u_p int phi0 dA and T_f = -rho w int phi0 r^2 dA,
    rho = (rho1 + rho2)/2 by Eq. (17) at phi = 0."""
    n = 64
    prm = O.make_params(sigma=0.01, rho1=1.0, rho2=0.5, theta_deg=90.0)
    s = O.OracleSim((n, n), prm)
    R, D = 9.0, 4.0
    up, w = np.array([0.02, -0.01]), 0.003
    s.set_particle(0, O.Particle(x=(30.3, 33.7), u=tuple(up), w=(0, 0, w), R=R, rho_p=2.0))
    s.init(np.zeros((n, n)), np.zeros((n, n)))
    F, T = s.particle_force(0)
    area, mom2 = CF.tanh_indicator_moments(R, D, dim=2)
    rho = 0.75
    np.testing.assert_allclose(F[:2], -rho * up * area, rtol=1e-7)
    np.testing.assert_allclose(T[2], -rho * w * mom2, rtol=1e-7)


def test_particle_update_constant_force():
    """Eqs. (26a), (28) by first-order explicit Euler with F_in from the last
    velocity change: for constant F_f the velocity obeys
    u^{n+1} - u^n = A + beta (u^n - u^{n-1}) with beta = rho/rho_p and
    A = F_f/M_p + (1 - rho/rho_p) g, whose closed form is checked; the position
    follows dx/dt = u_p (Eq. 26c)."""
    prm = O.make_params(rho1=1.0, rho2=0.2, g=(0.0, -1e-5, 0.0))
    part = O.Particle(x=(10.0, 20.0), u=(0.001, 0.0), R=5.0, rho_p=3.0)
    Ff = np.array([2e-3, 1e-3, 0.0])
    Tf = np.array([0.0, 0.0, 5e-3])
    Vp = math.pi * 25.0
    Mp = 3.0 * Vp
    Ip = 0.5 * Mp * 25.0
    rho = 0.6
    beta = rho / 3.0
    A_ = Ff[:2] / Mp + (1 - rho / 3.0) * np.array([0.0, -1e-5])
    x0, u0 = np.array(part.x[:2]), np.array(part.u[:2])
    nsteps = 25
    for _ in range(nsteps):
        part = O.particle_update(2, prm, part, Ff, Tf)
    for a in range(2):
        assert abs(part.u[a] - CF.constant_force_velocity(u0[a], A_[a], beta, nsteps)) < 1e-15
        assert abs(part.x[a] - CF.constant_force_position(x0[a], u0[a], A_[a], beta, nsteps)) < 1e-12
    alpha = Tf[2] / Ip
    assert abs(part.w[2] - CF.constant_force_velocity(0.0, alpha, beta, nsteps)) < 1e-15


def test_hmax_solver_geometry():
    """The equal-area H_max of Eqs. (40)-(41): at the solution the drop circle
    (radius r, centre k above the cylinder centre) minus the cylinder covers the
    initial area A0 (checked by counting points on a fine grid), and at
    theta = 90 deg k^2 = r^2 + Rp^2."""
    Rp, R0 = 50.0, 50.0
    A0 = CF.initial_drop_area(R0, Rp)
    for th in (30.0, 60.0, 90.0, 120.0):
        H, r, k = CF.hmax_on_cylinder(th, Rp, A0)
        h = 0.05
        xs = np.arange(-r - 1, r + 1, h)
        ys = np.arange(k - r - 1, k + r + 1, h)
        X, Y = np.meshgrid(xs, ys)
        inside = ((X ** 2 + (Y - k) ** 2) < r * r) & ((X ** 2 + Y ** 2) >= Rp * Rp)
        assert abs(inside.sum() * h * h / A0 - 1) < 2e-3
        assert abs(H - (r + k)) < 1e-12
        if th == 90.0:
            assert abs(k * k - (r * r + Rp * Rp)) < 1e-9
    # a more wetting drop is flatter
    hs = [CF.hmax_on_cylinder(t, Rp, A0)[0] for t in (30.0, 60.0, 90.0, 120.0)]
    assert all(a < b for a, b in zip(hs, hs[1:]))


def test_particle_interface_height_limits():
    """Sec. 4.4 closed form: a neutrally buoyant particle (Bo -> 0) sits at
    h = R_p cos(theta) (its contact line at the flat interface), and the
    problem is antisymmetric under swapping the phases and the sign of gravity:
    h(theta, -Bo) = -h(180 - theta, Bo)."""
    L, Rp = 256, 32.0
    for th in (45.0, 60.0, 90.0, 120.0):
        h, a = CF.particle_interface_height(L, Rp, th, 1e-9)
        assert abs(h - Rp * math.cos(math.radians(th))) < 1e-5 and abs(a) < 1e-6
        for Bo in (0.1, 0.3, 0.5):
            hp, ap = CF.particle_interface_height(L, Rp, th, Bo)
            hm, am = CF.particle_interface_height(L, Rp, 180.0 - th, -Bo)
            assert abs(hp + hm) < 1e-9 and abs(ap + am) < 1e-12
    # heavier particles sit lower; more wetting (smaller theta) pulls them into phase 1
    hs = [CF.particle_interface_height(L, Rp, 90.0, Bo)[0] for Bo in (0.1, 0.2, 0.4)]
    assert hs[0] < hs[1] < hs[2]
    hs = [CF.particle_interface_height(L, Rp, th, 0.2)[0] for th in (120.0, 90.0, 60.0)]
    assert hs[0] < hs[1] < hs[2]


def test_repulsion_invariants():
    """Particle-particle repulsion (Sec. 4.5, reading R19): Newton's third law
    (forces sum to zero), central and repulsive, zero beyond R_k + R_j + xi and
    continuous there, periodic minimum image, off when eps = 0."""
    rng = np.random.default_rng(3)
    n = (64, 48)
    p = O.make_params(rep_xi=3.0, rep_eps=0.5)
    parts = [O.Particle((rng.uniform(0, n[0]), rng.uniform(0, n[1])), R=rng.uniform(3, 6)) for _ in range(12)]
    F = O.repulsion(2, p, n, parts)
    assert np.abs(F.sum(axis=0)).max() < 1e-12 * max(np.abs(F).max(), 1.0)
    # a pair: radial, repulsive, range, continuity at the edge of the range
    for dist, expect in ((8.0, True), (10.5, True), (13.0 - 1e-7, True), (13.0 + 1e-9, False), (20.0, False)):
        a, b = O.Particle((20.0, 20.0), R=5.0), O.Particle((20.0 + dist * 0.6, 20.0 + dist * 0.8), R=5.0)
        Fa, Fb = O.repulsion(2, p, n, [a, b])
        assert np.allclose(Fa, -Fb, rtol=0, atol=1e-15)
        dx = np.array(a.x) - np.array(b.x)
        if expect:
            assert Fa @ dx > 0 and abs(Fa[0] * dx[1] - Fa[1] * dx[0]) < 1e-12 * np.abs(Fa).max() * dist
        else:
            assert np.abs(Fa).max() == 0.0
        if dist > 13.0 - 1e-3 and expect:
            assert np.abs(Fa).max() < 1e-12
    # across the periodic edge in x
    a, b = O.Particle((1.0, 10.0), R=4.0), O.Particle((n[0] - 6.0, 10.0), R=4.0)
    Fa, Fb = O.repulsion(2, p, n, [a, b])
    assert Fa[0] > 0 and Fb[0] < 0
    assert np.abs(O.repulsion(2, O.make_params(rep_xi=3.0, rep_eps=0.0), n, [a, b])).max() == 0.0


@pytest.mark.parametrize("shape,xp,rp", [((40, 48), (34.0, 12.0), 6.0), ((16, 18, 20), (14.5, 12.0, 11.0), 4.0)])
def test_own_contact_angle_superposes_eq9(shape, xp, rp):
    """A particle with its own contact angle (reading R18), in 2D and 3D: the
    oracle's mu_phi equals Eq. 9 with the total phi0 and no wetting, plus the
    wetting part of Eq. 9 of each solid with its own angle (the fixed disc or
    sphere at the simulation's 60 deg, the particle at 130 deg) -- the
    superposition the reading defines, evaluated with the pinned pointwise
    Eq. 9."""
    c = W.small_case(shape, seed=2, solid=True, theta_deg=60.0)
    prm = dict(c["params"])
    part = O.Particle(xp, R=rp, rho_p=2.0, theta_deg=130.0)
    phi = (1.0 - W.disc(c["shape"], part.x, part.R, prm["D"])) * c["phi"]
    o = O.OracleSim(c["shape"], O.make_params(**prm))
    o.set_particle(0, part)
    o.init(c["phi0"], phi)
    m = o.macros()
    ph, mu = m["phi"], m["mu"]
    p0_tot = o.phi0()
    p0_fix = c["phi0"]
    p0_par = p0_tot - p0_fix
    lphi = O.lap(ph)
    P = {th: O.make_params(**dict(prm, theta_deg=th)) for th in (90.0, 60.0, 130.0)}

    def eq9(params, p0, i):
        return O.mu_phi(params, ph.flat[i], p0.flat[i], lphi.flat[i], O_lap[id(p0)].flat[i])

    O_lap = {id(p0_tot): O.lap(p0_tot), id(p0_fix): O.lap(p0_fix), id(p0_par): O.lap(p0_par)}
    err = 0.0
    for i in range(ph.size):
        expect = eq9(P[90.0], p0_tot, i)
        expect += eq9(P[60.0], p0_fix, i) - eq9(P[90.0], p0_fix, i)
        expect += eq9(P[130.0], p0_par, i) - eq9(P[90.0], p0_par, i)
        err = max(err, abs(mu.flat[i] - expect))
    assert err < 1e-14, err
    # the same particle without its own angle reproduces the single-angle path
    o2 = O.OracleSim(c["shape"], O.make_params(**prm))
    o2.set_particle(0, O.Particle(xp, R=rp, rho_p=2.0))
    o2.init(c["phi0"], phi)
    mu2 = o2.macros()["mu"]
    ref = np.array([eq9(P[60.0], p0_tot, i) for i in range(ph.size)]).reshape(ph.shape)
    assert np.abs(mu2 - ref).max() < 1e-14


def test_walls_poiseuille_converges_second_order():
    """Box walls (reading R21, halfway bounce-back): a body-force-driven channel
    of ny rows between walls at y = -1/2 and ny - 1/2 approaches
    u(y) = F_b (y + 1/2)(ny - 1/2 - y) / (2 mu) with a second-order error."""
    errs = []
    for ny, steps in ((16, 20000), (32, 60000)):
        nx = 4
        prm = O.make_params(sigma=0.0, mu1=0.1, mu2=0.1, Fb=(1e-6, 0, 0))
        s = O.OracleSim((ny, nx), prm)
        s.set_walls(True)
        s.init(np.zeros((ny, nx)), np.zeros((ny, nx)))
        s.step(steps)
        u = s.macros()["u"][0][:, 0]
        y = np.arange(ny)
        ua = 1e-6 / (2 * 0.1) * (y + 0.5) * (ny - 0.5 - y)
        errs.append(np.abs(u - ua).max() / ua.max())
    assert errs[1] < 1e-3 and errs[0] / errs[1] > 3.5, errs


def test_walls_conserve_mass():
    """Bounce-back returns every population that would leave: sum phi is kept
    to round-off with walls (a drop next to them, random initial flow)."""
    c = W.small_case((40, 36), seed=3, solid=False, u_amp=0.01)
    s = O.OracleSim(c["shape"], O.make_params(**c["params"]))
    s.set_walls(True)
    s.init(c["phi0"], c["phi"], c["u"])
    m0 = s.diagnostics()["mass"]
    s.step(400)
    assert abs(s.diagnostics()["mass"] - m0) <= 1e-13 * np.abs(c["phi"]).sum()


def test_walls_give_a_right_contact_angle():
    """The mirrored stencil rows at a box wall (reading R21) mean zero normal
    gradient of phi there, i.e. a 90 degree contact angle: a half-ellipse of
    phase 1 resting on the bottom wall relaxes to a half-circle centred on the
    wall line y = -1/2 (a periodic image or a wrong mirror would pull the
    contact line away from 90 degrees)."""
    ny, nx = 24, 48
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    a, b = 14.0, 7.0
    r = np.sqrt(((x - 24.0) / a) ** 2 + ((y + 0.5) / b) ** 2)
    phi = np.tanh(2.0 * (1.0 - r) * math.sqrt(a * b) / 4.0)
    prm = O.make_params(sigma=0.03, D=4.0, M=0.1, rho1=1.0, rho2=1.0, mu1=0.1, mu2=0.1)
    s = O.OracleSim((ny, nx), prm)
    s.set_walls(True)
    s.init(np.zeros((ny, nx)), phi)
    s.step(4000)
    ph = s.macros()["phi"]
    pts = A.zero_contour_points(ph)
    pts = pts[pts[:, 1] > 4.0]  # away from the wall layer
    xc, yc, R = A.fit_circle(pts)
    theta = math.degrees(math.acos(max(-1.0, min(1.0, (-0.5 - yc) / R))))
    assert abs(theta - 90.0) < 0.5, (theta, xc, yc, R)
    assert abs(R - math.sqrt(a * b)) < 0.5, R
    # height above the wall line equals the half-width along the wall row
    col, row = ph[:, 24], ph[0, 24:]
    j = int(np.nonzero(col < 0)[0][0])
    height = j - 1 + col[j - 1] / (col[j - 1] - col[j]) + 0.5
    i = int(np.nonzero(row < 0)[0][0])
    half = i - 1 + row[i - 1] / (row[i - 1] - row[i])
    assert abs(height - half) < 0.2, (height, half)


def test_particle_wall_repulsion():
    """Particle-wall repulsion (Sec. 4.5, reading R22): the printed form with
    2 R_k, eps/2 and the mirror image across the nearest wall; a box wall and
    a circular wall through the same point with the same normal give the same
    force; zero beyond 2 R_k + xi; only the nearest wall acts."""
    n = (64, 48)
    R, xi, eps = 5.0, 3.0, 0.5
    p = O.make_params(rep_xi=xi, rep_eps=eps)
    # d' = 2 (y + 1/2): overlapping (d' < 2R), within xi, at the edge, beyond
    for y, expect in ((4.0, None), (5.2, None), (5.9, None), (6.0 + 1e-9, 0.0), (20.0, 0.0)):
        a = O.Particle((30.0, y), R=R)
        F = O.repulsion(2, p, n, [a], walls_y=True)[0]
        d = 2.0 * (y + 0.5)
        if expect is None:
            g = (2 * R + xi - d) ** 2 if d >= 2 * R else (2 * R - d)
            assert F[0] == 0.0 and abs(F[1] - d * g / (eps / 2)) <= 1e-13 * abs(F[1]) and F[1] > 0
        else:
            assert np.abs(F).max() == 0.0
        # the same wall as a huge circle centred above, tangent to y = -1/2 at x = 30
        Rw = 1e6
        pc = O.make_params(rep_xi=xi, rep_eps=eps, wall_circle=(30.0, Rw - 0.5, Rw))
        Fc = O.repulsion(2, pc, n, [a])[0]
        assert np.allclose(Fc, F, rtol=1e-8, atol=1e-12), (y, F, Fc)
    # top wall pushes down; only the nearest wall counts; off without walls
    a = O.Particle((30.0, n[1] - 6.0), R=R)
    assert O.repulsion(2, p, n, [a], walls_y=True)[0][1] < 0
    assert np.abs(O.repulsion(2, p, n, [a])[0]).max() == 0.0
    small = O.Particle((30.0, 4.0), R=2.0)  # both walls within range only when ny is tiny
    F1 = O.repulsion(2, p, (64, 12), [small], walls_y=True)[0]
    F2 = O.repulsion(2, p, (64, 1000), [small], walls_y=True)[0]
    assert np.array_equal(F1, F2)
    # circle: points to the centre, radial
    pc = O.make_params(rep_xi=xi, rep_eps=eps, wall_circle=(32.0, 24.0, 20.0))
    b = O.Particle((32.0 + 14.0 * 0.6, 24.0 + 14.0 * 0.8), R=R)
    Fb = O.repulsion(2, pc, n, [b])[0]
    r = np.array([0.6, 0.8])
    assert Fb[:2] @ r < 0 and abs(Fb[0] * r[1] - Fb[1] * r[0]) < 1e-12 * np.abs(Fb).max()


def test_particle_pair_balance_closed_form():
    """Two particles at an interface (Sec. 4.4, two-particle case): the closed
    form reduces to the single particle in a box of width L/2 when the gaps are
    equal (and F_lat = 0 there), swapping the gaps flips F_lat, the printed
    vertical balance sigma (sin a + sin b) + R_p dp (sin(theta - a) +
    sin(theta - b)) = pi sigma Bo holds, and Bo -> 0 leaves a flat interface."""
    L, R = 256.0, 16.0
    for theta in (60.0, 90.0, 120.0):
        for Bo in (0.05, 0.128, 0.3):
            half = CF.particle_pair_balance(L, R, theta, Bo, L / 4)
            h1, a1 = CF.particle_interface_height(L / 2, R, theta, Bo)
            assert abs(half["h"] - h1) < 1e-9 and abs(half["alpha"] - a1) < 1e-12
            assert abs(half["F_lat_over_sigma"]) < 1e-14
            for d in (24.0, 40.0, 52.0):
                r = CF.particle_pair_balance(L, R, theta, Bo, d)
                s = CF.particle_pair_balance(L, R, theta, Bo, L / 2 - d)
                assert abs(r["F_lat_over_sigma"] + s["F_lat_over_sigma"]) < 1e-12
                th = math.radians(theta)
                vert = (math.sin(r["alpha"]) + math.sin(r["beta"])
                        + R / r["Rc"] * (math.sin(th - r["alpha"]) + math.sin(th - r["beta"])))
                assert abs(vert - math.pi * Bo) < 1e-12 * max(1.0, math.pi * Bo)
            # the narrow gap attracts (capillary attraction of like particles)
            assert CF.particle_pair_balance(L, R, theta, Bo, 24.0)["F_lat_over_sigma"] < 0
    r = CF.particle_pair_balance(L, R, 70.0, 1e-9, 30.0)
    assert abs(r["h"] - R * math.cos(math.radians(70.0))) < 1e-5 and abs(r["F_lat_over_sigma"]) < 1e-8


def test_held_particle_components():
    """Reading R25: held components of a particle's motion keep their value
    under a force and torque, the free ones follow Newton-Euler."""
    p = O.make_params(g=(0.0, -1e-5, 0.0))
    base = O.Particle((10.0, 10.0), u=(0.01, 0.0, 0.0), w=(0.0, 0.0, 0.002), R=5.0, rho_p=2.0)
    free = O.particle_update(2, p, base, (1e-3, 2e-3, 0.0), (0.0, 0.0, 1e-3))
    held = O.particle_update(2, p, O.Particle((10.0, 10.0), u=(0.01, 0.0, 0.0), w=(0.0, 0.0, 0.002), R=5.0,
                                              rho_p=2.0, prescribed=2 | 16),
                             (1e-3, 2e-3, 0.0), (0.0, 0.0, 1e-3))
    assert held.u[0] == 0.01 and held.w[2] == 0.002
    assert held.u[1] == free.u[1] != 0.0
    assert free.u[0] != 0.01 and free.w[2] != 0.002
    assert held.x[0] == free.x[0] == 10.01


def test_walls_3d_poiseuille_and_mass():
    """Box walls in 3D (reading R21 with D3Q19/D3Q7): a body-force channel
    between walls at y = -1/2 and ny - 1/2, periodic in x and z, approaches
    u(y) = F_b (y + 1/2)(ny - 1/2 - y)/(2 mu), uniform in x and z; a drop next
    to the walls with random flow keeps sum phi to round-off."""
    ny = 16
    prm = O.make_params(sigma=0.0, mu1=0.1, mu2=0.1, Fb=(1e-6, 0, 0), d0=0.3)
    s = O.OracleSim((4, ny, 4), prm)
    s.set_walls(True)
    s.init(np.zeros((4, ny, 4)), np.zeros((4, ny, 4)))
    s.step(20000)
    u = s.macros()["u"][0]
    y = np.arange(ny)
    ua = 1e-6 / (2 * 0.1) * (y + 0.5) * (ny - 0.5 - y)
    assert np.abs(u - u[0:1, :, 0:1]).max() < 1e-15
    assert np.abs(u[0, :, 0] - ua).max() < 0.01 * ua.max()
    c = W.small_case((10, 14, 12), seed=3, solid=False, u_amp=0.01)
    c["params"] = dict(c["params"], d0=0.3)
    s = O.OracleSim(c["shape"], O.make_params(**c["params"]))
    s.set_walls(True)
    s.init(c["phi0"], c["phi"], c["u"])
    m0 = s.diagnostics()["mass"]
    s.step(200)
    assert abs(s.diagnostics()["mass"] - m0) <= 1e-13 * np.abs(c["phi"]).sum()


# ---- prescribed contact angle (Young's law through the wetting terms) --------------------

@pytest.mark.parametrize("theta,R,nx,ny", [(45.0, 30.0, 128, 48), (135.0, 16.0, 96, 64)])
def test_cap_at_the_prescribed_angle_stays_there(theta, R, nx, ny):
    """The wetting terms of the free energy (Eq. 8: 3 sigma cos(theta)/D
    phi0 phi (phi^2/3 + phi0^2 - 1) ... and its gradient term) make the
    prescribed theta the equilibrium angle of a drop on a wall (Young's law,
    Sec. 2.1; theta is the angle of phase 1, reading R16).  A drop cut from a
    circle that meets the flat indicator wall at theta keeps that angle: after
    4000 steps the fitted angle is within 2.5 deg of theta (measured 45.1 and
    137.3 deg; the D = 4 diffuse interface and the cap's distance from the
    equal-area equilibrium leave about 2 deg).  A wrong sign of cos(theta)
    would make the 45 deg wall repel the drop and the 135 deg wall attract it,
    moving each cap by tens of degrees."""
    c = W.cap_on_flat_wall(nx, ny, theta, R)
    a0, _ = A.contact_angle_flat(c["phi"], c["phi0"], c["params"]["D"])
    assert abs(a0 - theta) < 0.5, a0
    s = make(c)
    s.step(4000)
    a, info = A.contact_angle_flat(s.macros()["phi"], c["phi0"], c["params"]["D"])
    assert abs(a - theta) < 2.5, (a, info)


@pytest.mark.parametrize("theta_wet", [45.0, 135.0])
def test_semicircle_moves_toward_the_prescribed_angle(theta_wet):
    """The same semicircular drop (90 deg) on walls wetting at 45 and at 135 deg
    (Eq. 8): it spreads on the first and beads up on the second, monotonically,
    by more than 10 deg in 4000 steps (measured 90 -> 82.1 -> 75.5 and 90 ->
    100.1 -> 107.6 at 2000 and 4000 steps), never passing the prescribed angle.
    The direction pins the sign of the wetting terms; the amount, their
    size."""
    c = W.cap_on_flat_wall(96, 48, 90.0, 16.0, theta_wet=theta_wet)
    s = make(c)
    angles = []
    for _ in range(2):
        s.step(2000)
        angles.append(A.contact_angle_flat(s.macros()["phi"], c["phi0"], c["params"]["D"])[0])
    sign = 1.0 if theta_wet > 90.0 else -1.0
    steps = [sign * (angles[0] - 90.0), sign * (angles[1] - angles[0])]
    assert all(v > 0.5 for v in steps), angles
    assert sign * (angles[1] - 90.0) > 10.0, angles
    assert sign * (theta_wet - angles[1]) > 0.0, angles


@pytest.mark.parametrize("theta", [60.0, 120.0])
def test_drop_on_cylinder_moves_toward_hmax(theta):
    """A drop placed on a cylinder (Sec. 4.2 layout, reduced to a 96 x 96 box:
    cylinder radius 16, drop radius 14 centred on its top) relaxes toward the
    equal-area equilibrium height H_max of Eqs. (40)-(41) (closed form with
    reading R13): downward on a wetting cylinder (60 deg, H_max = 29.58 below
    the start 30.0) and upward on a non-wetting one (120 deg, H_max = 34.97),
    monotonically and by at least a quarter of the initial gap within 4000
    steps (measured 43 % and 57 %), without passing H_max."""
    Rp, R0, n = 16.0, 14.0, 96
    cyl = (n / 2.0, 32.0)
    c = W.drop_on_cylinder(n=n, Rp=Rp, cyl=cyl, R0=R0, theta_deg=theta, rho2=1.0, mu2=0.1)
    c["params"] = dict(c["params"], sigma=0.01, s0=1.0)
    Hth, _, _ = CF.hmax_on_cylinder(theta, Rp, CF.initial_drop_area(R0, Rp))
    H0 = A.drop_top_height(c["phi"], cyl[0], cyl[1])
    s = make(c)
    gaps = [abs(H0 - Hth)]
    for _ in range(2):
        s.step(2000)
        H = A.drop_top_height(s.macros()["phi"], cyl[0], cyl[1])
        assert (H - Hth) * (H0 - Hth) > 0.0, (H, Hth)  # still on the starting side
        gaps.append(abs(H - Hth))
    assert gaps[1] < gaps[0] and gaps[2] < gaps[1], gaps
    assert gaps[2] < 0.75 * gaps[0], gaps
