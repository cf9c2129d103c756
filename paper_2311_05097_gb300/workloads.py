"""Seeded synthetic inputs shared by the CUDA library's tests, the oracle's
tests and the benchmark.

This module holds geometry and initial conditions only (smooth indicators of
solids, tanh-profiled drops, parameter draws).  It contains none of the
time-stepping arithmetic of the method and imports neither the CUDA binding
nor the oracle.

Every array is float64, x-fastest: 2D shape (ny, nx), 3D shape (nz, ny, nx).
Cell (i, j[, k]) sits at coordinate (x, y[, z]) = (i, j[, k]).

Shapes follow the paper's experiments: the drop on a cylinder of Sec. 4.2
(initial fields of Eq. 39), porous media of Sec. 4.1, particles of Secs. 4.3-4.6.
The micro-CT image of Sec. 4.1 and the literature data of Secs. 4.2-4.3 are not
available; seeded synthetic stand-ins replace them.
"""
import math

import numpy as np


def smooth_indicator(zeta, D):
    """1/2 (1 + tanh(2 zeta / D)) for a signed distance zeta (positive inside)."""
    return 0.5 * (1.0 + np.tanh(2.0 * zeta / D))


def _coords(shape):
    if len(shape) == 2:
        ny, nx = shape
        y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64),
                           indexing="ij")
        return [x, y]
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return [x, y, z]


def _periodic_dist(shape, centre):
    """Minimum-image distance of every cell to ``centre`` on the periodic box."""
    X = _coords(shape)
    n = list(reversed(shape))
    d2 = np.zeros(shape)
    for a, xa in enumerate(X):
        d = xa - centre[a]
        d -= n[a] * np.floor(d / n[a] + 0.5)
        d2 += d * d
    return np.sqrt(d2)


def disc(shape, centre, R, D):
    """Smooth indicator of a disc / sphere of radius R (positive inside)."""
    return smooth_indicator(R - _periodic_dist(shape, centre), D)


def slab_walls(shape, thickness, D, axis=1):
    """Smooth indicator of a wall slab straddling the periodic boundary of ``axis``
    (x=0, y=1, z=2): cells [0, thickness) and [n - thickness, n) are solid."""
    X = _coords(shape)
    n = list(reversed(shape))[axis]
    y = X[axis]
    yc = -0.5
    d = y - yc
    d -= n * np.floor(d / n + 0.5)
    return smooth_indicator(thickness - np.abs(d), D)


def drop_field(shape, centre, R, D, phi0=None):
    """phi = (1 - phi0) tanh(2 (R - |x - x_c|) / D): phase 1 inside the drop,
    phase 2 outside, zero inside solids (the pattern of Eq. 39)."""
    phi = np.tanh(2.0 * (R - _periodic_dist(shape, centre)) / D)
    if phi0 is not None:
        phi = (1.0 - phi0) * phi
    return phi


# ---------------------------------------------------------------------------------------
# parameter sets (lattice units)
# ---------------------------------------------------------------------------------------

PAPER_DEFAULTS = dict(d0=0.4, s0=1.0, s1=1.0, s2=1.0, s3=1.0, s4=1.0, D=4.0, solid_eps=1e-3)


def params(**kw):
    d = dict(sigma=0.01, D=4.0, M=0.02, eta=0.0, rho1=1.0, rho2=1.0, mu1=0.1, mu2=0.1,
             d0=0.4, s0=1.0, s1=1.0, s2=1.0, s3=1.0, s4=1.0, theta_deg=90.0,
             Fb=(0.0, 0.0, 0.0), g=(0.0, 0.0, 0.0), solid_eps=1e-3, rep_xi=0.0, rep_eps=0.0,
             wall_circle=(0.0, 0.0, 0.0), phase_model=0)
    d.update(kw)
    return d


# ---------------------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------------------

def static_drop(n=128, R=25.0, D=4.0):
    """2D static drop, periodic box, no solid."""
    shape = (n, n)
    phi0 = np.zeros(shape)
    phi = drop_field(shape, ((n - 1) / 2.0, (n - 1) / 2.0), R, D)
    p = params(sigma=0.01, D=D, M=0.02, rho1=1.0, rho2=0.1, mu1=0.1, mu2=0.01)
    return dict(shape=shape, phi0=phi0, phi=phi, params=p, steps=2000, name="static_drop_2d")


def drop_on_cylinder(n=512, Rp=60.0, cyl=(256.0, 160.0), R0=50.0, wall=8, D=4.0,
                     theta_deg=60.0, rho2=1e-2, mu2=1e-3):
    """2D drop resting on a fixed cylinder between two wall slabs (Sec. 4.2 layout)."""
    shape = (n, n)
    phi0 = slab_walls(shape, wall, D, axis=1) + disc(shape, cyl, Rp, D)
    centre = (cyl[0], cyl[1] + Rp)
    phi = drop_field(shape, centre, R0, D, phi0)
    # sigma and M are those of Secs. 4.1-4.2 (sigma_12 = 0.001, M = 0.1);
    # density ratio 100 (viscosity ratio 100): at 1000 the scheme is not stable
    # next to wetting solids
    p = params(sigma=0.001, D=D, M=0.1, rho1=1.0, rho2=rho2, mu1=0.1, mu2=mu2,
               theta_deg=theta_deg, s0=1.6)
    return dict(shape=shape, phi0=phi0, phi=phi, params=p, steps=20000,
                name="drop_on_cylinder_2d")


def rsa_spheres(n, seed=0, rmin=8.0, rmax=16.0, porosity=0.6, reservoir=32, max_tries=20000):
    """Random sequential addition of non-overlapping spheres in the periodic cube,
    none in the reservoir x < ``reservoir``, until the solid fraction reaches
    1 - porosity or ``max_tries`` consecutive rejections (the packing jams).
    Returns (centres, radii)."""
    rng = np.random.default_rng(seed)
    cents = np.zeros((0, 3))
    radii = np.zeros(0)
    target = (1.0 - porosity) * n ** 3
    vol = 0.0
    fails = 0
    while vol < target and fails < max_tries:
        r = rng.uniform(rmin, rmax)
        c = np.array([rng.uniform(reservoir + r, n - r), rng.uniform(0, n), rng.uniform(0, n)])
        if len(radii):
            d = cents - c
            d[:, 1:] -= n * np.floor(d[:, 1:] / n + 0.5)
            if np.any((d * d).sum(1) < (radii + r + 1.0) ** 2):
                fails += 1
                continue
        fails = 0
        cents = np.vstack([cents, c])
        radii = np.append(radii, r)
        vol += 4.0 / 3.0 * math.pi * r ** 3
    return cents, radii


def spheres_indicator(shape, cents, radii, D):
    """phi0 of a union of spheres (zeta = max over spheres of R - |x - x_c|),
    evaluated in each sphere's periodic bounding box."""
    nz, ny, nx = shape
    zeta = np.full(shape, -1e9)
    reach = 10.0 * D
    for c, r in zip(cents, radii):
        h = int(math.ceil(r + reach))
        idx = []
        for a, n in ((2, nz), (1, ny), (0, nx)):
            lo = int(math.floor(c[a])) - h
            idx.append(np.arange(lo, lo + 2 * h + 2) % n)
        zz, yy, xx = np.meshgrid(*idx, indexing="ij")
        d2 = np.zeros(zz.shape)
        for a, g, n in ((0, xx, nx), (1, yy, ny), (2, zz, nz)):
            d = g - c[a]
            d -= n * np.floor(d / n + 0.5)
            d2 += d * d
        sub = r - np.sqrt(d2)
        cur = zeta[zz, yy, xx]
        zeta[zz, yy, xx] = np.maximum(cur, sub)
    return smooth_indicator(zeta, D)


def porous_drainage_3d(n=256, seed=0, D=4.0, invade=24, porosity=0.6):
    """3D drainage: random non-overlapping spheres (radius 8-16), phase 1
    (non-wetting, theta = 120 deg) initially fills x < ``invade``; body force
    pushes it in +x.  Density ratio 10 (see the note on stability below)."""
    shape = (n, n, n)
    cents, radii = rsa_spheres(n, seed=seed, porosity=porosity)
    phi0 = spheres_indicator(shape, cents, radii, D)
    x = np.arange(n, dtype=np.float64)[None, None, :]
    # phase-1 slab [0, invade) with smooth interfaces on both sides (periodic in x)
    dx = x - (invade - 1) / 2.0
    dx -= n * np.floor(dx / n + 0.5)
    phi = (1.0 - phi0) * np.tanh(2.0 * (invade / 2.0 - np.abs(dx)) / D)
    # d0 = 0.3: the D3Q7 rest weight 1 - 3 d0 must stay non-negative.
    # Density ratio 10 needs s0 = 1.9 and a solid viscosity cap of 10x
    # (solid_eps = 0.1): with s0 <= 1.6, or with a 100x or 1000x cap, the 3D
    # extension blows up next to the solids within 1000-1500 steps (the D3Q19
    # Hermite basis is not orthogonal, so very different relaxation rates couple)
    p = params(sigma=0.01, D=D, M=0.02, rho1=1.0, rho2=0.1, mu1=0.1, mu2=0.1, theta_deg=120.0,
               Fb=(1e-6, 0.0, 0.0), d0=0.3, solid_eps=0.1, s0=1.9)
    achieved = float((phi0 < 0.5).mean())
    return dict(shape=shape, phi0=phi0, phi=phi, params=p, steps=2000,
                name="porous_drainage_3d", porosity=achieved, spheres=len(radii))


def rsa_discs(shape, seed=0, rmin=6.0, rmax=12.0, porosity=0.7, clear=2.0, max_tries=20000):
    """Random sequential addition of non-overlapping discs in a box periodic in
    x and bounded in y (each disc at least ``clear`` from the ends of y),
    until the solid fraction reaches 1 - porosity or ``max_tries`` consecutive
    rejections.  Returns (centres (x, y), radii)."""
    rng = np.random.default_rng(seed)
    ny, nx = shape
    cents = np.zeros((0, 2))
    radii = np.zeros(0)
    target = (1.0 - porosity) * nx * ny
    area = 0.0
    fails = 0
    while area < target and fails < max_tries:
        r = rng.uniform(rmin, rmax)
        c = np.array([rng.uniform(0, nx), rng.uniform(r + clear, ny - r - clear)])
        if len(radii):
            d = cents - c
            d[:, 0] -= nx * np.floor(d[:, 0] / nx + 0.5)
            if np.any((d * d).sum(1) < (radii + r + 1.0) ** 2):
                fails += 1
                continue
        fails = 0
        cents = np.vstack([cents, c])
        radii = np.append(radii, r)
        area += math.pi * r * r
    return cents, radii


def porous_phase_separation_2d(n=256, theta_deg=90.0, seed=0, porosity=0.7, D=4.0):
    """Phase separation inside a 2D porous medium (the setting of Sec. 4.1,
    with random discs standing in for the micro-CT image): no-flux walls at
    both ends of y (periodic in x), phi = (1 - phi0) * U(-1, 1) per cell,
    equal densities and viscosities, sigma = 0.001, M = 0.1, D = 4."""
    shape = (n, n)
    cents, radii = rsa_discs(shape, seed=seed, porosity=porosity)
    x, y = _coords(shape)
    zeta = np.full(shape, -1e9)
    for c, r in zip(cents, radii):
        dx = x - c[0]
        dx -= n * np.floor(dx / n + 0.5)
        zeta = np.maximum(zeta, r - np.sqrt(dx * dx + (y - c[1]) ** 2))
    phi0 = smooth_indicator(zeta, D)
    rng = np.random.default_rng(seed + 1000)
    phi = (1.0 - phi0) * rng.uniform(-1.0, 1.0, shape)
    p = params(sigma=0.001, D=D, M=0.1, rho1=1.0, rho2=1.0, mu1=0.1, mu2=0.1, theta_deg=theta_deg, d0=0.4)
    return dict(shape=shape, phi0=phi0, phi=phi, params=p, walls_y=True,
                name="porous_phase_separation_2d", porosity=float((phi0 < 0.5).mean()), discs=len(radii))


def water_entry(nx=1024, ny=2048, depth=800, wall=8, R=40.0, gap=200.0, D=4.0):
    """2D water entry of a particle (density 2 rho1, theta 90 deg) dropped at
    -0.02 towards a liquid pool of depth ``depth`` resting on a wall slab;
    the fluid inside the particle starts at the particle's velocity."""
    shape = (ny, nx)
    phi0 = slab_walls(shape, wall, D, axis=1)
    y = _coords(shape)[1]
    surface = wall + depth
    particle = dict(x=(nx / 2.0, surface + gap, 0.0), u=(0.0, -0.02, 0.0), w=(0.0, 0.0, 0.0),
                    R=R, rho_p=2.0)
    ind = disc(shape, particle["x"], R, D)
    solid = phi0 + ind
    phi = (1.0 - solid) * np.tanh(2.0 * (surface - y) / D)
    u = np.stack([ind * particle["u"][0], ind * particle["u"][1]])
    # density ratio 10 (viscosity ratio 10): a particle moving through a light
    # gas at density ratio 100 or 1000 blows up within 100 steps with this scheme
    p = params(sigma=0.001, D=D, M=0.1, rho1=1.0, rho2=0.1, mu1=0.1, mu2=0.01,
               theta_deg=90.0, g=(0.0, -1e-6, 0.0), s0=1.6)
    return dict(shape=shape, phi0=phi0, phi=phi, u=u, params=p, particles=[particle], steps=50000,
                name="water_entry_2d")


def particle_balance(L=256, Rp=32.0, theta_deg=90.0, rho_p=1.1, sigma=0.01, g=2e-5, wall=8, D=4.0, M=0.1):
    """One free disc (radius Rp, density rho_p) half immersed at the flat
    interface between two fluids of equal density (rho_f = 1) in a box of
    width L, periodic in x, with wall slabs of ``wall`` cells below and above
    (Sec. 4.4 layout; sigma and g scaled together from the paper's 0.001 and
    2e-6, which keeps the Bond number and shortens the relaxation 10x).
    Gravity acts on the particle only."""
    ny = L + 2 * wall
    shape = (ny, L)
    phi0 = slab_walls(shape, wall, D, axis=1)
    y_if = ny / 2.0
    particle = dict(x=(L / 2.0, y_if, 0.0), u=(0.0, 0.0, 0.0), w=(0.0, 0.0, 0.0), R=Rp, rho_p=rho_p)
    ind = disc(shape, particle["x"], Rp, D)
    y = _coords(shape)[1]
    phi = (1.0 - phi0 - ind) * np.tanh(2.0 * (y_if - y) / D)
    p = params(sigma=sigma, D=D, M=M, rho1=1.0, rho2=1.0, mu1=0.1, mu2=0.1, theta_deg=theta_deg,
               g=(0.0, -g, 0.0))
    return dict(shape=shape, phi0=phi0, phi=phi, params=p, particles=[particle], L=L, Rp=Rp,
                rho_f=1.0, sigma=sigma, g=g, y_if=y_if, name="particle_balance_2d")


def particle_pair_balance(L=256, Rp=16.0, delta=24.0, theta_deg=90.0, rho_p=1.25, sigma=0.01, g=2e-5,
                          wall=8, D=3.0, M=0.1):
    """Two equal discs half immersed at the flat interface of two fluids of
    equal density, centres at L/2 -+ delta, in the box of ``particle_balance``
    (Sec. 4.4 two-particle case: R_p = 16, D = 3; sigma and g scaled together
    as there).  Each particle holds its horizontal translation and its
    rotation (moves only vertically); gravity acts on the particles only."""
    ny = L + 2 * wall
    shape = (ny, L)
    phi0 = slab_walls(shape, wall, D, axis=1)
    y_if = ny / 2.0
    parts = [dict(x=(L / 2.0 + s * delta, y_if, 0.0), u=(0.0, 0.0, 0.0), w=(0.0, 0.0, 0.0), R=Rp,
                  rho_p=rho_p, prescribed=2 | 16) for s in (-1.0, 1.0)]
    solid = phi0 + sum(disc(shape, q["x"], Rp, D) for q in parts)
    y = _coords(shape)[1]
    phi = (1.0 - solid) * np.tanh(2.0 * (y_if - y) / D)
    p = params(sigma=sigma, D=D, M=M, rho1=1.0, rho2=1.0, mu1=0.1, mu2=0.1, theta_deg=theta_deg,
               g=(0.0, -g, 0.0))
    return dict(shape=shape, phi0=phi0, phi=phi, params=p, particles=parts, L=L, Rp=Rp, delta=delta,
                rho_f=1.0, sigma=sigma, g=g, y_if=y_if, wall=wall, name="particle_pair_balance_2d")


def annulus_mixing(n=512, count=15, seed=4, D=5.0, omega=1e-4, g=1e-6, rep_xi=2.5, rep_eps=1e4):
    """Two fluid layers and ``count`` free wetting particles in the annulus
    between a fixed outer wall (radius n/2) and an inner cylinder (radius
    n/8) rotating at ``omega`` rad/step (Sec. 4.5 layout in lattice units,
    dx = 0.01 of the paper: R_p in [20, 30], rho_p in [0.95, 1.05], theta_k in
    [45, 135] deg, neutral walls, sigma = 0.001, equal fluid densities and
    viscosities, gravity on the particles, short-range particle-particle and
    particle-wall repulsion).  The inner cylinder is particle 0 with prescribed
    rotation."""
    rng = np.random.default_rng(seed)
    shape = (n, n)
    c = (n - 1) / 2.0
    r_out, r_in = n / 2.0, n / 8.0
    X, Y = _coords(shape)
    r = np.hypot(X - c, Y - c)
    phi0 = smooth_indicator(r - r_out, D)  # outer wall: solid outside r_out
    parts = [dict(x=(c, c, 0.0), u=(0.0, 0.0, 0.0), w=(0.0, 0.0, omega), R=r_in, rho_p=1.0,
                  prescribed=True)]
    placed = []
    tries = 0
    while len(placed) < count and tries < 100000:
        tries += 1
        R = rng.uniform(20.0, 30.0)
        rad = rng.uniform(r_in + R + 6.0, r_out - R - 6.0)
        ang = rng.uniform(0.0, 2.0 * math.pi)
        x, y = c + rad * math.cos(ang), c + rad * math.sin(ang)
        if all(math.hypot(x - q[0], y - q[1]) > R + q[2] + 6.0 for q in placed):
            placed.append((x, y, R))
    for x, y, R in placed:
        parts.append(dict(x=(x, y, 0.0), u=(0.0, 0.0, 0.0), w=(0.0, 0.0, 0.0), R=R,
                          rho_p=rng.uniform(0.95, 1.05), theta_deg=rng.uniform(45.0, 135.0)))
    solid = phi0.copy()
    for q in parts:
        solid = solid + disc(shape, q["x"], q["R"], D)
    phi = (1.0 - solid) * np.tanh(-2.0 * (Y - c) / D)
    # the outer wall also repels the particles (its phi0 = 1/2 circle)
    p = params(sigma=0.001, D=D, M=0.1, rho1=1.0, rho2=1.0, mu1=0.1, mu2=0.1, theta_deg=90.0,
               g=(0.0, -g, 0.0), rep_xi=rep_xi, rep_eps=rep_eps, wall_circle=(c, c, r_out))
    return dict(shape=shape, phi0=phi0, phi=phi, params=p, particles=parts, name="annulus_mixing_2d")


def channel_displacement(L=256, count=16, seed=5, D=5.0, Fb=3e-7, rep_xi=2.5, rep_eps=1e4,
                         particles=True, fluid1=True):
    """Displacement of a drop of fluid 1 out of a cavity by fluid 2 and free
    particles in a channel of height L and length 5L (Sec. 4.6 layout in
    lattice units, dx = 0.01 of the paper): periodic in x, no-flux box walls at
    both ends of y, a bottom wall of height L/4 with a large cavity (the circle
    of radius L centred at (L, L)) and a small one (radius L/4 centred at
    (9L/4, L/4); see the reading of its centre) holding the drop; ``count``
    particles R in [0.0625 L, 0.078 L], rho_p in [0.95, 1.05], theta_k in
    [80, 100] deg, most of them above the large cavity; fluid 2 drives with a
    body force Fb in x; equal densities, viscosity ratio 10 (mu1 = 0.5,
    mu2 = 0.05: at the paper's mu2 = 0.01 the scheme blows up within 500 steps
    in this geometry, even without particles or walls), sigma = 0.001,
    neutral walls.  ``particles`` / ``fluid1`` switch off the particles (the
    paper's case B) or the drop (case A)."""
    rng = np.random.default_rng(seed)
    shape = (L, 5 * L)
    X, Y = _coords(shape)
    xc_small = 9.0 * L / 4.0

    def ind(zeta):
        return smooth_indicator(zeta, D)

    # bottom wall below y = L/4, minus the two cavities (product of indicators)
    phi0 = (ind(L / 4.0 - Y) * ind(np.hypot(X - L, Y - L) - L)
            * ind(np.hypot(X - xc_small, Y - L / 4.0) - L / 4.0))
    parts = []
    if particles:
        placed = []
        tries = 0
        while len(placed) < count and tries < 200000:
            tries += 1
            R = rng.uniform(0.0625 * L, 0.078 * L)
            # three quarters above the large cavity, the rest upstream of the drop
            x = rng.uniform(0.35 * L, 1.65 * L) if len(placed) < 0.75 * count else rng.uniform(1.7 * L, 4.8 * L)
            y = rng.uniform(0.0, L - R - 4.0)
            xi, yi = int(round(x)) % shape[1], int(round(y))
            if yi < 0 or yi >= L:
                continue
            # clear of the solid (phi0 < 1e-3 on a ring just outside the particle)
            ang = np.linspace(0.0, 2 * math.pi, 32, endpoint=False)
            rx = (np.round(x + (R + 4.0) * np.cos(ang)).astype(int)) % shape[1]
            ry = np.round(y + (R + 4.0) * np.sin(ang)).astype(int)
            if np.any(ry < 0) or np.any(ry >= L) or np.any(phi0[ry, rx] > 1e-3) or phi0[yi, xi] > 1e-3:
                continue
            if any(math.hypot(x - q[0], y - q[1]) < R + q[2] + 6.0 for q in placed):
                continue
            placed.append((x, y, R))
        for x, y, R in placed:
            parts.append(dict(x=(x, y, 0.0), u=(0.0, 0.0, 0.0), w=(0.0, 0.0, 0.0), R=R,
                              rho_p=rng.uniform(0.95, 1.05), theta_deg=rng.uniform(80.0, 100.0)))
    solid = phi0.copy()
    for q in parts:
        solid = solid + disc(shape, q["x"], q["R"], D)
    if fluid1:
        phi = (1.0 - solid) * np.tanh(2.0 * (L / 4.0 - np.hypot(X - xc_small, Y - L / 4.0)) / D)
    else:
        phi = -(1.0 - solid)
    p = params(sigma=0.001, D=D, M=0.1, rho1=1.0, rho2=1.0, mu1=0.5, mu2=0.05, theta_deg=90.0,
               Fb=(Fb, 0.0, 0.0), rep_xi=rep_xi, rep_eps=rep_eps)
    return dict(shape=shape, phi0=phi0, phi=phi, params=p, particles=parts, walls_y=True,
                cavity=(2.0 * L, 2.5 * L), name="channel_displacement_2d")


def equal_area_cap_base(theta_deg, area):
    """Radius and base half-width of a circular cap of given area on a flat wall."""
    th = math.radians(theta_deg)
    # area of a cap of radius r and contact angle th: r^2 (th - sin th cos th)
    r = math.sqrt(area / (th - math.sin(th) * math.cos(th)))
    return r, r * math.sin(th)


def flat_wall_drop(L, theta_deg, rho_ratio, r0=None, wall=8, D=4.0, mu1=0.1, mu2=None,
                   sigma=0.01, M=0.1, s0=1.6):
    """A semicircular drop of radius r0 (default 0.3 L, limited so that the
    equilibrium base stays within 0.7 L) centred on the top face of a bottom
    wall slab in an L x L periodic box.  mu2 defaults to 0.1 r^(-2/3) for
    density ratio r (kinematic viscosity 0.1 r^(1/3) in phase 2)."""
    shape = (L, L)
    phi0 = slab_walls(shape, wall, D, axis=1)
    r0 = 0.3 * L if r0 is None else r0
    area = 0.5 * math.pi * r0 * r0
    _, half = equal_area_cap_base(theta_deg, area)
    clamped = False
    if 2.0 * half > 0.7 * L:
        # shrink the drop until the equilibrium base is 0.7 L
        scale = 0.7 * L / (2.0 * half)
        r0 *= scale
        clamped = True
    centre = ((L - 1) / 2.0, wall - 0.5)
    phi = drop_field(shape, centre, r0, D, phi0)
    if mu2 is None:
        mu2 = mu1 * rho_ratio ** (-2.0 / 3.0)
    # s0 (zeroth flow moment, a free rate of S_H in Eq. 38) = 1.6 keeps density
    # ratios up to 100 stable next to wetting walls (the paper's own runs use
    # s0 = 1 at density ratios <= 10)
    p = params(sigma=sigma, D=D, M=M, rho1=1.0, rho2=1.0 / rho_ratio, mu1=mu1, mu2=mu2,
               theta_deg=theta_deg, s0=s0)
    return dict(shape=shape, phi0=phi0, phi=phi, params=p, r0=r0, clamped=clamped,
                wall=wall)


def cap_on_flat_wall(nx, ny, theta_deg, R, wall=8, D=4.0, theta_wet=None, sigma=0.01, M=0.1,
                     rho_ratio=1.0, s0=1.0):
    """A drop of phase 1 on the bottom of two wall slabs (``wall`` cells each) of
    an nx x ny box, cut from a circle of radius R whose centre lies
    R cos(theta_deg) below the wall's phi0 = 1/2 level y_w = wall - 1/2, so
    that the circle meets that level at theta_deg (Young's construction; the
    equal-area equilibrium cap is not sought).  Distances in y are not
    periodic (the walls separate the periodic copies).  Density ratio
    rho_ratio (1: equal densities), mu2 = 0.1 rho_ratio^(-2/3) as in
    ``flat_wall_drop``; theta_wet (default theta_deg) is the prescribed angle
    of the walls."""
    shape = (ny, nx)
    phi0 = slab_walls(shape, wall, D, axis=1)
    x, y = _coords(shape)
    yc = wall - 0.5 - R * math.cos(math.radians(theta_deg))
    dx = x - (nx - 1) / 2.0
    dx -= nx * np.floor(dx / nx + 0.5)
    r = np.sqrt(dx * dx + (y - yc) ** 2)
    phi = (1.0 - phi0) * np.tanh(2.0 * (R - r) / D)
    p = params(sigma=sigma, D=D, M=M, rho1=1.0, rho2=1.0 / rho_ratio, mu1=0.1,
               mu2=0.1 * rho_ratio ** (-2.0 / 3.0), s0=s0,
               theta_deg=theta_deg if theta_wet is None else theta_wet)
    return dict(shape=shape, phi0=phi0, phi=phi, params=p, wall=wall)


def periodic_drop(L, rho_ratio, D=4.0, sigma=0.01, M=0.1, mu1=0.1, s0=1.6):
    """A drop of radius L/4 at the centre of an L x L periodic box without
    solids (mu2 as in ``flat_wall_drop``): a batch domain for either
    order-parameter lattice."""
    shape = (L, L)
    phi = drop_field(shape, ((L - 1) / 2.0, (L - 1) / 2.0), 0.25 * L, D)
    p = params(sigma=sigma, D=D, M=M, rho1=1.0, rho2=1.0 / rho_ratio, mu1=mu1,
               mu2=mu1 * rho_ratio ** (-2.0 / 3.0), s0=s0)
    return dict(shape=shape, phi0=np.zeros(shape), phi=phi, params=p)


def batch_cases(count=256, seed=1, sizes=(64, 128, 256, 512), max_ratio=100.0):
    """Parameter draws of the batched sweep: box side uniform over ``sizes``,
    contact angle uniform in [30, 150] deg, density ratio log-uniform in
    [1, max_ratio] (100: higher ratios next to wetting walls are not stable
    with this scheme).  Fields are produced lazily by ``flat_wall_drop``."""
    rng = np.random.default_rng(seed)
    L = rng.choice(np.array(sizes), size=count)
    theta = rng.uniform(30.0, 150.0, size=count)
    ratio = np.exp(rng.uniform(0.0, math.log(max_ratio), size=count))
    return [dict(L=int(L[i]), theta_deg=float(theta[i]), rho_ratio=float(ratio[i]))
            for i in range(count)]


# ---------------------------------------------------------------------------------------
# small cases for parity tests
# ---------------------------------------------------------------------------------------

def random_smooth(shape, seed, amp=1.0, modes=4):
    """Smooth periodic random field made of a few Fourier modes."""
    rng = np.random.default_rng(seed)
    X = _coords(shape)
    n = list(reversed(shape))
    f = np.zeros(shape)
    for _ in range(modes):
        k = [rng.integers(1, 3) for _ in range(len(shape))]
        ph = rng.uniform(0, 2 * math.pi)
        arg = sum(2 * math.pi * k[a] * X[a] / n[a] for a in range(len(shape)))
        f += rng.uniform(-1, 1) * np.sin(arg + ph)
    return amp * f / max(1.0, np.abs(f).max())


def wall_case(shape, seed=0, solid=True, theta_deg=60.0, u_amp=0.01, D=4.0):
    """2D box with no-flux walls at both ends of y: a drop cut by the top wall
    (a 90 degree contact line there), a solid disc close to the bottom wall and
    a smooth random initial flow.  Used by the wall parity tests."""
    rng = np.random.default_rng(seed)
    ny, nx = shape
    x, y = _coords(shape)

    def dist(cx, cy):  # periodic in x only: no image across a wall
        dx = x - cx
        dx -= nx * np.floor(dx / nx + 0.5)
        return np.sqrt(dx * dx + (y - cy) ** 2)

    phi0 = np.zeros(shape)
    if solid:
        phi0 = smooth_indicator(0.15 * min(nx, ny) - dist(nx * rng.uniform(0.2, 0.3), 0.22 * ny), D)
    phi = (1.0 - phi0) * np.tanh(2.0 * (0.25 * min(nx, ny) - dist(nx * rng.uniform(0.55, 0.65), 0.88 * ny)) / D)
    u = None
    if u_amp > 0:
        u = np.stack([random_smooth(shape, seed + 10 + a, amp=u_amp) for a in range(2)])
    p = params(sigma=0.01, D=D, M=0.02, rho1=1.0, rho2=0.1, mu1=0.1, mu2=0.01,
               theta_deg=theta_deg, d0=0.4)
    return dict(shape=shape, phi0=phi0, phi=phi, u=u, params=p)


def small_case(shape, seed=0, solid=True, theta_deg=60.0, rho_ratio=10.0, mu_ratio=10.0,
               D=4.0, u_amp=0.0):
    """A drop (and, with ``solid``, a disc/sphere solid) on a small periodic box
    with ragged sizes: used by the element-wise parity tests."""
    rng = np.random.default_rng(seed)
    dim = len(shape)
    n = list(reversed(shape))
    phi0 = np.zeros(shape)
    if solid:
        c = [n[a] * rng.uniform(0.25, 0.35) for a in range(dim)]
        phi0 = disc(shape, c, 0.18 * min(n), D)
    cd = [n[a] * rng.uniform(0.55, 0.7) for a in range(dim)]
    phi = drop_field(shape, cd, 0.22 * min(n), D, phi0)
    u = None
    if u_amp > 0:
        u = np.stack([random_smooth(shape, seed + 10 + a, amp=u_amp) for a in range(dim)])
    p = params(sigma=0.01, D=D, M=0.02, rho1=1.0, rho2=1.0 / rho_ratio, mu1=0.1,
               mu2=0.1 / mu_ratio, theta_deg=theta_deg, d0=0.4 if dim == 2 else 0.3)
    return dict(shape=shape, phi0=phi0, phi=phi, u=u, params=p)
