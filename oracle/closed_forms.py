"""Closed-form results from the paper and from textbook fluid mechanics used
to pin the oracle (and, in GPU tests, the CUDA library).

TEST INFRASTRUCTURE ONLY: see ``oracle/__init__.py``.
"""
import math

from scipy import integrate, optimize


def lens_area(r, R, k):
    """Area of the overlap of two circles of radii r and R whose centres are k apart."""
    if k >= r + R:
        return 0.0
    if k <= abs(R - r):
        return math.pi * min(r, R) ** 2
    d1 = (k * k + r * r - R * R) / (2.0 * k)
    d2 = (k * k - r * r + R * R) / (2.0 * k)
    h = math.sqrt(max(R * R - d2 * d2, 0.0))
    return r * r * math.acos(d1 / r) + R * R * math.acos(d2 / R) - k * h


def hmax_on_cylinder(theta_deg, Rp, A0):
    """Equilibrium height H_max = r + k of a 2D drop of area A0 on a cylinder of
    radius Rp (Eqs. 40-41, Sec. 4.2), with k^2 = r^2 + Rp^2 - 2 r Rp cos(theta).
    The square root term of Eq. (40) is read with its argument squared:
    k sqrt(Rp^2 - ((k^2 - r^2 + Rp^2)/(2k))^2), the chord term of a lens.
    Returns (H_max, r, k)."""
    th = math.radians(theta_deg)

    def k_of(r):
        return math.sqrt(r * r + Rp * Rp - 2.0 * r * Rp * math.cos(th))

    def resid(r):
        k = k_of(r)
        return math.pi * r * r - lens_area(r, Rp, k) - A0

    lo, hi = 1e-6, 10.0 * (math.sqrt(A0 / math.pi) + Rp)
    r = optimize.brentq(resid, lo, hi, xtol=1e-13, rtol=1e-15, maxiter=500)
    k = k_of(r)
    return r + k, r, k


def initial_drop_area(R0, Rp):
    """Area outside the cylinder of a drop of radius R0 centred on its surface."""
    return math.pi * R0 * R0 - lens_area(R0, Rp, Rp)


def taylor_green_rate(nu, k):
    """Decay rate of the velocity amplitude of a 2D Taylor-Green vortex: 2 nu k^2."""
    return 2.0 * nu * k * k


def tanh_indicator_moments(R, D, dim=2):
    """Integrals of the smooth indicator 1/2(1 + tanh(2 (R - r)/D)) over the
    plane (dim = 2) or space (dim = 3): returns (int phi0 dV, int phi0 r^2 dV)."""
    def s(r):
        return 0.5 * (1.0 + math.tanh(2.0 * (R - r) / D))
    top = R + 20.0 * D
    if dim == 2:
        a = integrate.quad(lambda r: s(r) * 2.0 * math.pi * r, 0.0, top, limit=400,
                           epsabs=1e-12, epsrel=1e-13)[0]
        b = integrate.quad(lambda r: s(r) * 2.0 * math.pi * r ** 3, 0.0, top, limit=400,
                           epsabs=1e-12, epsrel=1e-13)[0]
    else:
        a = integrate.quad(lambda r: s(r) * 4.0 * math.pi * r * r, 0.0, top, limit=400,
                           epsabs=1e-12, epsrel=1e-13)[0]
        # integral of (x^2 + y^2) phi0 over space = 2/3 int r^2 phi0 dV
        b = integrate.quad(lambda r: s(r) * 4.0 * math.pi * r ** 4, 0.0, top, limit=400,
                           epsabs=1e-12, epsrel=1e-13)[0] * 2.0 / 3.0
    return a, b


def constant_force_velocity(u0, A, beta, n):
    """Velocity after n explicit-Euler steps of
    u^{m+1} = u^m + A + beta (u^m - u^{m-1}), u^{-1} = u^0 (Eq. 26a with Eq. 28
    lagged by one step): u^n = u^0 + A/(1-beta) [n - beta (1 - beta^n)/(1 - beta)]."""
    return u0 + A / (1.0 - beta) * (n - beta * (1.0 - beta ** n) / (1.0 - beta))


def constant_force_position(x0, u0, A, beta, n):
    """x^n = x^0 + sum_{m<n} u^m for the velocities of ``constant_force_velocity``."""
    return x0 + sum(constant_force_velocity(u0, A, beta, m) for m in range(n))


def bond_number(rho_p, rho_f, Rp, g, sigma):
    """Bo = (rho_p - rho_f) R_p^2 |g| / sigma (Sec. 4.4)."""
    return (rho_p - rho_f) * Rp * Rp * g / sigma


def particle_interface_height(L, Rp, theta_deg, Bo):
    """Equilibrium of one wetting particle (2D disc) trapped at a fluid-fluid
    interface of equal densities under gravity, in a periodic box of width L
    (Sec. 4.4, after Mino et al.): the interface slope alpha at the contact
    point solves L/2 = R_p sin(theta - alpha) + L/(pi Bo) sin(alpha), and the
    downward distance from the far interface (at the box edge) to the particle
    centre is h = R_p cos(theta - alpha) + L/(pi Bo) (1 - cos(alpha)).
    Bo -> 0 gives alpha -> 0 and h -> R_p cos(theta).  Returns (h, alpha)."""
    th = math.radians(theta_deg)
    if Bo == 0.0:
        return Rp * math.cos(th), 0.0
    c = L / (math.pi * Bo)

    def f(a):
        return Rp * math.sin(th - a) + c * math.sin(a) - 0.5 * L

    a = optimize.brentq(f, -0.5 * math.pi + 1e-12, 0.5 * math.pi - 1e-12, xtol=1e-15, rtol=1e-15)
    return Rp * math.cos(th - a) + c * (1.0 - math.cos(a)), a



def particle_pair_balance(L, Rp, theta_deg, Bo, delta):
    """Equilibrium of two equal wetting particles (2D discs) at a fluid-fluid
    interface of equal densities under gravity, centres 2 delta apart in a
    periodic box of width L, allowed to move only vertically (Sec. 4.4, after
    Mino et al.).  The fluid carries both weights through one pressure jump,
    dp L = 2 pi sigma Bo, so every interface piece is an arc of radius
    R_c = sigma/dp = L/(2 pi Bo).  The slope angles alpha (wide gap, L - 2 delta)
    and beta (narrow gap, 2 delta) at the contact points follow from the arcs
    closing the gaps: L/2 - delta = R_p sin(theta - alpha) + R_c sin(alpha),
    delta = R_p sin(theta - beta) + R_c sin(beta).  The printed balances then
    give the lateral force F_lat = sigma (cos alpha - cos beta)
    + R_p (cos(theta - beta) - cos(theta - alpha)) dp (> 0: repulsive) and
    satisfy the vertical one identically.  h is the downward distance from the
    interface at the middle of the wide gap to the centres.
    Returns dict(h, F_lat_over_sigma, alpha, beta, Rc)."""
    th = math.radians(theta_deg)
    Rc = L / (2.0 * math.pi * Bo)

    def slope(gap_half):
        def f(a):
            return Rp * math.sin(th - a) + Rc * math.sin(a) - gap_half
        return optimize.brentq(f, -0.5 * math.pi + 1e-12, 0.5 * math.pi - 1e-12, xtol=1e-15, rtol=1e-15)

    a = slope(0.5 * L - delta)
    b = slope(delta)
    h = Rp * math.cos(th - a) + Rc * (1.0 - math.cos(a))
    f_lat = (math.cos(a) - math.cos(b)) + Rp / Rc * (math.cos(th - b) - math.cos(th - a))
    return dict(h=h, F_lat_over_sigma=f_lat, alpha=a, beta=b, Rc=Rc)