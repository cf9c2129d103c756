"""Pins of the oracle's lattice tables, equilibria, sources, collision matrix
and stencils against what the paper prints and what the mathematics fixes.

Each check is independent of the oracle's own code path: printed matrices
(golden fixture), defining moment identities, orthogonality of Hermite
polynomials, closed-form discrete derivatives of Fourier modes, the tanh
identities of Eq. (13), and variational consistency of Eqs. (9) and (19) with
the free energy of Eq. (8).
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "eq38_d2q9_matrices.txt")


def read_golden(cs2):
    blocks, cur = {}, None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("["):
            cur = line.strip("[]")
            blocks[cur] = []
            continue
        vals = {"0": 0.0, "1": 1.0, "-1": -1.0, "-cs2": -cs2, "cs4": cs2 * cs2}
        blocks[cur].append([vals[t] for t in line.split()])
    return np.array(blocks["M0"]), np.array(blocks["NH"])


@pytest.mark.parametrize("d0", [1.0 / 3.0, 0.4, 0.25])
def test_d2q9_matches_printed_matrices(d0):
    """M_H = N_H C_d M_0 (c = 1) with M_0, N_H as printed in Eq. (38)."""
    M0, NH = read_golden(d0)
    c, w, MH = O.lattice(O.D2Q9, d0)
    np.testing.assert_allclose(MH, NH @ M0, rtol=0, atol=1e-15)
    # velocity order: columns of the first-order rows of M_0
    np.testing.assert_array_equal(c[:, 0], M0[1])
    np.testing.assert_array_equal(c[:, 1], M0[2])
    # printed weights
    np.testing.assert_allclose(w[0], 1 - 2 * d0 + d0 * d0)
    np.testing.assert_allclose(w[1:5], (d0 - d0 * d0) / 2)
    np.testing.assert_allclose(w[5:], d0 * d0 / 4)


def hermite_rows_2d(c, cs2):
    cx, cy = c[:, 0].astype(float), c[:, 1].astype(float)
    hx, hy = cx * cx - cs2, cy * cy - cs2
    return np.array([np.ones_like(cx), cx, cy, hx, hy, cx * cy, cx * hy, cy * hx, hx * hy])


def hermite_rows_3d(c, cs2, q7=False):
    cx, cy, cz = (c[:, a].astype(float) for a in range(3))
    hx, hy, hz = cx * cx - cs2, cy * cy - cs2, cz * cz - cs2
    if q7:
        return np.array([np.ones_like(cx), cx, cy, cz, hx, hy, hz])
    return np.array([np.ones_like(cx), cx, cy, cz, hx, hy, hz, cx * cy, cx * cz, cy * cz,
                     cx * hy, cx * hz, cy * hx, cy * hz, cz * hx, cz * hy,
                     hx * hy, hx * hz, hy * hz])


@pytest.mark.parametrize("kind", [O.D2Q9, O.D3Q19, O.D3Q7])
@pytest.mark.parametrize("d0", [1.0 / 3.0, 0.4, 0.3])
def test_lattice_weights_isotropy(kind, d0):
    """sum w = 1, sum w c = 0, sum w c_a c_b = cs^2 delta_ab; for D2Q9 and
    D3Q19 also sum w c_a^2 c_b^2 = cs^4 (a != b), the identities that make the
    second moments of Eqs. (30), (32) and (33) come out as the paper states."""
    c, w, MH = O.lattice(kind, d0)
    cs2 = d0
    assert abs(w.sum() - 1) < 1e-15
    np.testing.assert_allclose(w @ c, 0, atol=1e-16)
    np.testing.assert_allclose((w[:, None, None] * c[:, :, None] * c[:, None, :]).sum(0),
                               cs2 * np.eye(3) * (np.arange(3) < (2 if kind == O.D2Q9 else 3)),
                               atol=1e-15)
    if kind != O.D3Q7:
        dim = 2 if kind == O.D2Q9 else 3
        for a in range(dim):
            for b in range(dim):
                if a != b:
                    assert abs((w * c[:, a] ** 2 * c[:, b] ** 2).sum() - cs2 * cs2) < 1e-15


def test_textbook_weights_at_one_third():
    """At d0 = 1/3 the weights reduce to the textbook D2Q9 / D3Q19 / D3Q7 sets."""
    _, w, _ = O.lattice(O.D2Q9, 1 / 3)
    np.testing.assert_allclose(w, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, atol=1e-16)
    _, w, _ = O.lattice(O.D3Q19, 1 / 3)
    np.testing.assert_allclose(w, [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12, atol=1e-16)
    _, w, _ = O.lattice(O.D3Q7, 1 / 3)
    np.testing.assert_allclose(w, [0.0] + [1 / 6] * 6, atol=1e-16)


@pytest.mark.parametrize("kind", [O.D2Q9, O.D3Q19, O.D3Q7])
def test_mh_rows_are_hermite_polynomials(kind):
    d0 = 0.4
    c, w, MH = O.lattice(kind, d0)
    if kind == O.D2Q9:
        ref = hermite_rows_2d(c, d0)
    else:
        ref = hermite_rows_3d(c, d0, q7=(kind == O.D3Q7))
    np.testing.assert_allclose(MH, ref, atol=1e-15)


@pytest.mark.parametrize("kind", [O.D2Q9, O.D3Q19])
def test_hermite_rows_orthogonal(kind):
    """Hermite moments are orthogonal under the lattice weights: M_H W M_H^T is
    diagonal.  A wrong entry of N_H breaks this.  D3Q19 has no corner
    velocities, so its quadrature misses the sixth-order moment c_x^2 c_y^2 c_z^2:
    pairs whose product contains it (third order with third order, fourth
    order with fourth order or with the diagonal second order) are not
    orthogonal and are not checked."""
    c, w, MH = O.lattice(kind, 0.4)
    G = MH @ np.diag(w) @ MH.T
    off = G - np.diag(np.diag(G))
    if kind == O.D3Q19:
        off = off.copy()
        off[10:16, 10:16] = 0.0
        off[16:, 16:] = 0.0
        off[4:7, 16:] = 0.0
        off[16:, 4:7] = 0.0
    assert np.abs(off).max() < 1e-15
    assert np.all(np.diag(G) > 0)


@pytest.mark.parametrize("kind", [O.D2Q9, O.D3Q19, O.D3Q7])
def test_bgk_reduction(kind):
    """All rates equal s => Lambda = s I (Eq. 37 reduces to BGK)."""
    Q = {O.D2Q9: 9, O.D3Q19: 19, O.D3Q7: 7}[kind]
    for s in (0.7, 1.0, 1.6):
        Lam = O.lambda_matrix(kind, 0.4, np.full(Q, s))
        np.testing.assert_allclose(Lam, s * np.eye(Q), atol=1e-13)


def test_lambda_conserves_and_relaxes_moments():
    """Lambda acts as diag(S) on Hermite moments: M_H Lambda = diag(S) M_H."""
    rng = np.random.default_rng(3)
    for kind, Q in ((O.D2Q9, 9), (O.D3Q19, 19), (O.D3Q7, 7)):
        S = rng.uniform(0.5, 1.8, Q)
        _, _, MH = O.lattice(kind, 0.4)
        Lam = O.lambda_matrix(kind, 0.4, S)
        np.testing.assert_allclose(MH @ Lam, np.diag(S) @ MH, atol=1e-12)


def moments(c, f, dim):
    c = c[:, :dim].astype(float)
    m0 = f.sum()
    m1 = c.T @ f
    m2 = np.einsum("i,ia,ib->ab", f, c, c)
    return m0, m1, m2


@pytest.mark.parametrize("kind,dim", [(O.D2Q9, 2), (O.D3Q7, 3)])
def test_feq1_and_source_moments(kind, dim):
    """Eq. (30): sum f1eq = phi, sum c f1eq = phi u, sum c c f1eq = eta mu cs^2 I;
    sum F1 = 0, sum c F1 = d_t(phi u)."""
    rng = np.random.default_rng(1)
    d0 = 0.4
    c, w, _ = O.lattice(kind, d0)
    for _ in range(20):
        phi, mu, eta = rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.1, 2)
        u = rng.uniform(-0.1, 0.1, 3)
        u[dim:] = 0
        f = O.feq1(kind, d0, phi, u, mu, eta)
        m0, m1, m2 = moments(c, f, dim)
        assert abs(m0 - phi) < 1e-14
        np.testing.assert_allclose(m1, phi * u[:dim], atol=1e-15)
        np.testing.assert_allclose(m2, eta * mu * d0 * np.eye(dim), atol=1e-14)
        G = rng.uniform(-1, 1, 3)
        G[dim:] = 0
        F = O.src1(kind, d0, G)
        m0, m1, _ = moments(c, F, dim)
        assert abs(m0) < 1e-15
        np.testing.assert_allclose(m1, G[:dim], atol=1e-15)


@pytest.mark.parametrize("kind,dim", [(O.D2Q9, 2), (O.D3Q19, 3)])
def test_feq2_moments(kind, dim):
    """Eq. (32): sum f2eq = 0, sum c f2eq = rho u,
    sum c c f2eq = P I + rho u u - (S u + u S)/2."""
    rng = np.random.default_rng(2)
    for d0 in (1 / 3, 0.4):
        c, w, _ = O.lattice(kind, d0)
        for _ in range(20):
            rho, P = rng.uniform(0.001, 2), rng.uniform(-0.1, 0.1)
            u, S = rng.uniform(-0.1, 0.1, 3), rng.uniform(-0.1, 0.1, 3)
            u[dim:] = 0
            S[dim:] = 0
            f = O.feq2(kind, d0, rho, u, S, P)
            m0, m1, m2 = moments(c, f, dim)
            ud, Sd = u[:dim], S[:dim]
            assert abs(m0) < 1e-14
            np.testing.assert_allclose(m1, rho * ud, atol=1e-15)
            ref = P * np.eye(dim) + rho * np.outer(ud, ud) - 0.5 * (np.outer(Sd, ud) + np.outer(ud, Sd))
            np.testing.assert_allclose(m2, ref, atol=1e-14)


@pytest.mark.parametrize("kind,dim", [(O.D2Q9, 2), (O.D3Q19, 3)])
def test_src2_moments(kind, dim):
    """Eq. (33): sum F2 = u.grad rho, sum c F2 = F + rho f,
    sum c c F2 = M2F + cs^2 (u.grad rho) I."""
    rng = np.random.default_rng(4)
    d0 = 0.4
    c, w, _ = O.lattice(kind, d0)
    for _ in range(20):
        u, gr, Ft = (rng.uniform(-0.1, 0.1, 3) for _ in range(3))
        for v in (u, gr, Ft):
            v[dim:] = 0
        M = rng.uniform(-0.1, 0.1, (dim, dim))
        M = 0.5 * (M + M.T)
        F = O.src2(kind, d0, u, gr, Ft, M)
        m0, m1, m2 = moments(c, F, dim)
        ugr = u[:dim] @ gr[:dim]
        assert abs(m0 - ugr) < 1e-15
        np.testing.assert_allclose(m1, Ft[:dim], atol=1e-15)
        np.testing.assert_allclose(m2, M + d0 * ugr * np.eye(dim), atol=1e-15)


# ---- stencils -----------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(16, 24), (8, 12, 20)])
def test_stencils_on_fourier_modes(shape):
    """On psi = sin(k x) the isotropic stencils give exactly sin(k) cos(k x) for
    d/dx and 2 (cos k - 1) sin(k x) for the Laplacian (2D: D2Q9 weights 1/9,
    1/36; 3D: D3Q19 weights 1/18, 1/36, cs^2 = 1/3)."""
    dim = len(shape)
    n = list(reversed(shape))
    grids = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    X = list(reversed(grids))
    for a in range(dim):
        k = 2 * math.pi * 3 / n[a]
        psi = np.sin(k * X[a])
        g = O.grad(psi)
        np.testing.assert_allclose(g[a], math.sin(k) * np.cos(k * X[a]), atol=1e-14)
        for b in range(dim):
            if b != a:
                np.testing.assert_allclose(g[b], 0, atol=1e-14)
        np.testing.assert_allclose(O.lap(psi), 2 * (math.cos(k) - 1) * psi, atol=1e-14)


@pytest.mark.parametrize("D", [4.0, 8.0])
def test_tanh_indicator_identities(D):
    """Eq. (13): for phi0 = (1 + tanh(2 zeta/D))/2, lap phi0 = 16/D^2 phi0 (1-phi0)(1-2phi0)
    and |grad phi0| = 4 phi0 (1-phi0)/D; the discrete stencils agree to O(1/D^2)."""
    n = 256
    x = np.arange(n, dtype=float)
    zeta = 60 - np.abs(x - n / 2)            # a slab, smooth on both faces
    phi0 = np.tile(0.5 * (1 + np.tanh(2 * zeta / D)), (4, 1))
    lap = O.lap(phi0)[0]
    g = O.grad(phi0)[0][0]
    p = phi0[0]
    lap_ref = 16 / D ** 2 * p * (1 - p) * (1 - 2 * p)
    g_ref = 4 * p * (1 - p) / D
    scale_l, scale_g = np.abs(lap_ref).max(), np.abs(g_ref).max()
    err_l = np.abs(lap - lap_ref).max() / scale_l
    err_g = np.abs(np.abs(g) - g_ref).max() / scale_g
    # leading truncation error of a second-order stencil ~ (2/D)^2 / 3 relative
    assert err_l < 0.6 * (2 / D) ** 2
    assert err_g < 0.6 * (2 / D) ** 2


def test_indicator_error_is_second_order():
    errs = []
    for D in (4.0, 8.0, 16.0):
        n = 512
        x = np.arange(n, dtype=float)
        zeta = 150 - np.abs(x - n / 2)
        p = 0.5 * (1 + np.tanh(2 * zeta / D))
        lap = O.lap(np.tile(p, (4, 1)))[0]
        ref = 16 / D ** 2 * p * (1 - p) * (1 - 2 * p)
        errs.append(np.abs(lap - ref).max() / np.abs(ref).max())
    assert 3.0 < errs[0] / errs[1] < 5.0
    assert 3.5 < errs[1] / errs[2] < 4.5


# ---- chemical potentials vs free energy ---------------------------------------------------

def uniform_energy_density(params, phi, phi0):
    """E_F per cell of a uniform state (all gradients vanish), via the oracle's
    diagnostics on a tiny periodic box."""
    s = O.OracleSim((4, 4), params)
    s.init(np.full((4, 4), phi0), np.full((4, 4), phi))
    return s.diagnostics()["E_F"] / 16.0


@pytest.mark.parametrize("theta", [30.0, 90.0, 135.0])
def test_mu_is_derivative_of_bulk_energy(theta):
    """Eq. (9) = d f / d phi and Eq. (19) = d f / d phi0 of the bulk part of Eq. (8)
    (uniform fields), checked by central differences of the energy."""
    p = O.make_params(sigma=0.013, D=3.7, theta_deg=theta)
    rng = np.random.default_rng(5)
    for _ in range(6):
        phi, phi0 = rng.uniform(-1, 1), rng.uniform(0, 1)
        h = 1e-5
        dfdphi = (uniform_energy_density(p, phi + h, phi0) -
                  uniform_energy_density(p, phi - h, phi0)) / (2 * h)
        dfdphi0 = (uniform_energy_density(p, phi, phi0 + h) -
                   uniform_energy_density(p, phi, phi0 - h)) / (2 * h)
        assert abs(O.mu_phi(p, phi, phi0, 0.0, 0.0) - dfdphi) < 1e-8
        assert abs(O.mu_phi0(p, phi, phi0, 0.0) - dfdphi0) < 1e-8


def test_mu_gradient_terms_are_variational():
    """The gradient terms of Eqs. (9), (19) are the first variations of the
    gradient terms of Eq. (8): for smooth periodic fields,
    d/de E_F[phi + e dphi] = sum mu dphi (and likewise for phi0), to the
    truncation error of the stencils."""
    n = 64
    p = O.make_params(sigma=0.01, D=4.0, theta_deg=50.0)
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    k = 2 * math.pi / n
    phi = 0.6 * np.sin(k * x) * np.cos(k * y)
    phi0 = 0.3 + 0.2 * np.cos(k * x + 0.3)
    dphi = np.cos(2 * k * y + 0.1)

    def E(ph, p0):
        s = O.OracleSim((n, n), p)
        s.init(p0, ph)
        return s.diagnostics()["E_F"]

    eps = 1e-4
    dE = (E(phi + eps * dphi, phi0) - E(phi - eps * dphi, phi0)) / (2 * eps)
    lap_phi, lap_phi0 = O.lap(phi), O.lap(phi0)
    mu = np.vectorize(lambda a, b, c, d: O.mu_phi(p, a, b, c, d))(phi, phi0, lap_phi, lap_phi0)
    assert abs(dE - (mu * dphi).sum()) < 2e-3 * abs(dE)
    dE0 = (E(phi, phi0 + eps * dphi) - E(phi, phi0 - eps * dphi)) / (2 * eps)
    mu0 = np.vectorize(lambda a, b, c: O.mu_phi0(p, a, b, c))(phi, phi0, lap_phi)
    assert abs(dE0 - (mu0 * dphi).sum()) < 2e-3 * abs(dE0)


def test_flat_equilibrium_profile_has_zero_mu():
    """With phi0 = 0, phi = tanh(2x/D) makes Eq. (9) vanish in the continuum; the
    discrete value is O(1/D^2) and falls by ~4 when D doubles."""
    errs = []
    for D in (4.0, 8.0, 16.0):
        p = O.make_params(sigma=0.01, D=D)
        n = 512
        x = np.arange(n, dtype=float)
        phi = np.tanh(2 * (150 - np.abs(x - n / 2)) / D)
        lap = O.lap(np.tile(phi, (4, 1)))[0]
        mu = np.array([O.mu_phi(p, a, 0.0, b, 0.0) for a, b in zip(phi, lap)])
        errs.append(np.abs(mu).max() / (3 * 0.01 / D))
    assert errs[0] < 0.1
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


def test_interface_normal():
    """The interface normal grad phi / |grad phi|: exactly the x axis on a flat
    profile in x (the stencil is symmetric in y), 0 in a uniform bulk, and
    along -r within a fraction of a degree across a circular drop (isotropic
    stencil)."""
    import math
    ny, nx = 16, 64
    x = np.arange(nx, dtype=float)
    phi = np.tile(np.tanh(2.0 * (x - 20.5) / 4.0) * np.tanh(2.0 * (52.5 - x) / 4.0), (ny, 1))
    s = O.OracleSim((ny, nx), O.make_params())
    s.init(np.zeros((ny, nx)), phi)
    n = s.normal()
    # across the interface (away from the bulk, where |grad phi| is round-off)
    assert np.abs(n[1][:, 15:26]).max() < 1e-14
    assert np.abs(np.abs(n[0][:, 15:26]) - 1.0).max() < 1e-12
    assert np.all(n[0][:, 15:26] > 0) and np.all(n[0][:, 48:57] < 0)
    s = O.OracleSim((8, 8), O.make_params())
    s.init(np.zeros((8, 8)), np.full((8, 8), -1.0))
    assert np.abs(s.normal()).max() == 0.0
    L = 96
    yy, xx = np.meshgrid(np.arange(L, dtype=float), np.arange(L, dtype=float), indexing="ij")
    r = np.hypot(xx - 47.5, yy - 47.5)
    s = O.OracleSim((L, L), O.make_params())
    s.init(np.zeros((L, L)), np.tanh(2.0 * (25.0 - r) / 4.0))
    n = s.normal()
    band = np.abs(r - 25.0) < 2.0
    ang = np.degrees(np.arccos(np.clip(-(n[0] * (xx - 47.5) + n[1] * (yy - 47.5)) / r, -1, 1)))
    assert ang[band].max() < 0.5, ang[band].max()
