"""Pins of the oracle's conservative Allen-Cahn option (reading R23: the
order-parameter lattice of Eq. 30 recovering
d_t phi + div(phi u) = div(M (grad phi - theta n)), theta = (2/D)(1 - phi^2),
n = grad phi / |grad phi|).  The paper prints no such scheme; what fixes it
is the continuous equation: the flat profile tanh(2 zeta / D) carries no flux,
far from an interface (theta n negligible) it is plain diffusion with
coefficient M, it is conservative, and it is advected by u.
"""
import math

import numpy as np

from oracle import oracle as O
from paper_2311_05097_gb300 import analysis as A
from paper_2311_05097_gb300 import workloads as W

NX, NY, D = 64, 4, 4.0
X = np.arange(NX, dtype=float)


def slab(centre, half=16.0, width=D):
    """A periodic slab of phase 1 of half-width ``half`` with tanh edges of width ``width``."""
    d = X - centre
    d -= NX * np.floor(d / NX + 0.5)
    return np.tanh(2.0 * (half - np.abs(d)) / width)


def sim(prm, phi, u=None):
    s = O.OracleSim((NY, NX), prm)
    s.init(np.zeros((NY, NX)), np.tile(phi, (NY, 1)), u)
    return s


def test_profile_relaxes_to_tanh_and_conserves_mass():
    """Too wide (2D) and too narrow (D/2) edges both relax to tanh(2 zeta/D):
    a dropped or mis-signed sharpening term would leave the width wrong."""
    prm = O.make_params(sigma=0.01, D=D, M=0.1, phase_model=1)
    for width in (2.0 * D, 0.5 * D):
        s = sim(prm, slab(32.0, width=width))
        m0 = s.diagnostics()["mass"]
        assert np.abs(slab(32.0, width=width) - slab(32.0)).max() > 0.25
        s.step(3000)
        ph = s.macros()["phi"]
        assert np.abs(ph - slab(32.0)).max() < 0.02, width
        assert np.abs(ph - ph[0]).max() < 1e-12  # stays one-dimensional
        assert abs(s.diagnostics()["mass"] - m0) < 1e-13 * NX * NY


def test_diffusion_rate_is_the_mobility():
    """With D so large that theta n is negligible the equation is
    d_t phi = M lap phi: a sine mode decays at M k^2 (s_1phi = 1/(M/cs^2 + 1/2))."""
    k = 2.0 * math.pi / NX
    A0, T = 1e-3, 400
    for M in (0.05, 0.2):
        prm = O.make_params(sigma=0.0, D=1e9, M=M, phase_model=1)
        s = sim(prm, A0 * np.sin(k * X))
        s.step(T)
        ph = s.macros()["phi"][0]
        amp = 2.0 / NX * np.sum(ph * np.sin(k * X))
        rate = -math.log(amp / A0) / T
        assert abs(rate / (M * k * k) - 1.0) < 0.01, (M, rate)


def test_profile_is_carried_by_a_uniform_flow():
    """Equal densities, sigma = 0, uniform u0: the slab moves by u0 t and keeps
    its tanh edges and |phi| <= 1 (the Cahn-Hilliard lattice with mu = 0 has no
    such restoring flux)."""
    u0 = 0.02
    u = np.stack([np.full((NY, NX), u0), np.zeros((NY, NX))])
    prm = O.make_params(sigma=0.0, D=D, M=0.05, phase_model=1)
    s = sim(prm, slab(32.0), u)
    s.step(800)
    ph = s.macros()["phi"][0]
    assert np.abs(ph - slab(32.0 + u0 * 800)).max() < 0.03
    assert np.abs(ph).max() <= 1.0 + 1e-9


def test_laplace_law_with_allen_cahn_interface():
    """The surface force of Eq. 16b with mu_phi of Eq. 9 on the Allen-Cahn
    profile still gives P_in - P_out = sigma/R in 2D (within 10 % at R = 16)."""
    R = 16.0
    c = W.static_drop(n=64, R=R)
    s = O.OracleSim(c["shape"], O.make_params(**dict(c["params"], phase_model=1)))
    s.init(c["phi0"], c["phi"])
    s.step(600)
    dps = []
    for _ in range(24):
        s.step(100)
        dps.append(A.laplace_jump(s.macros()["P"], (31.5, 31.5), R, 4.0))
    assert abs(float(np.mean(dps)) / (0.01 / R) - 1.0) < 0.1
