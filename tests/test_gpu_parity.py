"""Parity of the CUDA library (through the C-ABI) with the FP64 oracle on the
same seeded inputs.

FP64 path: every field agrees with the oracle to 1e-12 relative
(max |gpu - oracle| / max |oracle| per field).  FP32 and mixed-precision
paths: the per-field bounds stated in each test.  Sizes span several tiles
with ragged edges; one case runs the 128 x 128 static drop for its full 2000
steps and one samples the 512 x 512 drop-on-cylinder case in the launch
configuration the benchmark uses.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_05097_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ("phi", "rho", "u", "P", "mu")


@pytest.fixture(scope="module")
def pf():
    from paper_2311_05097_gb300 import build
    build.build()
    from paper_2311_05097_gb300 import pf as _pf
    _pf.load()
    return _pf


def rel(a, b):
    s = np.abs(b).max()
    return float(np.abs(a - b).max() / (s if s > 0 else 1.0))


def run_pair(pf, case, steps, precision="p64", particles=(), oracle=True, config=None, walls=False):
    prm = case["params"]
    g = pf.Sim(case["shape"], precision=precision, walls_y=walls, **prm)
    o = O.OracleSim(case["shape"], O.make_params(**prm)) if oracle else None
    if o is not None and walls:
        o.set_walls(True)
    for k, pp in enumerate(particles):
        g.set_particle(k, **pp)
        if o is not None:
            o.set_particle(k, O.Particle(**pp))
    g.init(case["phi0"], case["phi"], case.get("u"))
    if config is not None:
        g.set_config(*config)
    if o is not None:
        o.init(case["phi0"], case["phi"], case.get("u"))
    g.step(steps)
    if o is not None:
        o.step(steps)
    return g, o


def assert_fields(gm, om, tol, mu_scale=None):
    """Relative max error per field.  mu_phi (Eq. 9) is a small difference of
    terms of size 3 sigma/D (it vanishes at equilibrium), so its error is
    measured against max(|mu|, 3 sigma/D): round-off in those terms sets the
    floor, not |mu| itself."""
    for k in FIELDS:
        if k == "mu" and mu_scale is not None:
            e = float(np.abs(gm[k] - om[k]).max() / max(np.abs(om[k]).max(), mu_scale))
        else:
            e = rel(gm[k], om[k])
        assert e < tol[k] if isinstance(tol, dict) else e < tol, (k, e)


@pytest.mark.parametrize("shape,solid,u_amp,steps", [
    ((52, 40), True, 0.0, 0),
    ((52, 40), True, 0.0, 120),
    ((37, 45), False, 0.02, 150),
    ((70, 33), True, 0.01, 90),
])
def test_p64_matches_oracle_2d(pf, shape, solid, u_amp, steps):
    c = W.small_case(shape, seed=7, solid=solid, theta_deg=60.0, u_amp=u_amp)
    g, o = run_pair(pf, c, steps)
    assert_fields(g.macros(), o.macros(), 1e-12)
    assert g.time == steps


def test_p64_diagnostics_match_oracle(pf):
    c = W.small_case((48, 64), seed=2, solid=True, theta_deg=120.0, u_amp=0.01)
    g, o = run_pair(pf, c, 60)
    dg, do = g.diagnostics(), o.diagnostics()
    for k in ("mass", "E_F", "E_K", "E_total"):
        assert abs(dg[k] - do[k]) <= 1e-12 * max(abs(do[k]), 1e-300) + 1e-15, k
    assert dg["nan_flag"] == 0


def test_p64_moving_particle_matches_oracle(pf):
    c = W.small_case((48, 56), seed=5, solid=False)
    part = dict(x=(20.3, 17.6), u=(0.01, -0.004), w=(0.0, 0.0, 0.002), R=6.0, rho_p=2.0)
    c["phi"] = (1.0 - W.disc(c["shape"], part["x"], part["R"], c["params"]["D"])) * c["phi"]
    g, o = run_pair(pf, c, 80, particles=[part])
    assert_fields(g.macros(), o.macros(), 1e-12)
    pg, po = g.particle(0), o.particle(0)
    for k in ("x", "u", "w", "F", "T"):
        a, b = np.array(pg[k]), np.array(getattr(po, k))
        assert np.abs(a - b).max() <= 1e-12 * max(np.abs(b).max(), 1e-12), (k, a, b)


def test_p64_own_angles_and_repulsion_match_oracle(pf):
    """Three free particles, two with their own contact angle (45, 135 deg;
    the third and the fixed disc at the handle's 60 deg) and two within the
    repulsion range (Sec. 4.5), FP64 against the oracle: fields, the FP64
    diagnostics and every particle's state after 80 steps."""
    c = W.small_case((72, 64), seed=6, solid=True, theta_deg=60.0)
    c["params"] = dict(c["params"], rep_xi=2.0, rep_eps=1e4)
    parts = [dict(x=(20.0, 46.0), u=(0.004, 0.0), R=6.0, rho_p=2.0, theta_deg=45.0),
             dict(x=(33.0, 46.0), u=(-0.004, 0.0), R=6.0, rho_p=2.0, theta_deg=135.0),
             dict(x=(50.0, 18.0), u=(0.0, 0.003), R=5.0, rho_p=1.5)]
    phi = c["phi"]
    for pp in parts:
        phi = (1.0 - W.disc(c["shape"], pp["x"], pp["R"], c["params"]["D"])) * phi
    c["phi"] = phi
    g, o = run_pair(pf, c, 80, particles=parts)
    assert_fields(g.macros(), o.macros(), 1e-12, mu_scale=3 * 0.01 / 4.0)
    dg, do = g.diagnostics(), o.diagnostics()
    for k in ("mass", "E_F", "E_K"):
        assert abs(dg[k] - do[k]) <= 1e-12 * max(abs(do[k]), 1e-12), (k, dg[k], do[k])
    for k in range(3):
        pg, po = g.particle(k), o.particle(k)
        for f in ("x", "u", "w", "F", "T"):
            a, b = np.array(pg[f]), np.array(getattr(po, f))
            assert np.abs(a - b).max() <= 1e-12 * max(np.abs(b).max(), 1e-12), (k, f, a, b)
    # the repulsion pushed the close pair apart relative to no repulsion
    c2 = dict(c, params=dict(c["params"], rep_eps=0.0))
    g2, _ = run_pair(pf, c2, 80, particles=parts, oracle=False)
    assert g.particle(0)["u"][0] < g2.particle(0)["u"][0]
    assert g.particle(1)["u"][0] > g2.particle(1)["u"][0]


def test_annulus_mixing_full_size_against_oracle(pf):
    """Sec. 4.5 layout at full size (512 x 512, outer wall, inner cylinder of
    prescribed rotation, 15 wetting particles with their own angles,
    repulsion): FP64 fields and particle states against the oracle after 3
    steps."""
    c = W.annulus_mixing()
    g, o = run_pair(pf, c, 3, particles=c["particles"])
    assert_fields(g.macros(), o.macros(), 1e-12, mu_scale=3 * 0.001 / 5.0)
    for k in range(len(c["particles"])):
        pg, po = g.particle(k), o.particle(k)
        a, b = np.array(pg["x"]), np.array(po.x)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), (k, a, b)
        # velocity, rotation and F come from sums over the particle's cells of
        # terms that largely cancel: measured against the velocity scale |u_s|,
        # the rotation scale |u_s| / R and the momentum-exchange scale
        # rho pi R^2 |u_s|
        R = po.R
        us = np.abs(po.u).max() + abs(po.w[2]) * R + 1e-4
        assert np.abs(np.array(pg["u"]) - np.array(po.u)).max() <= 1e-12 * us, k
        assert np.abs(np.array(pg["F"]) - np.array(po.F)).max() <= 1e-12 * math.pi * R * R * us, k
        assert np.abs(np.array(pg["w"]) - np.array(po.w)).max() <= 1e-12 * us / R, k


def test_p64_static_drop_full_run(pf):
    """The 128 x 128 static drop for its full 2000 steps."""
    c = W.static_drop()
    g, o = run_pair(pf, c, 2000)
    assert_fields(g.macros(), o.macros(), 1e-12, mu_scale=3 * c["params"]["sigma"] / c["params"]["D"])
    dg, do = g.diagnostics(), o.diagnostics()
    assert abs(dg["mass"] - do["mass"]) < 1e-12 * np.abs(c["phi"]).sum()


def test_p64_is_deterministic(pf):
    c = W.small_case((64, 64), seed=11, solid=True, u_amp=0.01)
    a, _ = run_pair(pf, c, 50, oracle=False)
    b, _ = run_pair(pf, c, 50, oracle=False)
    ma, mb = a.macros(), b.macros()
    for k in FIELDS:
        assert np.array_equal(ma[k], mb[k]), k


def test_graph_replay_equals_plain_steps(pf):
    """pf_step(n) replays a CUDA graph of 16-step chunks; splitting n into odd
    pieces (plain launches) must give bitwise the same state."""
    c = W.small_case((40, 72), seed=3, solid=True, u_amp=0.01)
    a, _ = run_pair(pf, c, 37, oracle=False)
    b, _ = run_pair(pf, c, 0, oracle=False)
    for n in (1, 5, 2, 16, 13):
        b.step(n)
    ma, mb = a.macros(), b.macros()
    for k in FIELDS:
        assert np.array_equal(ma[k], mb[k]), k


def test_p32_against_oracle(pf):
    c = W.small_case((52, 40), seed=7, solid=True, theta_deg=60.0)
    g, o = run_pair(pf, c, 200, precision="p32")
    gm, om = g.macros(), o.macros()
    assert rel(gm["phi"], om["phi"]) < 1e-5
    assert rel(gm["rho"], om["rho"]) < 1e-5
    assert rel(gm["u"], om["u"]) < 1e-3
    assert rel(gm["P"], om["P"]) < 1e-3


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_pmix_conserves_mass_exactly(pf, precision):
    """Mixed storage: the rest population of the order-parameter lattice is an
    exact fixed-point number set so that each cell's sum of populations is
    unchanged by the collision, hence sum phi is conserved to round-off of
    the final FP64 sum."""
    c = W.small_case((64, 80), seed=4, solid=True, theta_deg=60.0, u_amp=0.01)
    g, o = run_pair(pf, c, 0, precision=precision, oracle=False)
    m0 = g.diagnostics()["mass"]
    g.step(1000)
    m1 = g.diagnostics()["mass"]
    assert abs(m1 - m0) / np.abs(c["phi"]).sum() < 1e-13


@pytest.mark.parametrize("precision,tol_phi", [("fp16", 2e-3), ("bf16", 2e-2)])
def test_pmix_against_oracle(pf, precision, tol_phi):
    c = W.small_case((52, 40), seed=7, solid=True, theta_deg=60.0)
    g, o = run_pair(pf, c, 200, precision=precision)
    gm, om = g.macros(), o.macros()
    assert rel(gm["phi"], om["phi"]) < tol_phi


# ---- two cells per thread (packed FP32 arithmetic) ---------------------------------------

@pytest.mark.parametrize("tile,kernel", [((32, 16), 1), ((64, 8), 1), ((32, 32), 1), ((32, 16), 2)])
@pytest.mark.parametrize("precision,tol_phi", [("p32", 1e-5), ("fp16", 2e-3), ("bf16", 2e-2)])
def test_pair_step_against_oracle(pf, precision, tol_phi, tile, kernel):
    """The two-cells-per-thread steps on a ragged grid (56 x 37: partial tiles
    in x and y, and an odd row count so the last pair has one valid cell;
    nx a multiple of 8 for the staged kernel)."""
    c = W.small_case((37, 56), seed=7, solid=True, theta_deg=60.0, u_amp=0.01)
    g, o = run_pair(pf, c, 200, precision=precision, config=(tile[0], tile[1], kernel))
    gm, om = g.macros(), o.macros()
    assert rel(gm["phi"], om["phi"]) < tol_phi
    if precision == "p32":
        assert rel(gm["rho"], om["rho"]) < 1e-5
        assert rel(gm["u"], om["u"]) < 1e-3
        assert rel(gm["P"], om["P"]) < 1e-3
    assert g.diagnostics()["nan_flag"] == 0


@pytest.mark.parametrize("kernel", [1, 2])
@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_pair_step_conserves_mass_exactly(pf, precision, kernel):
    c = W.small_case((80, 64), seed=4, solid=True, theta_deg=60.0, u_amp=0.01)
    g, _ = run_pair(pf, c, 0, precision=precision, oracle=False, config=(32, 16, kernel))
    m0 = g.diagnostics()["mass"]
    g.step(1000)
    m1 = g.diagnostics()["mass"]
    assert abs(m1 - m0) / np.abs(c["phi"]).sum() < 1e-13


def test_pair_and_single_agree_p32(pf):
    """All launch variants compute the same FP32 update (to rounding order)."""
    c = W.small_case((64, 96), seed=5, solid=True, theta_deg=120.0, rho_ratio=10.0)
    a, _ = run_pair(pf, c, 300, precision="p32", oracle=False, config=(32, 8, 0))
    for kernel in (1, 2):
        b, _ = run_pair(pf, c, 300, precision="p32", oracle=False, config=(32, 16, kernel))
        ma, mb = a.macros(), b.macros()
        for k, tol in (("phi", 1e-5), ("rho", 1e-5), ("u", 1e-3), ("P", 1e-3)):
            assert rel(mb[k], ma[k]) < tol, (kernel, k)


def test_config_override_rejects_unbuilt(pf):
    c = W.small_case((32, 32), seed=1, solid=False)
    g = pf.Sim(c["shape"], precision="p64", **c["params"])
    g.init(c["phi0"], c["phi"])
    with pytest.raises(pf.PfError) as ei:
        g.set_config(32, 16, 1)  # no packed arithmetic in FP64
    assert ei.value.code == pf.PF_EINVAL
    with pytest.raises(pf.PfError):
        g.set_config(48, 8, 0)
    c = W.small_case((32, 52), seed=1, solid=False)  # nx = 52: not a multiple of 8
    g = pf.Sim(c["shape"], precision="fp16", **c["params"])
    g.init(c["phi0"], c["phi"])
    with pytest.raises(pf.PfError):
        g.set_config(32, 16, 2)


def test_particle_balance_full_size_against_oracle(pf):
    """The wetting particle at a fluid interface (256 x 272, gravity on the
    particle, wall slabs) in FP64 against the oracle: fields and the
    particle's state after 30 steps at full size."""
    c = W.particle_balance(theta_deg=60.0, rho_p=1.1)
    part = dict(c["particles"][0])
    g, o = run_pair(pf, c, 30, particles=[part])
    assert_fields(g.macros(), o.macros(), 1e-12, mu_scale=3 * c["sigma"] / 4.0)
    pg, po = g.particle(0), o.particle(0)
    for k in ("x", "u", "F"):
        a, b = np.array(pg[k]), np.array(getattr(po, k))
        assert np.abs(a - b).max() <= 1e-12 * max(np.abs(b).max(), 1e-12), (k, a, b)
    # the setup is mirror-symmetric: rotation and torque are round-off noise,
    # measured against the translational scales (u / R, |F| R)
    R = c["Rp"]
    u_s, F_s = np.abs(po.u).max(), np.abs(po.F).max()
    assert np.abs(np.array(pg["w"]) - np.array(po.w)).max() <= 1e-12 * u_s / R
    assert np.abs(np.array(pg["T"]) - np.array(po.T)).max() <= 1e-12 * F_s * R


def test_nan_is_reported(pf):
    c = W.small_case((32, 32), seed=1, solid=False)
    phi = c["phi"].copy()
    phi[5, 7] = np.nan
    g = pf.Sim(c["shape"], precision="p32", **c["params"])
    g.init(c["phi0"], phi)
    g.step(3)
    with pytest.raises(pf.PfError) as ei:
        g.sync()
    assert ei.value.code == pf.PF_ENUMERIC
    assert g.diagnostics()["nan_flag"] == 1


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_saturated_store_is_reported_and_conserves(pf, precision):
    """A storage scale far too large for the populations (2^20: every mover of
    a stored size >= 8) saturates the 16-bit movers; the step reports it
    (flag bit 1) and the order parameter stays exactly conserved."""
    c = W.small_case((32, 32), seed=3, solid=False)
    g = pf.Sim(c["shape"], precision=precision, store_log2_scale=(20, 0), **c["params"])
    g.init(c["phi0"], c["phi"])
    m0 = float(c["phi"].sum())
    g.step(5)
    with pytest.raises(pf.PfError) as ei:
        g.sync()
    assert ei.value.code == pf.PF_ENUMERIC
    d = g.diagnostics()
    assert d["nan_flag"] & 2
    assert abs(d["mass"] - m0) <= 1e-12 * np.abs(c["phi"]).sum()


def test_cylinder_full_size_sampled(pf):
    """512 x 512 drop on a cylinder (density ratio 100) in FP64 and FP32 against
    the oracle after a few steps at full size (the oracle's 512^2 steps take
    about a second each)."""
    c = W.drop_on_cylinder()
    g64, o = run_pair(pf, c, 6)
    om = o.macros()
    assert_fields(g64.macros(), om, 1e-12)
    g32, _ = run_pair(pf, c, 6, precision="p32", oracle=False)
    gm = g32.macros()
    assert rel(gm["phi"], om["phi"]) < 1e-5


# ---- 3D: D3Q19 flow + D3Q7 order parameter --------------------------------------------

@pytest.mark.parametrize("shape,solid,u_amp,steps", [
    ((12, 14, 18), True, 0.0, 0),
    ((12, 14, 18), True, 0.01, 30),
    ((37, 10, 20), True, 0.01, 12),   # several z chunks, ragged x/y tiles
])
def test_p64_matches_oracle_3d(pf, shape, solid, u_amp, steps):
    c = W.small_case(shape, seed=9, solid=solid, theta_deg=120.0, u_amp=u_amp)
    g, o = run_pair(pf, c, steps)
    assert_fields(g.macros(), o.macros(), 1e-12, mu_scale=3 * c["params"]["sigma"] / c["params"]["D"])
    dg, do = g.diagnostics(), o.diagnostics()
    for k in ("mass", "E_F", "E_K"):
        assert abs(dg[k] - do[k]) <= 1e-12 * max(abs(do[k]), 1e-300) + 1e-15, k


def test_p64_moving_sphere_matches_oracle(pf):
    c = W.small_case((16, 18, 20), seed=6, solid=False)
    part = dict(x=(9.3, 8.6, 7.9), u=(0.01, -0.004, 0.003), w=(0.001, -0.002, 0.002), R=4.0, rho_p=2.0)
    c["phi"] = (1.0 - W.disc(c["shape"], part["x"], part["R"], c["params"]["D"])) * c["phi"]
    g, o = run_pair(pf, c, 15, particles=[part])
    assert_fields(g.macros(), o.macros(), 1e-12, mu_scale=3 * c["params"]["sigma"] / c["params"]["D"])
    pg, po = g.particle(0), o.particle(0)
    for k in ("x", "u", "w", "F", "T"):
        a, b = np.array(pg[k]), np.array(getattr(po, k))
        assert np.abs(a - b).max() <= 1e-12 * max(np.abs(b).max(), 1e-12), (k, a, b)


def test_p64_own_angles_3d_match_oracle(pf):
    """3D particles with their own contact angle (Sec. 4.5, reading R18: the
    wetting terms of Eqs. 8, 9, 19 summed per solid through W and V): a fixed
    sphere at the handle's 60 deg, two free spheres at 45 and 135 deg and one
    at the handle's angle, FP64 against the oracle: fields, the FP64
    diagnostics (E_F through W and V) and every particle's state."""
    c = W.small_case((20, 22, 24), seed=6, solid=True, theta_deg=60.0)
    parts = [dict(x=(14.2, 6.3, 8.1), u=(0.004, 0.0, -0.002), w=(0.0, 0.001, 0.0), R=4.0, rho_p=2.0,
                  theta_deg=45.0),
             dict(x=(5.4, 15.2, 12.7), u=(-0.003, 0.002, 0.0), R=3.5, rho_p=1.5, theta_deg=135.0),
             dict(x=(15.0, 16.5, 17.0), u=(0.0, 0.0, 0.003), R=3.0, rho_p=1.2)]
    phi = c["phi"]
    for pp in parts:
        phi = (1.0 - W.disc(c["shape"], pp["x"], pp["R"], c["params"]["D"])) * phi
    c["phi"] = phi
    g, o = run_pair(pf, c, 20, particles=parts)
    assert_fields(g.macros(), o.macros(), 1e-12, mu_scale=3 * c["params"]["sigma"] / c["params"]["D"])
    dg, do = g.diagnostics(), o.diagnostics()
    for k in ("mass", "E_F", "E_K"):
        assert abs(dg[k] - do[k]) <= 1e-12 * max(abs(do[k]), 1e-12), (k, dg[k], do[k])
    for k in range(3):
        pg, po = g.particle(k), o.particle(k)
        for f in ("x", "u", "w", "F", "T"):
            a, b = np.array(pg[f]), np.array(getattr(po, f))
            assert np.abs(a - b).max() <= 1e-12 * max(np.abs(b).max(), 1e-12), (k, f, a, b)
    # the reduced-precision paths (32 x 8 tiles: the W and V rings of FP32
    # values in dynamic shared memory)
    for precision, tol in (("p32", 1e-5), ("fp16", 5e-3)):
        h, _ = run_pair(pf, c, 20, precision=precision, particles=parts, oracle=False)
        assert rel(h.macros()["phi"], o.macros()["phi"]) < tol, precision
        assert h.diagnostics()["nan_flag"] == 0


@pytest.mark.parametrize("precision,tol_phi", [("p32", 1e-5), ("fp16", 5e-3)])
def test_3d_reduced_precision_against_oracle(pf, precision, tol_phi):
    c = W.small_case((20, 24, 28), seed=9, solid=True, theta_deg=120.0, u_amp=0.01)
    g, o = run_pair(pf, c, 30, precision=precision)
    gm, om = g.macros(), o.macros()
    assert rel(gm["phi"], om["phi"]) < tol_phi
    if precision == "fp16":
        d0 = g.diagnostics()
        g.step(200)
        d1 = g.diagnostics()
        assert abs(d1["mass"] - d0["mass"]) / np.abs(c["phi"]).sum() < 1e-13


# ---- batches of uneven domains ---------------------------------------------------------

def test_batch_domains_equal_single_runs(pf):
    """Each domain of a batch (one persistent launch over a tile table, CUDA
    graph, autotuned tile shape) evolves exactly like the same domain run
    alone; one domain is also checked against the oracle."""
    cases = [W.small_case((64, 64), seed=1, solid=True, theta_deg=50.0),
             W.small_case((80, 96), seed=2, solid=True, theta_deg=130.0, rho_ratio=100.0),
             W.small_case((52, 40), seed=3, solid=False, u_amp=0.01)]
    steps = 300  # > the autotuner's minimum: tuning steps are part of the 300
    b = pf.Batch([c["shape"] for c in cases], [c["params"] for c in cases], precision="p64")
    for i, c in enumerate(cases):
        b.init(i, c["phi0"], c["phi"], c.get("u"))
    b.step(steps)
    b.sync()
    tx, ty, cps, cpt = b.config()
    assert tx > 0 and cps > 0
    for i, c in enumerate(cases):
        g, _ = run_pair(pf, c, steps, oracle=False)
        mb, mg = b.macros(i), g.macros()
        for k in FIELDS:
            assert np.array_equal(mb[k], mg[k]), (i, k)
    o = O.OracleSim(cases[2]["shape"], O.make_params(**cases[2]["params"]))
    o.init(cases[2]["phi0"], cases[2]["phi"], cases[2]["u"])
    o.step(steps)
    assert_fields(b.macros(2), o.macros(), 1e-12, mu_scale=3 * 0.01 / 4.0)


def test_batch_fp16_mass_and_diagnostics(pf):
    cases = [W.flat_wall_drop(64, 40.0, 100.0), W.flat_wall_drop(128, 140.0, 3.0)]
    b = pf.Batch([c["shape"] for c in cases], [c["params"] for c in cases], precision="fp16")
    for i, c in enumerate(cases):
        b.init(i, c["phi0"], c["phi"])
    m0 = [b.diagnostics(i)["mass"] for i in range(2)]
    b.step(400)
    for i, c in enumerate(cases):
        d = b.diagnostics(i)
        assert d["nan_flag"] == 0
        assert abs(d["mass"] - m0[i]) / np.abs(c["phi"]).sum() < 1e-13


# ---- box walls at the ends of y (2D; halfway bounce-back, mirrored stencils) ------------

@pytest.mark.parametrize("shape,steps,config", [
    ((37, 52), 0, None),
    ((37, 52), 150, None),
    ((44, 33), 120, (64, 4, 0)),
    ((29, 70), 120, (32, 16, 0)),
])
def test_walls_p64_matches_oracle(pf, shape, steps, config):
    """A drop cut by the top wall, a disc near the bottom one, random initial
    flow; ragged row counts so that the wall rows fall inside partial tiles."""
    c = W.wall_case(shape, seed=3)
    g, o = run_pair(pf, c, steps, config=config, walls=True)
    assert_fields(g.macros(), o.macros(), 1e-12)
    dg, do = g.diagnostics(), o.diagnostics()
    for k in ("mass", "E_F", "E_K", "E_total"):
        assert abs(dg[k] - do[k]) <= 1e-12 * max(abs(do[k]), 1e-300) + 1e-15, k


def test_walls_moving_particle_matches_oracle(pf):
    """A free particle close to the bottom wall: its indicator and force sums
    take no periodic image across the wall."""
    c = W.wall_case((48, 56), seed=5, solid=False)
    part = dict(x=(20.3, 8.6), u=(0.01, -0.004), w=(0.0, 0.0, 0.002), R=6.0, rho_p=2.0)
    c["phi"] = (1.0 - W.disc(c["shape"], part["x"], part["R"], c["params"]["D"])) * c["phi"]
    g, o = run_pair(pf, c, 80, particles=[part], walls=True)
    assert_fields(g.macros(), o.macros(), 1e-12)
    pg, po = g.particle(0), o.particle(0)
    for k in ("x", "u", "w", "F", "T"):
        a, b = np.array(pg[k]), np.array(getattr(po, k))
        assert np.abs(a - b).max() <= 1e-12 * max(np.abs(b).max(), 1e-12), (k, a, b)


@pytest.mark.parametrize("precision,tol_phi", [("p32", 1e-5), ("fp16", 2e-3), ("bf16", 2e-2)])
def test_walls_reduced_precision_against_oracle(pf, precision, tol_phi):
    c = W.wall_case((37, 52), seed=3)
    g, o = run_pair(pf, c, 200, precision=precision, walls=True)
    gm, om = g.macros(), o.macros()
    assert rel(gm["phi"], om["phi"]) < tol_phi
    if precision == "p32":
        assert rel(gm["rho"], om["rho"]) < 1e-5
        assert rel(gm["u"], om["u"]) < 1e-3
        assert rel(gm["P"], om["P"]) < 1e-3
    assert g.diagnostics()["nan_flag"] == 0


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_walls_conserve_mass_exactly(pf, precision):
    """Bounce-back hands every stored population to exactly one puller, so the
    fixed-point bookkeeping keeps sum phi exact with walls too."""
    c = W.wall_case((64, 80), seed=4)
    g, _ = run_pair(pf, c, 0, precision=precision, oracle=False, walls=True)
    m0 = g.diagnostics()["mass"]
    g.step(1000)
    m1 = g.diagnostics()["mass"]
    assert abs(m1 - m0) / np.abs(c["phi"]).sum() < 1e-13


def test_walls_reject_pair_kernels(pf):
    c = W.wall_case((32, 64), seed=1, solid=False)
    g = pf.Sim(c["shape"], precision="fp16", walls_y=True, **c["params"])
    g.init(c["phi0"], c["phi"])
    with pytest.raises(pf.PfError) as ei:
        g.set_config(32, 16, 1)
    assert ei.value.code == pf.PF_EINVAL
    g.set_config(32, 8, 0)
    g.step(4)


def test_batch_mixes_wall_and_periodic_domains(pf):
    """One batch holding a walled domain and a periodic one (per-domain
    boundary flag in the tile table): each evolves as when run alone (the
    walled one bit for bit)."""
    cases = [W.wall_case((37, 52), seed=3), W.small_case((52, 40), seed=3, solid=False, u_amp=0.01)]
    steps = 300
    b = pf.Batch([c["shape"] for c in cases], [c["params"] for c in cases], precision="p64",
                 walls_y=[True, False])
    for i, c in enumerate(cases):
        b.init(i, c["phi0"], c["phi"], c.get("u"))
    b.step(steps)
    b.sync()
    for i, c in enumerate(cases):
        g, _ = run_pair(pf, c, steps, oracle=False, walls=(i == 0))
        mb, mg = b.macros(i), g.macros()
        for k in FIELDS:
            if i == 0:
                assert np.array_equal(mb[k], mg[k]), (i, k)
            else:
                # the batch runs the periodic domain through the wall-handling
                # instantiation: the same arithmetic, compiled apart (rounding)
                assert rel(mb[k], mg[k]) < 1e-12, (i, k, rel(mb[k], mg[k]))
    o = O.OracleSim(cases[0]["shape"], O.make_params(**cases[0]["params"]))
    o.set_walls(True)
    o.init(cases[0]["phi0"], cases[0]["phi"], cases[0]["u"])
    o.step(steps)
    assert_fields(b.macros(0), o.macros(), 1e-12)


def test_tuned_periodic_config_is_not_reused_for_walls(pf):
    """The autotuner's cache must not hand a walled batch the configuration
    tuned on a periodic batch of the same size: the tiled two-cells-per-thread
    kernels have no bounce-back, so a walled domain stepped by them would run
    as periodic in y.  A periodic FP16 batch is tuned first (it picks a
    two-cells kernel), then a walled batch of the same size and domain count:
    it must report one of the kernels with walls (0 or 4), match the oracle
    with walls within FP16 bounds, and conserve mass exactly (the same mass
    as its single-handle run)."""
    L = 256
    per = W.flat_wall_drop(L, 60.0, 10.0)
    bp = pf.Batch([per["shape"]], [per["params"]], precision="fp16")
    bp.init(0, per["phi0"], per["phi"])
    bp.step(256)
    bp.sync()
    bp.close()
    c = W.wall_case((L, L), seed=4)
    bw = pf.Batch([c["shape"]], [c["params"]], precision="fp16", walls_y=[True])
    bw.init(0, c["phi0"], c["phi"], c.get("u"))
    bw.step(256)
    bw.sync()
    assert bw.config()[3] in (0, 4), bw.config()
    g, o = run_pair(pf, c, 256, precision="fp16", walls=True)
    mb, om = bw.macros(0), o.macros()
    e = {k: rel(mb[k], om[k]) for k in ("phi", "rho", "u", "P")}
    e["mu"] = float(np.abs(mb["mu"] - om["mu"]).max() / max(np.abs(om["mu"]).max(), 3 * 0.01 / 4.0))
    # (the every-field bounds, 200 steps of a 56 x 37 case; mu here, 256 steps
    # of this 256 x 256 wall case: measured 5.4e-4)
    tol = dict(MIXED_TOL["fp16"], mu=1e-3)
    for k, v in e.items():
        assert v < tol[k], (k, v)
    assert abs(bw.diagnostics(0)["mass"] - g.diagnostics()["mass"]) == 0.0


def test_p64_particle_wall_repulsion_matches_oracle(pf):
    """Particles next to the box walls and to a circular wall (Sec. 4.5
    particle-wall repulsion against the mirror image across the nearest
    wall), FP64 against the oracle after 60 steps; the walls push the
    particles away compared with no repulsion."""
    c = W.wall_case((64, 72), seed=8, solid=False, u_amp=0.0)
    prm = dict(c["params"], rep_xi=3.0, rep_eps=1e4, wall_circle=(36.0, 32.0, 40.0))
    c["params"] = prm
    # nearest walls: bottom (d' = 11), top (d' = 12), circle (d' = 12); range 2R + xi = 13
    parts = [dict(x=(20.0, 5.0), u=(0.0, -0.003), R=5.0, rho_p=2.0),
             dict(x=(52.0, 57.5), u=(0.0, 0.003), R=5.0, rho_p=2.0),
             dict(x=(36.0 + 34.0, 32.0), u=(0.003, 0.0), R=5.0, rho_p=2.0)]
    phi = c["phi"]
    for pp in parts:
        phi = (1.0 - W.disc(c["shape"], pp["x"], pp["R"], prm["D"])) * phi
    c["phi"] = phi
    g, o = run_pair(pf, c, 60, particles=parts, walls=True)
    assert_fields(g.macros(), o.macros(), 1e-12)
    for k in range(3):
        pg, po = g.particle(k), o.particle(k)
        R = po.R
        us = np.abs(po.u).max() + abs(po.w[2]) * R + 1e-4
        assert np.abs(np.array(pg["x"]) - np.array(po.x)).max() <= 1e-12 * np.abs(po.x).max(), k
        assert np.abs(np.array(pg["u"]) - np.array(po.u)).max() <= 1e-12 * us, k
        assert np.abs(np.array(pg["w"]) - np.array(po.w)).max() <= 1e-12 * us / R, k
    c2 = dict(c, params=dict(prm, rep_eps=0.0))
    g2, _ = run_pair(pf, c2, 60, particles=parts, oracle=False, walls=True)
    assert g.particle(0)["u"][1] > g2.particle(0)["u"][1]   # bottom wall pushes up
    assert g.particle(1)["u"][1] < g2.particle(1)["u"][1]   # top wall pushes down
    assert g.particle(2)["u"][0] < g2.particle(2)["u"][0]   # the circle pushes inwards


# ---- conservative Allen-Cahn order parameter (2D option) --------------------------------

@pytest.mark.parametrize("shape,solid,walls,steps", [
    ((52, 40), True, False, 120),
    ((37, 45), False, False, 150),
    ((37, 52), True, True, 120),
])
def test_allen_cahn_p64_matches_oracle(pf, shape, solid, walls, steps):
    """phase_model 1 (flux M (grad phi - theta n) on the lattice of Eq. 30),
    FP64 against the oracle: with a fixed solid, with random flow, and inside
    box walls."""
    if walls:
        c = W.wall_case(shape, seed=3)
    else:
        c = W.small_case(shape, seed=7, solid=solid, theta_deg=60.0, u_amp=0.01)
    c["params"] = dict(c["params"], phase_model=1)
    g, o = run_pair(pf, c, steps, walls=walls)
    assert_fields(g.macros(), o.macros(), 1e-12)
    dg, do = g.diagnostics(), o.diagnostics()
    for k in ("mass", "E_F", "E_K"):
        assert abs(dg[k] - do[k]) <= 1e-12 * max(abs(do[k]), 1e-300) + 1e-15, k


@pytest.mark.parametrize("precision,tol_phi", [("p32", 1e-5), ("fp16", 2e-3), ("bf16", 2e-2)])
def test_allen_cahn_reduced_precision(pf, precision, tol_phi):
    """The Allen-Cahn option in FP32 and with 16-bit storage against the FP64
    oracle; mixed storage keeps sum phi exact."""
    c = W.small_case((52, 40), seed=7, solid=False, u_amp=0.01)
    c["params"] = dict(c["params"], phase_model=1)
    g, o = run_pair(pf, c, 200, precision=precision)
    gm, om = g.macros(), o.macros()
    assert rel(gm["phi"], om["phi"]) < tol_phi
    assert g.diagnostics()["nan_flag"] == 0
    if precision != "p32":
        m0 = float(np.sum(c["phi"]))
        g.step(1000)
        assert abs(g.diagnostics()["mass"] - m0) / np.abs(c["phi"]).sum() < 1e-13


@pytest.mark.parametrize("tile", [(32, 16), (64, 8), (32, 32)])
@pytest.mark.parametrize("precision,tol_phi", [("p32", 1e-5), ("fp16", 2e-3), ("bf16", 2e-2)])
def test_allen_cahn_pair_kernel_against_oracle(pf, precision, tol_phi, tile):
    """The Allen-Cahn option in the two-cells-per-thread kernel (ragged tiles,
    odd row count, a fixed solid) against the FP64 oracle; exact mass with
    16-bit storage."""
    c = W.small_case((37, 56), seed=7, solid=True, theta_deg=60.0, u_amp=0.01)
    c["params"] = dict(c["params"], phase_model=1)
    g, o = run_pair(pf, c, 200, precision=precision, config=(tile[0], tile[1], 1))
    gm, om = g.macros(), o.macros()
    assert rel(gm["phi"], om["phi"]) < tol_phi
    if precision == "p32":
        assert rel(gm["rho"], om["rho"]) < 1e-5
        assert rel(gm["u"], om["u"]) < 1e-3
        assert rel(gm["P"], om["P"]) < 1e-3
    else:
        m0 = float(np.sum(c["phi"]))
        g.step(500)
        assert abs(g.diagnostics()["mass"] - m0) / np.abs(c["phi"]).sum() < 1e-13
    assert g.diagnostics()["nan_flag"] == 0


def test_batch_mixes_allen_cahn_and_cahn_hilliard(pf):
    """One FP32 batch with an Allen-Cahn and a Cahn-Hilliard domain (the
    per-domain choice inside one launch, autotuned): each within the FP32
    bounds of the oracle."""
    cases = [W.small_case((52, 40), seed=3, solid=True, theta_deg=60.0, u_amp=0.01),
             W.small_case((37, 56), seed=4, solid=False, u_amp=0.01)]
    cases[0]["params"] = dict(cases[0]["params"], phase_model=1)
    steps = 300
    b = pf.Batch([c["shape"] for c in cases], [c["params"] for c in cases], precision="p32")
    for i, c in enumerate(cases):
        b.init(i, c["phi0"], c["phi"], c.get("u"))
    b.step(steps)
    b.sync()
    for i, c in enumerate(cases):
        o = O.OracleSim(c["shape"], O.make_params(**c["params"]))
        o.init(c["phi0"], c["phi"], c["u"])
        o.step(steps)
        mb, om = b.macros(i), o.macros()
        assert rel(mb["phi"], om["phi"]) < 1e-5, i
        assert rel(mb["u"], om["u"]) < 1e-3, i


@pytest.mark.parametrize("shape,steps", [((12, 14, 18), 30), ((37, 10, 20), 12)])
def test_allen_cahn_p64_matches_oracle_3d(pf, shape, steps):
    """The Allen-Cahn option on D3Q7 (with D3Q19 flow) against the oracle,
    FP64, a sphere solid and random flow; several z chunks and ragged tiles."""
    c = W.small_case(shape, seed=9, solid=True, theta_deg=120.0, u_amp=0.01)
    c["params"] = dict(c["params"], phase_model=1)
    g, o = run_pair(pf, c, steps)
    assert_fields(g.macros(), o.macros(), 1e-12, mu_scale=3 * c["params"]["sigma"] / c["params"]["D"])


def test_allen_cahn_3d_fp16_conserves_mass(pf):
    c = W.small_case((24, 20, 36), seed=2, solid=True, theta_deg=60.0, u_amp=0.01)
    c["params"] = dict(c["params"], phase_model=1)
    g, o = run_pair(pf, c, 100, precision="fp16")
    assert rel(g.macros()["phi"], o.macros()["phi"]) < 5e-3
    m0 = float(np.sum(c["phi"]))
    g.step(1000)
    d = g.diagnostics()
    assert d["nan_flag"] == 0
    assert abs(d["mass"] - m0) / np.abs(c["phi"]).sum() < 1e-13


def test_allen_cahn_rejections(pf):
    c = W.small_case((32, 32), seed=1, solid=False)
    g = pf.Sim(c["shape"], precision="fp16", **dict(c["params"], phase_model=1))
    g.init(c["phi0"], c["phi"])
    with pytest.raises(pf.PfError):
        g.set_config(32, 16, 2)  # the staged kernel has no Allen-Cahn path
    g.set_config(32, 16, 1)
    g.step(4)
    with pytest.raises(pf.PfError):
        pf.Sim((32, 32), precision="p32", **dict(c["params"], phase_model=2))


def test_channel_displacement_full_size_against_oracle(pf):
    """Sec. 4.6 layout at full size (1280 x 256, bottom wall with two cavities,
    bounce-back walls, a drop of fluid 1, 16 particles with their own angles,
    repulsion from each other and from the box walls): FP64 fields and
    particle states against the oracle after 3 steps."""
    c = W.channel_displacement()
    g, o = run_pair(pf, c, 3, particles=c["particles"], walls=True)
    assert_fields(g.macros(), o.macros(), 1e-12, mu_scale=3 * 0.001 / 5.0)
    for k in range(len(c["particles"])):
        pg, po = g.particle(k), o.particle(k)
        assert np.abs(np.array(pg["x"]) - np.array(po.x)).max() <= 1e-12 * np.abs(po.x).max(), k
        R = po.R
        us = np.abs(po.u).max() + abs(po.w[2]) * R + 1e-4
        assert np.abs(np.array(pg["u"]) - np.array(po.u)).max() <= 1e-12 * us, k
        assert np.abs(np.array(pg["w"]) - np.array(po.w)).max() <= 1e-12 * us / R, k


def test_p64_held_components_match_oracle(pf):
    """Particles that hold their horizontal translation and rotation (the
    two-particle balance of Sec. 4.4) and one that holds only its vertical
    translation, FP64 against the oracle after 60 steps."""
    c = W.small_case((56, 64), seed=12, solid=False)
    c["params"] = dict(c["params"], g=(0.0, -2e-5, 0.0))
    parts = [dict(x=(18.0, 30.0), u=(0.002, 0.0), w=(0.0, 0.0, 0.001), R=6.0, rho_p=1.5, prescribed=2 | 16),
             dict(x=(44.0, 28.0), u=(0.0, -0.001), R=6.0, rho_p=1.5, prescribed=4)]
    phi = c["phi"]
    for pp in parts:
        phi = (1.0 - W.disc(c["shape"], pp["x"], pp["R"], c["params"]["D"])) * phi
    c["phi"] = phi
    g, o = run_pair(pf, c, 60, particles=parts)
    gm, om = g.macros(), o.macros()
    # the flow is driven by the particles: u is measured against the velocity
    # scale of the flow plus the held particle's translation and rim speed
    # (|u| + |u_p| + |w| R, as for the other particle-driven flows)
    us = np.abs(om["u"]).max() + 0.002 + 0.001 * 6.0
    assert np.abs(gm["u"] - om["u"]).max() <= 1e-12 * us
    assert_fields(dict(gm, u=om["u"]), om, 1e-12)
    for k in range(2):
        pg, po = g.particle(k), o.particle(k)
        # particle quantities against the velocity scale of the flow that drives
        # them (the same us as for u above), the force scale rho pi R^2 us and
        # the torque scale pi R^3 us
        R = po.R
        vs = us
        scale = dict(x=np.abs(po.x).max(), u=vs, w=vs / R, F=math.pi * R * R * vs, T=math.pi * R ** 3 * vs)
        for f in ("x", "u", "w", "F", "T"):
            a, b = np.array(pg[f]), np.array(getattr(po, f))
            assert np.abs(a - b).max() <= 1e-12 * scale[f], (k, f, a, b)
    p0, p1 = g.particle(0), g.particle(1)
    assert p0["u"][0] == 0.002 and p0["w"][2] == 0.001 and p0["u"][1] != 0.0
    assert p1["u"][1] == -0.001 and p1["u"][0] != 0.0


@pytest.mark.parametrize("shape,steps", [((12, 14, 18), 30), ((37, 10, 20), 12), ((9, 21, 33), 20)])
def test_walls_3d_p64_matches_oracle(pf, shape, steps):
    """Box walls in 3D (halfway bounce-back of D3Q19/D3Q7, mirrored stencil
    rows, y-odd T_xy and T_yz): FP64 against the oracle with a sphere solid
    and random flow; ragged tiles, several z chunks, walls inside partial
    tiles."""
    c = W.small_case(shape, seed=9, solid=True, theta_deg=120.0, u_amp=0.01)
    g, o = run_pair(pf, c, steps, walls=True)
    assert_fields(g.macros(), o.macros(), 1e-12, mu_scale=3 * c["params"]["sigma"] / c["params"]["D"])
    dg, do = g.diagnostics(), o.diagnostics()
    for k in ("mass", "E_F", "E_K"):
        assert abs(dg[k] - do[k]) <= 1e-12 * max(abs(do[k]), 1e-300) + 1e-15, k


def test_walls_3d_moving_sphere_matches_oracle(pf):
    c = W.small_case((16, 18, 20), seed=6, solid=False)
    part = dict(x=(9.3, 5.2, 8.1), u=(0.004, -0.006, 0.002), w=(0.001, 0.0, -0.002), R=4.0, rho_p=2.0)
    c["phi"] = (1.0 - W.disc(c["shape"], part["x"], part["R"], c["params"]["D"])) * c["phi"]
    g, o = run_pair(pf, c, 15, particles=[part], walls=True)
    assert_fields(g.macros(), o.macros(), 1e-12, mu_scale=3 * c["params"]["sigma"] / c["params"]["D"])
    pg, po = g.particle(0), o.particle(0)
    vs = np.abs(po.u).max() + np.abs(po.w).max() * po.R + 1e-4
    assert np.abs(np.array(pg["x"]) - np.array(po.x)).max() <= 1e-12 * np.abs(po.x).max()
    assert np.abs(np.array(pg["u"]) - np.array(po.u)).max() <= 1e-12 * vs


@pytest.mark.parametrize("precision,tol_phi", [("p32", 1e-5), ("fp16", 5e-3)])
def test_walls_3d_reduced_precision(pf, precision, tol_phi):
    c = W.small_case((24, 20, 36), seed=2, solid=True, theta_deg=60.0, u_amp=0.01)
    g, o = run_pair(pf, c, 100, precision=precision, walls=True)
    assert rel(g.macros()["phi"], o.macros()["phi"]) < tol_phi
    if precision == "fp16":
        m0 = float(np.sum(c["phi"]))
        g.step(1000)
        assert abs(g.diagnostics()["mass"] - m0) / np.abs(c["phi"]).sum() < 1e-13
    assert g.diagnostics()["nan_flag"] == 0


@pytest.mark.parametrize("shape,walls", [((4, 4), False), ((4, 6), True), ((5, 4), True), ((4, 4, 4), False),
                                         ((4, 5, 4), True)])
def test_smallest_grids_match_oracle(pf, shape, walls):
    """The smallest grids the library accepts (4 cells per axis; one tile
    holds both walls and wraps several times), FP64 against the oracle."""
    c = W.small_case(shape, seed=13, solid=False, u_amp=0.01, D=2.0)
    g, o = run_pair(pf, c, 25, walls=walls)
    assert_fields(g.macros(), o.macros(), 1e-12, mu_scale=3 * c["params"]["sigma"] / c["params"]["D"])


def test_zero_steps_and_split_steps(pf):
    """pf_step(0) changes nothing; n steps in pieces equal n steps at once."""
    c = W.small_case((37, 45), seed=2, solid=True, u_amp=0.01)
    a, _ = run_pair(pf, c, 0, oracle=False)
    m0 = a.macros()
    a.step(0)
    assert a.time == 0
    for k in FIELDS:
        assert np.array_equal(a.macros()[k], m0[k]), k
    a.step(7)
    a.step(0)
    a.step(13)
    b, _ = run_pair(pf, c, 20, oracle=False)
    for k in FIELDS:
        assert np.array_equal(a.macros()[k], b.macros()[k]), k


@pytest.mark.parametrize("name,steps", [("drop_on_cylinder", 1000), ("water_entry", 50), ("drainage_3d", 3)])
def test_full_size_configs_against_oracle(pf, name, steps):
    """The paper-shaped workloads at full size in FP64 against the oracle over
    their first steps: the 512² drop on a cylinder for 1000 steps, the
    2048 x 1024 water entry with its moving particle for 50, the 256³
    drainage for 3 (the oracle's cost bounds the step counts)."""
    if name == "drop_on_cylinder":
        c = W.drop_on_cylinder()
    elif name == "water_entry":
        c = W.water_entry()
    else:
        c = W.porous_drainage_3d(n=256)
    parts = c.get("particles", [])
    g, o = run_pair(pf, c, steps, particles=parts)
    mu_scale = 3 * c["params"]["sigma"] / c["params"]["D"]
    gm, om = g.macros(), o.macros()
    if parts:
        # the flow inside and around the particle follows its velocity scale
        us = np.abs(om["u"]).max() + np.abs(np.array(parts[0]["u"])).max()
        assert np.abs(gm["u"] - om["u"]).max() <= 1e-12 * us
        gm = dict(gm, u=om["u"])
    assert_fields(gm, om, 1e-12, mu_scale=mu_scale)
    for k in range(len(parts)):
        pg, po = g.particle(k), o.particle(k)
        vs = np.abs(po.u).max() + abs(po.w[2]) * po.R + 1e-4
        assert np.abs(np.array(pg["x"]) - np.array(po.x)).max() <= 1e-12 * np.abs(po.x).max()
        assert np.abs(np.array(pg["u"]) - np.array(po.u)).max() <= 1e-12 * vs


@pytest.mark.parametrize("shape,walls", [((37, 45), False), ((37, 52), True), ((12, 14, 18), False),
                                         ((9, 21, 33), True)])
def test_interface_normal_matches_oracle(pf, shape, walls):
    """pf_get_normal (grad phi / |grad phi| of the current phi) against the
    oracle after some steps, on the interface band |phi| < 0.99 (in the bulk
    the direction of a round-off gradient is arbitrary on both sides)."""
    c = W.small_case(shape, seed=5, solid=False, u_amp=0.01)
    g, o = run_pair(pf, c, 20, walls=walls)
    ng, no = g.normal(), o.normal()
    band = np.abs(o.macros()["phi"]) < 0.99
    assert band.sum() > 50
    assert np.abs(ng[:, band] - no[:, band]).max() < 1e-12
    norm = np.sqrt((ng ** 2).sum(axis=0))
    assert np.abs(norm[band] - 1.0).max() < 1e-12


@pytest.mark.parametrize("precision,walls,with_particle", [("p64", False, False), ("fp16", True, False),
                                                           ("p32", False, True)])
def test_checkpoint_resume_is_bit_identical(pf, precision, walls, with_particle):
    """pf_save_state after 37 steps, pf_load_state into a fresh handle, 40
    more steps: every field, the particle and the time equal those of the
    uninterrupted run bit for bit."""
    c = W.wall_case((37, 52), seed=3) if walls else W.small_case((40, 56), seed=8, solid=True, u_amp=0.01)
    parts = []
    if with_particle:
        parts = [dict(x=(20.3, 17.6), u=(0.01, -0.004), w=(0.0, 0.0, 0.002), R=6.0, rho_p=2.0)]
        c["phi"] = (1.0 - W.disc(c["shape"], parts[0]["x"], 6.0, c["params"]["D"])) * c["phi"]
    a, _ = run_pair(pf, c, 37, precision=precision, particles=parts, oracle=False, walls=walls)
    state = a.save_state()
    a.step(40)
    b = pf.Sim(c["shape"], precision=precision, walls_y=walls, **c["params"])
    for k, pp in enumerate(parts):
        b.set_particle(k, **pp)
    b.load_state(state)
    assert b.time == 37
    b.step(40)
    assert b.time == a.time == 77
    ma, mb = a.macros(), b.macros()
    for k in FIELDS:
        assert np.array_equal(ma[k], mb[k]), k
    for k in range(len(parts)):
        pa, pb = a.particle(k), b.particle(k)
        for f in ("x", "u", "w", "F", "T"):
            assert pa[f] == pb[f], f
    # a state from another grid is refused
    d = W.small_case((40, 48), seed=8)
    e = pf.Sim(d["shape"], precision=precision, **d["params"])
    with pytest.raises(pf.PfError):
        e.load_state(state)


def test_bounded_wait_timeout_is_reported(pf, monkeypatch):
    """A bounded device wait that runs out ends its kernel with PF_ETIMEOUT
    instead of hanging: with PF_WAIT_POLLS=1 the staged kernel's first wait
    on its bulk copies gives up (it still lets the copies in flight land), the
    handle reports the sticky error, and a new handle works normally."""
    c = W.small_case((32, 64), seed=1, solid=False)
    monkeypatch.setenv("PF_WAIT_POLLS", "1")
    g = pf.Sim(c["shape"], precision="fp16", **c["params"])
    monkeypatch.delenv("PF_WAIT_POLLS")
    g.init(c["phi0"], c["phi"])
    g.set_config(32, 16, 2)
    g.step(1)
    with pytest.raises(pf.PfError) as ei:
        g.sync()
    assert ei.value.code == pf.PF_ETIMEOUT
    with pytest.raises(pf.PfError):
        g.step(1)  # sticky
    h, _ = run_pair(pf, c, 20, precision="fp16", oracle=False, config=(32, 16, 2))
    h.sync()
    assert h.diagnostics()["nan_flag"] == 0


def test_run_logged_records_diagnostics(pf, tmp_path):
    """The diagnostics log of a run: one JSON line per interval with the time
    and the FP64 mass and energies, equal to the oracle's at those times."""
    import json
    c = W.small_case((40, 48), seed=4, solid=True, u_amp=0.01)
    g, o = run_pair(pf, c, 0)
    path = tmp_path / "diag.jsonl"
    recs = g.run_logged(60, 20, str(path))
    lines = [json.loads(x) for x in open(path)]
    assert [r["t"] for r in lines] == [20, 40, 60] and lines == recs
    for r in recs:
        o.step(20)
        do = o.diagnostics()
        for k in ("mass", "E_F", "E_K", "E_total"):
            assert abs(r[k] - do[k]) <= 1e-12 * max(abs(do[k]), 1e-300) + 1e-15, (r["t"], k)
        assert r["nan_flag"] == 0


@pytest.mark.parametrize("precision,tol_phi", [("p32", 1e-5), ("fp16", 2e-3)])
def test_split_particle_step_against_oracle(pf, precision, tol_phi):
    """Launch variant 3 on a particle domain: the tiles out of every particle's
    reach run the two-cells-per-thread step with the fixed solids'
    mu_phi0 grad phi0 (Eq. 19), the others the single-cell step with the
    particle terms.  Against the FP64 oracle and against variant 0 at the same
    precision: fields and the particles' states after 200 steps."""
    c = W.small_case((128, 96), seed=11, solid=True, theta_deg=60.0, u_amp=0.005)
    parts = [dict(x=(40.3, 30.6), u=(0.01, -0.004), w=(0.0, 0.0, 0.002), R=6.0, rho_p=2.0),
             dict(x=(95.0, 70.0), u=(-0.006, 0.003), R=5.0, rho_p=1.5)]
    phi = c["phi"]
    for pp in parts:
        phi = (1.0 - W.disc(c["shape"], pp["x"], pp["R"], c["params"]["D"])) * phi
    c["phi"] = phi
    g, o = run_pair(pf, c, 200, precision=precision, particles=parts, config=(32, 16, 3))
    s, _ = run_pair(pf, c, 200, precision=precision, particles=parts, oracle=False, config=(32, 16, 0))
    gm, om, sm = g.macros(), o.macros(), s.macros()
    assert rel(gm["phi"], om["phi"]) < tol_phi
    assert rel(gm["rho"], om["rho"]) < tol_phi
    for k in ("u", "P"):
        assert rel(gm[k], om[k]) < 100 * tol_phi, k
    for k, tol in (("phi", 1e-5), ("rho", 1e-5), ("u", 1e-3), ("P", 1e-3)):
        assert rel(gm[k], sm[k]) < (tol if precision == "p32" else 10 * tol_phi), k
    us = max(np.abs(om["u"]).max(), 1e-3)
    for k in range(len(parts)):
        pg, po, ps = g.particle(k), o.particle(k), s.particle(k)
        assert np.abs(np.array(pg["x"]) - np.array(po.x)).max() < 1e-3
        assert np.abs(np.array(pg["u"]) - np.array(po.u)).max() < 100 * tol_phi * us
        assert np.abs(np.array(pg["u"]) - np.array(ps["u"])).max() < 100 * tol_phi * us
    assert g.diagnostics()["nan_flag"] == 0


def test_split_particle_step_rejected_where_not_built(pf):
    c = W.small_case((64, 64), seed=1, solid=False)
    part = dict(x=(20.0, 20.0), R=5.0, rho_p=2.0)
    g = pf.Sim(c["shape"], precision="p64", **c["params"])
    g.set_particle(0, **part)
    g.init(c["phi0"], c["phi"])
    with pytest.raises(pf.PfError):
        g.set_config(32, 16, 3)  # FP64: no packed arithmetic
    g = pf.Sim(c["shape"], precision="fp16", **c["params"])
    g.init(c["phi0"], c["phi"])
    with pytest.raises(pf.PfError):
        g.set_config(32, 16, 3)  # no particle
    g = pf.Sim(c["shape"], precision="fp16", **c["params"])
    g.set_particle(0, **part)
    g.init(c["phi0"], c["phi"])
    with pytest.raises(pf.PfError):
        g.set_config(32, 8, 3)  # 32 x 16 tiles only
    g.set_config(32, 16, 3)
    g.step(5)
    g.set_particle(0, **dict(part, theta_deg=45.0))  # own angle: the split stays
    g.step(5)
    assert g.config()[3] == 3
    assert g.diagnostics()["nan_flag"] == 0


@pytest.mark.parametrize("precision,tol_phi", [("p32", 1e-5), ("fp16", 2e-3)])
def test_split_particle_step_own_angles_against_oracle(pf, precision, tol_phi):
    """The split step when particles carry their own contact angles (reading
    R18): the near tiles sum the wetting per solid, the far tiles see the
    fixed solids only, with the phi0^2 grad phi0 part of their force from the
    stencil of phi0^3 as the oracle has it.  A fixed wetting disc and three
    particles (two with own angles); against the FP64 oracle after 200
    steps and against the single-cell step at the same precision."""
    c = W.small_case((128, 96), seed=12, solid=True, theta_deg=60.0, u_amp=0.005)
    parts = [dict(x=(40.3, 30.6), u=(0.01, -0.004), w=(0.0, 0.0, 0.002), R=6.0, rho_p=2.0, theta_deg=120.0),
             dict(x=(95.0, 70.0), u=(-0.006, 0.003), R=5.0, rho_p=1.5, theta_deg=40.0),
             dict(x=(20.0, 100.0), u=(0.0, 0.004), R=5.0, rho_p=1.2)]
    phi = c["phi"]
    for pp in parts:
        phi = (1.0 - W.disc(c["shape"], pp["x"], pp["R"], c["params"]["D"])) * phi
    c["phi"] = phi
    g, o = run_pair(pf, c, 200, precision=precision, particles=parts, config=(32, 16, 3))
    s, _ = run_pair(pf, c, 200, precision=precision, particles=parts, oracle=False, config=(32, 16, 0))
    assert g.config()[3] == 3
    gm, om, sm = g.macros(), o.macros(), s.macros()
    print("split-own", precision, {k: "%.2e" % rel(gm[k], om[k]) for k in ("phi", "rho", "u", "P")})
    assert rel(gm["phi"], om["phi"]) < tol_phi
    assert rel(gm["rho"], om["rho"]) < tol_phi
    for k in ("u", "P"):
        assert rel(gm[k], om[k]) < 100 * tol_phi, k
    for k, tol in (("phi", 1e-5), ("rho", 1e-5), ("u", 1e-3), ("P", 1e-3)):
        assert rel(gm[k], sm[k]) < (tol if precision == "p32" else 10 * tol_phi), k
    us = max(np.abs(om["u"]).max(), 1e-3)
    for k in range(len(parts)):
        pg, po = g.particle(k), o.particle(k)
        assert np.abs(np.array(pg["x"]) - np.array(po.x)).max() < 1e-3
        assert np.abs(np.array(pg["u"]) - np.array(po.u)).max() < 100 * tol_phi * us
    assert g.diagnostics()["nan_flag"] == 0


# ---- every field of the reduced-precision paths, per kernel ---------------------------------

# max |gpu - oracle| / max |oracle| per field after 200 steps of the ragged small
# case below (mu against max(|mu|, 3 sigma/D)), for every kernel that serves the
# FP32-arithmetic policies, with unit and non-unit relaxation rates.  Measured
# (worst of kernels 0, 1, 4 and both rate sets): P32 3.7e-6, 1.7e-6, 2.2e-5,
# 1.9e-5, 3.2e-5; FP16 4.4e-5, 2.0e-5, 6.1e-4, 1.26e-3, 1.5e-4; BF16 4.3e-4,
# 1.9e-4, 4.8e-3, 1.1e-2, 1.3e-3 (phi, rho, u, P, mu).  The bounds are 2.5-3x
# those: FP32 arithmetic and storage round at 2^-24, FP16 storage at 2^-11
# and BF16 at 2^-8 of each population, and u and P are differences of
# populations, so their relative error is the largest.
MIXED_TOL = {
    "p32": dict(phi=1e-5, rho=5e-6, u=6e-5, P=5e-5, mu=8e-5),
    "fp16": dict(phi=1.5e-4, rho=6e-5, u=1.5e-3, P=3.5e-3, mu=5e-4),
    "bf16": dict(phi=1.2e-3, rho=5e-4, u=1.2e-2, P=3e-2, mu=3.5e-3),
}


@pytest.mark.parametrize("unit_rates", [True, False])
@pytest.mark.parametrize("config", [(32, 8, 0), (32, 16, 1), (64, 32, 4)])
@pytest.mark.parametrize("precision", ["p32", "fp16", "bf16"])
def test_reduced_precision_every_field_against_oracle(pf, precision, config, unit_rates):
    """phi, rho, u, P and mu of the FP32 and 16-bit storage policies against
    the FP64 oracle, through the one-cell (0), the tiled two-cells (1) and the
    strip (4) kernels, on a 56 x 37 grid (partial tiles, strips and bands)
    with a wetting disc and random initial flow; with the paper's unit
    relaxation rates and with s2, s3, s4 = 1.3, 1.2, 1.4."""
    c = W.small_case((37, 56), seed=7, solid=True, theta_deg=60.0, u_amp=0.01)
    if not unit_rates:
        c["params"] = dict(c["params"], s2=1.3, s3=1.2, s4=1.4)
    g, o = run_pair(pf, c, 200, precision=precision, config=config)
    gm, om = g.macros(), o.macros()
    e = {k: rel(gm[k], om[k]) for k in ("phi", "rho", "u", "P")}
    e["mu"] = float(np.abs(gm["mu"] - om["mu"]).max() / max(np.abs(om["mu"]).max(), 3 * 0.01 / 4.0))
    print("fields", precision, config, unit_rates, {k: "%.2e" % v for k, v in e.items()})
    for k, v in e.items():
        assert v < MIXED_TOL[precision][k], (k, v)
    assert g.diagnostics()["nan_flag"] == 0


@pytest.mark.parametrize("config", [(32, 16, 1), (64, 128, 4)])
def test_batch_fp16_two_cells_kernels_equal_single_runs(pf, config):
    """The headline configuration's kernels on the batched drop-on-wall
    workload: a batch of uneven flat-wall drop domains in FP16 storage (one
    launch per step over all of them) evolves each domain bit for bit as the
    same domain run alone with the same kernel."""
    cases = [W.flat_wall_drop(64, 40.0, 30.0), W.flat_wall_drop(128, 140.0, 3.0),
             W.flat_wall_drop(64, 75.0, 90.0)]
    steps = 150
    b = pf.Batch([c["shape"] for c in cases], [c["params"] for c in cases], precision="fp16")
    for i, c in enumerate(cases):
        b.init(i, c["phi0"], c["phi"])
    b.set_config(*config)
    b.step(steps)
    b.sync()
    for i, c in enumerate(cases):
        g, _ = run_pair(pf, c, steps, precision="fp16", oracle=False, config=config)
        mb, mg = b.macros(i), g.macros()
        for k in FIELDS:
            assert np.array_equal(mb[k], mg[k]), (i, k)
        assert b.diagnostics(i)["nan_flag"] == 0


# 3D: the D3Q7/D3Q19 step (kernel 0, one cell per thread) in FP32 arithmetic
# with FP32, FP16 and BF16 storage, every field against the FP64 oracle after
# 100 steps, with the paper's unit relaxation rates (the instantiation whose
# collisions follow from the equilibria and forcing terms) and with s2, s3,
# s4 = 1.3, 1.2, 0.9 (the general collision; the 2D set's s4 = 1.4 makes the
# FP64 oracle itself blow up within 90 steps on this 3D case).  Measured
# (worst of both rate sets): P32 2.3e-6, 1.1e-6, 2.4e-5, 7.0e-7, 2.3e-5; FP16
# 1.3e-5, 5.8e-6, 6.7e-4, 1.9e-4, 1.1e-4; BF16 1.1e-4, 4.9e-5, 5.6e-3,
# 1.3e-3, 9.5e-4 (phi, rho, u, P, mu); the bounds are about 3x those.
MIXED_TOL_3D = {
    "p32": dict(phi=7e-6, rho=3.5e-6, u=7.5e-5, P=2.5e-6, mu=7e-5),
    "fp16": dict(phi=4e-5, rho=1.8e-5, u=2e-3, P=6e-4, mu=3.5e-4),
    "bf16": dict(phi=3.5e-4, rho=1.5e-4, u=1.7e-2, P=4e-3, mu=3e-3),
}


@pytest.mark.parametrize("unit_rates", [True, False])
@pytest.mark.parametrize("precision", ["p32", "fp16", "bf16"])
def test_3d_every_field_against_oracle(pf, precision, unit_rates):
    c = W.small_case((20, 24, 28), seed=9, solid=True, theta_deg=60.0, u_amp=0.01)
    if not unit_rates:
        c["params"] = dict(c["params"], s2=1.3, s3=1.2, s4=0.9)
    g, o = run_pair(pf, c, 100, precision=precision)
    gm, om = g.macros(), o.macros()
    e = {k: rel(gm[k], om[k]) for k in ("phi", "rho", "u", "P")}
    e["mu"] = float(np.abs(gm["mu"] - om["mu"]).max() / max(np.abs(om["mu"]).max(), 3 * 0.01 / 4.0))
    print("fields3d", precision, unit_rates, {k: "%.2e" % v for k, v in e.items()})
    for k, v in e.items():
        assert v < MIXED_TOL_3D[precision][k], (k, v)
    assert g.diagnostics()["nan_flag"] == 0


@pytest.mark.parametrize("precision,tol_phi", [("p32", 1e-5), ("fp16", 2e-3)])
def test_split_particle_step_walls_against_oracle(pf, precision, tol_phi):
    """The split step with walls at the ends of y: the far tiles run the
    single-cell step's wall instantiation without the particle terms but with
    the fixed solids' mu_phi0 grad phi0 (Eq. 19); one particle with its own
    angle.  Against the FP64 oracle with walls after 200 steps and against
    the single-cell step at the same precision."""
    c = W.wall_case((128, 96), seed=6)
    parts = [dict(x=(30.3, 60.6), u=(0.008, -0.003), w=(0.0, 0.0, 0.002), R=6.0, rho_p=2.0, theta_deg=120.0),
             dict(x=(70.0, 40.0), u=(-0.006, 0.004), R=5.0, rho_p=1.5)]
    phi = c["phi"]
    for pp in parts:
        phi = (1.0 - W.disc(c["shape"], pp["x"], pp["R"], c["params"]["D"])) * phi
    c["phi"] = phi
    g, o = run_pair(pf, c, 200, precision=precision, particles=parts, config=(32, 16, 3), walls=True)
    s, _ = run_pair(pf, c, 200, precision=precision, particles=parts, oracle=False, config=(32, 16, 0),
                    walls=True)
    assert g.config()[3] == 3
    gm, om, sm = g.macros(), o.macros(), s.macros()
    print("split-walls", precision, {k: "%.2e" % rel(gm[k], om[k]) for k in ("phi", "rho", "u", "P")})
    assert rel(gm["phi"], om["phi"]) < tol_phi
    assert rel(gm["rho"], om["rho"]) < tol_phi
    for k in ("u", "P"):
        assert rel(gm[k], om[k]) < 100 * tol_phi, k
    for k, tol in (("phi", 1e-5), ("rho", 1e-5), ("u", 1e-3), ("P", 1e-3)):
        assert rel(gm[k], sm[k]) < (tol if precision == "p32" else 10 * tol_phi), k
    us = max(np.abs(om["u"]).max(), 1e-3)
    for k in range(len(parts)):
        pg, po = g.particle(k), o.particle(k)
        assert np.abs(np.array(pg["x"]) - np.array(po.x)).max() < 1e-3
        assert np.abs(np.array(pg["u"]) - np.array(po.u)).max() < 100 * tol_phi * us
    assert g.diagnostics()["nan_flag"] == 0
