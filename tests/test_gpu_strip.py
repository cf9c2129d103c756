"""The strip step (kernel 4): two cells per thread on strips of 64 columns
marched in y, every input staged in shared memory by tensor copies, periodic
wrap in x through ghost columns.  Parity with the FP64 oracle on ragged
grids (partial strips, partial bands, partial segments, a domain narrower
than two ghost widths), exact mass with 16-bit storage, independence of the
segment length, agreement with the other two-cells kernel, ghost refill
after other kernels and after a checkpoint load, batches of uneven domains,
and a bounded wait that runs out."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_05097_gb300 import workloads as W

from test_gpu_parity import FIELDS, rel, run_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    from paper_2311_05097_gb300 import build
    build.build()
    from paper_2311_05097_gb300 import pf as _pf
    _pf.load()
    return _pf


# per-field bounds (max |gpu - oracle| / max |oracle|) after 200 steps: FP32
# storage, and 16-bit storage of the populations (FP16: 11 significant bits,
# BF16: 8) with FP32 arithmetic.  Measured on the five cases below (worst):
# P32 4.0e-6, 1.8e-6, 1.3e-5, 5.7e-6, 2.9e-5; FP16 5.4e-5, 2.5e-5, 6.9e-4,
# 2.0e-3, 2.5e-4; BF16 4.1e-4, 1.8e-4, 5.2e-3, 1.3e-2, 2.4e-3 (phi, rho, u, P,
# mu); the bounds are about 3x those.
TOL = {
    "p32": dict(phi=1.2e-5, rho=6e-6, u=5e-5, P=2e-5, mu=1e-4),
    "fp16": dict(phi=1.6e-4, rho=8e-5, u=2e-3, P=6e-3, mu=8e-4),
    "bf16": dict(phi=1.2e-3, rho=6e-4, u=1.6e-2, P=4e-2, mu=7e-3),
}


def field_errors(gm, om, mu_scale):
    e = {k: rel(gm[k], om[k]) for k in ("phi", "rho", "u", "P")}
    e["mu"] = float(np.abs(gm["mu"] - om["mu"]).max() / max(np.abs(om["mu"]).max(), mu_scale))
    return e


@pytest.mark.parametrize("shape,seg,rates", [((37, 136), 16, None), ((70, 96), 128, None), ((64, 64), 8, None),
                                             ((24, 10), 8, None), ((70, 96), 32, (1.3, 1.2, 1.4))])
@pytest.mark.parametrize("precision", ["p32", "fp16", "bf16"])
def test_strip_step_against_oracle(pf, precision, shape, seg, rates):
    """Ragged grids: 136 columns (two full strips and one of 8), 37 rows in
    segments of 16 (the last one partial, its last band partial); 96 x 70 in
    one segment (a partial strip and a partial band); 64 x 64 in eight
    one-band segments; 10 x 24 (every cell is copied into a ghost column on
    both sides).  The first four have the paper's unit relaxation rates (the
    instantiation that builds the order-parameter collision from the
    macroscopic fields); the last sets s2, s3, s4 = 1.3, 1.2, 1.4 (the general
    instantiation)."""
    c = W.small_case(shape, seed=7, solid=True, theta_deg=60.0, u_amp=0.01)
    if rates is not None:
        c["params"] = dict(c["params"], s2=rates[0], s3=rates[1], s4=rates[2])
    g, o = run_pair(pf, c, 200, precision=precision, config=(64, seg, 4))
    assert g.config()[3] == 4
    e = field_errors(g.macros(), o.macros(), 3 * c["params"]["sigma"] / c["params"]["D"])
    print("strip", precision, shape, seg, e)
    for k, v in e.items():
        assert v < TOL[precision][k], (k, v)
    assert g.diagnostics()["nan_flag"] == 0


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_strip_conserves_mass_exactly(pf, precision):
    c = W.small_case((80, 128), seed=4, solid=True, theta_deg=60.0, u_amp=0.01)
    g, _ = run_pair(pf, c, 0, precision=precision, oracle=False, config=(64, 32, 4))
    m0 = g.diagnostics()["mass"]
    g.step(1000)
    d = g.diagnostics()
    assert d["nan_flag"] == 0
    assert abs(d["mass"] - m0) / np.abs(c["phi"]).sum() < 1e-13


def test_strip_segments_are_bit_identical(pf):
    """Every cell computes phi, mu and w from the same inputs whether its row
    starts a segment or not: the segment length does not change the result."""
    c = W.small_case((70, 96), seed=3, solid=True, theta_deg=120.0, u_amp=0.01)
    a, _ = run_pair(pf, c, 150, precision="fp16", oracle=False, config=(64, 8, 4))
    b, _ = run_pair(pf, c, 150, precision="fp16", oracle=False, config=(64, 256, 4))
    ma, mb = a.macros(), b.macros()
    for k in FIELDS:
        assert np.array_equal(ma[k], mb[k]), k


def test_strip_and_pair_agree_p32(pf):
    """The strip step and the tiled two-cells step compute the same FP32
    update (to rounding order of the stencil sums)."""
    c = W.small_case((64, 96), seed=5, solid=True, theta_deg=120.0, rho_ratio=10.0)
    a, _ = run_pair(pf, c, 300, precision="p32", oracle=False, config=(32, 16, 1))
    b, _ = run_pair(pf, c, 300, precision="p32", oracle=False, config=(64, 128, 4))
    ma, mb = a.macros(), b.macros()
    for k, tol in (("phi", 1e-5), ("rho", 1e-5), ("u", 1e-3), ("P", 1e-3)):
        assert rel(mb[k], ma[k]) < tol, k


def test_strip_refills_ghosts_after_other_kernels(pf):
    """Steps of another kernel leave the ghost columns stale; switching to the
    strip step refills them first (a stale ghost would corrupt the columns
    next to x = 0 and x = nx - 1)."""
    c = W.small_case((64, 96), seed=6, solid=True, theta_deg=60.0, u_amp=0.01)
    a, _ = run_pair(pf, c, 100, precision="p32", oracle=False, config=(32, 16, 1))
    a.step(100)
    b, _ = run_pair(pf, c, 100, precision="p32", oracle=False, config=(32, 16, 1))
    b.set_config(64, 128, 4)
    b.step(100)
    ma, mb = a.macros(), b.macros()
    for k, tol in (("phi", 1e-5), ("rho", 1e-5), ("u", 1e-3), ("P", 1e-3)):
        assert rel(mb[k], ma[k]) < tol, k


def test_strip_resume_after_load_is_bit_identical(pf):
    """A checkpoint holds no ghost columns: the loaded handle refills them
    before its first strip step, and continues bit for bit."""
    c = W.small_case((70, 96), seed=8, solid=True, theta_deg=60.0, u_amp=0.01)
    a, _ = run_pair(pf, c, 120, precision="fp16", oracle=False, config=(64, 128, 4))
    b, _ = run_pair(pf, c, 60, precision="fp16", oracle=False, config=(64, 128, 4))
    st = b.save_state()
    h = pf.Sim(c["shape"], precision="fp16", **c["params"])
    h.init(c["phi0"], c["phi"])
    h.set_config(64, 128, 4)
    h.load_state(st)
    h.step(60)
    ma, mh = a.macros(), h.macros()
    for k in FIELDS:
        assert np.array_equal(ma[k], mh[k]), k


def test_batch_strip_equals_single_runs(pf):
    """A batch of uneven domains in one strip launch: each domain evolves
    exactly as when run alone with the same kernel; one against the oracle."""
    cases = [W.flat_wall_drop(64, 40.0, 30.0), W.flat_wall_drop(128, 140.0, 3.0),
             W.small_case((70, 96), seed=3, solid=True, theta_deg=120.0, u_amp=0.01)]
    steps = 200
    b = pf.Batch([c["shape"] for c in cases], [c["params"] for c in cases], precision="fp16")
    for i, c in enumerate(cases):
        b.init(i, c["phi0"], c["phi"], c.get("u"))
    b.set_config(64, 32, 4)
    b.step(steps)
    b.sync()
    for i, c in enumerate(cases):
        g, _ = run_pair(pf, c, steps, precision="fp16", oracle=False, config=(64, 32, 4))
        mb, mg = b.macros(i), g.macros()
        for k in FIELDS:
            assert np.array_equal(mb[k], mg[k]), (i, k)
    c = cases[2]
    o = O.OracleSim(c["shape"], O.make_params(**c["params"]))
    o.init(c["phi0"], c["phi"], c["u"])
    o.step(steps)
    e = field_errors(b.macros(2), o.macros(), 3 * c["params"]["sigma"] / c["params"]["D"])
    for k, v in e.items():
        assert v < TOL["fp16"][k], (k, v)


def test_headline_configuration_against_oracle(pf):
    """The batched benchmark's own configuration: drops on a flat wall slab
    (wetting angles 40, 140 and 75 deg, density ratios 30, 3 and 100, s0 = 1.6,
    unit rates otherwise), FP16 storage, one strip launch with 192-row
    segments (the 256 x 256 domain takes two segments per strip): every field
    of every domain against the FP64 oracle after 200 steps, within the FP16
    bounds of the strip step (measured worst: phi 3.4e-6, rho 1.3e-6,
    u 3.8e-4, P 6.4e-4, mu 1.9e-5)."""
    cases = [W.flat_wall_drop(64, 40.0, 30.0), W.flat_wall_drop(128, 140.0, 3.0),
             W.flat_wall_drop(256, 75.0, 100.0)]
    steps = 200
    b = pf.Batch([c["shape"] for c in cases], [c["params"] for c in cases], precision="fp16")
    b.init_all([c["phi0"] for c in cases], [c["phi"] for c in cases])
    b.set_config(64, 192, 4)
    b.step(steps)
    b.sync()
    assert b.config()[3] == 4
    assert b.diagnostics(0)["nan_flag"] == 0
    mb = b.macros_all()
    for i, c in enumerate(cases):
        o = O.OracleSim(c["shape"], O.make_params(**c["params"]))
        o.init(c["phi0"], c["phi"])
        o.step(steps)
        e = field_errors(mb[i], o.macros(), 3 * c["params"]["sigma"] / c["params"]["D"])
        print("headline case", i, {k: "%.2e" % v for k, v in e.items()})
        for k, v in e.items():
            assert v < TOL["fp16"][k], (i, k, v)


def test_strip_rejected_where_not_built(pf):
    """FP64 (no packed arithmetic), odd nx and a strip width other than 64
    are refused."""
    c = W.small_case((32, 64), seed=1, solid=False)
    g = pf.Sim(c["shape"], precision="p64", **c["params"])
    g.init(c["phi0"], c["phi"])
    with pytest.raises(pf.PfError):
        g.set_config(64, 128, 4)  # FP64: no packed arithmetic
    c = W.small_case((32, 65), seed=1, solid=False)
    g = pf.Sim(c["shape"], precision="fp16", **c["params"])
    g.init(c["phi0"], c["phi"])
    with pytest.raises(pf.PfError):
        g.set_config(64, 128, 4)  # odd nx
    c = W.small_case((32, 64), seed=1, solid=False)
    g = pf.Sim(c["shape"], precision="fp16", **c["params"])
    g.init(c["phi0"], c["phi"])
    with pytest.raises(pf.PfError):
        g.set_config(32, 128, 4)  # tile_x is the strip width, 64


def test_strip_bounded_wait_timeout_is_reported(pf, monkeypatch):
    """With PF_WAIT_POLLS=1 the strip step's first wait on its tensor copies
    gives up: the copies in flight still land (a second wait with the default
    bound), the kernel ends, the handle reports PF_ETIMEOUT, and a new handle
    works normally."""
    c = W.small_case((32, 64), seed=1, solid=False)
    monkeypatch.setenv("PF_WAIT_POLLS", "1")
    g = pf.Sim(c["shape"], precision="fp16", **c["params"])
    monkeypatch.delenv("PF_WAIT_POLLS")
    g.init(c["phi0"], c["phi"])
    g.set_config(64, 128, 4)
    g.step(1)
    with pytest.raises(pf.PfError) as ei:
        g.sync()
    assert ei.value.code == pf.PF_ETIMEOUT
    h, _ = run_pair(pf, c, 20, precision="fp16", oracle=False, config=(64, 128, 4))
    h.sync()
    assert h.diagnostics()["nan_flag"] == 0


# ---- walls at the ends of y (halfway bounce-back, mirrored stencil rows) ------------------------

@pytest.mark.parametrize("shape,seg,rates", [((37, 136), 16, None), ((70, 96), 128, None), ((5, 64), 8, None),
                                             ((24, 10), 8, None), ((37, 96), 16, (1.3, 1.2, 1.4))])
@pytest.mark.parametrize("precision", ["p32", "fp16", "bf16"])
def test_strip_walls_against_oracle(pf, precision, shape, seg, rates):
    """The wall case (a drop cut by the top wall, a disc near the bottom one,
    random initial flow) through the strip step: 37 rows in segments of 16
    (the top wall inside a partial band of a partial segment), 70 rows in one
    segment, 5 rows (fewer than a band: one band reaches beyond both walls),
    10 columns (every cell is also a ghost); unit rates and s2, s3, s4 = 1.3,
    1.2, 1.4."""
    c = W.wall_case(shape, seed=3)
    if rates is not None:
        c["params"] = dict(c["params"], s2=rates[0], s3=rates[1], s4=rates[2])
    g, o = run_pair(pf, c, 200, precision=precision, config=(64, seg, 4), walls=True)
    assert g.config()[3] == 4
    e = field_errors(g.macros(), o.macros(), 3 * c["params"]["sigma"] / c["params"]["D"])
    print("strip-walls", precision, shape, seg, rates, {k: "%.2e" % v for k, v in e.items()})
    for k, v in e.items():
        assert v < TOL[precision][k], (k, v)
    assert g.diagnostics()["nan_flag"] == 0


def test_strip_walls_agree_with_one_cell_kernel_p32(pf):
    """FP32 with walls: the strip step and the one-cell step (kernel 0, which
    has its own wall code) agree to rounding order."""
    c = W.wall_case((70, 96), seed=4)
    a, _ = run_pair(pf, c, 300, precision="p32", oracle=False, config=(32, 8, 0), walls=True)
    b, _ = run_pair(pf, c, 300, precision="p32", oracle=False, config=(64, 32, 4), walls=True)
    ma, mb = a.macros(), b.macros()
    for k, tol in (("phi", 1e-5), ("rho", 1e-5), ("u", 1e-3), ("P", 1e-3)):
        assert rel(mb[k], ma[k]) < tol, k


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_strip_walls_conserve_mass_exactly(pf, precision):
    c = W.wall_case((64, 80), seed=4)
    g, _ = run_pair(pf, c, 0, precision=precision, oracle=False, config=(64, 16, 4), walls=True)
    m0 = g.diagnostics()["mass"]
    g.step(1000)
    d = g.diagnostics()
    assert d["nan_flag"] == 0
    assert abs(d["mass"] - m0) / np.abs(c["phi"]).sum() < 1e-13


def test_strip_walls_segments_are_bit_identical(pf):
    c = W.wall_case((70, 96), seed=5)
    a, _ = run_pair(pf, c, 150, precision="fp16", oracle=False, config=(64, 8, 4), walls=True)
    b, _ = run_pair(pf, c, 150, precision="fp16", oracle=False, config=(64, 256, 4), walls=True)
    ma, mb = a.macros(), b.macros()
    for k in FIELDS:
        assert np.array_equal(ma[k], mb[k]), k


def test_batch_strip_mixes_wall_and_periodic_domains(pf):
    """A walled and a periodic domain in one strip launch (the wall
    instantiation serves both): each bit-identical to its single run with the
    same kernel and boundary."""
    cases = [W.wall_case((37, 52), seed=3), W.small_case((52, 40), seed=3, solid=True, u_amp=0.01)]
    steps = 200
    b = pf.Batch([c["shape"] for c in cases], [c["params"] for c in cases], precision="fp16",
                 walls_y=[True, False])
    for i, c in enumerate(cases):
        b.init(i, c["phi0"], c["phi"], c.get("u"))
    b.set_config(64, 32, 4)
    b.step(steps)
    b.sync()
    for i, c in enumerate(cases):
        g, _ = run_pair(pf, c, steps, precision="fp16", oracle=False, config=(64, 32, 4), walls=(i == 0))
        mb, mg = b.macros(i), g.macros()
        for k in FIELDS:
            assert np.array_equal(mb[k], mg[k]), (i, k)


def test_single_handle_autotune(pf):
    """pf_autotune times the candidates on a single simulation's live state:
    an even number of real steps (one more from an odd step), a kernel the
    handle can run, the oracle's result to the FP16 bounds 50 steps later,
    exact mass; a second handle of the same kind takes the
    cached choice without stepping."""
    c = W.small_case((96, 128), seed=2, solid=True, theta_deg=60.0, u_amp=0.01)
    g = pf.Sim(c["shape"], precision="fp16", **c["params"])
    g.init(c["phi0"], c["phi"], c["u"])
    m0 = g.diagnostics()["mass"]
    g.step(1)
    n = g.autotune()
    assert n > 0 and n % 2 == 1, n
    cfg = g.config()
    assert cfg[3] in (0, 1, 4), cfg
    g.step(50)
    o = O.OracleSim(c["shape"], O.make_params(**c["params"]))
    o.init(c["phi0"], c["phi"], c["u"])
    o.step(1 + n + 50)
    e = field_errors(g.macros(), o.macros(), 3 * c["params"]["sigma"] / c["params"]["D"])
    for k, v in e.items():
        assert v < TOL["fp16"][k], (k, v)
    assert abs(g.diagnostics()["mass"] - m0) / np.abs(c["phi"]).sum() < 1e-13
    h = pf.Sim(c["shape"], precision="fp16", **c["params"])
    h.init(c["phi0"], c["phi"], c["u"])
    assert h.autotune() == 0
    assert h.config() == cfg


def test_batch_init_all_and_macros_all_equal_per_domain_calls(pf):
    """pf_batch_init_all / pf_batch_get_macros_all (one wait for all domains)
    give the same state and fields as the per-domain calls, bit for bit."""
    cases = [W.flat_wall_drop(64, 40.0, 30.0), W.flat_wall_drop(128, 140.0, 3.0),
             W.small_case((70, 96), seed=3, solid=True, theta_deg=120.0, u_amp=0.01)]
    shapes = [c["shape"] for c in cases]
    params = [c["params"] for c in cases]
    a = pf.Batch(shapes, params, precision="fp16")
    for i, c in enumerate(cases):
        a.init(i, c["phi0"], c["phi"], c.get("u"))
    b = pf.Batch(shapes, params, precision="fp16")
    b.init_all([c["phi0"] for c in cases], [c["phi"] for c in cases],
               [c.get("u") if c.get("u") is not None else None for c in cases])
    for x in (a, b):
        x.set_config(64, 32, 4)
        x.step(40)
        x.sync()
    mb = b.macros_all()
    for i in range(len(cases)):
        ma = a.macros(i)
        for k in FIELDS:
            assert np.array_equal(ma[k], mb[i][k]), (i, k)


@pytest.mark.parametrize("ring", [None, "20000"])
def test_batch_init_all_copy_stream_and_device_inputs(pf, monkeypatch, ring):
    """pf_batch_init_all stages host inputs on its copy stream (the default
    ring, and one so small that it wraps at every domain, where the copy
    stream first waits for the kernels of the domains before) and reads
    device inputs in place; pf_batch_get_macros_all alternates two macro
    buffers (five domains: each reused).  Every field equals the per-domain
    calls' bit for bit."""
    import torch
    cases = [W.flat_wall_drop(64, 40.0, 30.0), W.flat_wall_drop(128, 140.0, 3.0),
             W.small_case((70, 96), seed=3, solid=True, theta_deg=120.0, u_amp=0.01),
             W.flat_wall_drop(64, 90.0, 10.0),
             W.small_case((40, 72), seed=4, solid=False, u_amp=0.02)]
    shapes = [c["shape"] for c in cases]
    params = [c["params"] for c in cases]
    us = [c.get("u") for c in cases]
    a = pf.Batch(shapes, params, precision="fp16")
    for i, c in enumerate(cases):
        a.init(i, c["phi0"], c["phi"], us[i])
    if ring:
        monkeypatch.setenv("PF_INIT_RING", ring)
    b = pf.Batch(shapes, params, precision="fp16")
    if ring:
        monkeypatch.delenv("PF_INIT_RING")
    b.init_all([c["phi0"] for c in cases], [c["phi"] for c in cases], us)
    d = pf.Batch(shapes, params, precision="fp16")
    dev = lambda x: None if x is None else torch.from_numpy(np.ascontiguousarray(x)).cuda()
    t0, t1, tu = ([dev(c["phi0"]) for c in cases], [dev(c["phi"]) for c in cases], [dev(x) for x in us])
    torch.cuda.synchronize()
    d.init_all(t0, t1, tu)
    for x in (a, b, d):
        x.set_config(64, 32, 4)
        x.step(30)
        x.sync()
    mb, md = b.macros_all(), d.macros_all()
    for i in range(len(cases)):
        ma = a.macros(i)
        for k in FIELDS:
            assert np.array_equal(ma[k], mb[i][k]), ("host", i, k)
            assert np.array_equal(ma[k], md[i][k]), ("device", i, k)
