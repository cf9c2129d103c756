"""pf_diagnostics_noalloc: FP64 diagnostics for callers that may not allocate
device memory (stream-captured work, fixed-budget loops, hosts whose device
memory belongs to another allocator).  Its scratch is a fixed device array, so
it must agree with pf_diagnostics, which uses library-allocated scratch, and
give the same answer when called twice in a row on the shared array.

Kept in its own file that pytest collects last."""
import ctypes as C

import numpy as np
import pytest

from paper_2311_05097_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    from paper_2311_05097_gb300 import build
    build.build()
    from paper_2311_05097_gb300 import pf as _pf
    _pf.load()
    return _pf


def device_fields(pf, sim, dim, N):
    import torch
    out = dict(phi=torch.empty(N, dtype=torch.float64, device="cuda"),
               rho=torch.empty(N, dtype=torch.float64, device="cuda"),
               u=torch.empty(dim * N, dtype=torch.float64, device="cuda"))
    sim.macros(out=out)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("shape,precision,walls", [((52, 40), "p64", False), ((48, 64), "fp16", False),
                                                   ((12, 14, 18), "p64", False), ((37, 52), "p64", True),
                                                   ((12, 14, 18), "p64", True)])
def test_noalloc_matches_pf_diagnostics(pf, shape, precision, walls):
    """Both entry points on the same fields, periodic boxes and boxes with
    walls at the ends of y (mirrored stencil rows in both)."""
    import torch
    if walls and len(shape) == 2:
        c = W.wall_case(shape, seed=2, solid=True, theta_deg=120.0, u_amp=0.01)
    else:
        c = W.small_case(shape, seed=2, solid=True, theta_deg=120.0, u_amp=0.01)
    sim = pf.Sim(c["shape"], precision=precision, walls_y=walls, **c["params"])
    sim.init(c["phi0"], c["phi"], c["u"])
    sim.step(25)
    ref = sim.diagnostics()
    N = int(np.prod(shape))
    dim = len(shape)
    f = device_fields(pf, sim, dim, N)
    # the library keeps the fixed indicator in the precision of its auxiliary
    # fields (FP32 unless the policy is FP64); the diagnostics read that copy
    p0 = c["phi0"] if precision == "p64" else c["phi0"].astype(np.float32).astype(np.float64)
    phi0 = torch.from_numpy(np.ascontiguousarray(p0).reshape(-1)).cuda()
    g = pf.make_grid(shape, walls_y=walls)
    p = pf.make_params(**c["params"])
    L = pf.load()
    ptr = lambda t: C.c_void_p(t.data_ptr())
    for call in range(2):  # two calls in a row share the static scratch
        host = (C.c_double * 4)()
        rc = L.pf_diagnostics_noalloc(C.byref(g), C.byref(p), ptr(f["phi"]), ptr(f["rho"]),
                                      ptr(f["u"]), ptr(phi0), host, pf.PF_HOST, None)
        assert rc == pf.PF_OK, pf.last_error()
        dev = torch.zeros(4, dtype=torch.float64, device="cuda")
        rc = L.pf_diagnostics_noalloc(C.byref(g), C.byref(p), ptr(f["phi"]), ptr(f["rho"]),
                                      ptr(f["u"]), ptr(phi0),
                                      C.cast(C.c_void_p(dev.data_ptr()), C.POINTER(C.c_double)),
                                      pf.PF_DEVICE, None)
        assert rc == pf.PF_OK, pf.last_error()
        torch.cuda.synchronize()
        d = dev.cpu().numpy()
        for k, name in enumerate(("mass", "E_F", "E_K", "E_total")):
            tol = 1e-12 * max(abs(ref[name]), 1e-300) + 1e-15
            assert abs(host[k] - ref[name]) <= tol, (call, name, host[k], ref[name])
            assert abs(d[k] - ref[name]) <= tol, (call, name, d[k], ref[name])


def test_noalloc_rejects_grids_beyond_its_scratch(pf):
    g = pf.make_grid((8192, 8193))  # 67,117,056 cells > PF_NOALLOC_MAX_CELLS
    p = pf.make_params()
    out = (C.c_double * 4)()
    L = pf.load()
    rc = L.pf_diagnostics_noalloc(C.byref(g), C.byref(p), C.c_void_p(1), C.c_void_p(1),
                                  C.c_void_p(1), C.c_void_p(1), out, pf.PF_HOST, None)
    assert rc == pf.PF_EINVAL
    assert "maximum" in pf.last_error()


def test_noalloc_rejects_unsupported_boundaries(pf):
    """Walls are accepted at the ends of y only, as in pf_create."""
    g = pf.make_grid((16, 16))
    g.periodic[0] = 0
    p = pf.make_params()
    out = (C.c_double * 4)()
    L = pf.load()
    rc = L.pf_diagnostics_noalloc(C.byref(g), C.byref(p), C.c_void_p(1), C.c_void_p(1),
                                  C.c_void_p(1), C.c_void_p(1), out, pf.PF_HOST, None)
    assert rc == pf.PF_EINVAL
    assert "periodic" in pf.last_error()
