"""Host-side checks of the C-ABI library that need no GPU: it builds for
sm_103a, loads, exports every entry point declared in include/pf.h, and
rejects invalid grids and parameters before touching the device."""
import ctypes as C
import os
import re

import pytest

from paper_2311_05097_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    from paper_2311_05097_gb300 import pf
    return pf


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pf_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("pf_create", "pf_init_fields", "pf_step", "pf_get_macros", "pf_particle_state",
              "pf_diagnostics", "pf_batch_create", "pf_batch_step", "pf_destroy", "pf_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    so = C.CDLL(lib.library_path())
    missing = [n for n in declared_symbols() if not hasattr(so, n)]
    assert not missing, missing


def test_params_default_and_validation(lib):
    p = lib.make_params()
    assert p.d0 == 0.4 and p.s0 == 1.0 and p.D == 4.0 and p.precision == lib.PF_P64
    L = lib.load()
    h = C.c_void_p()
    g = lib.make_grid((16, 16))
    bad = [dict(d0=0.6), dict(D=0.0), dict(M=-1.0), dict(rho2=0.0), dict(s3=2.0),
           dict(solid_eps=0.0), dict(mu1=0.0), dict(sigma=-0.1), dict(theta_deg=float('nan'))]
    for kw in bad:
        p = lib.make_params(**kw)
        rc = L.pf_create(C.byref(g), C.byref(p), C.byref(h))
        assert rc == lib.PF_EINVAL, kw
        assert lib.last_error() != ""
    p = lib.make_params(precision=7)
    assert L.pf_create(C.byref(g), C.byref(p), C.byref(h)) == lib.PF_EINVAL
    g2 = lib.make_grid((2, 16))
    p = lib.make_params()
    assert L.pf_create(C.byref(g2), C.byref(p), C.byref(h)) == lib.PF_EINVAL
    # walls only at the ends of y
    g3 = lib.make_grid((16, 16))
    g3.periodic[0] = 0
    assert L.pf_create(C.byref(g3), C.byref(p), C.byref(h)) == lib.PF_EINVAL
    assert "periodic" in lib.last_error()
    g3 = lib.make_grid((8, 16, 16), walls_y=True)
    g3.periodic[2] = 0
    assert L.pf_create(C.byref(g3), C.byref(p), C.byref(h)) == lib.PF_EINVAL


def test_null_handles_are_rejected(lib):
    L = lib.load()
    assert L.pf_step(None, 1) == lib.PF_EINVAL
    assert L.pf_sync(None) == lib.PF_EINVAL
    d = lib.pf_diag()
    assert L.pf_diagnostics(None, C.byref(d)) == lib.PF_EINVAL
    L.pf_destroy(None)
    L.pf_batch_destroy(None)
    assert L.pf_batch_create(0, None, None, None) == lib.PF_EINVAL
