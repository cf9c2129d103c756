"""Python binding of libpf (include/pf.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module converts
NumPy arrays / torch tensors to pointers and return codes to exceptions.
The library must have been built (``paper_2311_05097_gb300.build.build()``);
importing this module without it raises at load time -- there is no CPU
fallback.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

PF_OK, PF_EINVAL, PF_ENOMEM, PF_ECUDA, PF_ENUMERIC, PF_ETIMEOUT, PF_ESTATE = 0, -1, -2, -3, -4, -5, -6
PF_P64, PF_P32, PF_PMIX_FP16, PF_PMIX_BF16 = 0, 1, 2, 3
PF_HOST, PF_DEVICE = 0, 1
PF_MAX_PARTICLES = 64
PRECISIONS = {"p64": PF_P64, "p32": PF_P32, "fp16": PF_PMIX_FP16, "bf16": PF_PMIX_BF16}


class PfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libpf error %d: %s" % (code, msg))
        self.code = code


class pf_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("periodic", C.c_int * 3)]


class pf_params(C.Structure):
    _fields_ = [
        ("sigma", C.c_double), ("D", C.c_double), ("M", C.c_double), ("eta", C.c_double),
        ("rho1", C.c_double), ("rho2", C.c_double), ("mu1", C.c_double), ("mu2", C.c_double),
        ("d0", C.c_double), ("s0", C.c_double), ("s1", C.c_double), ("s2", C.c_double),
        ("s3", C.c_double), ("s4", C.c_double), ("theta_deg", C.c_double),
        ("Fb", C.c_double * 3), ("g", C.c_double * 3), ("solid_eps", C.c_double),
        ("rep_xi", C.c_double), ("rep_eps", C.c_double), ("wall_circle", C.c_double * 3),
        ("phase_model", C.c_int),
        ("precision", C.c_int), ("store_log2_scale", C.c_int * 2), ("stream", C.c_void_p),
    ]


class pf_particle(C.Structure):
    _fields_ = [("x", C.c_double * 3), ("u", C.c_double * 3), ("w", C.c_double * 3),
                ("R", C.c_double), ("rho_p", C.c_double), ("theta_deg", C.c_double),
                ("F", C.c_double * 3), ("T", C.c_double * 3), ("prescribed", C.c_int)]


class pf_diag(C.Structure):
    _fields_ = [("mass", C.c_double), ("E_F", C.c_double), ("E_K", C.c_double),
                ("E_total", C.c_double), ("nan_flag", C.c_int)]


_lib = None
_DP = C.POINTER(C.c_double)


def library_path():
    return _build.LIB


def load(build_if_missing=False):
    """Load libpf.so; raises if it is missing (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError("libpf.so is not built (%s); run paper_2311_05097_gb300.build.build()"
                               % path)
    L = C.CDLL(path)
    vp = C.c_void_p
    sig = {
        "pf_params_default": (C.c_int, [C.POINTER(pf_params)]),
        "pf_create": (C.c_int, [C.POINTER(pf_grid), C.POINTER(pf_params), C.POINTER(vp)]),
        "pf_init_fields": (C.c_int, [vp, vp, vp, vp, vp, C.c_int]),
        "pf_step": (C.c_int, [vp, C.c_int64]),
        "pf_autotune": (C.c_int, [vp, C.POINTER(C.c_int64)]),
        "pf_get_macros": (C.c_int, [vp, vp, vp, vp, vp, vp, C.c_int]),
        "pf_get_normal": (C.c_int, [vp, vp, C.c_int]),
        "pf_state_size": (C.c_int, [vp, C.POINTER(C.c_int64)]),
        "pf_save_state": (C.c_int, [vp, vp, C.c_int64]),
        "pf_load_state": (C.c_int, [vp, vp, C.c_int64]),
        "pf_particle_state": (C.c_int, [vp, C.c_int, C.POINTER(pf_particle), C.c_int]),
        "pf_num_particles": (C.c_int, [vp]),
        "pf_diagnostics": (C.c_int, [vp, C.POINTER(pf_diag)]),
        "pf_sync": (C.c_int, [vp]),
        "pf_time": (C.c_int64, [vp]),
        "pf_destroy": (None, [vp]),
        "pf_last_error": (C.c_char_p, []),
        "pf_batch_create": (C.c_int, [C.c_int, C.POINTER(pf_grid), C.POINTER(pf_params), C.POINTER(vp)]),
        "pf_batch_init": (C.c_int, [vp, C.c_int, vp, vp, vp, vp, C.c_int]),
        "pf_batch_step": (C.c_int, [vp, C.c_int64]),
        "pf_batch_get_macros": (C.c_int, [vp, C.c_int, vp, vp, vp, vp, vp, C.c_int]),
        "pf_batch_init_all": (C.c_int, [vp, vp, vp, vp, vp, C.c_int]),
        "pf_batch_get_macros_all": (C.c_int, [vp, vp, vp, vp, vp, vp, C.c_int]),
        "pf_batch_diagnostics": (C.c_int, [vp, C.c_int, C.POINTER(pf_diag)]),
        "pf_batch_sync": (C.c_int, [vp]),
        "pf_batch_cells": (C.c_int64, [vp]),
        "pf_get_config": (C.c_int, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                    C.POINTER(C.c_int)]),
        "pf_batch_config": (C.c_int, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                      C.POINTER(C.c_int)]),
        "pf_batch_set_config": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, C.c_int]),
        "pf_set_config": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, C.c_int]),
        "pf_batch_destroy": (None, [vp]),
        "pf_launch_count": (C.c_int64, []),
        "pf_diagnostics_noalloc": (C.c_int, [C.POINTER(pf_grid), C.POINTER(pf_params), vp, vp, vp, vp,
                                             C.POINTER(C.c_double), C.c_int, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(rc):
    if rc != PF_OK:
        raise PfError(rc, load().pf_last_error().decode())
    return rc


def last_error():
    return load().pf_last_error().decode()


def launch_count():
    return int(load().pf_launch_count())


def make_params(precision=PF_P64, stream=None, **kw):
    """pf_params from keyword arguments (library defaults for the rest)."""
    p = pf_params()
    _check(load().pf_params_default(C.byref(p)))
    for k, v in kw.items():
        if k in ("Fb", "g", "wall_circle"):
            v = tuple(v) + (0.0,) * (3 - len(v))
            setattr(p, k, (C.c_double * 3)(*v))
        elif k == "store_log2_scale":
            setattr(p, k, (C.c_int * 2)(*v))
        elif k == "eta":
            p.eta = float(v)
        elif k == "phase_model":
            p.phase_model = int(v)
        else:
            setattr(p, k, float(v))
    p.precision = PRECISIONS.get(precision, precision) if isinstance(precision, str) else precision
    p.stream = stream
    return p


def make_grid(shape, walls_y=False):
    """Grid of a (ny, nx) or (nz, ny, nx) box; walls_y: no-flux walls at both
    ends of y instead of periodicity."""
    g = pf_grid()
    if len(shape) == 2:
        g.dim, g.ny, g.nx, g.nz = 2, shape[0], shape[1], 1
    else:
        g.dim, g.nz, g.ny, g.nx = 3, shape[0], shape[1], shape[2]
    g.periodic = (C.c_int * 3)(1, 0 if walls_y else 1, 1)
    return g


def _ptr(a, where):
    """(pointer, keepalive) for a float64 array on host (numpy) or device (torch)."""
    if a is None:
        return None, None
    if where == PF_DEVICE:
        import torch
        assert isinstance(a, torch.Tensor) and a.is_cuda and a.dtype == torch.float64
        a = a.contiguous()
        return C.c_void_p(a.data_ptr()), a
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return C.c_void_p(a.ctypes.data), a


def _is_device(a):
    try:
        import torch
        return isinstance(a, torch.Tensor) and a.is_cuda
    except ImportError:
        return False


class Sim:
    """One domain advanced by libpf (pf_create ... pf_destroy): periodic, or
    with walls_y=True bounded by no-flux walls at both ends of y."""

    def __init__(self, shape, precision=PF_P64, stream=None, walls_y=False, **params):
        L = load()
        self.shape = tuple(shape)
        self.dim = len(shape)
        self.N = int(np.prod(shape))
        self._g = make_grid(shape, walls_y)
        self._p = make_params(precision=precision, stream=stream, **params)
        h = C.c_void_p()
        _check(L.pf_create(C.byref(self._g), C.byref(self._p), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().pf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_particle(self, k, x, u=(0, 0, 0), w=(0, 0, 0), R=10.0, rho_p=1.0, theta_deg=None,
                     prescribed=False):
        """Add or overwrite particle k; theta_deg None keeps the handle's angle;
        prescribed: True keeps the given u, w (e.g. a rotating cylinder), or
        the bit flags of held components (2, 4, 8: x, y, z translation;
        16: rotation)."""
        pp = pf_particle()
        pp.x = (C.c_double * 3)(*(tuple(x) + (0.0,) * (3 - len(x))))
        pp.u = (C.c_double * 3)(*(tuple(u) + (0.0,) * (3 - len(u))))
        pp.w = (C.c_double * 3)(*(tuple(w) + (0.0,) * (3 - len(w))))
        pp.R, pp.rho_p = float(R), float(rho_p)
        pp.theta_deg = float("nan") if theta_deg is None else float(theta_deg)
        pp.prescribed = int(prescribed)
        _check(load().pf_particle_state(self._h, int(k), C.byref(pp), 1))

    def particle(self, k):
        pp = pf_particle()
        _check(load().pf_particle_state(self._h, int(k), C.byref(pp), 0))
        return dict(x=list(pp.x), u=list(pp.u), w=list(pp.w), R=pp.R, rho_p=pp.rho_p,
                    theta_deg=pp.theta_deg, prescribed=int(pp.prescribed), F=list(pp.F), T=list(pp.T))

    def init(self, phi0, phi, u=None, P=None):
        where = PF_DEVICE if _is_device(phi) else PF_HOST
        keep = [_ptr(a, where) for a in (phi0, phi, u, P)]
        _check(load().pf_init_fields(self._h, *[k[0] for k in keep], where))

    def set_config(self, tile_x, tile_y, kernel=0, ctas_per_sm=0):
        """Fix the launch configuration (after init); kernel 0, 1, 2 or 3 as in pf.h."""
        _check(load().pf_set_config(self._h, int(tile_x), int(tile_y), int(kernel), int(ctas_per_sm)))

    def config(self):
        """(tile_x, tile_y, ctas_per_sm, kernel) of the step launches; -1 before tuning."""
        a, b, c, d = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        _check(load().pf_get_config(self._h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)))
        return a.value, b.value, c.value, d.value

    def step(self, n=1):
        _check(load().pf_step(self._h, int(n)))

    def autotune(self):
        """Time the autotuner's candidates on the live state (or take the cached
        choice) and keep the fastest; returns the time steps that took."""
        n = C.c_int64(0)
        _check(load().pf_autotune(self._h, C.byref(n)))
        return n.value

    def sync(self):
        _check(load().pf_sync(self._h))

    @property
    def time(self):
        return int(load().pf_time(self._h))

    def macros(self, out=None):
        """Fields at the current time as numpy arrays (or into torch CUDA
        tensors given in ``out``: dict of phi, rho, u, P, mu)."""
        if out is not None:
            ptrs = [C.c_void_p(out[k].data_ptr()) if k in out else None
                    for k in ("phi", "rho", "u", "P", "mu")]
            _check(load().pf_get_macros(self._h, *ptrs, PF_DEVICE))
            return out
        N, sh = self.N, self.shape
        phi, rho, P, mu = (np.empty(N) for _ in range(4))
        u = np.empty(self.dim * N)
        _check(load().pf_get_macros(self._h, *[C.c_void_p(a.ctypes.data) for a in (phi, rho, u, P, mu)],
                                    PF_HOST))
        return dict(phi=phi.reshape(sh), rho=rho.reshape(sh), u=u.reshape((self.dim,) + sh),
                    P=P.reshape(sh), mu=mu.reshape(sh))

    def run_logged(self, n, every, path=None):
        """Advance n steps, taking the FP64 diagnostics every ``every`` steps;
        returns the records (dicts with t, mass, E_F, E_K, E_total, nan_flag)
        and, with ``path``, appends each as one JSON line to that file."""
        import json
        recs = []
        done = 0
        while done < n:
            k = min(every, n - done)
            self.step(k)
            done += k
            d = self.diagnostics()
            rec = dict(t=int(self.time), **{key: (float(v) if key != "nan_flag" else int(v)) for key, v in d.items()})
            recs.append(rec)
            if path:
                with open(path, "a") as f:
                    f.write(json.dumps(rec) + "\n")
        return recs

    def save_state(self):
        """The run's state as bytes (pf_save_state)."""
        n = C.c_int64()
        _check(load().pf_state_size(self._h, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(load().pf_save_state(self._h, buf, n.value))
        return buf.raw

    def load_state(self, state):
        """Continue from bytes written by save_state (same grid, precision and
        particle count)."""
        buf = C.create_string_buffer(bytes(state), len(state))
        _check(load().pf_load_state(self._h, buf, len(state)))

    def normal(self):
        """Interface normal grad phi / |grad phi| (dim, *shape) as a numpy array."""
        n = np.empty(self.dim * self.N)
        _check(load().pf_get_normal(self._h, C.c_void_p(n.ctypes.data), PF_HOST))
        return n.reshape((self.dim,) + self.shape)

    def diagnostics(self):
        d = pf_diag()
        _check(load().pf_diagnostics(self._h, C.byref(d)))
        return dict(mass=d.mass, E_F=d.E_F, E_K=d.E_K, E_total=d.E_total, nan_flag=d.nan_flag)


class Batch:
    """Many independent domains of uneven size advanced together (pf_batch_*);
    walls_y: one flag for all domains or one per domain."""

    def __init__(self, shapes, params_list, precision=PF_PMIX_FP16, stream=None, walls_y=False):
        L = load()
        n = len(shapes)
        self.shapes = [tuple(s) for s in shapes]
        self.dim = len(shapes[0])
        wl = list(walls_y) if isinstance(walls_y, (list, tuple)) else [walls_y] * n
        G = (pf_grid * n)(*[make_grid(s, w) for s, w in zip(shapes, wl)])
        P = (pf_params * n)(*[make_params(precision=precision, stream=stream, **pp)
                               for pp in params_list])
        h = C.c_void_p()
        _check(L.pf_batch_create(n, G, P, C.byref(h)))
        self._h = h
        self.n = n

    def close(self):
        if getattr(self, "_h", None):
            load().pf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, i, phi0, phi, u=None, P=None):
        where = PF_DEVICE if _is_device(phi) else PF_HOST
        keep = [_ptr(a, where) for a in (phi0, phi, u, P)]
        _check(load().pf_batch_init(self._h, int(i), *[k[0] for k in keep], where))

    def init_all(self, phi0s, phis, us=None):
        """pf_batch_init_all: every domain from lists of arrays (host or device)."""
        where = PF_DEVICE if _is_device(phis[0]) else PF_HOST
        n = len(self.shapes)
        keep = []

        def table(arrs):
            if arrs is None:
                return None
            t = (C.c_void_p * n)()
            for i, a in enumerate(arrs):
                p, k = _ptr(a, where)
                keep.append(k)
                t[i] = p.value if p is not None else None
            keep.append(t)
            return C.cast(t, C.c_void_p)

        _check(load().pf_batch_init_all(self._h, table(phi0s), table(phis), table(us), None, where))

    def macros_all(self):
        """pf_batch_get_macros_all: the fields of every domain (host arrays)."""
        n = len(self.shapes)
        outs = []
        tabs = [(C.c_void_p * n)() for _ in range(5)]
        for i, sh in enumerate(self.shapes):
            N = int(np.prod(sh))
            phi, rho, P, mu = (np.empty(N) for _ in range(4))
            u = np.empty(self.dim * N)
            for t, a in zip(tabs, (phi, rho, u, P, mu)):
                t[i] = a.ctypes.data
            outs.append(dict(phi=phi.reshape(sh), rho=rho.reshape(sh), u=u.reshape((self.dim,) + sh),
                             P=P.reshape(sh), mu=mu.reshape(sh)))
        _check(load().pf_batch_get_macros_all(self._h, *[C.cast(t, C.c_void_p) for t in tabs], PF_HOST))
        return outs

    def step(self, n=1):
        _check(load().pf_batch_step(self._h, int(n)))

    def sync(self):
        _check(load().pf_batch_sync(self._h))

    def cells(self):
        return int(load().pf_batch_cells(self._h))

    def config(self):
        """(tile_x, tile_y, ctas_per_sm, kernel) of the step launches."""
        a, b, c, d = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        _check(load().pf_batch_config(self._h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)))
        return a.value, b.value, c.value, d.value

    def set_config(self, tile_x, tile_y, kernel=0, ctas_per_sm=0):
        _check(load().pf_batch_set_config(self._h, int(tile_x), int(tile_y), int(kernel), int(ctas_per_sm)))

    def macros(self, i):
        sh = self.shapes[i]
        N = int(np.prod(sh))
        phi, rho, P, mu = (np.empty(N) for _ in range(4))
        u = np.empty(self.dim * N)
        _check(load().pf_batch_get_macros(self._h, int(i),
                                          *[C.c_void_p(a.ctypes.data) for a in (phi, rho, u, P, mu)],
                                          PF_HOST))
        return dict(phi=phi.reshape(sh), rho=rho.reshape(sh), u=u.reshape((self.dim,) + sh),
                    P=P.reshape(sh), mu=mu.reshape(sh))

    def diagnostics(self, i):
        d = pf_diag()
        _check(load().pf_batch_diagnostics(self._h, int(i), C.byref(d)))
        return dict(mass=d.mass, E_F=d.E_F, E_K=d.E_K, E_total=d.E_total, nan_flag=d.nan_flag)
