"""ctypes wrapper of the FP64 CPU oracle (``pf_oracle.c``).

TEST INFRASTRUCTURE ONLY: see ``oracle/__init__.py``.  Argument marshalling
only; every number is computed in the C code.
"""
import ctypes as C
import math

import numpy as np

from . import build_oracle

_lib = None


class OrcParams(C.Structure):
    _fields_ = [
        ("sigma", C.c_double), ("D", C.c_double), ("M", C.c_double), ("eta", C.c_double),
        ("rho1", C.c_double), ("rho2", C.c_double), ("mu1", C.c_double), ("mu2", C.c_double),
        ("d0", C.c_double), ("s0", C.c_double), ("s1", C.c_double), ("s2", C.c_double),
        ("s3", C.c_double), ("s4", C.c_double), ("theta_deg", C.c_double),
        ("Fb", C.c_double * 3), ("g", C.c_double * 3), ("solid_eps", C.c_double),
        ("rep_xi", C.c_double), ("rep_eps", C.c_double), ("wall_circle", C.c_double * 3),
        ("phase_model", C.c_int),
    ]


class OrcParticle(C.Structure):
    _fields_ = [
        ("x", C.c_double * 3), ("u", C.c_double * 3), ("w", C.c_double * 3),
        ("R", C.c_double), ("rho_p", C.c_double),
        ("u_prev", C.c_double * 3), ("w_prev", C.c_double * 3),
        ("F", C.c_double * 3), ("T", C.c_double * 3),
        ("theta_deg", C.c_double), ("prescribed", C.c_int),
    ]


D2Q9, D3Q19, D3Q7 = 0, 1, 2

_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int)


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = C.CDLL(path)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(OrcParams)]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_num_threads.restype = C.c_int
        L.orc_init.argtypes = [C.c_void_p, _DP, _DP, _DP, _DP]
        L.orc_step.argtypes = [C.c_void_p, C.c_long]
        L.orc_macros.argtypes = [C.c_void_p, _DP, _DP, _DP, _DP, _DP]
        L.orc_diagnostics.argtypes = [C.c_void_p, _DP]
        L.orc_get_f.argtypes = [C.c_void_p, _DP, _DP]
        L.orc_get_phi0.argtypes = [C.c_void_p, _DP]
        L.orc_normal.argtypes = [C.c_void_p, _DP]
        L.orc_set_particle.argtypes = [C.c_void_p, C.c_int, C.POINTER(OrcParticle)]
        L.orc_set_particle.restype = C.c_int
        L.orc_get_particle.argtypes = [C.c_void_p, C.c_int, C.POINTER(OrcParticle)]
        L.orc_get_particle.restype = C.c_int
        L.orc_num_particles.argtypes = [C.c_void_p]
        L.orc_num_particles.restype = C.c_int
        L.orc_lattice.argtypes = [C.c_int, C.c_double, _IP, _DP, _DP]
        L.orc_lattice.restype = C.c_int
        L.orc_feq1.argtypes = [C.c_int, C.c_double, C.c_double, _DP, C.c_double, C.c_double, _DP]
        L.orc_src1.argtypes = [C.c_int, C.c_double, _DP, _DP]
        L.orc_feq2.argtypes = [C.c_int, C.c_double, C.c_double, _DP, _DP, C.c_double, _DP]
        L.orc_src2.argtypes = [C.c_int, C.c_double, _DP, _DP, _DP, _DP, _DP]
        L.orc_lambda.argtypes = [C.c_int, C.c_double, _DP, _DP]
        L.orc_rates.argtypes = [C.c_int, C.c_int] + [C.c_double] * 6 + [_DP]
        L.orc_grad.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _DP, _DP]
        L.orc_lap.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _DP, _DP]
        L.orc_mu_phi.argtypes = [C.POINTER(OrcParams)] + [C.c_double] * 4
        L.orc_mu_phi.restype = C.c_double
        L.orc_mu_phi0.argtypes = [C.POINTER(OrcParams)] + [C.c_double] * 3
        L.orc_mu_phi0.restype = C.c_double
        L.orc_particle_update.argtypes = [C.c_int, C.POINTER(OrcParams), C.POINTER(OrcParticle),
                                          _DP, _DP]
        L.orc_particle_force.argtypes = [C.c_void_p, C.c_int, _DP, _DP]
        L.orc_set_walls.argtypes = [C.c_void_p, C.c_int]
        L.orc_set_walls.restype = C.c_int
        L.orc_repulsion.argtypes = [C.c_int, C.POINTER(OrcParams), _IP, C.c_int, C.c_int,
                                    C.POINTER(OrcParticle), _DP]
        _lib = L
    return _lib


def _p(a):
    """Pointer to a contiguous float64 numpy array (or None)."""
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


def _arr(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        a = np.ascontiguousarray(np.resize(a, n))
    return a


def make_params(**kw):
    """Oracle parameters from keyword arguments (paper defaults for the rest)."""
    d = dict(sigma=0.01, D=4.0, M=0.02, eta=0.0, rho1=1.0, rho2=1.0, mu1=0.1, mu2=0.1,
             d0=0.4, s0=1.0, s1=1.0, s2=1.0, s3=1.0, s4=1.0, theta_deg=90.0,
             Fb=(0.0, 0.0, 0.0), g=(0.0, 0.0, 0.0), solid_eps=1e-3, rep_xi=0.0, rep_eps=0.0,
             wall_circle=(0.0, 0.0, 0.0), phase_model=0)
    d.update(kw)
    p = OrcParams()
    for k, v in d.items():
        if k in ("Fb", "g", "wall_circle"):
            v = tuple(v) + (0.0,) * (3 - len(v))
            setattr(p, k, (C.c_double * 3)(*v))
        elif k == "phase_model":
            p.phase_model = int(v)
        else:
            setattr(p, k, float(v))
    return p


class Particle:
    """Plain particle record (FP64) mirroring the oracle's struct."""

    def __init__(self, x, u=(0, 0, 0), w=(0, 0, 0), R=10.0, rho_p=1.0, theta_deg=None, prescribed=False):
        # prescribed: False/True (all of u and w held) or the bit flags of the
        # held components (2, 4, 8: x, y, z translation; 16: rotation)
        self.theta_deg = float("nan") if theta_deg is None else float(theta_deg)
        self.prescribed = int(prescribed)
        self.x = list(x) + [0.0] * (3 - len(x))
        self.u = list(u) + [0.0] * (3 - len(u))
        self.w = list(w) + [0.0] * (3 - len(w))
        self.R = float(R)
        self.rho_p = float(rho_p)
        self.F = [0.0] * 3
        self.T = [0.0] * 3
        self.u_prev = list(self.u)
        self.w_prev = list(self.w)

    def to_c(self):
        c = OrcParticle()
        for k in ("x", "u", "w", "u_prev", "w_prev", "F", "T"):
            setattr(c, k, (C.c_double * 3)(*getattr(self, k)))
        c.R, c.rho_p = self.R, self.rho_p
        c.theta_deg = self.theta_deg
        c.prescribed = int(self.prescribed)
        return c

    @classmethod
    def from_c(cls, c):
        p = cls(list(c.x), list(c.u), list(c.w), c.R, c.rho_p)
        p.theta_deg = c.theta_deg
        p.prescribed = int(c.prescribed)
        p.u_prev, p.w_prev = list(c.u_prev), list(c.w_prev)
        p.F, p.T = list(c.F), list(c.T)
        return p


class OracleSim:
    """One periodic domain advanced by the FP64 oracle."""

    def __init__(self, shape, params):
        L = lib()
        self.dim = len(shape)
        if self.dim == 2:
            ny, nx = shape
            nz = 1
        else:
            nz, ny, nx = shape
        self.shape = tuple(shape)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.N = nx * ny * nz
        self.params = params
        self._h = L.orc_create(self.dim, nx, ny, nz, C.byref(params))
        if not self._h:
            raise ValueError("oracle: bad grid")
        self.Q1 = 9 if self.dim == 2 else 7
        self.Q2 = 9 if self.dim == 2 else 19

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_destroy(self._h)
            self._h = None

    def init(self, phi0, phi, u=None, P=None):
        phi0 = _arr(phi0).reshape(-1)
        phi = _arr(phi).reshape(-1)
        u = None if u is None else _arr(u).reshape(-1)
        P = None if P is None else _arr(P).reshape(-1)
        lib().orc_init(self._h, _p(phi0), _p(phi), _p(u), _p(P))

    def step(self, n=1):
        lib().orc_step(self._h, int(n))

    def macros(self):
        N, sh = self.N, self.shape
        phi, rho, P, mu = (np.empty(N) for _ in range(4))
        u = np.empty(self.dim * N)
        lib().orc_macros(self._h, _p(phi), _p(rho), _p(u), _p(P), _p(mu))
        return dict(phi=phi.reshape(sh), rho=rho.reshape(sh), u=u.reshape((self.dim,) + sh),
                    P=P.reshape(sh), mu=mu.reshape(sh))

    def diagnostics(self):
        out = np.empty(4)
        lib().orc_diagnostics(self._h, _p(out))
        return dict(mass=out[0], E_F=out[1], E_K=out[2], E_total=out[3])

    def distributions(self):
        f1 = np.empty(self.Q1 * self.N)
        f2 = np.empty(self.Q2 * self.N)
        lib().orc_get_f(self._h, _p(f1), _p(f2))
        return f1.reshape((self.Q1,) + self.shape), f2.reshape((self.Q2,) + self.shape)

    def normal(self):
        """Interface normal grad phi / |grad phi| (dim, *shape)."""
        n = np.empty(self.dim * self.N)
        lib().orc_normal(self._h, _p(n))
        return n.reshape((self.dim,) + self.shape)

    def phi0(self):
        a = np.empty(self.N)
        lib().orc_get_phi0(self._h, _p(a))
        return a.reshape(self.shape)

    def set_walls(self, wall_y=True):
        """Walls at the ends of y (reading R21); call before init."""
        if lib().orc_set_walls(self._h, 1 if wall_y else 0) != 0:
            raise ValueError("walls are 2D only")

    def set_particle(self, k, part):
        c = part.to_c()
        if lib().orc_set_particle(self._h, int(k), C.byref(c)) != 0:
            raise IndexError(k)

    def particle(self, k):
        c = OrcParticle()
        if lib().orc_get_particle(self._h, int(k), C.byref(c)) != 0:
            raise IndexError(k)
        return Particle.from_c(c)

    def particle_force(self, k):
        F = np.empty(3)
        T = np.empty(3)
        lib().orc_particle_force(self._h, int(k), _p(F), _p(T))
        return F, T


# ---- per-cell building blocks --------------------------------------------------------

def lattice(kind, d0):
    c = (C.c_int * (19 * 3))()
    w = np.empty(19)
    MH = np.empty(19 * 19)
    Q = lib().orc_lattice(kind, d0, c, _p(w), _p(MH))
    cc = np.array(c[: Q * 3], dtype=int).reshape(Q, 3)
    return cc, w[:Q].copy(), MH[: Q * Q].reshape(Q, Q).copy()


def _q(kind):
    return {D2Q9: 9, D3Q19: 19, D3Q7: 7}[kind]


def feq1(kind, d0, phi, u, mu, eta):
    out = np.empty(_q(kind))
    lib().orc_feq1(kind, d0, phi, _p(_arr(u, 3)), mu, eta, _p(out))
    return out


def src1(kind, d0, G):
    out = np.empty(_q(kind))
    lib().orc_src1(kind, d0, _p(_arr(G, 3)), _p(out))
    return out


def feq2(kind, d0, rho, u, S, P):
    out = np.empty(_q(kind))
    lib().orc_feq2(kind, d0, rho, _p(_arr(u, 3)), _p(_arr(S, 3)), P, _p(out))
    return out


def src2(kind, d0, u, gradrho, Ftot, M2F):
    out = np.empty(_q(kind))
    lib().orc_src2(kind, d0, _p(_arr(u, 3)), _p(_arr(gradrho, 3)), _p(_arr(Ftot, 3)),
                   _p(_arr(M2F).reshape(-1).copy()), _p(out))
    return out


def lambda_matrix(kind, d0, S):
    Q = _q(kind)
    out = np.empty(Q * Q)
    lib().orc_lambda(kind, d0, _p(_arr(S)), _p(out))
    return out.reshape(Q, Q)


def rates(kind, k, s0, s1, s2a, s2b, s3, s4):
    out = np.empty(_q(kind))
    lib().orc_rates(kind, k, s0, s1, s2a, s2b, s3, s4, _p(out))
    return out


def grad(psi):
    psi = _arr(psi)
    dim = psi.ndim
    shp = psi.shape if dim == 3 else (1,) + psi.shape
    nz, ny, nx = shp
    out = np.empty(dim * psi.size)
    lib().orc_grad(dim, nx, ny, nz, _p(psi.reshape(-1).copy()), _p(out))
    return out.reshape((dim,) + psi.shape)


def lap(psi):
    psi = _arr(psi)
    dim = psi.ndim
    shp = psi.shape if dim == 3 else (1,) + psi.shape
    nz, ny, nx = shp
    out = np.empty(psi.size)
    lib().orc_lap(dim, nx, ny, nz, _p(psi.reshape(-1).copy()), _p(out))
    return out.reshape(psi.shape)


def mu_phi(params, phi, phi0, lap_phi, lap_phi0):
    return lib().orc_mu_phi(C.byref(params), phi, phi0, lap_phi, lap_phi0)


def mu_phi0(params, phi, phi0, lap_phi):
    return lib().orc_mu_phi0(C.byref(params), phi, phi0, lap_phi)


def particle_update(dim, params, part, Ff, Tf):
    c = part.to_c()
    lib().orc_particle_update(dim, C.byref(params), C.byref(c), _p(_arr(Ff, 3)), _p(_arr(Tf, 3)))
    return Particle.from_c(c)


def repulsion(dim, params, n, parts, walls_y=False):
    """Repulsion force on each particle (np x 3), readings R19 and R22; n is
    (nx, ny[, nz]); walls_y: box walls at the ends of y."""
    arr = (OrcParticle * max(len(parts), 1))(*[q.to_c() for q in parts])
    nn = (C.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
    out = np.zeros(3 * max(len(parts), 1))
    lib().orc_repulsion(dim, C.byref(params), nn, 1 if walls_y else 0, len(parts), arr, _p(out))
    return out[:3 * len(parts)].reshape(len(parts), 3)


def num_threads():
    return lib().orc_num_threads()


def deg(x):
    return x * math.pi / 180.0
