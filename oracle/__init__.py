"""CPU FP64 oracle of the entropic lattice Boltzmann method (ELBM) with the
relaxation-rate formula of Zhao & Yong.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
path (the CUDA library ``paper_1904_00866_gb300`` and its binding) never
imports it and shares no code with it.

This module is argument marshalling (ctypes + numpy) around the plain C
oracle in ``elbm_oracle.c``; every arithmetic step lives there and cites the
equation it follows.  Parity status of each function, and what pins it, is
stated in the tests (``tests/test_oracle_*.py``).
"""
import ctypes
import os

import numpy as np

from . import build as _build

D2Q9, D3Q27, D1Q3 = 0, 1, 2
FORMULA, ROOT, SECANT = 0, 1, 2
LATTICES = {"D2Q9": D2Q9, "D3Q27": D3Q27, "D1Q3": D1Q3}
MODES = {"formula": FORMULA, "root": ROOT, "secant": SECANT}

F_DEGENERATE, F_ACCEPT_STAR, F_FORMULA, F_ACCEPT_TWO = 1, 2, 4, 8
F_VIOLATION, F_ROOT_CAP, F_NO_ROOT = 16, 32, 64


class Stats(ctypes.Structure):
    _fields_ = [
        ("mass", ctypes.c_double),
        ("momentum", ctypes.c_double * 3),
        ("kinetic_energy", ctypes.c_double),
        ("h_total", ctypes.c_double),
        ("alpha_min", ctypes.c_double),
        ("alpha_max", ctypes.c_double),
        ("alpha_sum", ctypes.c_double),
        ("n_nodes", ctypes.c_longlong),
        ("n_degenerate", ctypes.c_longlong),
        ("n_accept_star", ctypes.c_longlong),
        ("n_formula", ctypes.c_longlong),
        ("n_accept_two", ctypes.c_longlong),
        ("n_violations", ctypes.c_longlong),
        ("n_root_iters", ctypes.c_longlong),
        ("n_root_cap", ctypes.c_longlong),
        ("n_no_root", ctypes.c_longlong),
    ]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if name == "momentum" else v
        return d


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    L = ctypes.CDLL(path)
    L.orc_lattice.argtypes = [ctypes.c_int, _ip, _dp]
    L.orc_lattice.restype = ctypes.c_int
    L.orc_lattice_dim.argtypes = [ctypes.c_int]
    L.orc_lattice_q.argtypes = [ctypes.c_int]
    L.orc_equilibrium.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp]
    L.orc_entropy.argtypes = [ctypes.c_int, _dp]
    L.orc_entropy.restype = ctypes.c_double
    L.orc_delta_h.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double]
    L.orc_delta_h.restype = ctypes.c_double
    L.orc_delta_h_bound.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double]
    L.orc_delta_h_bound.restype = ctypes.c_double
    L.orc_delta_h_literal.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double]
    L.orc_delta_h_literal.restype = ctypes.c_double
    L.orc_alpha_max.argtypes = [ctypes.c_int, _dp, _dp]
    L.orc_alpha_max.restype = ctypes.c_double
    L.orc_collide_node.argtypes = [ctypes.c_int, _dp, ctypes.c_double,
                                   ctypes.c_int, ctypes.c_int, _dp, _dp, _ip,
                                   _ip]
    L.orc_step.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double, ctypes.c_int,
                                                ctypes.c_int, _dp, _dp, _dp,
                                                ctypes.POINTER(Stats),
                                                ctypes.c_int]
    L.orc_init_equilibrium.argtypes = [ctypes.c_int] * 4 + [_dp, _dp, _dp]
    L.orc_moments.argtypes = [ctypes.c_int] * 4 + [_dp, _dp, _dp]
    L.orc_enstrophy.argtypes = [ctypes.c_int] * 4 + [_dp]
    L.orc_enstrophy.restype = ctypes.c_double
    _lib = L
    return L


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def lattice_id(lattice):
    return LATTICES[lattice] if isinstance(lattice, str) else int(lattice)


def lattice(lat):
    """(c, w): velocities as (q, 3) int array and weights as (q,) array."""
    lat = lattice_id(lat)
    c = np.zeros((27, 3), dtype=np.int32)
    w = np.zeros(27)
    q = lib().orc_lattice(lat, c.ctypes.data_as(_ip), _ptr(w))
    if q < 0:
        raise ValueError("unknown lattice")
    return c[:q].astype(np.int64), w[:q].copy()


def dim(lat):
    return lib().orc_lattice_dim(lattice_id(lat))


def equilibrium(lat, rho, u):
    lat = lattice_id(lat)
    q = lib().orc_lattice_q(lat)
    uu = np.zeros(3)
    uu[: len(u)] = u
    feq = np.zeros(q)
    if lib().orc_equilibrium(lat, float(rho), _ptr(uu), _ptr(feq)):
        raise ValueError("equilibrium undefined (rho <= 0 or |u| >= 1)")
    return feq


def entropy(lat, f):
    return lib().orc_entropy(lattice_id(lat), _ptr(_f64(f)))


def delta_h(f, x, alpha):
    f, x = _f64(f), _f64(x)
    return lib().orc_delta_h(len(f), _ptr(f), _ptr(x), float(alpha))


def delta_h_bound(f, x, alpha):
    f, x = _f64(f), _f64(x)
    return lib().orc_delta_h_bound(len(f), _ptr(f), _ptr(x), float(alpha))


def delta_h_literal(lat, f, feq, alpha):
    return lib().orc_delta_h_literal(lattice_id(lat), _ptr(_f64(f)),
                                     _ptr(_f64(feq)), float(alpha))


def alpha_max(f, feq):
    f, feq = _f64(f), _f64(feq)
    return lib().orc_alpha_max(len(f), _ptr(f), _ptr(feq))


def collide_node(lat, f, beta, mode="formula", secant_iters=1):
    """One Eq. (1) collision.  Returns (f_tilde, alpha, flags, iters)."""
    lat = lattice_id(lat)
    f = _f64(f)
    ft = np.zeros_like(f)
    a = ctypes.c_double()
    fl = ctypes.c_int()
    it = ctypes.c_int()
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    if lib().orc_collide_node(lat, _ptr(f), float(beta), m, int(secant_iters),
                              _ptr(ft), ctypes.byref(a), ctypes.byref(fl),
                              ctypes.byref(it)):
        raise ValueError("invalid node state")
    return ft, a.value, fl.value, it.value


def beta_from_nu(nu):
    """Eq. (2) with dt = 1 and c_s^2 = 1/3."""
    cs2 = 1.0 / 3.0
    return cs2 / (2.0 * nu + cs2)


class Lattice:
    """A periodic lattice advanced by the oracle.  f is SoA (q, nz, ny, nx)."""

    def __init__(self, lat, nx, ny=1, nz=1, nu=None, beta=None):
        self.lat = lattice_id(lat)
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.q = lib().orc_lattice_q(self.lat)
        self.d = lib().orc_lattice_dim(self.lat)
        if beta is None:
            beta = beta_from_nu(nu)
        self.beta = float(beta)
        self.f = np.zeros((self.q, self.nz, self.ny, self.nx))
        self.step_count = 0

    @property
    def n(self):
        return self.nx * self.ny * self.nz

    def init_fields(self, rho, u):
        rho = _f64(np.broadcast_to(rho, (self.nz, self.ny, self.nx)))
        u = _f64(u).reshape(self.d, self.nz, self.ny, self.nx)
        if lib().orc_init_equilibrium(self.lat, self.nx, self.ny, self.nz,
                                      _ptr(rho), _ptr(u), _ptr(self.f)):
            raise ValueError("invalid initial fields")
        self.step_count = 0

    def set_populations(self, f):
        self.f = _f64(f).reshape(self.q, self.nz, self.ny, self.nx).copy()

    def step(self, nsteps=1, mode="formula", secant_iters=1, threads=0,
             alpha_map=False, stats=False):
        """Advance nsteps.  Returns (alpha maps, stats list) as requested."""
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        out = np.empty_like(self.f)
        maps, st = [], []
        for _ in range(int(nsteps)):
            amap = np.empty((self.nz, self.ny, self.nx)) if alpha_map else None
            s = Stats() if stats else None
            rc = lib().orc_step(self.lat, self.nx, self.ny, self.nz, self.beta,
                                m, int(secant_iters), _ptr(self.f), _ptr(out),
                                _ptr(amap) if amap is not None else None,
                                ctypes.byref(s) if s is not None else None,
                                int(threads))
            if rc:
                raise ValueError("oracle step failed (non-positive population"
                                 " or |u| >= 1)")
            self.f, out = out, self.f
            self.step_count += 1
            if alpha_map:
                maps.append(amap)
            if stats:
                st.append(s.as_dict())
        return maps, st

    def moments(self):
        rho = np.empty((self.nz, self.ny, self.nx))
        u = np.empty((self.d, self.nz, self.ny, self.nx))
        lib().orc_moments(self.lat, self.nx, self.ny, self.nz, _ptr(self.f),
                          _ptr(rho), _ptr(u))
        return rho, u

    def enstrophy(self):
        return lib().orc_enstrophy(self.lat, self.nx, self.ny, self.nz,
                                   _ptr(self.f))
