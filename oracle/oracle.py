"""ctypes wrapper of the plain FP64 CPU oracle (``lp_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: this module and the library it builds may be used by
``tests/``, by ``__graft_entry__.smoke()`` and by the CPU-baseline leg of
``bench.py``. The CUDA library never calls it and shares no code with it.

Every function follows the paper (Zepeda & Samulyak, arXiv 2206.14061):
neighbour search and stencils (Sec. 3.1 items 5-6, mirrors item 9), GFD
least-squares fits by Householder QR (Sec. 3.1 item 7), the mu(I) closure
(Sec. 2.2-2.3, with R = dN/dphi) and the explicit step (Sec. 3.1 items 8, 10).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lp_oracle.cpp")
_LIB = os.path.join(_HERE, "liblp_oracle.so")
_lock = threading.Lock()
_lib = None

MIRROR_BIT = 0x80000000
GHOST_BIT = 0x40000000  # ghost particle: entry reflected through the particle


class OrcParams(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in (
        "mu_s", "mu_2", "I0", "d", "rho_s", "phi_c", "phi_min", "phi_max", "alpha", "beta",
        "h", "radius", "gx", "gy", "gz", "floor_z", "dt")] + [
        ("mirror_mode", ctypes.c_int32), ("free_surface", ctypes.c_int32),
        ("time_scheme", ctypes.c_int32), ("pad", ctypes.c_int32),
        ("period_x", ctypes.c_double), ("period_y", ctypes.c_double)]


class OrcDiag(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "n_gas", "n_inertial", "n_quasistatic", "n_over_c", "n_below_floor",
        "n_rank_deficient", "min_stencil", "max_stencil", "n_ghosts")]


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (FP64, no FMA contraction, OpenMP)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call([
                "g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                "-o", tmp, _SRC])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
        vp = ctypes.c_void_p
        L.orc_neighbors.argtypes = [i64, vp, vp, vp, vp, d, ctypes.c_int, d, i32, ctypes.c_int,
                                    ctypes.c_int, vp, vp, ctypes.c_int]
        L.orc_neighbors.restype = ctypes.c_int
        L.orc_fit.argtypes = [i64, vp, vp, vp, vp, vp, i32, ctypes.c_int, vp, vp, d, d, vp, vp,
                              ctypes.c_int]
        L.orc_fit.restype = ctypes.c_int
        L.orc_closure.argtypes = [i64, vp, P(OrcParams), vp]
        L.orc_closure.restype = None
        L.orc_mui_stress.argtypes = [i64, P(OrcParams), vp, vp, vp, vp, vp, vp, vp]
        L.orc_mui_stress.restype = None
        L.orc_step.argtypes = [i64] + [vp] * 7 + [P(OrcParams), ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_int, ctypes.c_int, P(OrcDiag)]
        L.orc_step.restype = ctypes.c_int
        L.orc_step_detail.argtypes = [i64] + [vp] * 7 + [P(OrcParams), ctypes.c_int,
                                                         ctypes.c_int] + [vp] * 8
        L.orc_step_detail.restype = ctypes.c_int
        L.orc_step_tangent.argtypes = [i64] + [vp] * 7 + [P(OrcParams), ctypes.c_int,
                                                          ctypes.c_int, ctypes.c_int,
                                                          ctypes.c_int, vp]
        L.orc_step_tangent.restype = ctypes.c_int
        L.orc_step_stencils.argtypes = [i64, vp, vp, vp, P(OrcParams), ctypes.c_int, i32, vp,
                                        vp, ctypes.c_int]
        L.orc_step_stencils.restype = ctypes.c_int
        L.orc_ghost_state.argtypes = [i64, vp, vp, P(OrcParams), vp, vp]
        L.orc_ghost_state.restype = None
        L.orc_max_threads.argtypes = []
        L.orc_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def params(**kw) -> OrcParams:
    p = OrcParams()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def max_threads() -> int:
    return lib().orc_max_threads()


def neighbors(x, y, z, radius=None, r_const=0.0, mirror_mode=0, floor_z=0.0, cap=256,
              keep_nearest=False, brute=True, nthreads=0):
    """Stencils (Sec. 3.1 items 5-6). Returns (nbr [n, cap] int32, cnt [n], n_overflow).

    Entries are particle indices j, or j | 0x80000000 for the floor mirror of j;
    real particles come first, each group in ascending index order.
    keep_nearest: False / 0 keeps all (cnt may exceed cap: overflow), True / 1
    the cap nearest, 2 the first cap of the octant-balanced ordering (Sec. 3.1
    item 6)."""
    x, y, z = _f64(x), _f64(y), _f64(z)
    n = x.size
    rad = None if radius is None else _f64(radius)
    nbr = np.zeros((n, cap), dtype=np.int32)
    cnt = np.zeros(n, dtype=np.int32)
    over = lib().orc_neighbors(n, _p(x), _p(y), _p(z), _p(rad), float(r_const), int(mirror_mode),
                               float(floor_z), int(cap), int(keep_nearest), int(bool(brute)),
                               _p(nbr), _p(cnt), int(nthreads))
    return nbr, cnt, over


def fit(x, y, z, nbr, cnt, fields, mirror_sign, h, floor_z=0.0, nthreads=0):
    """GFD least-squares derivatives (Sec. 3.1 item 7) of nf fields.

    fields: [nf, n]. Returns (coeffs [n, nf, 9], rank [n]); coefficient order
    d/dx, d/dy, d/dz, d2/dx2, d2/dy2, d2/dz2, d2/dxdy, d2/dxdz, d2/dydz."""
    x, y, z = _f64(x), _f64(y), _f64(z)
    fields = _f64(np.atleast_2d(fields))
    nf, n = fields.shape
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    cnt = np.ascontiguousarray(cnt, dtype=np.int32)
    ms = _f64(mirror_sign)
    if nbr.ndim != 2 or nbr.shape[0] != n or cnt.shape != (n,) or ms.shape != (nf,):
        raise ValueError("fit: nbr must be [n, cap], cnt [n], mirror_sign [nf]")
    if x.size != n or y.size != n or z.size != n:
        raise ValueError("fit: positions and fields must have the same length")
    coeffs = np.zeros((n, nf, 9))
    rank = np.zeros(n, dtype=np.int32)
    lib().orc_fit(n, _p(x), _p(y), _p(z), _p(nbr), _p(cnt), nbr.shape[1], nf, _p(fields), _p(ms),
                  float(h), float(floor_z), _p(coeffs), _p(rank), int(nthreads))
    return coeffs, rank


def closure(phi, p: OrcParams):
    """M, N, S, R, mu at the given solid fractions (Sec. 2.3). Returns [n, 5]."""
    phi = _f64(np.atleast_1d(phi))
    out = np.zeros((phi.size, 5))
    lib().orc_closure(phi.size, _p(phi), ctypes.byref(p), _p(out))
    return out


def mui_stress(V, grad_u, p: OrcParams):
    """Pointwise mu(I) stress (Sec. 2.2): returns gdot [n,6], |gdot|, P, eta, regime."""
    V = _f64(V)
    n = V.size
    G = _f64(np.asarray(grad_u).reshape(n, 9))
    gd = np.zeros((n, 6)); gn = np.zeros(n); P = np.zeros(n); eta = np.zeros(n)
    reg = np.zeros(n, dtype=np.int8)
    lib().orc_mui_stress(n, ctypes.byref(p), _p(V), _p(G), _p(gd), _p(gn), _p(P), _p(eta), _p(reg))
    return gd, gn, P, eta, reg


FIELDS = ("x", "y", "z", "u", "v", "w", "V")


def step_stencils(x, y, z, p: OrcParams, brute: bool = True, cap: int = 256, nthreads: int = 0):
    """Stencils one step uses (Sec. 3.1 items 5-6 and 9): the neighbour lists
    and, with p.free_surface, the ghost entries (code | GHOST_BIT: the point
    reflection of entry `code` through the particle). Returns (nbr, cnt, over)."""
    x, y, z = _f64(x), _f64(y), _f64(z)
    n = x.size
    nbr = np.zeros((n, cap), dtype=np.int32)
    cnt = np.zeros(n, dtype=np.int32)
    over = lib().orc_step_stencils(n, _p(x), _p(y), _p(z), ctypes.byref(p), int(bool(brute)),
                                   cap, _p(nbr), _p(cnt), int(nthreads))
    return nbr, cnt, over


def ghost_state(phi, gnorm, p: OrcParams):
    """Solid fraction and |gdot| of the ghost particles of fluid particles with
    solid fraction phi and |gdot| gnorm (Sec. 3.1 item 9)."""
    phi, gnorm = _f64(phi), _f64(gnorm)
    phi_g, gn_g = np.zeros(phi.size), np.zeros(phi.size)
    lib().orc_ghost_state(phi.size, _p(phi), _p(gnorm), ctypes.byref(p), _p(phi_g), _p(gn_g))
    return phi_g, gn_g


def step(state: dict, p: OrcParams, nsteps: int, rebuild_every: int = 1, brute: bool = True,
         nthreads: int = 0):
    """nsteps explicit LP steps. state: dict of x,y,z,u,v,w,V arrays. Returns (new state, diag)."""
    s = {k: _f64(state[k]).copy() for k in FIELDS}
    dg = OrcDiag()
    lib().orc_step(s["x"].size, *[_p(s[k]) for k in FIELDS], ctypes.byref(p), int(nsteps),
                   int(rebuild_every), int(bool(brute)), int(nthreads), ctypes.byref(dg))
    return s, {k: getattr(dg, k) for k, _ in OrcDiag._fields_}


def step_detail(state: dict, p: OrcParams, brute: bool = True, nthreads: int = 0):
    """Per-particle intermediates of one step at `state` (nothing advanced)."""
    s = {k: _f64(state[k]) for k in FIELDS}
    n = s["x"].size
    out = dict(gdot=np.zeros((n, 6)), gnorm=np.zeros(n), gradV=np.zeros((n, 3)),
               lapdiv=np.zeros((n, 3)), div=np.zeros(n), grad_gnorm=np.zeros((n, 3)),
               acc=np.zeros((n, 3)), regime=np.zeros(n, dtype=np.int8))
    nrd = lib().orc_step_detail(n, *[_p(s[k]) for k in FIELDS], ctypes.byref(p), int(bool(brute)),
                                int(nthreads), *[_p(out[k]) for k in (
                                    "gdot", "gnorm", "gradV", "lapdiv", "div", "grad_gnorm",
                                    "acc", "regime")])
    out["n_rank_deficient"] = nrd
    return out


def step_tangent(state: dict, p: OrcParams, nsteps: int, rebuild_every: int = 1,
                 brute: bool = True, nthreads: int = 0):
    """Tangent-linear run. Returns (final state, tangent [3 (mu_s, mu_2, I0), 7 fields, n])."""
    s = {k: _f64(state[k]).copy() for k in FIELDS}
    n = s["x"].size
    tan = np.zeros((3, 7, n))
    lib().orc_step_tangent(n, *[_p(s[k]) for k in FIELDS], ctypes.byref(p), int(nsteps),
                           int(rebuild_every), int(bool(brute)), int(nthreads), _p(tan))
    return s, tan
