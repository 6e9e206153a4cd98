"""Thin Python binding of the C ABI declared in ``include/lp.h``.

Argument marshalling only: torch supplies device memory and streams, every
step of the LP path runs in the CUDA library ``_lib/liblp.so``. If the
library is missing or a call fails, an exception is raised; there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import torch  # loads the CUDA runtime that liblp.so shares

from . import build as _build

LP_OK = 0
LP_ERR_INVALID_ARG = 1
LP_ERR_STENCIL_OVERFLOW = 2
LP_ERR_NONFINITE = 3
LP_ERR_TIMEOUT = 4
LP_ERR_CUDA = 5
LP_ERR_OOM = 6
LP_ERR_UNIMPLEMENTED = 7
LP_TIME_PAPER = 0
LP_TIME_HEUN = 1
LP_FP64 = 0
LP_MIXED = 1
LP_MIXED_FF = 2
LP_MIRROR_NONE = 0
LP_MIRROR_NOSLIP = 1
LP_MIRROR_FREESLIP = 2
LP_MAX_CAP = 64
LP_KEEP_ALL = 0
LP_KEEP_NEAREST = 1
LP_KEEP_OCTANTS = 2
LP_LAUNCH_KERNELS = 0
LP_LAUNCH_GRAPH = 1
LP_LAUNCH_PERSISTENT = 2
MIRROR_BIT = 0x80000000

_vp = ctypes.c_void_p


class LpCtxDesc(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("max_columns", ctypes.c_int32),
                ("max_particles", ctypes.c_int64), ("cap", ctypes.c_int32), ("pad", ctypes.c_int32)]


class LpParticles(ctypes.Structure):
    _fields_ = [(k, _vp) for k in ("x", "y", "z", "u", "v", "w", "V")] + [
        ("n", ctypes.c_int64), ("column_offsets", ctypes.POINTER(ctypes.c_int32)),
        ("ncolumns", ctypes.c_int32), ("pad", ctypes.c_int32)]


class LpMui(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("mu_s", "mu_2", "I0", "d", "rho_s")]


class LpEos(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("phi_c", "phi_min", "phi_max", "alpha", "beta")]


class LpParams(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("h", "radius", "gx", "gy", "gz", "floor_z")] + [
        (k, ctypes.c_int32) for k in ("mirror_mode", "precision", "rebuild_every", "launch_mode")] + [
        ("skin", ctypes.c_double), ("free_surface", ctypes.c_int32),
        ("time_scheme", ctypes.c_int32), ("period_x", ctypes.c_double),
        ("period_y", ctypes.c_double), ("keep_lists", ctypes.c_int32), ("pad", ctypes.c_int32)]


class LpNeighbors(ctypes.Structure):
    _fields_ = [("nbr", _vp), ("cnt", _vp), ("n", ctypes.c_int64), ("cap", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class LpDiag(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_uint32), ("min_stencil", ctypes.c_int32),
                ("max_stencil", ctypes.c_int32), ("pad", ctypes.c_int32)] + [
        (k, ctypes.c_int64) for k in ("n_overflow", "n_fallback", "n_gas", "n_quasistatic",
                                      "n_over_c", "n_nonfinite", "n_below_floor",
                                      "n_stencil_rows", "n_stencils", "n_ghosts")]


class LpTuning(ctypes.Structure):
    _fields_ = [("block_neighbors", ctypes.c_int32), ("block_pass1", ctypes.c_int32),
                ("block_pass2", ctypes.c_int32), ("launch_mode", ctypes.c_int32),
                ("ms_per_step", ctypes.c_double), ("from_table", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class LpError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().lp_status_string(status).decode() if _lib is not None else str(status)
        super().__init__(f"{where}: {msg} (status {status})")


_lib = None

_P = ctypes.POINTER
_SIGS = {
    "lp_version": ([], ctypes.c_char_p),
    "lp_status_string": ([ctypes.c_int32], ctypes.c_char_p),
    "lp_ctx_create": ([_P(LpCtxDesc), _P(_vp)], ctypes.c_int32),
    "lp_ctx_destroy": ([_vp], ctypes.c_int32),
    "lp_ctx_sync": ([_vp, _vp, _P(LpDiag)], ctypes.c_int32),
    "lp_ctx_profile": ([_vp, ctypes.c_int32], ctypes.c_int32),
    "lp_ctx_set_wait_limit": ([_vp, ctypes.c_int64, ctypes.c_int32], ctypes.c_int32),
    "lp_ctx_set_adjoint_memory": ([_vp, ctypes.c_int64], ctypes.c_int32),
    "lp_ctx_phase_times": ([_vp, _vp, _P(ctypes.c_double), _P(ctypes.c_int64),
                            _P(ctypes.c_int64)], ctypes.c_int32),
    "lp_ctx_set_tuning": ([_vp, _P(LpTuning)], ctypes.c_int32),
    "lp_autotune": ([_vp, _P(LpParticles), _P(LpMui), _P(LpEos), _P(LpParams), ctypes.c_double,
                     ctypes.c_int32, ctypes.c_char_p, _P(LpTuning), _vp], ctypes.c_int32),
    "lp_build_neighbors": ([_vp, _P(LpParticles), _vp, ctypes.c_double, ctypes.c_int32,
                            ctypes.c_double, ctypes.c_int32, ctypes.c_int32, _P(LpNeighbors), _vp],
                           ctypes.c_int32),
    "lp_neighbors_export": ([_vp, _P(LpNeighbors), _vp, _vp, _vp], ctypes.c_int32),
    "lp_fit_derivatives": ([_vp, _P(LpParticles), _P(LpNeighbors), _P(_vp), _P(ctypes.c_double),
                            ctypes.c_int32, ctypes.c_double, ctypes.c_double, _vp, ctypes.c_int32,
                            _vp], ctypes.c_int32),
    "lp_fit_derivatives_noalloc": ([ctypes.c_int64, _vp, _vp, _vp, _vp, _vp, ctypes.c_int32,
                                    _P(_vp), _P(ctypes.c_double), ctypes.c_int32, ctypes.c_double,
                                    ctypes.c_double, _vp, ctypes.c_int32, _vp, _P(LpDiag)],
                                   ctypes.c_int32),
    "lp_mui_stress": ([_vp, _P(LpMui), _P(LpEos), ctypes.c_int64, _vp, _vp, _vp, _vp, _vp, _vp,
                       _vp, _vp], ctypes.c_int32),
    "lp_step": ([_vp, _P(LpParticles), _P(LpMui), _P(LpEos), _P(LpParams), ctypes.c_double,
                 ctypes.c_int32, _vp], ctypes.c_int32),
    "lp_step_adjoint": ([_vp, _P(LpParticles), _P(LpMui), _P(LpEos), _P(LpParams),
                         ctypes.c_double, ctypes.c_int32, ctypes.c_int32, _P(LpParticles), _vp,
                         _P(LpParticles), _vp], ctypes.c_int32),
}


def header_functions() -> list[str]:
    """Names of the functions declared in include/lp.h."""
    text = open(os.path.join(_build.INCLUDE, "lp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lp_[a-z_]+)\s*\(", text)))


def lib(build_if_missing: bool = False):
    """Load liblp.so (built in-tree). Raises if it is missing."""
    global _lib
    if _lib is None:
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(
                f"CUDA library {_build.LIB} is not built; run paper_2206_14061_gb300.build.build()")
        L = ctypes.CDLL(_build.LIB)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(status: int, where: str):
    if status != LP_OK:
        raise LpError(status, where)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t: torch.Tensor, name: str, dtype=torch.float64) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor of {dtype}")
    return t


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


FIELDS = ("x", "y", "z", "u", "v", "w", "V")


def _host(t: torch.Tensor, name: str) -> torch.Tensor:
    if (not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.float64
            or not t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CPU tensor of torch.float64")
    return t


def _particles(state: dict, column_offsets=None, need_state=True, allow_host=False):
    n = state["x"].numel()
    p = LpParticles()
    host = allow_host and not state["x"].is_cuda
    for k in FIELDS:
        if k in state and state[k] is not None:
            t = _host(state[k], k) if host else _dev(state[k], k)
            if t.numel() != n:
                raise ValueError("all particle arrays must have the same length")
            setattr(p, k, t.data_ptr())
        elif need_state or k in ("x", "y", "z"):
            raise ValueError(f"missing particle array {k}")
    p.n = n
    keep = None
    if column_offsets is None:
        p.ncolumns = 1
    else:
        keep = np.ascontiguousarray(np.asarray(column_offsets, dtype=np.int32))
        p.ncolumns = keep.size - 1
        p.column_offsets = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    return p, keep


def mui_struct(m) -> LpMui:
    return LpMui(*(float(m[k]) for k in ("mu_s", "mu_2", "I0", "d", "rho_s")))


def eos_struct(e) -> LpEos:
    return LpEos(*(float(e[k]) for k in ("phi_c", "phi_min", "phi_max", "alpha", "beta")))


def params_struct(q) -> LpParams:
    return LpParams(float(q["h"]), float(q["radius"]), float(q["gx"]), float(q["gy"]),
                    float(q["gz"]), float(q.get("floor_z", 0.0)), int(q.get("mirror_mode", 1)),
                    int(q.get("precision", LP_FP64)), int(q.get("rebuild_every", 1)),
                    int(q.get("launch_mode", LP_LAUNCH_KERNELS)), float(q.get("skin", 0.0)),
                    int(q.get("free_surface", 0)), int(q.get("time_scheme", 0)),
                    float(q.get("period_x", 0.0)), float(q.get("period_y", 0.0)),
                    int(q.get("keep_lists", 0)), 0)


class Context:
    """An lp_ctx: the library's workspace on one device."""

    def __init__(self, max_particles: int, max_columns: int = 1, cap: int = LP_MAX_CAP,
                 device: int | None = None):
        L = lib()
        if device is None:
            device = torch.cuda.current_device()
        d = LpCtxDesc(int(device), int(max_columns), int(max_particles), int(cap), 0)
        h = ctypes.c_void_p()
        _check(L.lp_ctx_create(ctypes.byref(d), ctypes.byref(h)), "lp_ctx_create")
        self.handle = h
        self.device = device
        self.cap = cap

    def sync(self, stream=None, raise_on_error: bool = True) -> dict:
        dg = LpDiag()
        st = lib().lp_ctx_sync(self.handle, _stream(stream), ctypes.byref(dg))
        out = {k: getattr(dg, k) for k, _ in LpDiag._fields_ if k != "pad"}
        out["status"] = st
        if raise_on_error:
            _check(st, "lp_ctx_sync")
        return out

    def set_wait_limit(self, max_spins: int = 1 << 25, extra_arrivals: int = 0):
        _check(lib().lp_ctx_set_wait_limit(self.handle, int(max_spins), int(extra_arrivals)),
               "lp_ctx_set_wait_limit")

    def set_adjoint_memory(self, max_bytes: int = -1):
        """Device memory lp_step_adjoint may keep for a whole run's data
        (-1: half of the free memory; 0: re-run each checkpoint segment)."""
        _check(lib().lp_ctx_set_adjoint_memory(self.handle, int(max_bytes)),
               "lp_ctx_set_adjoint_memory")

    def profile(self, enable: bool = True):
        _check(lib().lp_ctx_profile(self.handle, int(bool(enable))), "lp_ctx_profile")

    def phase_times(self, stream=None) -> dict:
        """Device ms per phase (sort, neighbors, pass1, pass2), kernel launches
        and steps since the last call."""
        ms = (ctypes.c_double * 4)()
        la, stp = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().lp_ctx_phase_times(self.handle, _stream(stream), ms, ctypes.byref(la),
                                        ctypes.byref(stp)), "lp_ctx_phase_times")
        return dict(ms=dict(zip(("sort", "neighbors", "pass1", "pass2"), list(ms))),
                    launches=la.value, steps=stp.value)

    def close(self):
        if getattr(self, "handle", None):
            lib().lp_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Neighbors:
    """Library-owned stencils (valid until the next search or step on the context)."""

    def __init__(self, ctx: Context, s: LpNeighbors):
        self.ctx = ctx
        self.s = s

    def export(self, stream=None):
        n, cap = self.s.n, self.s.cap
        nbr = np.zeros((n, cap), dtype=np.int32)
        cnt = np.zeros(n, dtype=np.int32)
        _check(lib().lp_neighbors_export(self.ctx.handle, ctypes.byref(self.s),
                                         nbr.ctypes.data_as(_vp), cnt.ctypes.data_as(_vp),
                                         _stream(stream)), "lp_neighbors_export")
        return nbr, cnt


def lp_build_neighbors(ctx: Context, x, y, z, radius=None, r_const=0.0, mirror_mode=1,
                       floor_z=0.0, cap=LP_MAX_CAP, keep_nearest=False, column_offsets=None,
                       stream=None) -> Neighbors:
    """keep_nearest: False / LP_KEEP_ALL, True / LP_KEEP_NEAREST or
    LP_KEEP_OCTANTS (octant-balanced truncation)."""
    p, keep = _particles(dict(x=x, y=y, z=z), column_offsets, need_state=False)
    if radius is not None:
        _dev(radius, "radius")
    s = LpNeighbors()
    _check(lib().lp_build_neighbors(ctx.handle, ctypes.byref(p), _ptr(radius), float(r_const),
                                    int(mirror_mode), float(floor_z), int(cap),
                                    int(keep_nearest), ctypes.byref(s), _stream(stream)),
           "lp_build_neighbors")
    return Neighbors(ctx, s)


def lp_fit_derivatives(ctx: Context, x, y, z, nb: Neighbors, fields, mirror_sign, h,
                       floor_z=0.0, precision=LP_FP64, out=None, stream=None) -> torch.Tensor:
    p, keep = _particles(dict(x=x, y=y, z=z), None, need_state=False)
    nf = len(fields)
    for i, f in enumerate(fields):
        _dev(f, f"fields[{i}]")
    fp = (_vp * nf)(*[f.data_ptr() for f in fields])
    ms = (ctypes.c_double * nf)(*[float(v) for v in mirror_sign])
    if out is None:
        out = torch.empty((x.numel(), nf, 9), dtype=torch.float64, device=x.device)
    _dev(out, "out")
    _check(lib().lp_fit_derivatives(ctx.handle, ctypes.byref(p), ctypes.byref(nb.s), fp, ms, nf,
                                    float(h), float(floor_z), _ptr(out), int(precision),
                                    _stream(stream)), "lp_fit_derivatives")
    return out


NOALLOC_MAX_PARTICLES = 1 << 20


def lp_fit_derivatives_noalloc(x, y, z, nbr, cnt, cap, fields, mirror_sign, h, out,
                               floor_z=0.0, precision=LP_FP64, stream=None, diag=False):
    """The fit without a context and without any device allocation by the
    library: stencils nbr (int32, k-major [cap, n] or flat) and cnt (int32, n)
    and the output `out` ([n, nf, 9] float64) are all supplied by the caller.
    With diag=True the call waits for the stream and returns (out, counts),
    counts holding n_fallback and flags; otherwise it returns out."""
    n = x.numel()
    for t, nm in ((x, "x"), (y, "y"), (z, "z")):
        _dev(t, nm)
    _dev(nbr, "nbr", torch.int32)
    _dev(cnt, "cnt", torch.int32)
    _dev(out, "out")
    nf = len(fields)
    for i, f in enumerate(fields):
        _dev(f, f"fields[{i}]")
    fp = (_vp * nf)(*[f.data_ptr() for f in fields])
    ms = (ctypes.c_double * nf)(*[float(v) for v in mirror_sign])
    dg = LpDiag() if diag else None
    _check(lib().lp_fit_derivatives_noalloc(n, _ptr(x), _ptr(y), _ptr(z), _ptr(nbr), _ptr(cnt),
                                            int(cap), fp, ms, nf, float(h), float(floor_z),
                                            _ptr(out), int(precision), _stream(stream),
                                            ctypes.byref(dg) if diag else None),
           "lp_fit_derivatives_noalloc")
    if diag:
        return out, {"n_fallback": dg.n_fallback, "flags": dg.flags}
    return out


def lp_mui_stress(ctx: Context, mui: dict, eos: dict, V, grad_u, stream=None) -> dict:
    n = V.numel()
    _dev(V, "V")
    _dev(grad_u, "grad_u")
    dev = V.device
    out = dict(gdot=torch.empty((n, 6), dtype=torch.float64, device=dev),
               gdot_norm=torch.empty(n, dtype=torch.float64, device=dev),
               P=torch.empty(n, dtype=torch.float64, device=dev),
               eta=torch.empty(n, dtype=torch.float64, device=dev),
               regime=torch.empty(n, dtype=torch.int8, device=dev))
    m, e = mui_struct(mui), eos_struct(eos)
    _check(lib().lp_mui_stress(ctx.handle, ctypes.byref(m), ctypes.byref(e), n, _ptr(V),
                               _ptr(grad_u), _ptr(out["gdot"]), _ptr(out["gdot_norm"]),
                               _ptr(out["P"]), _ptr(out["eta"]), _ptr(out["regime"]),
                               _stream(stream)), "lp_mui_stress")
    return out


def _mui_array(mui, ncol):
    if isinstance(mui, dict):
        mui = [mui] * ncol
    if len(mui) != ncol:
        raise ValueError("one mu(I) parameter set per column is required")
    return (LpMui * ncol)(*[mui_struct(m) for m in mui])


def lp_step(ctx: Context, state: dict, mui, eos: dict, params: dict, dt: float, nsteps: int,
            column_offsets=None, stream=None):
    """nsteps LP steps in place on the tensors of `state`: all CUDA tensors,
    or all CPU tensors (pinned for asynchronous copies), which the library
    copies to the device and back on `stream`; read them after the stream
    has finished."""
    p, keep = _particles(state, column_offsets, allow_host=True)
    ma = _mui_array(mui, p.ncolumns)
    e, q = eos_struct(eos), params_struct(params)
    _check(lib().lp_step(ctx.handle, ctypes.byref(p), ma, ctypes.byref(e), ctypes.byref(q),
                         float(dt), int(nsteps), _stream(stream)), "lp_step")


def lp_autotune(ctx: Context, state: dict, mui, eos: dict, params: dict, dt: float,
                steps_per_trial: int = 5, table_path: str | None = None, column_offsets=None,
                stream=None) -> dict:
    """Pick block sizes and the launch mode for this workload (applied to ctx)."""
    p, keep = _particles(state, column_offsets)
    ma = _mui_array(mui, p.ncolumns)
    e, q = eos_struct(eos), params_struct(params)
    t = LpTuning()
    _check(lib().lp_autotune(ctx.handle, ctypes.byref(p), ma, ctypes.byref(e), ctypes.byref(q),
                             float(dt), int(steps_per_trial),
                             table_path.encode() if table_path else None, ctypes.byref(t),
                             _stream(stream)), "lp_autotune")
    return {k: getattr(t, k) for k, _ in LpTuning._fields_ if k != "pad"}


def lp_ctx_set_tuning(ctx: Context, block_neighbors=128, block_pass1=128, block_pass2=128,
                      launch_mode=LP_LAUNCH_GRAPH):
    t = LpTuning(int(block_neighbors), int(block_pass1), int(block_pass2), int(launch_mode), 0.0,
                 0, 0)
    _check(lib().lp_ctx_set_tuning(ctx.handle, ctypes.byref(t)), "lp_ctx_set_tuning")


def lp_step_adjoint(ctx: Context, initial: dict, mui, eos: dict, params: dict, dt: float,
                    nsteps: int, checkpoint_every: int, seed: dict, want_initial: bool = False,
                    stream=None):
    """dL/d(mu_s, mu_2, I0) (and optionally dL/d initial state) for the seed dL/d final state."""
    p, keep = _particles(initial, None)
    sp, keep2 = _particles(seed, None)
    ma = _mui_array(mui, 1)
    e, q = eos_struct(eos), params_struct(params)
    dmui = torch.zeros(3, dtype=torch.float64, device=initial["x"].device)
    gi = None
    gp = None
    if want_initial:
        gi = {k: torch.zeros_like(initial[k]) for k in FIELDS}
        gp, _ = _particles(gi, None)
    _check(lib().lp_step_adjoint(ctx.handle, ctypes.byref(p), ma, ctypes.byref(e),
                                 ctypes.byref(q), float(dt), int(nsteps), int(checkpoint_every),
                                 ctypes.byref(sp), _ptr(dmui),
                                 ctypes.byref(gp) if gp is not None else None, _stream(stream)),
           "lp_step_adjoint")
    return dmui, gi
