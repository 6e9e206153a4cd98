"""Verlet candidate lists kept across lp_step calls (lp_params.keep_lists).

A run of single-step calls that keeps its lists gives the bits of one call of
the same steps (both search once, then filter); a particle moved beyond
skin/2 between calls forces a search (the result then equals a fresh
context's up to summation order); a change of particle count or columns, or
another entry point in between, drops the lists.
"""
import math

import numpy as np
import pytest

from paper_2206_14061_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_14061_gb300 import build
    build.build()
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def capi(dev):
    from paper_2206_14061_gb300 import capi as C
    C.lib()
    return C


def T(a, dev):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)


def _dicts(pd):
    mui = {k: pd[k] for k in ("mu_s", "mu_2", "I0", "d", "rho_s")}
    eos = {k: pd[k] for k in ("phi_c", "phi_min", "phi_max", "alpha", "beta")}
    return mui, eos


def _prm(pd, **kw):
    q = dict(h=pd["h"], radius=pd["radius"], gx=pd["gx"], gy=pd["gy"], gz=pd["gz"],
             floor_z=pd["floor_z"], mirror_mode=pd["mirror_mode"], precision=0, rebuild_every=1,
             launch_mode=0, skin=0.1 * pd["h"], free_surface=0, time_scheme=0,
             period_x=pd.get("period_x", 0.0), period_y=pd.get("period_y", 0.0), keep_lists=1)
    q.update(kw)
    return q


def _cube():
    wl = W.cube(16)
    s = dict(wl.state)
    s["u"] = 20.0 * s["z"]
    return s, W.param_dict(wl)


def _layer():
    wl = W.periodic_layer(n_xy=12)
    L, h = wl.extra["L"], wl.h
    pd = W.param_dict(wl)
    th = math.radians(30)
    pd.update(gx=9.81 * math.sin(th), gz=-9.81 * math.cos(th), period_x=L, period_y=L)
    s = dict(wl.state)
    s["x"] = np.mod(s["x"] + 0.5 * h, L)
    s["u"] = np.full(wl.n, 0.5)
    return s, pd


def _calls(capi, dev, ctx, state, pd, steps, per_call, **kw):
    st = {k: T(state[k], dev) for k in capi.FIELDS}
    m, eos = _dicts(pd)
    done = 0
    while done < steps:
        k = min(per_call, steps - done)
        capi.lp_step(ctx, st, m, eos, _prm(pd, **kw), pd["dt"], k)
        done += k
    ctx.sync()
    return {k: st[k].cpu().numpy() for k in capi.FIELDS}


@pytest.mark.parametrize("case", ["cube", "layer_ghosts"])
def test_kept_lists_match_one_long_call(dev, capi, case):
    s0, pd = _cube() if case == "cube" else _layer()
    n = s0["x"].size
    fs = 1 if case == "layer_ghosts" else 0
    for prec in (0, 2):
        one = _calls(capi, dev, capi.Context(n, cap=64), s0, pd, 6, 6, precision=prec,
                     free_surface=fs)
        many = _calls(capi, dev, capi.Context(n, cap=64), s0, pd, 6, 1, precision=prec,
                      free_surface=fs)
        for k in one:
            assert np.array_equal(one[k], many[k]), (case, prec, k)
        # without keep_lists each single-step call searches afresh: same stencils
        fresh = _calls(capi, dev, capi.Context(n, cap=64), s0, pd, 6, 1, precision=prec,
                       free_surface=fs, keep_lists=0)
        for k in one:
            assert np.allclose(fresh[k], one[k], rtol=1e-12, atol=1e-14), (case, prec, k)


def test_moved_particles_force_a_search(dev, capi):
    s0, pd = _cube()
    n = s0["x"].size
    ctx = capi.Context(n, cap=64)
    s1 = _calls(capi, dev, ctx, s0, pd, 2, 1)
    # move every tenth particle by 0.4 h (> skin / 2) between the calls
    s1m = {k: v.copy() for k, v in s1.items()}
    s1m["x"][::10] += 0.4 * pd["h"]
    kept = _calls(capi, dev, ctx, s1m, pd, 3, 1)
    ref = _calls(capi, dev, capi.Context(n, cap=64), s1m, pd, 3, 1, keep_lists=0)
    for k in kept:
        assert np.allclose(kept[k], ref[k], rtol=1e-11, atol=1e-14), k


def test_lists_dropped_on_new_particles_or_other_calls(dev, capi):
    s0, pd = _cube()
    n = s0["x"].size
    ctx = capi.Context(n, cap=64)
    _calls(capi, dev, ctx, s0, pd, 2, 1)
    # fewer particles: no reuse, the bits of a fresh context
    sub = {k: v[: n - 100].copy() for k, v in s0.items()}
    a = _calls(capi, dev, ctx, sub, pd, 2, 1)
    b = _calls(capi, dev, capi.Context(n, cap=64), sub, pd, 2, 1)
    for k in a:
        assert np.array_equal(a[k], b[k]), ("count", k)
    # another entry point between two calls drops the lists as well
    _calls(capi, dev, ctx, s0, pd, 1, 1)
    capi.lp_build_neighbors(ctx, T(s0["x"], dev), T(s0["y"], dev), T(s0["z"], dev),
                            r_const=pd["radius"], mirror_mode=1, floor_z=0.0, cap=64)
    a = _calls(capi, dev, ctx, s0, pd, 2, 1)
    b = _calls(capi, dev, capi.Context(n, cap=64), s0, pd, 2, 1)
    for k in a:
        assert np.array_equal(a[k], b[k]), ("other call", k)
