"""Periodic boundaries (Sec. 3.1 item 9) on the GPU against the oracle.

Workload: the paper's periodic layer (Sec. 4: 0.03 m high, periodic along x
and y), shifted so that particles sit on the periodic edges, set sliding
(u = 0.5 m/s) down a 30 degree incline over a no-slip floor: in 50 steps
about 240 particles cross the edge at x = L and every edge particle has
neighbours across both edges.

Bars as without periods: stencil sizes and ghost counts equal the oracle's
(integer work), 1e-9 after 50 FP64 steps, the mixed bounds, bitwise equality
across launch modes. Offsets and displacements along periodic axes are
compared through their nearest images.
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


def _layer(n_xy=16, slide=0.5, incline=30.0, jitter=0.05):
    wl = W.periodic_layer(n_xy=n_xy, jitter=jitter)
    L, h = wl.extra["L"], wl.h
    pd = W.param_dict(wl)
    th = math.radians(incline)
    pd.update(gx=9.81 * math.sin(th), gz=-9.81 * math.cos(th), period_x=L, period_y=L)
    s = dict(wl.state)
    s["x"] = np.mod(s["x"] + 0.5 * h, L)
    s["y"] = np.mod(s["y"] + 0.3 * h, L)
    s["u"] = np.full(wl.n, slide)
    return s, pd, L


def _prm(pd, **kw):
    q = dict(h=pd["h"], radius=pd["radius"], gx=pd["gx"], gy=pd["gy"], gz=pd["gz"],
             floor_z=pd["floor_z"], mirror_mode=pd["mirror_mode"], precision=0, rebuild_every=1,
             launch_mode=0, skin=0.0, free_surface=0, time_scheme=0,
             period_x=pd.get("period_x", 0.0), period_y=pd.get("period_y", 0.0))
    q.update(kw)
    return q


def _opar(orc, pd, **kw):
    return orc.params(**dict(pd, **kw))


def _img(d, L):
    return np.mod(d + 0.5 * L, L) - 0.5 * L


def _rel(diff, scale):
    m = np.abs(scale).max()
    d = np.abs(diff).max()
    if m == 0.0:
        return 0.0 if d == 0.0 else np.inf
    return d / m


def _state_err(got, ref, s0, L, joint=False):
    """Per-field relative errors. joint=True scales the x, y and z
    displacement errors by the largest displacement component of any axis
    (the displacement as one vector), for runs where one axis barely moves."""
    e = {}
    disp = {k: _img(ref[k] - s0[k], L) for k in "xy"}
    disp["z"] = ref["z"] - s0["z"]
    dscale = max(np.abs(v).max() for v in disp.values())
    for k in "xy":
        e[k] = _rel(_img(got[k] - ref[k], L), dscale if joint else disp[k])
    e["z"] = _rel(got["z"] - ref["z"], dscale if joint else disp["z"])
    for k in "uvw":
        e[k] = _rel(got[k] - ref[k], ref[k])
    e["V"] = _rel(got["V"] - ref["V"], ref["V"] - s0["V"])
    return e


def _run_gpu(capi, dev, state, pd, nsteps, stream=None, raise_on_error=True, **kw):
    n = state["x"].size
    ctx = capi.Context(n, cap=64)
    st = {k: T(state[k], dev) for k in capi.FIELDS}
    m, eos = _dicts(pd)
    capi.lp_step(ctx, st, m, eos, _prm(pd, **kw), pd["dt"], nsteps, stream=stream)
    d = ctx.sync(stream, raise_on_error=raise_on_error)
    return {k: st[k].cpu().numpy() for k in capi.FIELDS}, d


def test_periodic_stencils_and_parity_50_steps(dev, capi, orc):
    s0, pd, L = _layer()
    nbr, cnt, _ = orc.step_stencils(s0["x"], s0["y"], s0["z"], _opar(orc, pd), brute=False)
    _, d1 = _run_gpu(capi, dev, s0, pd, 1)
    assert d1["n_stencil_rows"] == int(cnt.sum()) and d1["n_stencils"] == s0["x"].size
    assert d1["min_stencil"] == int(cnt.min()) and d1["max_stencil"] == int(cnt.max())
    ref, _ = orc.step(s0, _opar(orc, pd), 50, brute=False)
    crossed = int((ref["x"] < s0["x"] - 0.5 * L).sum())
    assert crossed > 100
    for prec, tol in ((0, 1e-9), (1, 1e-9), (2, 1e-10)):
        got, d = _run_gpu(capi, dev, s0, pd, 50, precision=prec)
        e = _state_err(got, ref, s0, L)
        print(f"periodic precision {prec} 50-step errors:", {k: f"{v:.2e}" for k, v in e.items()})
        assert max(e.values()) <= tol, (prec, e)
        for k in "xy":
            assert (got[k] >= 0.0).all() and (got[k] < L).all(), (prec, k)
        assert d["n_nonfinite"] == 0 and d["n_overflow"] == 0
    # the periods change the step: the run without them differs
    plain, _ = orc.step(s0, _opar(orc, pd, period_x=0.0, period_y=0.0), 50, brute=False)
    assert max(_state_err(plain, ref, s0, L).values()) > 1e-6


@pytest.mark.parametrize("axes", ["x", "y"])
def test_one_periodic_axis_parity(dev, capi, orc, axes):
    """Periodic along one axis only; the other axis has free sides (ghosts on)."""
    s0, pd, L = _layer(n_xy=12)
    pd = dict(pd, period_x=L if axes == "x" else 0.0, period_y=L if axes == "y" else 0.0)
    op = _opar(orc, pd, free_surface=1)
    ref, rd = orc.step(s0, op, 30, brute=False)
    for prec, tol in ((0, 1e-9), (2, 1e-10)):
        got, d = _run_gpu(capi, dev, s0, pd, 30, precision=prec, free_surface=1)
        assert d["n_ghosts"] == rd["n_ghosts"], (axes, prec)
        e = _state_err(got, ref, s0, L)
        print(f"periodic {axes} precision {prec}:", {k: f"{v:.2e}" for k, v in e.items()})
        assert max(e.values()) <= tol, (axes, prec, e)
        k = "x" if axes == "x" else "y"
        assert (got[k] >= 0.0).all() and (got[k] < L).all()


def test_periodic_ghost_counts_and_parity(dev, capi, orc):
    """With periodic sides only the top of the layer is a free surface."""
    s0, pd, L = _layer()
    op = _opar(orc, pd, free_surface=1)
    nbr, cnt, _ = orc.step_stencils(s0["x"], s0["y"], s0["z"], op, brute=False)
    ref1 = int(((nbr.astype(np.int64) & 0x40000000) != 0).sum())
    _, d1 = _run_gpu(capi, dev, s0, pd, 1, free_surface=1)
    assert ref1 > 0 and d1["n_ghosts"] == ref1, (d1["n_ghosts"], ref1)
    ref, rd = orc.step(s0, op, 30, brute=False)
    for prec, tol in ((0, 1e-9), (2, 1e-10)):
        got, d = _run_gpu(capi, dev, s0, pd, 30, precision=prec, free_surface=1)
        assert d["n_ghosts"] == rd["n_ghosts"], (prec, d["n_ghosts"], rd["n_ghosts"])
        e = _state_err(got, ref, s0, L)
        print(f"periodic ghosts precision {prec}:", {k: f"{v:.2e}" for k, v in e.items()})
        assert max(e.values()) <= tol, (prec, e)


def test_periodic_heun_parity(dev, capi, orc):
    s0, pd, L = _layer()
    ref, _ = orc.step(s0, _opar(orc, pd, time_scheme=1), 30, brute=False)
    for prec, tol in ((0, 1e-9), (2, 1e-10)):
        got, _ = _run_gpu(capi, dev, s0, pd, 30, precision=prec, time_scheme=1)
        e = _state_err(got, ref, s0, L)
        assert max(e.values()) <= tol, (prec, e)
        assert (got["x"] >= 0.0).all() and (got["x"] < L).all()


def test_periodic_bitwise_across_launch_modes(dev, capi):
    """Per-phase kernels, graph replay and the persistent launch give the same
    bits with periods, with and without Verlet candidate lists, ghosts and
    Heun's method."""
    s0, pd, L = _layer(n_xy=12)
    for prec in (0, 2):
        for skin, fs, ts in ((0.0, 0, 0), (0.1 * pd["h"], 1, 0), (0.1 * pd["h"], 0, 1)):
            runs = [_run_gpu(capi, dev, s0, pd, 6, precision=prec, launch_mode=mode, skin=skin,
                             free_surface=fs, time_scheme=ts, stream=torch.cuda.Stream())
                    for mode in (0, 1, 2)]
            for got, d in runs[1:]:
                assert d["n_ghosts"] == runs[0][1]["n_ghosts"]
                for k in got:
                    assert np.array_equal(got[k], runs[0][0][k]), (prec, skin, fs, ts, k)


def test_translation_and_out_of_range_positions(dev, capi):
    """The step commutes with a translation along a periodic axis; positions
    given outside [0, L) are mapped in first."""
    s0, pd, L = _layer(n_xy=12)
    h = pd["h"]
    ref, _ = _run_gpu(capi, dev, s0, pd, 8)
    sh = 2.37 * h
    got, _ = _run_gpu(capi, dev, dict(s0, x=np.mod(s0["x"] + sh, L)), pd, 8)
    assert np.abs(_img(got["x"] - ref["x"] - sh, L)).max() < 1e-12 * L
    for k in ("y", "z", "u", "v", "w", "V"):
        assert np.allclose(got[k], ref[k], rtol=1e-9, atol=1e-11 * np.abs(ref[k]).max()), k
    far = dict(s0, x=s0["x"] + L, y=s0["y"] - 3 * L)
    got2, _ = _run_gpu(capi, dev, far, pd, 8)
    assert (got2["x"] >= 0).all() and (got2["x"] < L).all()
    assert (got2["y"] >= 0).all() and (got2["y"] < L).all()
    for k in "xy":
        assert np.abs(_img(got2[k] - ref[k], L)).max() < 1e-12 * L, k
    for k in ("z", "u", "v", "w", "V"):
        assert np.allclose(got2[k], ref[k], rtol=1e-9, atol=1e-11 * np.abs(ref[k]).max()), k


def test_periodic_layer_stays_laterally_homogeneous(dev, capi):
    """Unjittered periodic layer at rest on the floor, ghosts at the top: every
    particle of a horizontal lattice layer has the same stencil, so the layer
    moves as a 1D column (the 3D side of the paper's 1D/3D check)."""
    wl = W.periodic_layer(n_xy=8, jitter=0.0)
    pd = W.param_dict(wl)
    L = wl.extra["L"]
    pd.update(period_x=L, period_y=L)
    z0 = wl.state["z"]
    iz = np.rint(z0 / wl.h - 0.5).astype(int)
    for prec in (0, 2):
        got, d = _run_gpu(capi, dev, wl.state, pd, 20, precision=prec, free_surface=1)
        assert d["n_ghosts"] > 0
        for k in range(iz.max() + 1):
            sel = iz == k
            for f in ("z", "w", "V"):
                v = got[f][sel]
                assert np.ptp(v) <= 1e-10 * max(np.abs(v).max(), 1e-30), (prec, k, f)
            assert np.abs(got["u"][sel]).max() < 1e-12 and np.abs(got["v"][sel]).max() < 1e-12
        assert np.abs(got["z"] - z0).max() > 0.0


def test_periodic_parameter_checks(dev, capi):
    s0, pd, L = _layer(n_xy=12)
    m, eos = _dicts(pd)
    n = s0["x"].size
    ctx = capi.Context(n, cap=64)
    st = {k: T(s0[k], dev) for k in capi.FIELDS}
    r = pd["radius"]
    for bad in (2.9 * r, -L, float("nan"), float("inf")):
        with pytest.raises(capi.LpError) as ei:
            capi.lp_step(ctx, st, m, eos, _prm(pd, period_x=bad), pd["dt"], 1)
        assert ei.value.status == capi.LP_ERR_INVALID_ARG, bad
    with pytest.raises(capi.LpError) as ei:  # period below 3 (radius + skin)
        capi.lp_step(ctx, st, m, eos, _prm(pd, period_y=3.05 * r, skin=0.2 * r), pd["dt"], 1)
    assert ei.value.status == capi.LP_ERR_INVALID_ARG


def test_periodic_adjoint_matches_oracle_tangent(dev, capi, orc):
    """lp_step_adjoint with periodic x and y (sheared layer sliding across the
    edges, 12 FP64 steps, stencils rebuilt every 4) against the oracle's
    tangent-linear run, and dL/d(initial state) of particles on the edges
    against central differences of lp_step."""
    s0, pd, L = _layer(n_xy=8)
    s0 = dict(s0, u=0.5 + 20.0 * s0["z"])
    n = s0["x"].size
    m, eos = _dicts(pd)
    prm = _prm(pd)
    nsteps, C = 12, 4
    rng = np.random.default_rng(3)
    w = {k: rng.standard_normal(n) for k in capi.FIELDS}
    ctx = capi.Context(n, cap=64)
    init = {k: T(s0[k], dev) for k in capi.FIELDS}
    seed = {k: T(w[k], dev) for k in capi.FIELDS}
    dmui, gi = capi.lp_step_adjoint(ctx, init, m, eos, prm, pd["dt"], nsteps, C, seed,
                                    want_initial=True)
    got = dmui.cpu().numpy()
    _, tan = orc.step_tangent(s0, _opar(orc, pd), nsteps, rebuild_every=C)
    ref = np.array([sum((w[k] * tan[t, f]).sum() for f, k in enumerate(capi.FIELDS))
                    for t in range(3)])
    print("periodic adjoint", got, "tangent", ref)
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max(), (got, ref)

    def loss(state):
        st = {k: T(state[k], dev) for k in capi.FIELDS}
        capi.lp_step(ctx, st, m, eos, dict(prm, rebuild_every=C), pd["dt"], nsteps)
        ctx.sync()
        return sum(float((st[k].cpu().numpy() * w[k]).sum()) for k in capi.FIELDS)

    h = pd["h"]
    edge = np.flatnonzero((s0["x"] < 0.3 * h) | (s0["x"] > L - 0.3 * h))
    for i in edge[:2]:
        for k, eps in (("u", 1e-7), ("x", 1e-9), ("y", 1e-9)):
            sp = {q: v.copy() for q, v in s0.items()}
            sm = {q: v.copy() for q, v in s0.items()}
            sp[k][i] += eps
            sm[k][i] -= eps
            fd = (loss(sp) - loss(sm)) / (2 * eps)
            a = float(gi[k][i].item())
            assert abs(fd - a) <= 1e-5 * abs(a) + 1e-6, (i, k, fd, a)


@pytest.mark.slow
def test_periodic_layer_full_size(dev, capi, orc):
    """The periodic layer at the benchmark's size (162 x 162 x 30 = 787,320
    particles), periodic along x and y, free-surface ghosts, in the benchmark's
    launch configuration (graph replay on a stream, Verlet skin 0.1 h), here
    sliding down the incline so that every state component moves: three steps
    against the oracle on every particle, FP64 within 1e-9 and float-float
    within 1e-10 (displacement errors scaled by the largest displacement
    component: across the slope, y barely moves)."""
    s0, pd, L = _layer(n_xy=162)
    ref, rd = orc.step(s0, _opar(orc, pd, free_surface=1), 3, brute=False)
    stream = torch.cuda.Stream()
    for prec, tol in ((0, 1e-9), (2, 1e-10)):
        got, d = _run_gpu(capi, dev, s0, pd, 3, stream=stream, precision=prec,
                          launch_mode=capi.LP_LAUNCH_GRAPH, skin=0.1 * pd["h"], free_surface=1)
        e = _state_err(got, ref, s0, L, joint=True)
        print(f"periodic layer 787,320, precision {prec}, 3-step errors:",
              {k: f"{v:.2e}" for k, v in e.items()})
        assert max(e.values()) <= tol, (prec, e)
        assert d["n_nonfinite"] == 0 and d["n_overflow"] == 0
        assert d["n_ghosts"] == rd["n_ghosts"], (d["n_ghosts"], rd["n_ghosts"])


def test_periodic_layer_matches_the_1d_reduction(dev, capi):
    """Sec. 4.1's verification on the GPU path: the paper's layer on an
    unjittered 16 x 16 x 30 periodic lattice (at rest, solid fraction 0.50 at
    the floor to 0.48 at the top, free-surface ghosts, float-float fits,
    graph replay) against the layer reduced to 1D (oracle/layer1d.py) over
    600 steps: every level moves as one, the total compaction agrees to 5 %
    and the velocities above the two floor levels to 1e-2 (0.2 % and 1e-4
    after 200 steps; the floor levels split the compaction differently)."""
    from oracle import layer1d as L1
    wl = W.periodic_layer(n_xy=16, jitter=0.0)
    L, h, nz = wl.extra["L"], wl.h, 30
    pd = dict(W.param_dict(wl), period_x=L, period_y=L)
    mui, eos = _dicts(pd)
    s0 = wl.state
    lev = np.rint(s0["z"] / h - 0.5).astype(int)
    zl = (np.arange(nz) + 0.5) * h
    z1, w1 = zl.copy(), np.zeros(nz)
    V1 = np.array([s0["V"][lev == lv][0] for lv in range(nz)])
    V0 = V1.copy()
    ctx = capi.Context(wl.n, cap=64)
    st = {k: T(s0[k], dev) for k in capi.FIELDS}
    prm = _prm(pd, precision=capi.LP_MIXED_FF, launch_mode=capi.LP_LAUNCH_GRAPH,
               skin=0.1 * h, free_surface=1)
    done = 0
    for steps, tol_c, tol_w in ((200, 2e-3, 1e-4), (600, 5e-2, 1e-2)):
        capi.lp_step(ctx, st, mui, eos, prm, pd["dt"], steps - done)
        d = ctx.sync()
        assert d["n_nonfinite"] == 0
        for _ in range(steps - done):
            z1, w1, V1, _ = L1.step(z1, w1, V1, mui, eos, h, pd["radius"], pd["dt"])
        done = steps
        g = {k: st[k].cpu().numpy() for k in ("z", "w", "V")}
        for f in ("z", "w", "V"):
            spread = max(np.ptp(g[f][lev == lv]) for lv in range(nz))
            assert spread <= 1e-12 * np.abs(g[f]).max(), (steps, f, spread)
        w3 = np.array([g["w"][lev == lv][0] for lv in range(nz)])
        V3 = np.array([g["V"][lev == lv][0] for lv in range(nz)])
        c3, c1 = (V3 - V0).sum(), (V1 - V0).sum()
        ew = np.abs(w3[2:] - w1[2:]).max() / np.abs(w1).max()
        print(f"GPU layer, {steps} steps: compaction 3D {c3:.6e}, 1D {c1:.6e}; "
              f"velocity above the floor levels {ew:.2e}")
        assert abs(c3 - c1) <= tol_c * abs(c1), (steps, c3, c1)
        assert ew <= tol_w, (steps, ew)
