"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs.

Bars: neighbour sets bit-exact (canonical sorted order); FP64 derivatives
within 1e-11 relative per coefficient class (max |diff| / max |oracle|);
state after 50 FP64 steps within 1e-9 relative (displacement, velocity and
change of V each normalised by the oracle's largest value). The mixed-precision
path is held to the bounds stated in each test.
"""
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
             launch_mode=0, skin=0.0)
    q.update(kw)
    return q


# ------------------------------------------------------------ neighbours ---

def test_neighbors_bitexact_cube_with_mirrors(dev, capi, orc):
    wl = W.cube(20)
    x, y, z = (wl.state[k] for k in "xyz")
    ref, rcnt, over = orc.neighbors(x, y, z, r_const=wl.radius, mirror_mode=1, cap=64, brute=True)
    assert over == 0
    ctx = capi.Context(wl.n, cap=64)
    nb = capi.lp_build_neighbors(ctx, T(x, dev), T(y, dev), T(z, dev), r_const=wl.radius,
                                 mirror_mode=1, cap=64)
    d = ctx.sync()
    got, gcnt = nb.export()
    assert np.array_equal(gcnt, rcnt)
    assert np.array_equal(got, ref[:, :64])
    assert d["min_stencil"] == rcnt.min() and d["max_stencil"] == rcnt.max()


def test_neighbors_keep_nearest_per_particle_radius(dev, capi, orc):
    x, y, z, rad, _, _ = W.sweep_lattice(n_side=18, nfields=1)
    ref, rcnt, _ = orc.neighbors(x, y, z, radius=rad, mirror_mode=1, cap=48, keep_nearest=True)
    ctx = capi.Context(x.size, cap=64)
    nb = capi.lp_build_neighbors(ctx, T(x, dev), T(y, dev), T(z, dev), radius=T(rad, dev),
                                 mirror_mode=1, cap=48, keep_nearest=True)
    ctx.sync()
    got, gcnt = nb.export()
    assert np.array_equal(gcnt, rcnt)
    assert np.array_equal(got, ref[:, :48])
    assert gcnt.max() == 48 and gcnt.min() >= 1


def test_neighbors_octant_balanced_per_particle_radius(dev, capi, orc):
    """Octant-balanced truncation (Sec. 3.1 item 6) bit-exact against the
    oracle, with floor mirrors and per-particle radii; an unknown rule is
    rejected on the host."""
    x, y, z, rad, _, _ = W.sweep_lattice(n_side=18, nfields=1)
    ref, rcnt, _ = orc.neighbors(x, y, z, radius=rad, mirror_mode=1, cap=48, keep_nearest=2)
    near, _, _ = orc.neighbors(x, y, z, radius=rad, mirror_mode=1, cap=48, keep_nearest=1)
    ctx = capi.Context(x.size, cap=64)
    X = [T(a, dev) for a in (x, y, z)]
    nb = capi.lp_build_neighbors(ctx, *X, radius=T(rad, dev), mirror_mode=1, cap=48,
                                 keep_nearest=capi.LP_KEEP_OCTANTS)
    ctx.sync()
    got, gcnt = nb.export()
    assert np.array_equal(gcnt, rcnt)
    assert np.array_equal(got, ref[:, :48])
    assert not np.array_equal(ref, near)
    with pytest.raises(capi.LpError) as e:
        capi.lp_build_neighbors(ctx, *X, radius=T(rad, dev), mirror_mode=1, cap=48,
                                keep_nearest=3)
    assert e.value.status == capi.LP_ERR_INVALID_ARG


def test_neighbors_stay_within_columns(dev, capi, orc):
    wl = W.columns(ncol=5, n_lo=300, n_hi=1500, only=[0, 1, 2, 3, 4])
    x, y, z = (wl.state[k] for k in "xyz")
    offs = wl.column_offsets
    ctx = capi.Context(wl.n, max_columns=8, cap=64)
    nb = capi.lp_build_neighbors(ctx, T(x, dev), T(y, dev), T(z, dev), r_const=wl.radius,
                                 mirror_mode=1, cap=64, column_offsets=offs)
    ctx.sync()
    got, gcnt = nb.export()
    for c in range(len(offs) - 1):
        b, e = offs[c], offs[c + 1]
        ref, rcnt, _ = orc.neighbors(x[b:e], y[b:e], z[b:e], r_const=wl.radius, mirror_mode=1,
                                     cap=64)
        assert np.array_equal(gcnt[b:e], rcnt)
        g = got[b:e].astype(np.int64) & 0xFFFFFFFF
        r = ref[:, :64].astype(np.int64) & 0xFFFFFFFF
        mask = np.arange(64)[None, :] < rcnt[:, None]
        gi = np.where(mask, (g & 0x7FFFFFFF) - b, 0)
        ri = np.where(mask, r & 0x7FFFFFFF, 0)
        assert np.array_equal(gi, ri)
        assert np.array_equal(np.where(mask, g >> 31, 0), np.where(mask, r >> 31, 0))


def test_neighbor_overflow_is_reported(dev, capi):
    wl = W.cube(8)
    ctx = capi.Context(wl.n, cap=64)
    capi.lp_build_neighbors(ctx, *(T(wl.state[k], dev) for k in "xyz"), r_const=wl.radius,
                            mirror_mode=1, cap=8)
    with pytest.raises(capi.LpError) as e:
        ctx.sync()
    assert e.value.status == capi.LP_ERR_STENCIL_OVERFLOW
    assert ctx.sync()["status"] == 0  # cleared


# ------------------------------------------------------------------ fits ---

def _class_err(got, ref):
    """max |diff| / max |ref| per field and class (first / second derivatives)."""
    out = []
    for f in range(ref.shape[1]):
        for sl in (slice(0, 3), slice(3, 9)):
            r = ref[:, f, sl]
            out.append(np.abs(got[:, f, sl] - r).max() / np.abs(r).max())
    return max(out)


@pytest.fixture(scope="module")
def sweep(dev, capi, orc):
    x, y, z, rad, fields, spec = W.sweep_lattice(n_side=24)
    ctx = capi.Context(x.size, cap=64)
    X = [T(a, dev) for a in (x, y, z)]
    nb = capi.lp_build_neighbors(ctx, *X, radius=T(rad, dev), mirror_mode=0, cap=48,
                                 keep_nearest=True)
    ctx.sync()
    nbr, cnt = nb.export()
    ref, rank = orc.fit(x, y, z, nbr, cnt, fields, [1.0] * 4, 1e-3)
    return dict(x=x, y=y, z=z, fields=fields, ctx=ctx, X=X, nb=nb, ref=ref, rank=rank, nbr=nbr,
                cnt=cnt)


def test_fit_fp64_parity(dev, capi, sweep):
    F = [T(f, dev) for f in sweep["fields"]]
    got = capi.lp_fit_derivatives(sweep["ctx"], *sweep["X"], sweep["nb"], F, [1.0] * 4, 1e-3,
                                  precision=capi.LP_FP64)
    sweep["ctx"].sync()
    err = _class_err(got.cpu().numpy(), sweep["ref"])
    assert err <= 1e-11, err


def test_fit_mixed_error_bound(dev, capi, sweep):
    F = [T(f, dev) for f in sweep["fields"]]
    got = capi.lp_fit_derivatives(sweep["ctx"], *sweep["X"], sweep["nb"], F, [1.0] * 4, 1e-3,
                                  precision=capi.LP_MIXED)
    sweep["ctx"].sync()
    err = _class_err(got.cpu().numpy(), sweep["ref"])
    print(f"mixed-precision fit: max class error vs FP64 oracle = {err:.3e}")
    # one FP64 refinement contracts the FP32 error by about kappa(G) u_32; on
    # this +-0.2h lattice (kappa(G) up to ~1e4) that leaves a few 1e-6
    assert err <= 1e-5, err


def test_fit_mixed_ff_error_bound(dev, capi, sweep):
    """Float-float fit (moments, factor, right-hand sides on FP32 pairs): its
    error is about 2^-44 kappa(G), far below the FP32-plus-refinement mode."""
    F = [T(f, dev) for f in sweep["fields"]]
    got = capi.lp_fit_derivatives(sweep["ctx"], *sweep["X"], sweep["nb"], F, [1.0] * 4, 1e-3,
                                  precision=capi.LP_MIXED_FF)
    sweep["ctx"].sync()
    err = _class_err(got.cpu().numpy(), sweep["ref"])
    print(f"float-float fit: max class error vs FP64 oracle = {err:.3e}")
    assert err <= 1e-9, err


def test_fit_mixed_ff_mirrors_and_field_groups(dev, capi, orc):
    """Floor mirrors with even, odd and zero mirror signs, five fields (a full
    and a partial group of three): float-float against the oracle."""
    x, y, z, rad, fields, spec = W.sweep_lattice(n_side=14, nfields=5, index=7)
    ctx = capi.Context(x.size, cap=64)
    X = [T(a, dev) for a in (x, y, z)]
    nb = capi.lp_build_neighbors(ctx, *X, radius=T(rad, dev), mirror_mode=1, floor_z=0.0, cap=48,
                                 keep_nearest=True)
    ctx.sync()
    nbr, cnt = nb.export()
    assert (nbr < 0).any()  # some entries are floor mirrors (bit 31)
    ms = [1.0, -1.0, 0.0, 1.0, -1.0]
    ref, _ = orc.fit(x, y, z, nbr, cnt, fields, ms, 1e-3)
    got = capi.lp_fit_derivatives(ctx, *X, nb, [T(f, dev) for f in fields], ms, 1e-3,
                                  precision=capi.LP_MIXED_FF).cpu().numpy()
    ctx.sync()
    err = _class_err(got, ref)
    print(f"float-float fit with mirrors: max class error = {err:.3e}")
    assert err <= 1e-9, err


def test_fit_mixed_ff_limits(dev, capi, orc):
    """Float-float fit at the field limit (16 fields: five groups of three and
    one of one) against the oracle; 17 fields and an empty set."""
    x, y, z, rad, fields, _ = W.sweep_lattice(n_side=10, nfields=16, index=9)
    ctx = capi.Context(x.size, cap=64)
    X = [T(a, dev) for a in (x, y, z)]
    nb = capi.lp_build_neighbors(ctx, *X, radius=T(rad, dev), mirror_mode=0, cap=48,
                                 keep_nearest=True)
    ctx.sync()
    nbr, cnt = nb.export()
    ref, _ = orc.fit(x, y, z, nbr, cnt, fields, [1.0] * 16, 1e-3)
    F = [T(f, dev) for f in fields]
    got = capi.lp_fit_derivatives(ctx, *X, nb, F, [1.0] * 16, 1e-3,
                                  precision=capi.LP_MIXED_FF).cpu().numpy()
    ctx.sync()
    err = _class_err(got, ref)
    assert err <= 1e-9, err
    with pytest.raises(capi.LpError) as e:
        capi.lp_fit_derivatives(ctx, *X, nb, F + F[:1], [1.0] * 17, 1e-3,
                                precision=capi.LP_MIXED_FF)
    assert e.value.status == capi.LP_ERR_INVALID_ARG
    # n = 0: nothing to do, no error
    E = [torch.zeros(0, dtype=torch.float64, device=dev) for _ in range(3)]
    nb0 = capi.lp_build_neighbors(ctx, *E, r_const=2.2e-3, mirror_mode=0, cap=48)
    out = capi.lp_fit_derivatives(ctx, *E, nb0, [E[0]], [1.0], 1e-3,
                                  precision=capi.LP_MIXED_FF)
    ctx.sync()
    assert out.shape == (0, 1, 9)


def test_fit_fallback_matches_oracle_projection(dev, capi, orc):
    """Sparse clouds (m < 9) and planar stencils take the pivoted-QR path; the
    fitted values A c (unique even when the basic solution is not) match."""
    rng = np.random.default_rng(21)
    n = 600
    x = rng.uniform(0, 0.03, n)
    y = rng.uniform(0, 0.03, n)
    z = np.where(rng.uniform(size=n) < 0.5, 0.005, rng.uniform(0, 0.03, n))
    f = np.stack([np.sin(100 * x) + y * 50, np.cos(70 * y) * z * 30])
    r = 0.0042
    ctx = capi.Context(n, cap=64)
    X = [T(a, dev) for a in (x, y, z)]
    nb = capi.lp_build_neighbors(ctx, *X, r_const=r, mirror_mode=0, cap=64)
    ctx.sync()
    nbr, cnt = nb.export()
    assert (cnt < 9).any()
    ref, rank = orc.fit(x, y, z, nbr, cnt, f, [1, 1], 1e-3)
    for prec in (capi.LP_FP64, capi.LP_MIXED_FF):
        got = capi.lp_fit_derivatives(ctx, *X, nb, [T(a, dev) for a in f], [1, 1], 1e-3,
                                      precision=prec).cpu().numpy()
        d = ctx.sync()
        assert d["n_fallback"] > 0
        _check_projection(x, y, z, f, nbr, cnt, got, ref, n, 1e-9 if prec == capi.LP_FP64 else 1e-7)


def test_fit_skips_out_of_range_entries(dev, capi):
    """A stencil entry whose index is outside [0, n) is skipped as if absent:
    every precision mode gives the bits of the same stencil without it, both
    in the Cholesky path and in the pivoted-QR fallback (sparse stencils)."""
    rng = np.random.default_rng(23)
    n = 600
    x = rng.uniform(0, 0.03, n)
    y = rng.uniform(0, 0.03, n)
    z = np.where(rng.uniform(size=n) < 0.5, 0.005, rng.uniform(0, 0.03, n))
    f = np.stack([np.sin(100 * x) + y * 50, np.cos(70 * y) * z * 30])
    ctx = capi.Context(n, cap=64)
    X = [T(a, dev) for a in (x, y, z)]
    F = [T(a, dev) for a in f]
    nb = capi.lp_build_neighbors(ctx, *X, r_const=0.0042, mirror_mode=0, cap=64)
    ctx.sync()
    nbr, cnt = nb.export()
    bad = nbr.copy()
    bcnt = cnt.copy()
    hit = np.flatnonzero((np.arange(n) % 3 == 0) & (cnt < 64))
    for i in hit:  # insert an out-of-range index in the middle of the stencil
        k = cnt[i] // 2
        bad[i, k + 1:cnt[i] + 1] = nbr[i, k:cnt[i]]
        bad[i, k] = n + 7 + i
        bcnt[i] += 1
    assert (cnt[hit] < 9).any() and (cnt[hit] >= 9).any()

    def own(nb_rows, c):
        t = torch.tensor(np.ascontiguousarray(nb_rows.T).ravel(), dtype=torch.int32, device=dev)
        tc = torch.tensor(c, dtype=torch.int32, device=dev)
        return (t, tc), capi.Neighbors(ctx, capi.LpNeighbors(t.data_ptr(), tc.data_ptr(), n, 64,
                                                              0))
    keep_a, nb_a = own(nbr, cnt)
    keep_b, nb_b = own(bad, bcnt)
    for prec in (capi.LP_FP64, capi.LP_MIXED, capi.LP_MIXED_FF):
        a = capi.lp_fit_derivatives(ctx, *X, nb_a, F, [1, 1], 1e-3, precision=prec).cpu().numpy()
        da = ctx.sync()
        b = capi.lp_fit_derivatives(ctx, *X, nb_b, F, [1, 1], 1e-3, precision=prec).cpu().numpy()
        db = ctx.sync()
        assert da["n_fallback"] == db["n_fallback"] > 0, prec
        assert np.array_equal(a, b), prec


def _check_projection(x, y, z, f, nbr, cnt, got, ref, n, tol):
    h = 1e-3
    for i in range(n):
        m = cnt[i]
        if m == 0:
            continue
        j = nbr[i, :m]
        dx, dy, dz = (x[j] - x[i]) / h, (y[j] - y[i]) / h, (z[j] - z[i]) / h
        A = np.stack([dx, dy, dz, dx * dx / 2, dy * dy / 2, dz * dz / 2, dx * dy, dx * dz,
                      dy * dz], 1)
        sc = np.array([h] * 3 + [h * h] * 6)
        for q in range(2):
            fa = A @ (got[i, q] * sc)
            fb = A @ (ref[i, q] * sc)
            b = f[q, j] - f[q, i]
            assert np.abs(fa - fb).max() <= tol * (np.abs(b).max() + 1e-30), (i, q)


# ----------------------------------------------------------------- mu(I) ---

def test_mui_stress_parity(dev, capi, orc):
    rng = np.random.default_rng(5)
    n = 5000
    phi = rng.uniform(0.3, 0.62, n)
    G = rng.standard_normal((n, 9)) * 20
    pd = W.param_dict(W.cube(4))
    mui, eos = _dicts(pd)
    ctx = capi.Context(16)
    out = capi.lp_mui_stress(ctx, mui, eos, T(1 / phi, dev), T(G, dev))
    ctx.sync()
    gd, gn, P, eta, reg = orc.mui_stress(1 / phi, G, orc.params(**pd))
    assert np.array_equal(out["regime"].cpu().numpy(), reg)
    for a, b in ((out["gdot"], gd), (out["gdot_norm"], gn), (out["P"], P), (out["eta"], eta)):
        a = a.cpu().numpy()
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


# ------------------------------------------------------------------ step ---

def _rel(diff, scale):
    """max |diff| / max |scale|; exact agreement required where scale is 0."""
    m = np.abs(scale).max()
    d = np.abs(diff).max()
    if m == 0.0:
        return 0.0 if d == 0.0 else np.inf
    return d / m


def _state_err(got, ref, s0):
    e = {}
    for k in "xyz":
        e[k] = _rel((got[k] - s0[k]) - (ref[k] - s0[k]), ref[k] - s0[k])
    for k in "uvw":
        e[k] = _rel(got[k] - ref[k], ref[k])
    e["V"] = _rel((got["V"] - s0["V"]) - (ref["V"] - s0["V"]), ref["V"] - s0["V"])
    return e


def _run_gpu(capi, dev, wl, pd, nsteps, prec=0, offsets=None, mui=None, stream=None, **kw):
    ctx = capi.Context(wl.n, max_columns=1 if offsets is None else len(offsets) - 1, cap=64)
    st = {k: T(wl.state[k], dev) for k in capi.FIELDS}
    m, eos = _dicts(pd)
    capi.lp_step(ctx, st, mui if mui is not None else m, eos, _prm(pd, precision=prec, **kw),
                 pd["dt"], nsteps, column_offsets=offsets, stream=stream)
    d = ctx.sync(stream)
    return {k: st[k].cpu().numpy() for k in capi.FIELDS}, d


def test_step_fp64_parity_50_steps(dev, capi, orc):
    wl = W.cube(20)
    pd = W.param_dict(wl)
    ref, rd = orc.step(wl.state, orc.params(**pd), 50, brute=False)
    got, d = _run_gpu(capi, dev, wl, pd, 50)
    e = _state_err(got, ref, wl.state)
    print("FP64 50-step errors:", {k: f"{v:.2e}" for k, v in e.items()})
    assert max(e.values()) <= 1e-9, e
    assert d["n_nonfinite"] == 0 and d["n_overflow"] == 0


def test_step_mixed_error_bound(dev, capi, orc):
    wl = W.cube(20)
    pd = W.param_dict(wl)
    ref, _ = orc.step(wl.state, orc.params(**pd), 50, brute=False)
    got, d = _run_gpu(capi, dev, wl, pd, 50, prec=1)
    e = _state_err(got, ref, wl.state)
    print("MIXED 50-step errors:", {k: f"{v:.2e}" for k, v in e.items()})
    assert max(e.values()) <= 1e-9, e


def test_step_mixed_ff_error_bound(dev, capi, orc):
    """Float-float mode (no FP64 on stencil rows) against the FP64 oracle."""
    wl = W.cube(20)
    pd = W.param_dict(wl)
    ref, _ = orc.step(wl.state, orc.params(**pd), 50, brute=False)
    got, d = _run_gpu(capi, dev, wl, pd, 50, prec=2)
    e = _state_err(got, ref, wl.state)
    print("MIXED_FF 50-step errors:", {k: f"{v:.2e}" for k, v in e.items()})
    assert max(e.values()) <= 1e-10, e
    assert d["n_nonfinite"] == 0


def test_step_graph_replay_is_bitwise_identical(dev, capi):
    wl = W.cube(12)
    pd = W.param_dict(wl)
    s = torch.cuda.Stream()
    a, _ = _run_gpu(capi, dev, wl, pd, 12, stream=s, launch_mode=0)
    b, _ = _run_gpu(capi, dev, wl, pd, 12, stream=s, launch_mode=1)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_step_persistent_launch_is_bitwise_identical(dev, capi):
    """One cooperative persistent launch per step (phases separated by a grid
    barrier) gives exactly the per-phase kernels' result, for one column and
    for a batch of columns."""
    wl = W.cube(12)
    pd = W.param_dict(wl)
    a, _ = _run_gpu(capi, dev, wl, pd, 6, launch_mode=0)
    b, d = _run_gpu(capi, dev, wl, pd, 6, launch_mode=2)
    assert d["status"] == 0 and d["flags"] == 0
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    wc = W.columns(ncol=6, n_lo=300, n_hi=3000, only=list(range(6)))
    pc = W.param_dict(wc)
    mui_c = [dict(_dicts(pc)[0], mu_s=float(m)) for m in wc.mu_s_col]
    for prec in (0, 1, 2):
        a, _ = _run_gpu(capi, dev, wc, pc, 5, prec=prec, offsets=wc.column_offsets, mui=mui_c,
                        launch_mode=0, rebuild_every=2)
        b, _ = _run_gpu(capi, dev, wc, pc, 5, prec=prec, offsets=wc.column_offsets, mui=mui_c,
                        launch_mode=2, rebuild_every=2)
        for k in a:
            assert np.array_equal(a[k], b[k]), (prec, k)
    # with Verlet candidate lists the persistent kernel takes the search
    # branch from the device flag and filters every step
    for prec in (0, 1, 2):
        a, _ = _run_gpu(capi, dev, wc, pc, 6, prec=prec, offsets=wc.column_offsets, mui=mui_c,
                        launch_mode=0, skin=0.1 * pc["h"])
        b, d = _run_gpu(capi, dev, wc, pc, 6, prec=prec, offsets=wc.column_offsets, mui=mui_c,
                        launch_mode=2, skin=0.1 * pc["h"])
        assert d["status"] == 0 and d["flags"] == 0
        for k in a:
            assert np.array_equal(a[k], b[k]), ("skin", prec, k)


def test_persistent_phase_times(dev, capi):
    """With profiling on, a persistent launch times its own phases (marks
    after the grid barriers): all four are positive, their sum stays within
    the launch's wall time, and the state is still the per-phase kernels'."""
    wc = W.columns(ncol=6, n_lo=3000, n_hi=9000, only=list(range(6)))
    pc = W.param_dict(wc)
    mui_c = [dict(_dicts(pc)[0], mu_s=float(m)) for m in wc.mu_s_col]
    m, eos = _dicts(pc)
    ctx = capi.Context(wc.n, max_columns=8, cap=64)
    a, _ = _run_gpu(capi, dev, wc, pc, 4, prec=2, offsets=wc.column_offsets, mui=mui_c,
                    launch_mode=0, skin=0.1 * pc["h"])
    st = {k: T(wc.state[k], dev) for k in capi.FIELDS}
    ctx.profile(True)
    ctx.phase_times()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    capi.lp_step(ctx, st, mui_c, eos, _prm(pc, precision=2, launch_mode=2, skin=0.1 * pc["h"]),
                 pc["dt"], 4, column_offsets=wc.column_offsets)
    e1.record()
    pt = ctx.phase_times()
    ctx.profile(False)
    d = ctx.sync()
    assert d["status"] == 0 and d["flags"] == 0
    wall = e0.elapsed_time(e1)
    print("persistent phase ms:", pt["ms"], "wall ms:", wall)
    assert all(v > 0.0 for v in pt["ms"].values()), pt
    assert sum(pt["ms"].values()) <= wall * 1.001 + 0.05, (pt, wall)
    for k in capi.FIELDS:
        assert np.array_equal(st[k].cpu().numpy(), a[k]), k


def test_autotune_choices_and_table(dev, capi, tmp_path):
    """The tuner returns valid block sizes and a launch mode, leaves the
    caller's particles unchanged, and the chosen block sizes do not change a
    single bit of the step (each particle's arithmetic is the same)."""
    wc = W.columns(ncol=8, n_lo=500, n_hi=4000, only=list(range(8)))
    pc = W.param_dict(wc)
    mui_c = [dict(_dicts(pc)[0], mu_s=float(m)) for m in wc.mu_s_col]
    m, eos = _dicts(pc)
    ctx = capi.Context(wc.n, max_columns=8, cap=64)
    st = {k: T(wc.state[k], dev) for k in capi.FIELDS}
    table = str(tmp_path / "tuning.txt")
    t1 = capi.lp_autotune(ctx, st, mui_c, eos, _prm(pc, precision=1), pc["dt"], 3,
                          table_path=table, column_offsets=wc.column_offsets)
    for k in ("block_neighbors", "block_pass1", "block_pass2"):
        assert t1[k] in (64, 128, 256)
    assert t1["launch_mode"] in (1, 2) and t1["ms_per_step"] > 0 and t1["from_table"] == 0
    for k in capi.FIELDS:
        assert np.array_equal(st[k].cpu().numpy(), wc.state[k]), k
    t2 = capi.lp_autotune(ctx, st, mui_c, eos, _prm(pc, precision=1), pc["dt"], 3,
                          table_path=table, column_offsets=wc.column_offsets)
    assert t2["from_table"] == 1
    for k in ("block_neighbors", "block_pass1", "block_pass2", "launch_mode"):
        assert t2[k] == t1[k]
    ref, _ = _run_gpu(capi, dev, wc, pc, 4, prec=1, offsets=wc.column_offsets, mui=mui_c)
    for bs in (64, 256):
        ctx2 = capi.Context(wc.n, max_columns=8, cap=64)
        capi.lp_ctx_set_tuning(ctx2, bs, bs, bs)
        s2 = {k: T(wc.state[k], dev) for k in capi.FIELDS}
        capi.lp_step(ctx2, s2, mui_c, eos, _prm(pc, precision=1), pc["dt"], 4,
                     column_offsets=wc.column_offsets)
        ctx2.sync()
        for k in capi.FIELDS:
            assert np.array_equal(s2[k].cpu().numpy(), ref[k]), (bs, k)


def test_step_verlet_skin_matches_full_search(dev, capi, orc):
    """Candidate lists within radius + skin, filtered every step with the
    exact test, give the stencils of a full search: the same state (up to the
    row order inside a stencil), including when the displacement test
    triggers new searches during the run."""
    wl = W.cube(16)
    pd = W.param_dict(wl)
    ref, _ = _run_gpu(capi, dev, wl, pd, 20, launch_mode=0)
    s = torch.cuda.Stream()
    for skin, mode in ((0.1 * pd["h"], 0), (0.1 * pd["h"], 1), (2e-4 * pd["h"], 1),
                       (0.1 * pd["h"], 2), (2e-4 * pd["h"], 2)):
        got, d = _run_gpu(capi, dev, wl, pd, 20, launch_mode=mode, skin=skin, stream=s)
        assert d["n_overflow"] == 0
        e = _state_err(got, ref, wl.state)
        assert max(e.values()) <= 1e-12, (skin, mode, e)
    orc_ref, _ = orc.step(wl.state, orc.params(**pd), 20, brute=False)
    e = _state_err(got, orc_ref, wl.state)
    assert max(e.values()) <= 1e-9, e


def test_step_verlet_skin_under_shear_drift(dev, capi):
    """Gas-regime shear flow u = G z (no stresses, so no instability): pairs
    drift across the stencil radius and particles move beyond skin/2, so the
    candidate lists are searched again during the run; the state equals the
    full-search run's."""
    wl = W.cube(14)
    s = dict(wl.state)
    s["u"] = 50.0 * s["z"]
    s["V"] = np.full(wl.n, 1.0 / 0.3)  # phi below phi_min: gas, a = g
    wl.state = s
    pd = dict(W.param_dict(wl), mirror_mode=0, gz=0.0)
    ref, _ = _run_gpu(capi, dev, wl, pd, 40, launch_mode=0)
    moved = np.abs(ref["x"] - s["x"]).max() / pd["h"]
    assert moved > 0.1  # several searches were needed with skin 0.1h
    for mode in (0, 1, 2):
        got, d = _run_gpu(capi, dev, wl, pd, 40, launch_mode=mode, skin=0.1 * pd["h"],
                          stream=torch.cuda.Stream())
        e = _state_err(got, ref, s)
        assert max(e.values()) <= 1e-12, (mode, e)
        # stencils built by the filter (the persistent launch filters every step)
        print("mode", mode, "stencils built per particle-step:", d["n_stencils"] / (40 * wl.n))
        assert wl.n <= d["n_stencils"] <= 40 * wl.n
        if mode == 2:
            assert d["n_stencils"] == 40 * wl.n


def test_step_verlet_filter_skipping_under_slow_shear(dev, capi, orc):
    """Slow gas-regime shear u = G z over 200 steps: particles keep their
    stencils while their candidates provably stay on one side of the radius,
    and are filtered again before any pair can cross it; pairs do cross (the
    oracle's stencils of the first and last states differ), and the state
    equals the full-search run's."""
    wl = W.cube(14)
    s = dict(wl.state)
    s["u"] = 1.0 * s["z"]  # 0.003h relative drift of pairs 1.5h apart over the run
    s["V"] = np.full(wl.n, 1.0 / 0.3)  # gas: a = g
    wl.state = s
    pd = dict(W.param_dict(wl), mirror_mode=0, gz=0.0)
    nsteps = 200
    ref, _ = _run_gpu(capi, dev, wl, pd, nsteps, launch_mode=0)
    p = orc.params(**pd)
    n0, c0, _ = orc.step_stencils(s["x"], s["y"], s["z"], p, brute=False)
    n1, c1, _ = orc.step_stencils(ref["x"], ref["y"], ref["z"], p, brute=False)
    changed = sum(set(n0[i, :c0[i]].tolist()) != set(n1[i, :c1[i]].tolist())
                  for i in range(wl.n))
    print("particles whose stencil changed over the run:", changed)
    assert changed > 0.03 * wl.n
    for mode in (0, 1):
        got, d = _run_gpu(capi, dev, wl, pd, nsteps, launch_mode=mode, skin=0.1 * pd["h"],
                          stream=torch.cuda.Stream())
        e = _state_err(got, ref, s)
        built = d["n_stencils"] / (nsteps * wl.n)
        print("mode", mode, "stencils built per particle-step:", built, "errors:", e)
        assert max(e.values()) <= 1e-12, (mode, e)
        assert built < 0.99, built


def test_step_verlet_filter_skipped_at_rest(dev, capi):
    """A lattice at rest without gravity stays bitwise at rest; with candidate
    lists the first step filters every particle and the later steps keep the
    stencils (no particle moved), with the same state as the full search."""
    wl = W.cube(12)
    s = dict(wl.state)
    s["u"] = np.zeros(wl.n)
    wl.state = s
    pd = dict(W.param_dict(wl), gz=0.0)
    ref, _ = _run_gpu(capi, dev, wl, pd, 10, launch_mode=0)
    for mode in (0, 1):
        got, d = _run_gpu(capi, dev, wl, pd, 10, launch_mode=mode, skin=0.1 * pd["h"],
                          stream=torch.cuda.Stream())
        for k in capi.FIELDS:
            assert np.array_equal(got[k], ref[k]) and np.array_equal(got[k], s[k]), (mode, k)
        assert wl.n <= d["n_stencils"] <= 1.01 * wl.n, (mode, d["n_stencils"])


def test_persistent_bounded_wait_reports_timeout(dev, capi):
    """A grid barrier that waits for blocks that do not exist gives up after
    its spin limit: the kernel ends, lp_ctx_sync reports LP_ERR_TIMEOUT, and
    the same context then runs a normal step (no GPU fault, no hang)."""
    wl = W.cube(10)
    pd = W.param_dict(wl)
    m, eos = _dicts(pd)
    ctx = capi.Context(wl.n, cap=64)
    st = {k: T(wl.state[k], dev) for k in capi.FIELDS}
    ctx.set_wait_limit(max_spins=2000, extra_arrivals=1)
    capi.lp_step(ctx, st, m, eos, _prm(pd, launch_mode=2), pd["dt"], 1)
    d = ctx.sync(raise_on_error=False)
    assert d["status"] == capi.LP_ERR_TIMEOUT and d["flags"] & 0x4
    ctx.set_wait_limit()
    st = {k: T(wl.state[k], dev) for k in capi.FIELDS}
    capi.lp_step(ctx, st, m, eos, _prm(pd, launch_mode=2), pd["dt"], 2)
    assert ctx.sync()["status"] == 0
    ref, _ = _run_gpu(capi, dev, wl, pd, 2, launch_mode=0)
    for k in capi.FIELDS:
        assert np.array_equal(st[k].cpu().numpy(), ref[k]), k


def test_step_rebuild_period_matches_oracle(dev, capi, orc):
    wl = W.cube(10)
    pd = W.param_dict(wl)
    for R, steps in ((3, 10), (5, 10)):
        ref, _ = orc.step(wl.state, orc.params(**pd), steps, rebuild_every=R)
        got, _ = _run_gpu(capi, dev, wl, pd, steps, rebuild_every=R)
        e = _state_err(got, ref, wl.state)
        assert max(e.values()) <= 1e-9, (R, e)


def test_step_columns_match_oracle_per_column(dev, capi, orc):
    wl = W.columns(ncol=4, n_lo=400, n_hi=2500, only=[0, 1, 2, 3])
    pd = W.param_dict(wl)
    mui_c = [dict(_dicts(pd)[0], mu_s=float(m)) for m in wl.mu_s_col]
    got, _ = _run_gpu(capi, dev, wl, pd, 10, offsets=wl.column_offsets, mui=mui_c)
    offs = wl.column_offsets
    for c in range(len(offs) - 1):
        b, e = offs[c], offs[c + 1]
        sc = {k: v[b:e] for k, v in wl.state.items()}
        ref, _ = orc.step(sc, orc.params(**dict(pd, mu_s=float(wl.mu_s_col[c]))), 10)
        err = _state_err({k: got[k][b:e] for k in got}, ref, sc)
        assert max(err.values()) <= 1e-9, (c, err)


def test_step_all_three_regimes(dev, capi, orc):
    """A sheared 12^3 cube on the no-slip floor whose solid fraction
    0.47 + 0.14 sin(2 pi x/L) cos(2 pi y/L + 0.3) spans the gas (phi <= 0.35),
    inertial and quasi-static (phi > 0.59) regimes: every branch of the
    acceleration (Sec. 2.2-2.3) and the regime decision run in one step. A
    soft quasi-static law (beta = 0.1 m^2/s^2, alpha = -beta phi_max) keeps the
    regime boundaries sane over the 30 steps (a 1e-15 perturbation of the
    start grows to about 3e-13 on the oracle). FP64 and float-float, kernels
    and graph replay, against the oracle on every particle."""
    h = 1e-3
    x, y, z = W.lattice_box(12, 12, 12, h, 0.05, np.random.default_rng(31))
    L = 12 * h
    phi = 0.47 + 0.14 * np.sin(2 * np.pi * x / L) * np.cos(2 * np.pi * y / L + 0.3)
    st = dict(x=x, y=y, z=z, u=z * (1 + 0.2 * np.sin(2 * np.pi * y / L)),
              v=0.4 * z * np.cos(2 * np.pi * x / L), w=np.zeros(x.size), V=1 / phi)
    pd = dict(W.param_dict(W.cube(12)), beta=0.1, alpha=-0.1 * 0.59)
    ref, rd = orc.step(st, orc.params(**pd), 30, brute=False)
    assert rd["n_gas"] > 0 and rd["n_quasistatic"] > 0 and rd["n_inertial"] > 0
    wl = W.Workload("three_regimes", h, pd["radius"], pd["dt"], st)
    for prec, tol in ((0, 1e-9), (2, 1e-10)):
        for mode in (capi.LP_LAUNCH_KERNELS, capi.LP_LAUNCH_GRAPH):
            got, d = _run_gpu(capi, dev, wl, pd, 30, prec=prec, launch_mode=mode,
                              stream=torch.cuda.Stream())
            assert d["n_nonfinite"] == 0
            assert d["n_gas"] == rd["n_gas"] and d["n_quasistatic"] == rd["n_quasistatic"], (
                prec, mode, d["n_gas"], d["n_quasistatic"], rd["n_gas"], rd["n_quasistatic"])
            e = _state_err(got, ref, st)
            print(f"three regimes, precision {prec}, mode {mode}:",
                  {k: f"{v:.2e}" for k, v in e.items()})
            assert max(e.values()) <= tol, (prec, mode, e)


def test_step_edge_cases(dev, capi, orc):
    pd = W.param_dict(W.cube(2))
    # empty set: no work, no error
    ctx = capi.Context(8)
    empty = {k: torch.zeros(0, dtype=torch.float64, device=dev) for k in capi.FIELDS}
    m, eos = _dicts(pd)
    capi.lp_step(ctx, empty, m, eos, _prm(pd), pd["dt"], 3)
    ctx.sync()
    # one particle near the floor: only its own mirror (m = 1 < 9, QR path)
    one = dict(x=np.array([0.0]), y=np.array([0.0]), z=np.array([0.4e-3]),
               u=np.array([0.01]), v=np.array([0.0]), w=np.array([-0.02]),
               V=np.array([1 / 0.585]))
    wl1 = W.Workload("one", pd["h"], pd["radius"], pd["dt"], one)
    ref, _ = orc.step(one, orc.params(**pd), 5)
    for prec in (0, 2):
        got, d = _run_gpu(capi, dev, wl1, pd, 5, prec=prec)
        assert d["n_fallback"] > 0
        for k in capi.FIELDS:
            assert np.allclose(got[k], ref[k], rtol=1e-12, atol=1e-18), (prec, k)
    # a few particles (one partial group of fit threads), float-float and FP64
    few = W.cube(3)
    pf = W.param_dict(few)
    ref, _ = orc.step(few.state, orc.params(**pf), 3)
    for prec, tol in ((0, 1e-9), (2, 1e-10)):
        got, _ = _run_gpu(capi, dev, few, pf, 3, prec=prec)
        e = _state_err(got, ref, few.state)
        assert max(e.values()) <= tol, (prec, e)
    # invalid arguments are rejected on the host
    with pytest.raises(capi.LpError) as e:
        capi.lp_step(ctx, {k: T(one[k], dev) for k in capi.FIELDS}, m, eos,
                     _prm(pd, rebuild_every=0), pd["dt"], 1)
    assert e.value.status == capi.LP_ERR_INVALID_ARG


@pytest.mark.slow
def test_derivative_sweep_full_size(dev, capi, orc):
    """Derivative-operator sweep at full size: 126^3 = 2,000,376 particles,
    jitter +-0.2h, radius U(1.8h, 2.6h), the 48 nearest, four fields.
    Stencils bit-exact on every particle; FP64 derivatives within 1e-11 of
    the oracle; the mixed mode's error and both modes' error against the
    analytic derivatives are reported."""
    x, y, z, rad, fields, spec = W.sweep_lattice(n_side=126)
    n = x.size
    ref_nbr, ref_cnt, _ = orc.neighbors(x, y, z, radius=rad, mirror_mode=0, cap=48,
                                        keep_nearest=True, brute=False)
    ctx = capi.Context(n, cap=64)
    X = [T(a, dev) for a in (x, y, z)]
    nb = capi.lp_build_neighbors(ctx, *X, radius=T(rad, dev), mirror_mode=0, cap=48,
                                 keep_nearest=True)
    ctx.sync()
    got_nbr, got_cnt = nb.export()
    assert np.array_equal(got_cnt, ref_cnt)
    assert np.array_equal(got_nbr, ref_nbr[:, :48])
    interior = ((x > 3e-3) & (x < 123e-3) & (y > 3e-3) & (y < 123e-3) & (z > 3e-3) &
                (z < 123e-3))
    assert got_cnt[interior].min() >= 16 and got_cnt.max() == 48
    ref, _ = orc.fit(x, y, z, ref_nbr, ref_cnt, fields, [1.0] * 4, 1e-3)
    F = [T(f, dev) for f in fields]
    g64 = capi.lp_fit_derivatives(ctx, *X, nb, F, [1.0] * 4, 1e-3,
                                  precision=capi.LP_FP64).cpu().numpy()
    gmx = capi.lp_fit_derivatives(ctx, *X, nb, F, [1.0] * 4, 1e-3,
                                  precision=capi.LP_MIXED).cpu().numpy()
    gff = capi.lp_fit_derivatives(ctx, *X, nb, F, [1.0] * 4, 1e-3,
                                  precision=capi.LP_MIXED_FF).cpu().numpy()
    ctx.sync()
    e64, emx, eff = _class_err(g64, ref), _class_err(gmx, ref), _class_err(gff, ref)
    # analytic derivatives of the seeded fields (interior particles)
    inner = ((x > 10e-3) & (x < 116e-3) & (y > 10e-3) & (y < 116e-3) & (z > 10e-3) & (z < 116e-3))
    ana = np.zeros((inner.sum(), 4, 9))
    for f, (a, kv, ph) in enumerate(spec):
        for k in range(len(a)):
            arg = kv[k, 0] * x[inner] + kv[k, 1] * y[inner] + kv[k, 2] * z[inner] + ph[k]
            c, s_ = np.cos(arg), np.sin(arg)
            for q in range(3):
                ana[:, f, q] += a[k] * kv[k, q] * c
            pairs = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))
            for q, (i1, i2) in enumerate(pairs):
                ana[:, f, 3 + q] -= a[k] * kv[k, i1] * kv[k, i2] * s_
    ea = _class_err(ref[inner], ana)
    print(f"sweep 2,000,376: FP64 vs oracle {e64:.2e}, mixed vs oracle {emx:.2e}, "
          f"float-float vs oracle {eff:.2e}, oracle vs analytic {ea:.2e}")
    assert e64 <= 1e-11, e64
    assert emx <= 1e-5, emx
    assert eff <= 1e-9, eff


@pytest.mark.slow
def test_derivative_sweep_octant_balanced_full_size(dev, capi, orc):
    """The 2,000,376-particle sweep with octant-balanced stencils: bit-exact
    against the oracle on every particle, FP64 derivatives within 1e-11 and
    float-float within 1e-9 of the oracle on those stencils. The error of
    both truncation rules against the analytic derivatives is reported, in
    the interior and near the faces."""
    x, y, z, rad, fields, spec = W.sweep_lattice(n_side=126)
    ref_nbr, ref_cnt, _ = orc.neighbors(x, y, z, radius=rad, mirror_mode=0, cap=48,
                                        keep_nearest=2, brute=False)
    ctx = capi.Context(x.size, cap=64)
    X = [T(a, dev) for a in (x, y, z)]
    nb = capi.lp_build_neighbors(ctx, *X, radius=T(rad, dev), mirror_mode=0, cap=48,
                                 keep_nearest=capi.LP_KEEP_OCTANTS)
    ctx.sync()
    got_nbr, got_cnt = nb.export()
    assert np.array_equal(got_cnt, ref_cnt)
    assert np.array_equal(got_nbr, ref_nbr[:, :48])
    ref, _ = orc.fit(x, y, z, ref_nbr, ref_cnt, fields, [1.0] * 4, 1e-3)
    F = [T(f, dev) for f in fields]
    g64 = capi.lp_fit_derivatives(ctx, *X, nb, F, [1.0] * 4, 1e-3,
                                  precision=capi.LP_FP64).cpu().numpy()
    gff = capi.lp_fit_derivatives(ctx, *X, nb, F, [1.0] * 4, 1e-3,
                                  precision=capi.LP_MIXED_FF).cpu().numpy()
    ctx.sync()
    e64, eff = _class_err(g64, ref), _class_err(gff, ref)
    nb1 = capi.lp_build_neighbors(ctx, *X, radius=T(rad, dev), mirror_mode=0, cap=48,
                                  keep_nearest=capi.LP_KEEP_NEAREST)
    g1 = capi.lp_fit_derivatives(ctx, *X, nb1, F, [1.0] * 4, 1e-3,
                                 precision=capi.LP_FP64).cpu().numpy()
    ctx.sync()
    ana = np.zeros((x.size, 4, 9))
    for f, (a, kv, ph) in enumerate(spec):
        for k in range(len(a)):
            arg = kv[k, 0] * x + kv[k, 1] * y + kv[k, 2] * z + ph[k]
            c, s_ = np.cos(arg), np.sin(arg)
            for q in range(3):
                ana[:, f, q] += a[k] * kv[k, q] * c
            pairs = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))
            for q, (i1, i2) in enumerate(pairs):
                ana[:, f, 3 + q] -= a[k] * kv[k, i1] * kv[k, i2] * s_
    L = 126e-3
    dmin = np.minimum.reduce([x, y, z, L - x, L - y, L - z])
    for name, sel in (("faces (< 2h)", dmin < 2e-3), ("interior", dmin > 5e-3)):
        print(f"sweep vs analytic, {name}: nearest {_class_err(g1[sel], ana[sel]):.3e}, "
              f"octant-balanced {_class_err(g64[sel], ana[sel]):.3e}")
    print(f"octant-balanced sweep: FP64 vs oracle {e64:.2e}, float-float vs oracle {eff:.2e}")
    assert e64 <= 1e-11, e64
    assert eff <= 1e-9, eff


def test_columns_smallest_four_match_oracle(dev, capi, orc):
    """The batched workload's four smallest columns, advanced together on
    the GPU (FP64 and float-float modes), against the oracle run column by
    column (30 steps: inside the stable horizon at h = 1e-3)."""
    full = W.columns()
    sizes = np.diff(full.column_offsets)
    four = sorted(np.argsort(sizes)[:4].tolist())
    wl = W.columns(only=four)
    pd = W.param_dict(wl)
    mui_c = [dict(_dicts(pd)[0], mu_s=float(m)) for m in wl.mu_s_col]
    offs = wl.column_offsets
    refs = []
    for c in range(4):
        b, e = offs[c], offs[c + 1]
        sc = {k: v[b:e] for k, v in wl.state.items()}
        refs.append((sc, orc.step(sc, orc.params(**dict(pd, mu_s=float(wl.mu_s_col[c]))), 30,
                                  brute=False)[0]))
    for prec, tol in ((0, 1e-9), (2, 1e-10)):
        got, d = _run_gpu(capi, dev, wl, pd, 30, prec=prec, offsets=offs, mui=mui_c,
                          launch_mode=1, stream=torch.cuda.Stream())
        assert d["n_nonfinite"] == 0
        for c in range(4):
            b, e = offs[c], offs[c + 1]
            err = _state_err({k: got[k][b:e] for k in got}, refs[c][1], refs[c][0])
            assert max(err.values()) <= tol, (prec, c, err)


def test_ragged_columns_with_empty_and_single_particle_columns(dev, capi, orc):
    """A batch whose columns include an empty one and a one-particle one (its
    only stencil entry is its own floor mirror: the QR path), between two
    ordinary columns: every launch mode gives the oracle's per-column result,
    FP64 and float-float."""
    wl = W.columns(ncol=3, n_lo=300, n_hi=900, only=[0, 1, 2])
    offs0 = wl.column_offsets
    one = dict(x=np.array([0.0]), y=np.array([0.0]), z=np.array([0.4e-3]), u=np.array([0.01]),
               v=np.array([0.0]), w=np.array([-0.02]), V=np.array([1 / 0.585]))
    parts = [{k: v[offs0[c]:offs0[c + 1]] for k, v in wl.state.items()} for c in range(3)]
    cols = [parts[0], {k: np.zeros(0) for k in one}, one, parts[1], parts[2]]
    state = {k: np.concatenate([c[k] for c in cols]) for k in capi.FIELDS}
    offs = np.concatenate([[0], np.cumsum([c["x"].size for c in cols])]).astype(np.int32)
    mus = [0.33, 0.38, 0.41, 0.36, 0.44]
    pd = W.param_dict(wl)
    mui_c = [dict(_dicts(pd)[0], mu_s=m) for m in mus]
    nst = 6
    refs = [orc.step(c, orc.params(**dict(pd, mu_s=mus[k])), nst, brute=False)[0]
            if c["x"].size else None for k, c in enumerate(cols)]
    wlr = W.Workload("ragged", pd["h"], pd["radius"], pd["dt"], state)
    for prec, tol in ((0, 1e-9), (2, 1e-10)):
        for mode in (0, 1, 2):
            got, d = _run_gpu(capi, dev, wlr, pd, nst, prec=prec, offsets=offs, mui=mui_c,
                              launch_mode=mode, stream=torch.cuda.Stream())
            assert d["status"] == 0 and d["n_nonfinite"] == 0 and d["n_fallback"] > 0
            for k, c in enumerate(cols):
                if refs[k] is None:
                    continue
                b, e = offs[k], offs[k + 1]
                if c["x"].size == 1:  # displacement of one particle: compare the values
                    for f in capi.FIELDS:
                        assert np.allclose(got[f][b:e], refs[k][f], rtol=1e-12, atol=1e-18), (
                            prec, mode, f)
                    continue
                err = _state_err({f: got[f][b:e] for f in got}, refs[k], c)
                assert max(err.values()) <= tol, (prec, mode, k, err)


@pytest.mark.slow
def test_columns_smallest_four_500_steps(dev, capi, orc):
    """The batched workload's stated length: its four smallest columns (about
    2,100 particles each) advanced together for 500 steps on the GPU, from
    solid fraction 0.5 with free-surface ghosts (the start that keeps this
    spacing inside its stable horizon, about 700 steps), in FP64 and
    float-float, against the oracle run column by column. A 1e-14 relative
    perturbation of the start grows to about 2.5e-11 of the displacement over
    these 500 steps on the oracle, so the bar stays 1e-9."""
    full = W.columns()
    sizes = np.diff(full.column_offsets)
    four = sorted(np.argsort(sizes)[:4].tolist())
    wl = W.columns(only=four)
    wl.state = dict(wl.state, V=np.full(wl.n, 1.0 / 0.5))
    pd = dict(W.param_dict(wl), free_surface=1)
    mui_c = [dict(_dicts(pd)[0], mu_s=float(m)) for m in wl.mu_s_col]
    offs = wl.column_offsets
    refs = []
    for c in range(4):
        b, e = offs[c], offs[c + 1]
        sc = {k: v[b:e] for k, v in wl.state.items()}
        refs.append((sc, orc.step(sc, orc.params(**dict(pd, mu_s=float(wl.mu_s_col[c]))), 500,
                                  brute=False)[0]))
    for prec in (0, 2):
        got, d = _run_gpu(capi, dev, wl, pd, 500, prec=prec, offsets=offs, mui=mui_c,
                          launch_mode=1, skin=0.1 * pd["h"], free_surface=1,
                          stream=torch.cuda.Stream())
        assert d["n_nonfinite"] == 0 and d["n_ghosts"] > 0
        for c in range(4):
            b, e = offs[c], offs[c + 1]
            err = _state_err({k: got[k][b:e] for k in got}, refs[c][1], refs[c][0])
            print(f"column {c}, precision {prec}, 500-step errors:",
                  {k: f"{v:.2e}" for k, v in err.items()})
            assert max(err.values()) <= 1e-9, (prec, c, err)


@pytest.mark.slow
def test_columns_full_batch_bench_configuration(dev, capi, orc):
    """The batched workload at full size (256 columns, 4.79M particles) in the
    benchmark's launch configuration: float-float fits, the autotuned
    schedule, Verlet skin 0.1h, one lp_step call of 10 steps. Graph replay and
    the persistent launch give the same bits. Six columns spread over the size
    range (the two smallest, the quartiles and the largest) each match the
    oracle run on that column alone within 1e-10, and each equals, bit for
    bit, the same column stepped alone on the GPU: a column's result does not
    depend on the batch around it."""
    wl = W.columns()
    pd = W.param_dict(wl)
    offs = wl.column_offsets
    ncol = len(offs) - 1
    sizes = np.diff(offs)
    order = np.argsort(sizes, kind="stable")
    pick = sorted({int(order[0]), int(order[1]), int(order[ncol // 4]), int(order[ncol // 2]),
                   int(order[3 * ncol // 4]), int(order[-1])})
    m, eos = _dicts(pd)
    mui_c = [dict(m, mu_s=float(mu)) for mu in wl.mu_s_col]
    stream = torch.cuda.Stream()
    nst = 10
    prm = _prm(pd, precision=2, launch_mode=capi.LP_LAUNCH_GRAPH, skin=0.1 * pd["h"])
    ctx = capi.Context(wl.n, max_columns=ncol, cap=64)
    init = {k: T(wl.state[k], dev) for k in capi.FIELDS}
    tune = capi.lp_autotune(ctx, init, mui_c, eos, prm, pd["dt"], 3, column_offsets=offs,
                            stream=stream)
    print("autotuned schedule:", tune)
    outs = {}
    for mode in (capi.LP_LAUNCH_GRAPH, capi.LP_LAUNCH_PERSISTENT):
        st = {k: v.clone() for k, v in init.items()}
        with torch.cuda.stream(stream):
            capi.lp_step(ctx, st, mui_c, eos, dict(prm, launch_mode=mode), pd["dt"], nst,
                         column_offsets=offs, stream=stream)
        d = ctx.sync(stream)
        assert d["n_nonfinite"] == 0 and d["n_overflow"] == 0, (mode, d)
        outs[mode] = {k: st[k].cpu().numpy() for k in capi.FIELDS}
    for k in capi.FIELDS:
        assert np.array_equal(outs[capi.LP_LAUNCH_GRAPH][k], outs[capi.LP_LAUNCH_PERSISTENT][k]), k
    got = outs[capi.LP_LAUNCH_GRAPH]
    for c in pick:
        b, e = int(offs[c]), int(offs[c + 1])
        sc = {k: v[b:e] for k, v in wl.state.items()}
        ref, _ = orc.step(sc, orc.params(**dict(pd, mu_s=float(wl.mu_s_col[c]))), nst,
                          brute=False)
        gc = {k: got[k][b:e] for k in got}
        err = _state_err(gc, ref, sc)
        print(f"column {c} ({e - b} particles) 10-step errors:",
              {k: f"{v:.2e}" for k, v in err.items()})
        assert max(err.values()) <= 1e-10, (c, err)
        alone = W.Workload("column", pd["h"], pd["radius"], pd["dt"], sc)
        ga, da = _run_gpu(capi, dev, alone, pd, nst, prec=2, mui=mui_c[c],
                          launch_mode=capi.LP_LAUNCH_GRAPH, skin=0.1 * pd["h"], stream=stream)
        assert da["n_nonfinite"] == 0
        for k in capi.FIELDS:
            assert np.array_equal(ga[k], gc[k]), (c, k)


@pytest.mark.slow
def test_columns_full_batch_500_steps(dev, capi, orc):
    """The batch at its stated length in the benchmark's `full_length`
    configuration: all 256 columns (4.79M particles) from solid fraction 0.5
    with free-surface ghosts, float-float, Verlet skin 0.1h, the autotuned
    launch, 500 steps in one call. No value turns non-finite, and the four
    smallest columns match the oracle run on each column alone within 1e-9,
    as in the four-column batch. (Not bit for bit against a smaller batch: the
    Verlet search is flagged by any particle of the batch, and a search
    re-sorts the particles and so the order of each stencil's sums.)"""
    full = W.columns()
    pd = dict(W.param_dict(full), free_surface=1)
    offs = full.column_offsets
    ncol = len(offs) - 1
    sizes = np.diff(offs)
    four = sorted(np.argsort(sizes)[:4].tolist())
    m, eos = _dicts(pd)
    mui_c = [dict(m, mu_s=float(mu)) for mu in full.mu_s_col]
    stream = torch.cuda.Stream()
    prm = _prm(pd, precision=2, launch_mode=capi.LP_LAUNCH_GRAPH, skin=0.1 * pd["h"],
               free_surface=1)
    ctx = capi.Context(full.n, max_columns=ncol, cap=64)
    state0 = dict(full.state, V=np.full(full.n, 2.0))
    init = {k: T(state0[k], dev) for k in capi.FIELDS}
    tune = capi.lp_autotune(ctx, init, mui_c, eos, prm, pd["dt"], 3, column_offsets=offs,
                            stream=stream)
    st = {k: v.clone() for k, v in init.items()}
    with torch.cuda.stream(stream):
        capi.lp_step(ctx, st, mui_c, eos, dict(prm, launch_mode=tune["launch_mode"]), pd["dt"],
                     500, column_offsets=offs, stream=stream)
    d = ctx.sync(stream)
    assert d["n_nonfinite"] == 0 and d["n_ghosts"] > 0
    got = {k: st[k].cpu().numpy() for k in capi.FIELDS}
    for c in four:
        b, e = int(offs[c]), int(offs[c + 1])
        sc = {k: v[b:e] for k, v in state0.items()}
        gc = {k: got[k][b:e] for k in got}
        ref, _ = orc.step(sc, orc.params(**dict(pd, mu_s=float(full.mu_s_col[c]))), 500,
                          brute=False)
        err = _state_err(gc, ref, sc)
        print(f"column {c} ({e - b} particles) in the full batch, 500 steps:",
              {k: f"{v:.2e}" for k, v in err.items()})
        assert max(err.values()) <= 1e-9, (c, err)


@pytest.mark.slow
def test_large_column_sampled_particles(dev, capi, orc):
    """The headline column scaled up at the same spacing (R = 0.06 m, h = R/150,
    21.2M particles: indices past 2^24), 10 float-float steps with graph replay
    and Verlet skin 0.1h, as the benchmark's large-column line runs them, from
    the spreading flow u_r = 0.5 m/s (r/R)(z/H) (at rest only the particles
    near the floor would leave free fall within 10 steps). A
    particle's state after 10 steps depends only on particles within
    10 x 2 x 2.2h = 44h of it (each step's two fit passes reach 2.2h each), so
    the oracle computes sampled particles one by one: on the ball of radius 50h
    around each, 10 steps. Their displacements, velocities and changes of V
    match within 1e-9 of the ball's largest."""
    wl = W.cylinder(R=0.06, spacing_div=150, index=2)
    pd = W.param_dict(wl)
    assert wl.n > (1 << 24)
    H, R, h = 0.12, 0.06, pd["h"]
    st = dict(wl.state)
    st["u"] = 0.5 * st["x"] / R * (st["z"] / H)
    st["v"] = 0.5 * st["y"] / R * (st["z"] / H)
    wl.state = st
    got, d = _run_gpu(capi, dev, wl, pd, 10, prec=2, launch_mode=capi.LP_LAUNCH_GRAPH,
                      skin=0.1 * pd["h"], stream=torch.cuda.Stream())
    assert d["n_nonfinite"] == 0
    s0 = wl.state
    x, y, z = s0["x"], s0["y"], s0["z"]
    r = np.sqrt(x * x + y * y)
    picks = [int(np.argmin((x - 0.0) ** 2 + (y - 0.0) ** 2 + (z - 0.5 * H) ** 2)),  # centre
             int(np.argmin(x * x + y * y + z * z)),                               # floor
             int(np.argmin((r - R) ** 2 + (z - H) ** 2)),                         # top rim
             wl.n - 1, (1 << 24) + 12345]                                         # late indices
    for i in picks:
        ball = np.nonzero((x - x[i]) ** 2 + (y - y[i]) ** 2 + (z - z[i]) ** 2
                          <= (50 * h) ** 2)[0]
        sub = {k: v[ball] for k, v in s0.items()}
        ref, _ = orc.step(sub, orc.params(**pd), 10, brute=False)
        j = int(np.nonzero(ball == i)[0][0])
        # (far from the floor the ball is still in exact free fall: no change
        # of x, y or V anywhere in it, and then none is allowed here either)
        rel = lambda a, sc: 0.0 if a == 0.0 else (a / sc if sc > 0.0 else np.inf)
        err = {}
        for k in "xyzV":
            scale = np.abs(ref[k] - sub[k]).max()
            err[k] = rel(abs((got[k][i] - s0[k][i]) - (ref[k][j] - sub[k][j])), scale)
        for k in "uvw":
            err[k] = rel(abs(got[k][i] - ref[k][j]), np.abs(ref[k]).max())
        print(f"particle {i} ({ball.size} in its ball):", {k: f"{v:.2e}" for k, v in err.items()})
        assert max(err.values()) <= 1e-9, (i, err)


@pytest.mark.slow
def test_step_full_size_cylinder(dev, capi, orc):
    """The column of radius 0.02 m at spacing R/50 (785k particles), three FP64
    steps in the launch configuration the benchmark uses, against the oracle on
    every particle."""
    wl = W.cylinder()
    pd = W.param_dict(wl)
    ref, _ = orc.step(wl.state, orc.params(**pd), 3, brute=False)
    got, d = _run_gpu(capi, dev, wl, pd, 3, launch_mode=0)
    e = _state_err(got, ref, wl.state)
    print("cylinder 3-step FP64 errors:", {k: f"{v:.2e}" for k, v in e.items()})
    assert max(e.values()) <= 1e-9, e
    gotm, _ = _run_gpu(capi, dev, wl, pd, 3, prec=1)
    em = _state_err(gotm, ref, wl.state)
    print("cylinder 3-step MIXED errors:", {k: f"{v:.2e}" for k, v in em.items()})
    assert max(em.values()) <= 1e-9, em
    gotf, _ = _run_gpu(capi, dev, wl, pd, 3, prec=2)
    ef = _state_err(gotf, ref, wl.state)
    print("cylinder 3-step MIXED_FF errors:", {k: f"{v:.2e}" for k, v in ef.items()})
    assert max(ef.values()) <= 1e-10, ef


@pytest.mark.slow
def test_step_full_size_cylinder_20_steps(dev, capi, orc):
    """The full column (785k particles), 20 steps in one lp_step call (graph
    replay, Verlet skin 0.1h), FP64 and float-float, against the oracle's
    20-step run on every particle. Between steps 10 and 20 the column starts
    to blow up: the inertial-regime equations grow short waves at this
    spacing, and the largest speed goes from about 3e-4 to about 9 m/s at a
    few particles (9 above 0.1 m/s; all still inertial, displacements below
    0.01h). A 1e-15 relative perturbation of the start grows to about 1.5e-12
    of each field's scale on the oracle over these 20 steps, so the bars stay
    1e-9 (FP64) and 1e-10 (float-float)."""
    wl = W.cylinder()
    pd = W.param_dict(wl)
    ref, rd = orc.step(wl.state, orc.params(**pd), 20, brute=False)
    print(f"oracle after 20 steps: max|u| {np.abs(ref['u']).max():.3e} m/s, "
          f"max|w| {np.abs(ref['w']).max():.3e} m/s")
    for prec, tol in ((0, 1e-9), (2, 1e-10)):
        got, d = _run_gpu(capi, dev, wl, pd, 20, prec=prec, launch_mode=capi.LP_LAUNCH_GRAPH,
                          skin=0.1 * pd["h"], stream=torch.cuda.Stream())
        assert d["n_nonfinite"] == 0
        e = _state_err(got, ref, wl.state)
        print(f"cylinder 20-step precision {prec} errors:",
              {k: f"{v:.2e}" for k, v in e.items()},
              {k: d[k] for k in ("n_gas", "n_quasistatic", "n_fallback")})
        assert max(e.values()) <= tol, (prec, e)


@pytest.mark.slow
def test_step_full_size_cylinder_bench_configuration(dev, capi, orc):
    """The benchmark's exact launch configuration on the full column (785k
    particles): float-float fits, graph replay, Verlet skin 0.1h, two lp_step
    calls of 10 steps from the initial state (the benchmark's restart). Both
    calls give the same bits, within 1e-10 of the oracle's 10-step run on
    every particle."""
    wl = W.cylinder()
    pd = W.param_dict(wl)
    ref, _ = orc.step(wl.state, orc.params(**pd), 10, brute=False)
    ctx = capi.Context(wl.n, cap=64)
    m, eos = _dicts(pd)
    init = {k: T(wl.state[k], dev) for k in capi.FIELDS}
    st = {k: v.clone() for k, v in init.items()}
    stream = torch.cuda.Stream()
    prm = _prm(pd, precision=2, launch_mode=1, skin=0.1 * pd["h"])
    outs = []
    with torch.cuda.stream(stream):
        for call in range(2):
            for k in capi.FIELDS:
                st[k].copy_(init[k])
            capi.lp_step(ctx, st, m, eos, prm, pd["dt"], 10, stream=stream)
            d = ctx.sync(stream)
            assert d["n_nonfinite"] == 0
            outs.append({k: st[k].cpu().numpy() for k in capi.FIELDS})
    for k in capi.FIELDS:
        assert np.array_equal(outs[0][k], outs[1][k]), k
    e = _state_err(outs[0], ref, wl.state)
    print("cylinder 10-step bench configuration errors:", {k: f"{v:.2e}" for k, v in e.items()})
    assert max(e.values()) <= 1e-10, e
