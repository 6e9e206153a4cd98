"""Pins of the oracle's periodic boundaries (Sec. 3.1 item 9: along one or two
horizontal axes a particle near one edge sees the particles near the opposite
edge as neighbours). Checked against what the geometry fixes:
- neighbour sets equal a periodic KD-tree's (scipy, boxsize), by brute force
  and by the grid scan, floor mirrors included;
- the step commutes with a translation along a periodic axis;
- a periodic layer of identical columns stays laterally homogeneous (the
  paper's 3D periodic layer reproduces its 1D computation);
- rigid translation wraps positions back into [0, L);
- with periodic sides only the top of a layer is a free surface (ghosts).
"""
import numpy as np
import pytest

from paper_2206_14061_gb300 import workloads as W

MB, GB, IDX = 0x80000000, 0x40000000, 0x3FFFFFFF


def _p(orc, L, **kw):
    d = dict(W.MUI)
    d.update(W.EOS)
    d.update(h=1e-3, radius=2.2e-3, gx=0.0, gy=0.0, gz=-9.81, floor_z=0.0, dt=1e-5,
             mirror_mode=1, period_x=L, period_y=L)
    d.update(kw)
    return orc.params(**d)


def _layer(nxy, nz, h, jitter, seed):
    x, y, z = W.lattice_box(nxy, nxy, nz, h, jitter, np.random.default_rng(seed))
    L = nxy * h
    return np.mod(x, L), np.mod(y, L), z, L


def _state(x, y, z, u=None):
    n = x.size
    zero = np.zeros(n)
    return dict(x=x, y=y, z=z, u=zero.copy() if u is None else u, v=zero.copy(), w=zero.copy(),
                V=np.full(n, 1 / 0.585))


def _sets(nbr, cnt):
    return [set(int(v) for v in nbr[i, :cnt[i]].astype(np.int64) & 0xFFFFFFFF)
            for i in range(cnt.size)]


def test_periodic_neighbours_match_periodic_kdtree(orc):
    spatial = pytest.importorskip("scipy.spatial")
    h, r = 1e-3, 2.2e-3
    x, y, z, L = _layer(8, 6, h, 0.2, 7)
    n = x.size
    pts = np.stack([x, y, z], 1)
    mir = np.stack([x, y, -z], 1)
    big = 100.0  # z is not periodic
    tree = spatial.cKDTree(np.concatenate([pts, mir]) + np.array([0, 0, 50.0]),
                           boxsize=[L, L, big])
    ref = []
    for i in range(n):
        s = set()
        for j in tree.query_ball_point(pts[i] + np.array([0, 0, 50.0]), r):
            if j == i:
                continue
            s.add(j if j < n else (j - n) | MB)
        ref.append(s)
    for brute in (True, False):
        nbr, cnt, over = orc.step_stencils(x, y, z, _p(orc, L, free_surface=0), brute=brute)
        assert over == 0
        assert _sets(nbr, cnt) == ref, brute


def test_step_commutes_with_periodic_translation(orc):
    h = 1e-3
    x, y, z, L = _layer(7, 5, h, 0.05, 3)
    s0 = _state(x, y, z, u=20.0 * z)
    p = _p(orc, L)
    ref, _ = orc.step(s0, p, 6, brute=True)
    shift = 2.37 * h
    s1 = dict(s0, x=np.mod(x + shift, L))
    got, _ = orc.step(s1, p, 6, brute=True)
    dx = np.mod(got["x"] - ref["x"] - shift + 0.5 * L, L) - 0.5 * L
    assert np.abs(dx).max() < 1e-12 * L
    for k in ("y", "z", "u", "v", "w", "V"):
        assert np.allclose(got[k], ref[k], rtol=1e-10, atol=1e-12 * np.abs(ref[k]).max()), k


def test_periodic_layer_stays_laterally_homogeneous(orc):
    """Unjittered periodic layer under gravity on the floor, free top with
    ghosts: every particle of a horizontal lattice layer sees the same
    stencil, so the layer moves as a 1D column."""
    h = 1e-3
    x, y, z, L = _layer(6, 8, h, 0.0, 0)
    s, d = orc.step(_state(x, y, z), _p(orc, L, free_surface=1), 20, brute=True)
    assert d["n_ghosts"] > 0
    iz = np.rint(z / h - 0.5).astype(int)
    moved = 0.0
    for k in range(8):
        sel = iz == k
        for f in ("z", "w", "V"):
            v = s[f][sel]
            assert np.ptp(v) <= 1e-12 * max(np.abs(v).max(), 1e-30), (k, f, np.ptp(v))
        assert np.abs(s["u"][sel]).max() < 1e-12 and np.abs(s["v"][sel]).max() < 1e-12
        moved = max(moved, np.abs(s["z"][sel] - z[sel]).max())
    assert moved > 0.0


def test_rigid_translation_wraps_positions(orc):
    h = 1e-3
    x, y, z, L = _layer(6, 4, h, 0.05, 5)
    n, nst = x.size, 9
    U = np.array([41.0, -23.0, 0.0])  # a few h per step: crosses the edges
    st = _state(x, y, z + 0.01)
    st.update(u=np.full(n, U[0]), v=np.full(n, U[1]))
    for scheme in (0, 1):
        s, _ = orc.step(st, _p(orc, L, gz=0.0, mirror_mode=0, time_scheme=scheme), nst)
        t = nst * 1e-5
        for c, k in enumerate("xy"):
            assert (s[k] >= 0).all() and (s[k] < L).all(), (scheme, k)
            ex = np.mod(st[k] + U[c] * t, L)
            dd = np.mod(s[k] - ex + 0.5 * L, L) - 0.5 * L
            assert np.abs(dd).max() < 1e-12, (scheme, k)
        assert np.allclose(s["u"], U[0], rtol=1e-13)


def test_periodic_sides_carry_no_ghosts(orc):
    h = 1e-3
    x, y, z, L = _layer(7, 6, h, 0.05, 11)
    nbr, cnt, _ = orc.step_stencils(x, y, z, _p(orc, L, free_surface=1), brute=True)
    iz = np.rint(z / h - 0.5).astype(int)
    has = np.array([(nbr[i, :cnt[i]].astype(np.int64) & GB).any() for i in range(x.size)])
    assert has[iz == 5].all()
    assert not has[iz < 5].any()


def test_tangent_linear_with_periods_matches_central_differences(orc):
    """The dual-number tangent run (the reference of the GPU adjoint) with
    periodic x and y, on a sheared layer sliding across the edges."""
    import math
    h = 1e-3
    x, y, z, L = _layer(8, 30, h, 0.05, 5)
    x, y = np.mod(x + 0.5 * h, L), np.mod(y + 0.3 * h, L)
    st = _state(x, y, z, u=0.5 + 20.0 * z)
    th = math.radians(30)
    kw = dict(gx=9.81 * math.sin(th), gz=-9.81 * math.cos(th))
    p = _p(orc, L, **kw)
    nst = reb = 8
    _, tan = orc.step_tangent(st, p, nst, rebuild_every=reb)
    for kix, name in enumerate(("mu_s", "mu_2", "I0")):
        eps = 1e-5
        sp_, _ = orc.step(st, _p(orc, L, **dict(kw, **{name: getattr(p, name) + eps})), nst,
                          rebuild_every=reb)
        sm_, _ = orc.step(st, _p(orc, L, **dict(kw, **{name: getattr(p, name) - eps})), nst,
                          rebuild_every=reb)
        for f, key in enumerate(("u", "v", "w", "V")):
            fd = (sp_[key] - sm_[key]) / (2 * eps)
            t = tan[kix, 3 + f]
            assert np.abs(t).max() > 0
            assert np.abs(fd - t).max() <= 1e-5 * np.abs(t).max(), (name, key)
