"""The 3D oracle's periodic layer against the layer reduced to one dimension
(Sec. 4.1: the 3D code with periodic boundaries in both transverse directions
is verified against a reduced 1D computation of the same granular layer).

The 1D code (oracle/layer1d.py) is written independently of the 3D oracle.
Its own pins: its closure equals the 3D oracle's, its fit is exact on
quadratics, and a layer far above the floor falls freely with its density
unchanged. The comparison then runs the paper's layer (0.03 m high, at rest,
solid fraction 0.50 at the floor to 0.48 at the top, free surface on top,
no-slip floor) on an unjittered 7 x 7 x 30 periodic lattice and in 1D, step
for step. Both blow up long before the paper's final heights (the
inertial-regime equations grow short waves: test_oracle_stability.py), so the
comparison covers their first 600 steps.

The two discretisations differ where the velocity has a kink, at the floor
(mirror w* = -w): the 3D stencil of a floor particle weights the level above
nine times more than the level two above, the 1D stencil weighs them
equally. They split the compaction differently between the two floor levels
but agree on the layer's total compaction (the sum of V - V0 over the levels,
the layer height up to a factor) and on the motion above the floor levels."""
import numpy as np

from oracle import layer1d as L1
from paper_2206_14061_gb300 import workloads as W

H_LAYER = 0.03


def _phi0(z):
    return 0.50 + (0.48 - 0.50) * (z / H_LAYER)


def test_layer1d_closure_matches_the_3d_oracle(orc):
    mui, eos = dict(W.MUI), dict(W.EOS)
    phi = np.linspace(0.36, 0.589, 40)
    ref = orc.closure(phi, orc.params(**mui, **eos))
    for k, f in enumerate(phi):
        M, N, S, R = L1.closure(f, mui, eos)
        assert np.allclose([M, N, S, R], ref[k, :4], rtol=1e-13, atol=0), f


def test_layer1d_fit_exact_on_quadratics():
    h = 1e-3
    off = np.array([-2.1, -0.9, 1.05, 1.9, 0.4]) * h
    a, b, c = 0.3, -2.0, 7e3
    s = a + b * off + 0.5 * c * off * off
    d1, d2 = L1.fit(off, s - a, h)
    assert abs(d1 - b) <= 1e-12 * abs(b) and abs(d2 - c) <= 1e-10 * abs(c)


def test_layer1d_free_fall_above_the_floor():
    h, r, dt = 1e-3, 2.2e-3, 1e-5
    z = (np.arange(20) + 0.5) * h + 0.1
    w = np.zeros(z.size)
    V = 1.0 / _phi0(z - 0.1)
    V0 = V.copy()
    for k in range(5):
        z, w, V, _ = L1.step(z, w, V, dict(W.MUI), dict(W.EOS), h, r, dt)
    assert np.allclose(w, -9.81 * 5 * dt, rtol=1e-13, atol=0)
    assert np.array_equal(V, V0)


def test_periodic_layer_matches_the_1d_reduction(orc):
    h, r, dt, nxy, nz = 1e-3, 2.2e-3, 1e-5, 7, 30
    x, y, z = W.lattice_box(nxy, nxy, nz, h, 0.0, np.random.default_rng(0))
    Lp = nxy * h
    x, y = np.mod(x, Lp), np.mod(y, Lp)
    n = x.size
    st = dict(x=x, y=y, z=z, u=np.zeros(n), v=np.zeros(n), w=np.zeros(n), V=1.0 / _phi0(z))
    mui, eos = dict(W.MUI), dict(W.EOS)
    p = orc.params(**mui, **eos, h=h, radius=r, gx=0.0, gy=0.0, gz=-9.81, floor_z=0.0, dt=dt,
                   mirror_mode=1, free_surface=1, period_x=Lp, period_y=Lp)
    zl = (np.arange(nz) + 0.5) * h
    z1, w1, V1 = zl.copy(), np.zeros(nz), 1.0 / _phi0(zl)
    V0 = V1.copy()
    lev = np.rint(z / h - 0.5).astype(int)
    done = 0
    for steps, tol_c, tol_w in ((200, 2e-3, 1e-4), (600, 5e-2, 1e-2)):
        st, _ = orc.step(st, p, steps - done, brute=False)
        for _ in range(steps - done):
            z1, w1, V1, _ = L1.step(z1, w1, V1, mui, eos, h, r, dt)
        done = steps
        # every level of the 3D layer moves as one (unjittered periodic lattice)
        for f in ("z", "w", "V"):
            spread = max(np.ptp(st[f][lev == lv]) for lv in range(nz))
            assert spread <= 1e-12 * np.abs(st[f]).max(), (steps, f, spread)
        w3 = np.array([st["w"][lev == lv][0] for lv in range(nz)])
        V3 = np.array([st["V"][lev == lv][0] for lv in range(nz)])
        c3, c1 = (V3 - V0).sum(), (V1 - V0).sum()
        ew = np.abs(w3[2:] - w1[2:]).max() / np.abs(w1).max()
        print(f"{steps} steps: compaction 3D {c3:.6e}, 1D {c1:.6e}; "
              f"velocity above the floor levels {ew:.2e}")
        assert abs(c3 - c1) <= tol_c * abs(c1), (steps, c3, c1)
        assert ew <= tol_w, (steps, ew)
