"""Pins of the oracle's time integration (Sec. 3.1 items 8 and 10).

The paper's step is first order in time (it says so and plans a second-order
scheme); time_scheme = 1 is Heun's method. Both are checked against what the
mathematics fixes: the observed order under step halving on a smooth problem
(a sheared inertial block over a short horizon, stencils frozen), and rest and
exact rigid translation.
"""
import numpy as np

from paper_2206_14061_gb300 import workloads as W


def _p(orc, **kw):
    d = dict(W.MUI)
    d.update(W.EOS)
    d.update(h=1e-3, radius=2.2e-3, gx=0.0, gy=0.0, gz=0.0, floor_z=0.0, dt=1e-5,
             mirror_mode=0)
    d.update(kw)
    return orc.params(**d)


def _block(n=7, h=1e-3):
    """Sheared block in the inertial regime (solid fraction 0.585 +- 0.002) with
    smooth velocity perturbations: smooth in time over the short horizon used
    here."""
    x, y, z = W.lattice_box(n, n, n, h, 0.05, np.random.default_rng(9))
    L = n * h
    phi = 0.585 + 0.002 * np.sin(2 * np.pi * x / L) * np.cos(2 * np.pi * z / L)
    return dict(x=x, y=y, z=z, u=20.0 * z + 0.01 * np.sin(2 * np.pi * y / L),
                v=0.01 * np.cos(2 * np.pi * x / L), w=np.zeros(x.size), V=1.0 / phi)


def _orders(orc, scheme):
    """Observed order per field from the last two step-halvings (8, 16, 32 and
    64 steps over 8e-5 s, stencils frozen over the run)."""
    s0 = _block()
    T = 8e-5
    out = []
    for steps in (8, 16, 32, 64):
        s, d = orc.step(s0, _p(orc, dt=T / steps, time_scheme=scheme, gz=-9.81), steps,
                        rebuild_every=steps, brute=True)
        assert d["n_gas"] == 0 and d["n_quasistatic"] == 0
        out.append(s)
    res = {}
    for f in ("x", "u", "v", "w", "V"):
        e = [np.abs(out[a][f] - out[a + 1][f]).max() for a in range(3)]
        res[f] = np.log2(e[1] / e[2])
    return res


def test_paper_step_is_first_order_in_time(orc):
    p = _orders(orc, 0)
    print("paper step observed orders", p)
    assert all(0.8 < v < 1.2 for v in p.values()), p


def test_heun_is_second_order_in_time(orc):
    p = _orders(orc, 1)
    print("Heun observed orders", p)
    assert all(1.8 < v < 2.2 for v in p.values()), p


def test_heun_rest_and_rigid_translation(orc):
    s0 = _block()
    zero = np.zeros(s0["x"].size)
    s0.update(u=zero.copy(), v=zero.copy(), w=zero.copy(), V=np.full(zero.size, 1 / 0.585))
    s1, _ = orc.step(s0, _p(orc, time_scheme=1), 5)
    for k in s0:
        assert np.array_equal(s0[k], s1[k]), k
    U = np.array([0.3, -0.2, 0.1])
    n, nst = s0["x"].size, 7
    st = dict(s0, u=np.full(n, U[0]), v=np.full(n, U[1]), w=np.full(n, U[2]))
    s2, _ = orc.step(st, _p(orc, time_scheme=1), nst)
    t = nst * 1e-5
    for c, k in enumerate("xyz"):
        assert np.allclose(s2[k] - st[k], U[c] * t, rtol=1e-9, atol=1e-17)
    assert np.allclose(s2["u"], U[0], rtol=1e-13)


def test_heun_tangent_linear_matches_central_differences(orc):
    """The dual-number tangent run with Heun's method (the reference of the
    GPU adjoint for that scheme) on a sheared 8^3 cube."""
    wl = W.cube(8)
    st = dict(wl.state)
    st["u"] = 20.0 * st["z"]
    pd = W.param_dict(wl)
    nst = reb = 8
    p = orc.params(**dict(pd, time_scheme=1))
    _, tan = orc.step_tangent(st, p, nst, rebuild_every=reb)
    for kix, name in enumerate(("mu_s", "mu_2", "I0")):
        eps = 1e-5
        sp_, _ = orc.step(st, orc.params(**dict(pd, time_scheme=1, **{name: pd[name] + eps})),
                          nst, rebuild_every=reb)
        sm_, _ = orc.step(st, orc.params(**dict(pd, time_scheme=1, **{name: pd[name] - eps})),
                          nst, rebuild_every=reb)
        for f, key in enumerate(("u", "v", "w", "V")):
            fd = (sp_[key] - sm_[key]) / (2 * eps)
            t = tan[kix, 3 + f]
            assert np.abs(t).max() > 0
            assert np.abs(fd - t).max() <= 1e-5 * np.abs(t).max(), (name, key)
