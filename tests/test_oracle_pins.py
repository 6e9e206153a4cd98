"""Pins of the CPU oracle against what the paper and mathematics fix.

Nothing here compares the oracle with itself: neighbour sets are checked
against scipy's KD-tree and a numpy selection, the least-squares solver against
numpy's lstsq, the Taylor fit against exactness on quadratics and its
convergence order, the closure against finite differences and the paper's
primitive relations, and the combined momentum equation against the divergence
of the stress built from the primitive relations (Sec. 2.1-2.2).
"""
import math

import numpy as np
import pytest

from paper_2206_14061_gb300 import workloads as W

MB = 0x80000000


def _sets(nbr, cnt):
    out = []
    for i in range(cnt.size):
        row = nbr[i, :cnt[i]].astype(np.int64) & 0xFFFFFFFF
        out.append(set(int(v) for v in row))
    return out


# ----------------------------------------------------------- neighbours ---

def test_neighbors_match_kdtree_with_mirrors(orc):
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(7)
    h = 1e-3
    x, y, z = W.lattice_box(11, 11, 11, h, 0.2, rng)
    r = 2.2 * h
    nbr, cnt, over = orc.neighbors(x, y, z, r_const=r, mirror_mode=1, brute=True)
    assert over == 0
    n = x.size
    pts = np.stack([x, y, z], 1)
    mir = np.stack([x, y, -z], 1)
    # keep clear of rounding ties at the sphere boundary
    d2 = ((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1)
    d2m = ((pts[:, None, :] - mir[None, :, :]) ** 2).sum(-1)
    assert np.abs(d2 - r * r).min() > 1e-12 * r * r
    assert np.abs(d2m - r * r).min() > 1e-12 * r * r
    tree = spatial.cKDTree(np.concatenate([pts, mir]))
    got = _sets(nbr, cnt)
    for i in range(n):
        ref = set()
        for j in tree.query_ball_point(pts[i], r):
            if j == i:
                continue
            ref.add(j if j < n else (j - n) | MB)
        assert got[i] == ref, i


def test_neighbors_keep_nearest_matches_sorting(orc):
    rng = np.random.default_rng(11)
    h = 1e-3
    x, y, z = W.lattice_box(10, 10, 10, h, 0.2, rng)
    rad = rng.uniform(1.8 * h, 2.6 * h, size=x.size)
    cap = 48
    nbr, cnt, _ = orc.neighbors(x, y, z, radius=rad, mirror_mode=1, cap=cap, keep_nearest=True)
    pts = np.stack([x, y, z], 1)
    for i in range(0, x.size, 7):
        cand = []
        for j in range(x.size):
            dd = np.sum((pts[j] - pts[i]) ** 2)
            if j != i and dd <= rad[i] ** 2:
                cand.append((dd, j, 0))
            ddm = (x[j] - x[i]) ** 2 + (y[j] - y[i]) ** 2 + (-z[j] - z[i]) ** 2
            if ddm <= rad[i] ** 2:
                cand.append((ddm, j, 1))
        cand.sort()
        ref = set(j | (MB if m else 0) for _, j, m in cand[:cap])
        got = set(int(v) & 0xFFFFFFFF for v in nbr[i, :cnt[i]])
        assert cnt[i] == min(cap, len(cand))
        assert got == ref


def _octant_reference(x, y, z, rad, i, cap):
    """Octant-balanced selection for particle i written with numpy: all
    candidates (real and floor mirrors) within rad[i]; each one's round is its
    rank, nearest first (ties by index, real before mirror), among the
    candidates in its own octant (bit 0: dx >= 0, bit 1: dy >= 0, bit 2:
    dz >= 0); the first cap by (round, distance, index, mirror) are kept."""
    j = np.arange(x.size)
    rows = []
    for mir, zz in ((0, z), (1, -z)):
        dx, dy, dz = x - x[i], y - y[i], zz - z[i]
        d2 = (dx * dx + dy * dy) + dz * dz
        ok = d2 <= rad[i] ** 2
        if mir == 0:
            ok &= j != i
        oc = (dx >= 0).astype(int) + 2 * (dy >= 0) + 4 * (dz >= 0)
        rows += [(d2[k], k, mir, oc[k]) for k in np.flatnonzero(ok)]
    rows.sort()
    seen = [0] * 8
    keyed = []
    for d2, k, mir, oc in rows:
        keyed.append((seen[oc], d2, k, mir, oc))
        seen[oc] += 1
    keyed.sort()
    return keyed[:cap], rows


def test_neighbors_octant_balanced_matches_numpy(orc):
    """Sec. 3.1 item 6: the kept entries of a truncated stencil should lie in
    all directions. Against a numpy restatement of the selection; every
    octant that has candidates keeps at least min(its candidates,
    floor(cap / 8)) of them, so a one-sided cut never starves a direction the
    way a nearest-only cut does near a face."""
    rng = np.random.default_rng(12)
    h = 1e-3
    x, y, z = W.lattice_box(10, 10, 10, h, 0.2, rng)
    rad = rng.uniform(1.8 * h, 2.6 * h, size=x.size)
    cap = 48
    nbr, cnt, _ = orc.neighbors(x, y, z, radius=rad, mirror_mode=1, cap=cap, keep_nearest=2)
    near, _, _ = orc.neighbors(x, y, z, radius=rad, mirror_mode=1, cap=cap, keep_nearest=True)
    differs = 0
    for i in range(0, x.size, 5):
        kept, allc = _octant_reference(x, y, z, rad, i, cap)
        ref = set(k | (MB if m else 0) for _, _, k, m, _ in kept)
        got = set(int(v) & 0xFFFFFFFF for v in nbr[i, :cnt[i]])
        assert cnt[i] == min(cap, len(allc))
        assert got == ref, i
        n_oct = np.bincount([r[3] for r in allc], minlength=8)
        k_oct = np.bincount([r[4] for r in kept], minlength=8)
        assert (k_oct >= np.minimum(n_oct, cap // 8)).all(), (i, n_oct, k_oct)
        differs += got != set(int(v) & 0xFFFFFFFF for v in near[i, :cnt[i]])
    assert differs > 0  # truncation happens and the two rules differ


def test_grid_search_equals_brute_force(orc):
    rng = np.random.default_rng(3)
    n = 3000
    x, y = rng.uniform(0, 0.02, n), rng.uniform(0, 0.02, n)
    z = rng.uniform(0, 0.01, n)
    rad = rng.uniform(1.0e-3, 1.6e-3, n)
    a = orc.neighbors(x, y, z, radius=rad, mirror_mode=1, brute=True)
    b = orc.neighbors(x, y, z, radius=rad, mirror_mode=1, brute=False)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[0], b[0])
    for keep in (1, 2):
        a = orc.neighbors(x, y, z, radius=rad, mirror_mode=1, cap=16, keep_nearest=keep)
        b = orc.neighbors(x, y, z, radius=rad, mirror_mode=1, cap=16, keep_nearest=keep,
                          brute=False)
        assert np.array_equal(a[1], b[1]) and np.array_equal(a[0], b[0])


# ------------------------------------------------------------- GFD fits ---

def _ball_stencil(rng, m, h, r=2.2):
    pts = []
    while len(pts) < m:
        p = rng.uniform(-r, r, 3)
        if 0.3 < np.linalg.norm(p) <= r:
            pts.append(p)
    return np.array(pts) * h


def _quad(rng):
    c = rng.standard_normal(10)

    def f(x, y, z):
        return (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * x + c[5] * y * y + c[6] * z * z
                + c[7] * x * y + c[8] * x * z + c[9] * y * z)

    def d(x, y, z):  # exact derivatives at (x, y, z)
        one = np.ones_like(x)
        return np.stack([c[1] + 2 * c[4] * x + c[7] * y + c[8] * z,
                         c[2] + 2 * c[5] * y + c[7] * x + c[9] * z,
                         c[3] + 2 * c[6] * z + c[8] * x + c[9] * y,
                         2 * c[4] * one, 2 * c[5] * one, 2 * c[6] * one,
                         c[7] * one, c[8] * one, c[9] * one], 1)
    return f, d


def test_fit_reproduces_quadratics(orc):
    """A quadratic field is inside the 9-term basis: derivatives exact to rounding."""
    rng = np.random.default_rng(5)
    h = 1e-3
    x, y, z = W.lattice_box(9, 9, 9, h, 0.05, rng)
    nbr, cnt, _ = orc.neighbors(x, y, z, r_const=2.2 * h, mirror_mode=0)
    fs, ds = zip(*[_quad(rng) for _ in range(3)])
    fields = np.stack([f(x / h, y / h, z / h) for f in fs])
    coeffs, rank = orc.fit(x, y, z, nbr, cnt, fields, [1, 1, 1], h)
    assert (rank == 9).all()
    scale = np.array([1 / h] * 3 + [1 / h ** 2] * 6)
    for q in range(3):
        ref = ds[q](x / h, y / h, z / h) * scale
        err = np.abs(coeffs[:, q, :] - ref) / np.abs(ref).max()
        assert err.max() < 1e-12, err.max()


def test_fit_mirror_parity_quadratics(orc):
    """Floor mirrors carry s(x, y, -z) = +s for even fields and -s for odd ones."""
    rng = np.random.default_rng(6)
    h = 1e-3
    x, y, z = W.lattice_box(8, 8, 5, h, 0.05, rng)
    nbr, cnt, _ = orc.neighbors(x, y, z, r_const=2.2 * h, mirror_mode=1)
    assert (nbr[:, :] < 0).any()
    c = rng.standard_normal(6)
    even = c[0] * x / h + c[1] * (y / h) ** 2 + c[2] * (z / h) ** 2 + c[3] * x * y / h ** 2
    odd = (z / h) * (c[4] + c[5] * x / h)
    coeffs, _ = orc.fit(x, y, z, nbr, cnt, np.stack([even, odd]), [1.0, -1.0], h)
    X, Y, Z = x / h, y / h, z / h
    zero, one = np.zeros_like(X), np.ones_like(X)
    ref_e = np.stack([c[0] + c[3] * Y, 2 * c[1] * Y + c[3] * X, 2 * c[2] * Z, zero,
                      2 * c[1] * one, 2 * c[2] * one, c[3] * one, zero, zero], 1)
    ref_o = np.stack([c[5] * Z, zero, c[4] + c[5] * X, zero, zero, zero, zero, c[5] * one,
                      zero], 1)
    sc = np.array([1 / h] * 3 + [1 / h ** 2] * 6)
    for q, ref in ((0, ref_e), (1, ref_o)):
        err = np.abs(coeffs[:, q, :] - ref * sc).max() / np.abs(ref * sc).max()
        assert err < 1e-12, (q, err)


def test_fit_matches_numpy_lstsq(orc):
    """Householder QR gives the textbook least-squares solution (numpy lstsq)."""
    rng = np.random.default_rng(8)
    h = 1.0
    for m in (9, 12, 30, 48):
        off = _ball_stencil(rng, m, h)
        x = np.concatenate([[0.0], off[:, 0]])
        y = np.concatenate([[0.0], off[:, 1]])
        z = np.concatenate([[0.0], off[:, 2]]) + 10.0
        nbr = np.zeros((m + 1, 64), np.int32)
        nbr[0, :m] = np.arange(1, m + 1)
        cnt = np.zeros(m + 1, np.int32)
        cnt[0] = m
        b = rng.standard_normal((2, m + 1))
        coeffs, rank = orc.fit(x, y, z, nbr, cnt, b, [1, 1], h)
        dx, dy, dz = off[:, 0], off[:, 1], off[:, 2]
        A = np.stack([dx, dy, dz, dx * dx / 2, dy * dy / 2, dz * dz / 2, dx * dy, dx * dz,
                      dy * dz], 1)
        for q in range(2):
            ref = np.linalg.lstsq(A, b[q, 1:] - b[q, 0], rcond=None)[0]
            assert np.abs(coeffs[0, q] - ref).max() <= 1e-11 * np.abs(ref).max()


def test_fit_rank_deficient_gives_projection(orc):
    """Planar and tiny stencils: the basic solution still gives the LS projection."""
    rng = np.random.default_rng(9)
    for m, planar in ((20, True), (6, False)):
        off = _ball_stencil(rng, m, 1.0)
        if planar:
            off[:, 2] = 0.0
        x = np.concatenate([[0.0], off[:, 0]])
        y = np.concatenate([[0.0], off[:, 1]])
        z = np.concatenate([[0.0], off[:, 2]]) + 5.0
        nbr = np.zeros((m + 1, 32), np.int32)
        nbr[0, :m] = np.arange(1, m + 1)
        cnt = np.zeros(m + 1, np.int32)
        cnt[0] = m
        b = rng.standard_normal(m + 1)
        coeffs, rank = orc.fit(x, y, z, nbr, cnt, b[None], [1], 1.0)
        dx, dy, dz = off[:, 0], off[:, 1], off[:, 2]
        A = np.stack([dx, dy, dz, dx * dx / 2, dy * dy / 2, dz * dz / 2, dx * dy, dx * dz,
                      dy * dz], 1)
        assert rank[0] == np.linalg.matrix_rank(A)
        ref = np.linalg.lstsq(A, b[1:] - b[0], rcond=None)[0]
        assert np.allclose(A @ coeffs[0, 0], A @ ref, atol=1e-12)
        assert np.count_nonzero(coeffs[0, 0]) <= rank[0]


def test_fit_second_order_convergence(orc):
    """First derivatives converge at O(h^2) on jittered lattices; second at O(h^2)
    on an exact lattice (Sec. 3.1: second-order accurate in space)."""
    k = np.array([0.9, -0.6, 0.7]) * 20.0

    def run(n, jitter):
        h = 0.1 / n
        rng = np.random.default_rng(n)
        x, y, z = W.lattice_box(n, n, n, h, jitter, rng)
        nbr, cnt, _ = orc.neighbors(x, y, z, r_const=2.2 * h, brute=False)
        ph = k[0] * x + k[1] * y + k[2] * z
        coeffs, _ = orc.fit(x, y, z, nbr, cnt, np.sin(ph)[None], [1], h)
        c = np.cos(ph)
        s = np.sin(ph)
        ref = np.stack([k[0] * c, k[1] * c, k[2] * c, -k[0] ** 2 * s, -k[1] ** 2 * s,
                        -k[2] ** 2 * s, -k[0] * k[1] * s, -k[0] * k[2] * s, -k[1] * k[2] * s], 1)
        inner = ((np.abs(x - 0.05) < 0.02) & (np.abs(y - 0.05) < 0.02)
                 & (np.abs(z - 0.05) < 0.02))
        e = np.abs(coeffs[inner, 0, :] - ref[inner])
        return e[:, :3].max() / np.abs(k).max(), e[:, 3:].max() / (np.abs(k).max() ** 2)

    g1, _ = run(10, 0.1)
    g2, _ = run(20, 0.1)
    g3, _ = run(40, 0.1)
    assert math.log2(g1 / g2) > 1.8 and math.log2(g2 / g3) > 1.8, (g1, g2, g3)
    _, h1 = run(10, 0.0)
    _, h2 = run(20, 0.0)
    _, h3 = run(40, 0.0)
    assert math.log2(h1 / h2) > 1.8 and math.log2(h2 / h3) > 1.8, (h1, h2, h3)


# -------------------------------------------------------------- closure ---

def _p(orc, **kw):
    d = dict(W.MUI)
    d.update(W.EOS)
    d.update(h=1e-3, radius=2.2e-3, gx=0.0, gy=0.0, gz=-9.81, floor_z=0.0, dt=1e-5,
             mirror_mode=1)
    d.update(kw)
    return orc.params(**d)


def test_closure_matches_mu_of_I_and_derivatives(orc):
    p = _p(orc)
    a = p.phi_c - p.phi_min
    phi = np.linspace(0.36, 0.59, 41)
    out = orc.closure(phi, p)
    M, N, S, R, mu = out.T
    # mu(I) of Sec. 2.2 with I = (phi_c - phi)/a (Eq. for phi(I))
    I = (p.phi_c - phi) / a
    mu_I = p.mu_s + (p.mu_2 - p.mu_s) / (p.I0 / I + 1.0)
    assert np.allclose(mu, mu_I, rtol=1e-14)
    assert np.allclose(-N / M, mu_I, rtol=1e-14)
    # S = dM/dphi and R = dN/dphi (central differences)
    eps = 1e-6
    up = orc.closure(phi + eps, p)
    dn = orc.closure(phi - eps, p)
    assert np.allclose(S, (up[:, 0] - dn[:, 0]) / (2 * eps), rtol=1e-7)
    assert np.allclose(R, (up[:, 1] - dn[:, 1]) / (2 * eps), rtol=1e-7)


def test_mu_limits_with_paper_parameters(orc):
    golden = {}
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.txt")
    for line in open(path):
        line = line.split("#")[0].split()
        if line:
            golden[line[0]] = float(line[1])
    mu_s = math.tan(math.radians(golden["mu_s_deg"]))
    mu_2 = math.tan(math.radians(golden["mu_2_deg"]))
    p = _p(orc, mu_s=mu_s, mu_2=mu_2, I0=golden["I0"], d=golden["d"], rho_s=golden["phi_s"],
           phi_c=golden["phi_c"], phi_min=golden["phi_min"], phi_max=0.599)
    a = p.phi_c - p.phi_min
    # I -> 0 at phi_c: mu_s ; I = I0 : (mu_s + mu_2)/2 ; I -> infinity : mu_2
    mu = orc.closure([p.phi_c - 1e-12, p.phi_c - a * p.I0, p.phi_c - 1e9], p)[:, 4]
    assert abs(mu[0] - mu_s) < 1e-10
    assert abs(mu[1] - 0.5 * (mu_s + mu_2)) < 1e-14
    assert abs(mu[2] - mu_2) < 1e-8


def test_mui_stress_primitive_relations(orc):
    """P, I and tau from the pointwise closure satisfy the paper's defining
    relations: I = 2|gdot| d / sqrt(P/phi_s) equals (phi_c - phi)/a, and
    |tau| = eta |gdot| = mu(I) P (friction law); simple shear u = (G y, 0, 0)
    has |gdot| = G/2."""
    p = _p(orc)
    rng = np.random.default_rng(1)
    n = 200
    phi = rng.uniform(0.36, 0.589, n)
    G = rng.standard_normal((n, 9)) * 30.0
    gd, gn, P, eta, reg = orc.mui_stress(1.0 / phi, G, p)
    assert (reg == 1).all()
    a = p.phi_c - p.phi_min
    I = 2 * gn * p.d / np.sqrt(P / p.rho_s)
    assert np.allclose(I, (p.phi_c - phi) / a, rtol=1e-12)
    mu_I = p.mu_s + (p.mu_2 - p.mu_s) / (p.I0 / I + 1.0)
    assert np.allclose(eta * gn, mu_I * P, rtol=1e-12)
    # gdot is trace-free and symmetric part of grad u minus div/3
    assert np.allclose(gd[:, 0] + gd[:, 1] + gd[:, 2], 0, atol=1e-12)
    Gm = G.reshape(n, 3, 3)
    assert np.allclose(gd[:, 3], 0.5 * (Gm[:, 0, 1] + Gm[:, 1, 0]))
    shear = np.zeros((1, 9))
    shear[0, 1] = 40.0
    _, gn1, _, _, _ = orc.mui_stress(np.array([1 / 0.5]), shear, p)
    assert abs(gn1[0] - 20.0) < 1e-12
    # regimes of the pressure law (Sec. 2.2.1)
    phis = np.array([0.30, 0.35, 0.5, 0.59, 0.595, 0.61])
    _, _, P2, eta2, reg2 = orc.mui_stress(1 / phis, np.tile(G[:1], (6, 1)), p)
    assert list(reg2) == [0, 0, 1, 1, 2, 2]
    assert P2[0] == 0 and P2[1] == 0
    assert np.allclose(P2[4:], p.rho_s * (p.alpha + p.beta * phis[4:]))
    assert (eta2[[0, 1, 4, 5]] == 0).all()


# ----------------------------------------------------------------- step ---

def _state(x, y, z, u=None, v=None, w=None, V=None):
    n = x.size
    z0 = np.zeros(n)
    return dict(x=x, y=y, z=z, u=z0.copy() if u is None else u, v=z0.copy() if v is None else v,
                w=z0.copy() if w is None else w, V=np.full(n, 1 / 0.585) if V is None else V)


def test_rest_state_without_gravity_is_unchanged(orc):
    rng = np.random.default_rng(2)
    x, y, z = W.lattice_box(6, 6, 6, 1e-3, 0.05, rng)
    s0 = _state(x, y, z)
    s1, _ = orc.step(s0, _p(orc, gz=0.0), 5)
    for k in s0:
        assert np.array_equal(s0[k], s1[k]), k


def test_free_fall_and_rigid_translation(orc):
    rng = np.random.default_rng(4)
    h = 1e-3
    x, y, z = W.lattice_box(6, 6, 6, h, 0.05, rng)
    x, y, z = x, y, z + 0.01
    n = x.size
    p = _p(orc, mirror_mode=0)
    nst = 7
    s1, _ = orc.step(_state(x, y, z), p, nst)
    t = nst * p.dt
    assert np.allclose(s1["w"], p.gz * t, rtol=1e-13, atol=0)
    assert np.allclose(s1["z"] - z, 0.5 * p.gz * t * t, rtol=1e-9, atol=1e-18)
    assert np.array_equal(s1["V"], np.full(n, 1 / 0.585))
    # uniform velocity, no gravity: gdot = 0, x advances by u t
    U = np.array([0.3, -0.2, 0.1])
    st = _state(x, y, z, np.full(n, U[0]), np.full(n, U[1]), np.full(n, U[2]))
    s2, _ = orc.step(st, _p(orc, mirror_mode=0, gz=0.0), nst)
    for c, k in enumerate("xyz"):
        assert np.allclose(s2[k] - st[k], U[c] * t, rtol=1e-9, atol=1e-17)
    assert np.allclose(s2["u"], U[0], rtol=1e-13)


def test_mass_equation_under_uniform_dilation(orc):
    """Sec. 2.1 Eq. 1 in V = 1/phi, discretised by the first difference
    equation of Sec. 3.1 item 8: V^{n+1} = V^n + dt V^n DIV(u^n). Under the
    uniform dilation u = c (x - x0) the fit of a linear field is exact, so
    DIV u = 3c and one step gives V^n (1 + 3 c dt). The dilation has no
    deviatoric part (gdot = 0), so no stress acts: u keeps its values and x
    moves to x0 + (1 + c dt)(x - x0), where the same field is
    u = c/(1 + c dt) (x - x0): the second step gives V^1 (1 + 3 c dt/(1 + c dt))."""
    rng = np.random.default_rng(21)
    h = 1e-3
    x, y, z = W.lattice_box(7, 7, 7, h, 0.05, rng)
    z = z + 0.01
    c = 150.0
    x0 = np.array([3.1e-3, 3.7e-3, 1.35e-2])
    V0 = 1.0 / 0.585
    st = _state(x, y, z, c * (x - x0[0]), c * (y - x0[1]), c * (z - x0[2]),
                np.full(x.size, V0))
    p = _p(orc, mirror_mode=0, gz=0.0)
    cdt = c * p.dt
    s1, d1 = orc.step(st, p, 1)
    assert d1["n_inertial"] == x.size
    V1 = V0 * (1.0 + 3.0 * cdt)
    assert np.abs(s1["V"] / V1 - 1.0).max() <= 1e-14
    for k, o in zip("uvw", range(3)):
        assert np.abs(s1[k] - st[k]).max() <= 1e-12 * c * h
    s2, _ = orc.step(s1, p, 1)
    V2 = V1 * (1.0 + 3.0 * cdt / (1.0 + cdt))
    assert np.abs(s2["V"] / V2 - 1.0).max() <= 1e-14


@pytest.mark.parametrize("mode", [1, 2])
def test_floor_mirror_velocity_signs(orc, mode):
    """Solid boundary (Sec. 3.1 item 9) with the floor at z = 0: a mirror at
    z* = -z_j carries u* = -u_j on every component for the no-slip floor
    (mode 1) and only the normal component reversed for free slip (mode 2).
    The field u = (G1 z, G2 z, G3 z) is zero on the floor, so its odd
    extension is the same linear field and every no-slip stencil fits it
    exactly: gdot_xz = G1/2, gdot_yz = G2/2 and dw/dz = gdot_zz + div/3 = G3
    in the floor layer. Free slip reverses w alone: dw/dz stays exact, while
    the even extension of G1 z and G2 z (|z|-shaped) spoils gdot_xz and
    gdot_yz in stencils that hold mirrors."""
    rng = np.random.default_rng(22)
    h = 1e-3
    x, y, z = W.lattice_box(7, 7, 5, h, 0.05, rng)
    G = np.array([40.0, -25.0, 10.0])
    st = _state(x, y, z, G[0] * z, G[1] * z, G[2] * z)
    p = _p(orc, mirror_mode=mode, gz=0.0)
    nbr, cnt, _ = orc.step_stencils(x, y, z, p)
    has_mirror = np.array([(nbr[i, :cnt[i]].astype(np.int64) & MB).any() for i in range(x.size)])
    assert has_mirror.sum() >= 49
    det = orc.step_detail(st, p)
    gd = det["gdot"][has_mirror]
    scale = np.abs(G).max()
    err_xz = np.abs(gd[:, 4] - G[0] / 2).max() / scale
    err_yz = np.abs(gd[:, 5] - G[1] / 2).max() / scale
    dwdz = gd[:, 2] + det["div"][has_mirror] / 3
    assert np.abs(dwdz - G[2]).max() <= 1e-12 * scale
    if mode == 1:
        assert max(err_xz, err_yz) <= 1e-12
        assert np.abs(det["div"][has_mirror] - G[2]).max() <= 1e-12 * scale
    else:
        assert min(err_xz, err_yz) > 1e-3


def _analytic_accel(pts, prm, G, eps_u, kk, phi0, dphi, gvec):
    """a_i = (1/(phi_s phi)) d_j sigma_ij + g_i with sigma = -P I + tau built
    from the primitive relations of Sec. 2.2: gdot = D - div/3 I, P from the
    Bagnold form, I from its definition, mu(I), tau = mu P gdot/|gdot|."""
    sp = pytest.importorskip("sympy")
    X, Y, Z = sp.symbols("X Y Z", real=True)
    u = sp.Matrix([G * Y + eps_u * sp.sin(kk * Z) + 0.3 * eps_u * sp.sin(kk * X),
                   eps_u * sp.sin(kk * X) + 0.2 * eps_u * sp.cos(kk * Y),
                   eps_u * sp.cos(kk * Y) - 0.25 * eps_u * sp.sin(kk * Z)])
    phi = phi0 + dphi * sp.sin(kk * X) * sp.cos(kk * Y) + 0.5 * dphi * sp.sin(kk * Z)
    xs = (X, Y, Z)
    Gr = sp.Matrix(3, 3, lambda a, b: sp.diff(u[a], xs[b]))
    D = (Gr + Gr.T) / 2
    div = Gr.trace()
    gd = D - div / 3 * sp.eye(3)
    gn = sp.sqrt(sum(gd[a, b] ** 2 for a in range(3) for b in range(3)) / 2)
    aa = prm["phi_c"] - prm["phi_min"]
    P = prm["rho_s"] * (2 * aa * prm["d"] * gn / (prm["phi_c"] - phi)) ** 2
    I = 2 * gn * prm["d"] / sp.sqrt(P / prm["rho_s"])
    mu = prm["mu_s"] + (prm["mu_2"] - prm["mu_s"]) / (prm["I0"] / I + 1)
    sig = -P * sp.eye(3) + mu * P / gn * gd
    acc = [sum(sp.diff(sig[a, b], xs[b]) for b in range(3)) / (prm["rho_s"] * phi) + gvec[a]
           for a in range(3)]
    fu = sp.lambdify(xs, list(u), "numpy")
    fphi = sp.lambdify(xs, phi, "numpy")
    fa = sp.lambdify(xs, acc, "numpy")
    x, y, z = pts
    uu = [np.broadcast_to(c, x.shape).astype(float) for c in fu(x, y, z)]
    aa_ = np.stack([np.broadcast_to(c, x.shape).astype(float) for c in fa(x, y, z)], 1)
    return uu, fphi(x, y, z), aa_


@pytest.mark.slow
def test_momentum_equation_matches_divergence_of_stress(orc):
    """The combined system of Sec. 2.3 (through M, N, S, R and the GFD fits)
    reproduces (1/(phi_s phi)) div sigma + g with sigma from the primitive
    relations, converging at second order under refinement."""
    L = 0.02
    prm = dict(W.MUI, **W.EOS)
    gvec = (0.0, 0.0, -9.81)
    errs = []
    for n in (12, 24):
        h = L / n
        rng = np.random.default_rng(n)
        x, y, z = W.lattice_box(n, n, n, h, 0.0, rng)
        (u, v, w), phi, a_ref = _analytic_accel((x, y, z), prm, 60.0, 0.05, math.pi / L, 0.52,
                                                0.03, gvec)
        st = _state(x, y, z + 0.05, u, v, w, 1.0 / phi)
        p = _p(orc, h=h, radius=2.2 * h, mirror_mode=0)
        det = orc.step_detail(st, p, brute=False)
        assert (det["regime"] == 1).all()
        inner = ((np.abs(x - L / 2) < L / 4) & (np.abs(y - L / 2) < L / 4)
                 & (np.abs(z - L / 2) < L / 4))
        e = np.abs(det["acc"][inner] - a_ref[inner]).max()
        errs.append(e / np.abs(a_ref[inner] - np.array(gvec)).max())
    assert errs[1] < 0.05
    assert math.log2(errs[0] / errs[1]) > 1.7, errs


def test_quasistatic_and_gas_accelerations(orc):
    """Quasi-static: sigma = -phi_s(alpha + beta phi) I gives a = beta grad V / V + g
    (Sec. 2.2.1 with Eq. 2-4); gas: a = g."""
    h = 1e-3
    rng = np.random.default_rng(12)
    x, y, z = W.lattice_box(8, 8, 8, h, 0.05, rng)
    z = z + 0.02
    c = np.array([3.0, -2.0, 1.5])
    # V linear in x, so its quadratic fit is exact; phi = 1/V stays above phi_max
    V = 1 / 0.595 + 0.004 * (c[0] * x + c[1] * y + c[2] * z - 0.04) / 0.01
    phi = 1 / V
    st = _state(x, y, z, V=V)
    p = _p(orc, mirror_mode=0)
    det = orc.step_detail(st, p)
    assert (det["regime"] == 2).all()
    # a = (1/(phi_s phi)) d_i(-phi_s (alpha + beta phi)) + g = -(beta/phi) grad phi + g,
    # grad phi = -grad V / V^2
    gphi = -(0.004 * c / 0.01)[None, :] / V[:, None] ** 2
    a_ref = -(p.beta / phi[:, None]) * gphi + np.array([0, 0, p.gz])
    assert np.allclose(det["acc"], a_ref, rtol=1e-10, atol=1e-10)
    det2 = orc.step_detail(_state(x, y, z, V=np.full(x.size, 1 / 0.3)), p)
    assert (det2["regime"] == 0).all()
    assert np.array_equal(det2["acc"], np.tile([0.0, 0.0, p.gz], (x.size, 1)))


def test_hydrostatic_layer_is_at_rest_to_second_order(orc):
    """A quasi-static layer in hydrostatic balance (Sec. 2.2.1 with Eq. 2-4):
    with a = beta grad V / V + g, the profile V(z) = V_b exp(-g_z z / beta)
    makes a = 0 exactly. On the lattice the quadratic fit of V leaves a
    residual acceleration that falls as h^2 (order > 1.7 from h to h/2), and
    every particle stays quasi-static. beta = 1 m^2/s^2 gives the profile
    enough curvature (k h = 0.01) for the truncation error to stand above
    rounding; interior particles only (the faces have one-sided stencils)."""
    beta = 1.0
    k = 9.81 / beta
    res = []
    for nside, h in ((8, 1e-3), (16, 5e-4)):
        rng = np.random.default_rng(21)
        x, y, z = W.lattice_box(nside, nside, nside, h, 0.05, rng)
        z = z + 0.02
        V = (1 / 0.64) * np.exp(k * (z - 0.02))
        assert (1 / V).min() > 0.59  # quasi-static throughout
        p = _p(orc, h=h, radius=2.2 * h, mirror_mode=0, beta=beta, alpha=-beta * 0.59)
        det = orc.step_detail(_state(x, y, z, V=V), p)
        assert (det["regime"] == 2).all()
        L = nside * h
        inner = ((x > 2.2 * h) & (x < L - 2.2 * h) & (y > 2.2 * h) & (y < L - 2.2 * h)
                 & (z > 0.02 + 2.2 * h) & (z < 0.02 + L - 2.2 * h))
        assert inner.sum() >= 8
        res.append(np.abs(det["acc"][inner]).max())
    # the residual is 1e-4 of g at h = 1e-3 (3.9e-4 m/s^2), and it falls as h^2
    assert res[0] < 1e-3, res
    assert math.log2(res[0] / res[1]) > 1.7, res


def test_rotation_covariance(orc):
    """Rotating the column by 90 degrees about z rotates every output."""
    rng = np.random.default_rng(13)
    h = 1e-3
    x, y, z = W.lattice_box(7, 7, 7, h, 0.05, rng)
    x, y = x - 3.5 * h, y - 3.5 * h
    u = 20 * z * (1 + 0.3 * np.sin(300 * x))
    v = 5 * z * np.cos(200 * y)
    w = 3 * x * y / h
    V = 1 / (0.57 + 0.01 * np.sin(500 * (x + 2 * y)))
    a = _state(x, y, z, u, v, w, V)
    b = _state(-y, x, z, -v, u, w, V)
    p = _p(orc)
    sa, _ = orc.step(a, p, 3)
    sb, _ = orc.step(b, p, 3)
    tol = lambda r: 1e-11 * np.abs(r).max() + 1e-300
    assert np.abs(sb["x"] + sa["y"]).max() <= tol(sa["y"]) + 1e-16
    assert np.abs(sb["y"] - sa["x"]).max() <= tol(sa["x"]) + 1e-16
    assert np.abs(sb["u"] + sa["v"]).max() <= tol(sa["v"])
    assert np.abs(sb["v"] - sa["u"]).max() <= tol(sa["u"])
    assert np.abs(sb["w"] - sa["w"]).max() <= tol(sa["w"])
    assert np.abs(sb["V"] - sa["V"]).max() <= tol(sa["V"])


def test_tangent_linear_matches_central_differences(orc):
    """Forward-mode derivatives w.r.t. (mu_s, mu_2, I0) equal central finite
    differences of the same frozen-topology forward run."""
    rng = np.random.default_rng(14)
    h = 1e-3
    x, y, z = W.lattice_box(6, 6, 6, h, 0.05, rng)
    u = 20.0 * z
    st = _state(x, y, z, u=u)
    nst, reb = 8, 8
    p = _p(orc)
    _, tan = orc.step_tangent(st, p, nst, rebuild_every=reb)
    names = ("mu_s", "mu_2", "I0")
    for kix, name in enumerate(names):
        eps = 1e-5  # large enough that FD round-off (ulp(V)/eps) stays below 1e-6 relative
        pp = _p(orc, **{name: getattr(p, name) + eps})
        pm = _p(orc, **{name: getattr(p, name) - eps})
        sp_, _ = orc.step(st, pp, nst, rebuild_every=reb)
        sm_, _ = orc.step(st, pm, nst, rebuild_every=reb)
        for f, key in enumerate(("u", "v", "w", "V")):
            fd = (sp_[key] - sm_[key]) / (2 * eps)
            t = tan[kix, 3 + f]
            scale = np.abs(t).max()
            assert scale > 0
            assert np.abs(fd - t).max() <= 1e-5 * scale, (name, key, np.abs(fd - t).max(), scale)
