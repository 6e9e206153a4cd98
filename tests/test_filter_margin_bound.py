"""The rounding bound behind filter skipping between Verlet searches
(paper_2206_14061_gb300/csrc/nbr_bodies.cuh, filter_body). The filter forms
a pair's squared distance in FP32 from FP32 positions relative to the column
grid's origin (with the floor-mirror height and the nearest image along a
periodic axis), and takes |d^2 - r^2| minus the bound e2f as a lower bound of
the exact |d^2 - r^2|; the margin m r / (2 r^2 + m) then bounds |d - r| from
below. Here the same FP32 operations run in numpy float32 (IEEE single, round
to nearest) on random pairs within 2r, far from the origin as well as near
it, and the bound must hold for every pair."""
import numpy as np

F = np.float32


def _bound(cmax, rf, r2f):
    ec = F(2.0 ** -24) * (F(6.0) * cmax + F(6.0) * rf)
    return (ec * (F(7.0) * rf + F(3.0) * ec) + F(16.0) * F(2.0 ** -24) * r2f) * F(1.0 + 2.0 ** -10)


def _min_image_f(d, L):
    return np.where(np.abs(d) > F(0.5) * L, d - np.copysign(L, d), d).astype(F)


def _pairs(rng, n, r, span, mirror, period):
    """Particle i anywhere in [0, span)^3 (grid frame), j within 2r of i (or
    of i's mirror image through the floor, or across the periodic edge)."""
    xi = rng.uniform(0.0, span, (n, 3))
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    d = u * rng.uniform(0.0, 2.0 * r, n)[:, None]
    xj = xi + d
    if mirror:  # j is the mirror of a particle at (x, y, f2 - z)
        xj[:, 2] = 2.0 * mirror - xj[:, 2]
    if period:
        xj[:, 0] = np.mod(xj[:, 0], period)
        xi[:, 0] = np.mod(xi[:, 0], period)
    return xi, xj


def _check(rng, span, r, mirror=0.0, period=0.0, n=200000):
    xi, xj = _pairs(rng, n, r, span, mirror, period)
    ox = -rng.uniform(0.0, 4.0 * r)  # the grid origin sits below the particles
    pi = (xi - ox).astype(F)
    pj = (xj - ox).astype(F)
    rf, r2f = F(r), F(r * r)
    fz2 = F(2.0 * (mirror - ox)) if mirror else F(0.0)
    Lf = F(period)
    cmax = np.maximum(np.abs(pi).max(axis=1), abs(fz2))
    if period:
        cmax = np.maximum(cmax, Lf)
    cmax = cmax.astype(F)
    dxf = (pj[:, 0] - pi[:, 0]).astype(F)
    dyf = (pj[:, 1] - pi[:, 1]).astype(F)
    if period:
        dxf = _min_image_f(dxf, Lf)
    dzf = (((fz2 - pj[:, 2]).astype(F) - pi[:, 2]).astype(F) if mirror
           else (pj[:, 2] - pi[:, 2]).astype(F))
    d2f = ((dxf * dxf).astype(F) + (dyf * dyf).astype(F)).astype(F)
    d2f = (d2f + (dzf * dzf).astype(F)).astype(F)
    # the exact squared distance of the FP64 positions (nearest image, mirror)
    dx = xj[:, 0] - xi[:, 0]
    if period:
        dx = np.where(np.abs(dx) > 0.5 * period, dx - np.copysign(period, dx), dx)
    dz = (2.0 * mirror - xj[:, 2] - xi[:, 2]) if mirror else (xj[:, 2] - xi[:, 2])
    d2 = dx * dx + (xj[:, 1] - xi[:, 1]) ** 2 + dz * dz
    near = d2 <= 4.0 * r * r
    e2f = _bound(cmax, rf, r2f)
    # the lower bound of |d^2 - r^2| the filter takes, formed as in FP32
    m = np.abs((d2f - r2f).astype(F)) - e2f
    exact = np.abs(d2 - r * r)
    assert np.all(m[near] <= exact[near]), (span, mirror, period)
    # and the margin bounds |d - r| from below
    mm = np.maximum(m, F(0.0)).astype(F)
    marg = (mm * rf / (F(2.0) * r2f + mm) * F(1.0 - 2.0 ** -20)).astype(np.float64)
    assert np.all(marg[near] <= np.abs(np.sqrt(d2[near]) - r)), (span, mirror, period)
    return float(np.median(e2f / r2f))


def test_margin_bound_near_and_far_from_the_origin():
    rng = np.random.default_rng(20220628)
    h = 1e-3
    r = 2.2 * h
    for span in (10 * h, 110 * h, 1000 * h, 4000 * h):
        rel = _check(rng, span, r)
        assert rel < 1e-2  # a small fraction of r^2 (0.4 % at 4000h from the origin)


def test_margin_bound_with_floor_mirrors_and_periods():
    rng = np.random.default_rng(7)
    h = 4e-4
    r = 2.2 * h
    _check(rng, 100 * h, r, mirror=0.0)
    _check(rng, 100 * h, r, mirror=2.0 * h)
    _check(rng, 162 * h, r, period=162 * h)
    _check(rng, 30 * h, r, mirror=0.0, period=30 * h)
