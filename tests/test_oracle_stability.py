"""Short-wave growth of the inertial-regime equations (Sec. 2.3), on the oracle.

The explicit step blows up on every long run (column, cube, periodic layer),
at a rate that grows as the lattice is refined and does not depend on dt. This
file pins the cause to the continuum equations themselves, not to the
discretisation, by comparing the oracle with a linearisation written out by
hand from the paper's constitutive relations.

Linearise Sec. 2.3's system about a uniform simple shear u0 = (G y, 0, 0) at
uniform solid fraction phi (inertial regime, no gravity, gdot0 = G/2 (e_x e_y +
e_y e_x), |gdot0| = G/2). A plane wave (du, dV) exp(i k.x) obeys

    du_t = -V k^2 B du - (|gdot0|/V)(S |gdot0| I + R gdot0) (i k) dV,
    dV_t = V (i k) . du,

with k = |k| k^ and the principal symbol (the stress perturbation
2 M |gdot0| d|gdot| I + N d|gdot| gdot0 + N |gdot0| dgdot, with
d|gdot| = gdot0 : dgdot / (2 |gdot0|))

    B = M k^ (k^ . gdot0) + N/(2|gdot0|) (gdot0 k^)(k^ . gdot0)
        + N |gdot0| (I/2 + k^ k^/6).

Along the extension axis k^ = (1, 1, 0)/sqrt 2 of this shear,
k^ . B k^ = |gdot0| (M + 7 N / 6) = |M| |gdot0| (7 mu / 6 - 1): since M < 0
(the inertial pressure grows with |gdot|), the pressure term is
anti-diffusive and wins whenever mu(I) < 6/7. The growth rate then scales as
k^2: the problem is ill-posed in Hadamard's sense, and no time step cures it.
Both parameter sets in use have mu(I) < 0.75 for every phi in the inertial
range (mu_2 = 0.64 in the benchmark set; mu(I = 1) = 0.745 with the paper's
tan 30, tan 50, I0 = 2.65), so both are ill-posed there.

The tests seed the fastest eigenmode of this 4 x 4 system on a jittered
lattice, run the oracle, and project the interior state on the left
eigenvector: the measured rate must match the analytic one (the GFD operators
of Sec. 3.1 item 7 converge to the continuum symbol as k h -> 0), scale as
k^2, and vanish once mu is raised above 6/7.
"""
import math

import numpy as np
import pytest

from paper_2206_14061_gb300 import workloads as W

H = 1e-3
PHI = 0.585


def _closure(mui, phi):
    """M, N, S, R of Sec. 2.3 (R = dN/dphi) at solid fraction phi."""
    a = W.EOS["phi_c"] - W.EOS["phi_min"]
    c = W.EOS["phi_c"] - phi
    M = -4 * a * a * mui["d"] ** 2 / c ** 2
    S = -8 * a * a * mui["d"] ** 2 / c ** 3
    mu = (a * mui["mu_s"] * mui["I0"] + mui["mu_2"] * c) / (a * mui["I0"] + c)
    dmu = -a * mui["I0"] * (mui["mu_2"] - mui["mu_s"]) / (a * mui["I0"] + c) ** 2
    return M, -M * mu, S, -S * mu - M * dmu, mu


def _system(mui, G, kvec):
    """The 4 x 4 matrix of the linearised system above (du, dV)."""
    M, N, S, R, _ = _closure(mui, PHI)
    V = 1.0 / PHI
    g0 = np.array([[0.0, G / 2, 0.0], [G / 2, 0.0, 0.0], [0.0, 0.0, 0.0]])
    gn = G / 2
    k = np.linalg.norm(kvec)
    kh = kvec / k
    B = (M * np.outer(kh, kh @ g0) + N / (2 * gn) * np.outer(g0 @ kh, kh @ g0)
         + N * gn * (0.5 * np.eye(3) + np.outer(kh, kh) / 6.0))
    A = np.zeros((4, 4), complex)
    A[:3, :3] = -V * k * k * B
    A[:3, 3] = -(gn / V) * (S * gn * np.eye(3) + R * g0) @ (1j * kvec)
    A[3, :3] = V * 1j * kvec
    return A


def _growth(orc, mui, lam_h, G=100.0, nsteps=80, dt=1e-6, eps=1e-4):
    """Measured and analytic growth rate of the fastest mode with wavelength
    lam_h lattice spacings along (1, 1, 0)."""
    m = int(lam_h * 2 + 24)
    rng = np.random.default_rng(31)
    x, y, z = W.lattice_box(m, m, 10, H, 0.05, rng)
    z = z + 0.01
    kvec = (2 * math.pi / (lam_h * H)) * np.array([1.0, 1.0, 0.0]) / math.sqrt(2)
    A = _system(mui, G, kvec)
    ev, Rv = np.linalg.eig(A)
    # fastest mode that moves the material (a mode of dV alone is steady)
    moving = np.linalg.norm(Rv[:3], axis=0) > 1e-6 * np.linalg.norm(Rv, axis=0)
    i = int(np.argmax(np.where(moving, ev.real, -np.inf)))
    lam = ev[i]
    evl, Lv = np.linalg.eig(A.T)
    ell = Lv[:, int(np.argmin(np.abs(evl - lam)))]
    r = Rv[:, i] / np.abs(Rv[:3, i]).max()
    E = np.exp(1j * (x * kvec[0] + y * kvec[1]))
    V0 = 1.0 / PHI
    u0 = G * y
    pert = np.real(eps * np.outer(E, r))
    st = dict(x=x, y=y, z=z, u=u0 + pert[:, 0], v=pert[:, 1], w=pert[:, 2], V=V0 + pert[:, 3])
    p = orc.params(**mui, **W.EOS, h=H, radius=2.2 * H, gx=0.0, gy=0.0, gz=0.0, floor_z=0.0,
                   dt=dt, mirror_mode=0, free_surface=0)
    L = m * H
    inner = ((x > 8 * H) & (x < L - 8 * H) & (y > 8 * H) & (y < L - 8 * H)
             & (z > 0.013) & (z < 0.017))
    amp = []
    for it in range(nsteps + 1):
        f = np.stack([st["u"] - u0, st["v"], st["w"], st["V"] - V0], 1)[inner]
        amp.append(abs(ell @ (2 * (f * np.conj(E[inner])[:, None]).mean(0))))
        if it < nsteps:
            st, dg = orc.step(st, p, 1, brute=False)
            assert dg["n_inertial"] == x.size
    t = np.arange(nsteps + 1) * dt
    return np.polyfit(t, np.log(amp), 1)[0], lam.real


def test_symbol_along_the_extension_axis():
    """k^.B k^ = |M||gdot0|(7 mu/6 - 1) along (1, 1, 0) (the closed form in
    the module docstring), and the 4 x 4 system's fastest mode grows for both
    parameter sets (mu < 6/7) and not for mu = 1."""
    kvec = 628.0 * np.array([1.0, 1.0, 0.0]) / math.sqrt(2)
    for mui in (dict(W.MUI), dict(W.PAPER_MUI)):
        M, N, S, R, mu = _closure(mui, PHI)
        A = _system(mui, 100.0, kvec)
        kh = kvec / np.linalg.norm(kvec)
        Bkk = -(kh @ A[:3, :3] @ kh).real / ((1 / PHI) * 628.0 ** 2)
        assert Bkk == pytest.approx(abs(M) * 50.0 * (7 * mu / 6 - 1), rel=1e-12)
        assert mu < 6 / 7 and np.linalg.eigvals(A).real.max() > 0
    one = dict(W.MUI, mu_s=1.0, mu_2=1.0)
    assert np.linalg.eigvals(_system(one, 100.0, kvec)).real.max() <= 1e-6


def test_mu_stays_below_six_sevenths_in_the_inertial_range():
    """mu(I) for phi in (phi_min, phi_max], I = (phi_c - phi)/a <= 1, stays
    below 6/7 for both parameter sets (Sec. 2.2 rational law)."""
    for mui in (dict(W.MUI), dict(W.PAPER_MUI)):
        phi = np.linspace(W.EOS["phi_min"] + 1e-9, W.EOS["phi_max"], 1001)
        mu = np.array([_closure(mui, f)[4] for f in phi])
        assert mu.max() < 0.75 < 6 / 7


def test_oracle_growth_matches_linearisation(orc):
    """The oracle's growth rate of the seeded mode at wavelength 16 h matches
    the analytic rate within the GFD discretisation error (k h = 0.39)."""
    rate, ref = _growth(orc, dict(W.MUI), 16)
    assert ref > 0
    assert 0.75 * ref <= rate <= 1.05 * ref, (rate, ref)


def test_oracle_growth_scales_with_k_squared(orc):
    """Halving the wavelength multiplies the growth rate by about four (the
    analytic ratio is 4.0; the discrete operators lose some of it at the
    shorter wave): a short-wave instability, which no time step removes."""
    r12, a12 = _growth(orc, dict(W.MUI), 12)
    r24, a24 = _growth(orc, dict(W.MUI), 24)
    assert a12 / a24 == pytest.approx(4.0, rel=0.02)
    assert 3.0 <= r12 / r24 <= 4.5, (r12, r24)


def test_oracle_paper_parameters_grow_and_mu_above_six_sevenths_does_not(orc):
    """The paper's own parameters (Sec. 4) give the same growth; with a
    constant mu = 1 > 6/7 the oracle's mode no longer grows (its moving modes decay)."""
    rate, ref = _growth(orc, dict(W.PAPER_MUI), 16)
    assert ref > 0 and 0.75 * ref <= rate <= 1.05 * ref, (rate, ref)
    one = dict(W.MUI, mu_s=1.0, mu_2=1.0)
    rate1, ref1 = _growth(orc, one, 16)
    assert ref1 < 0
    assert rate1 <= 0.02 * ref, (rate1, ref1, ref)
