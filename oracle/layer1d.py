"""The LP step reduced to one space dimension: a horizontally infinite granular
layer on a no-slip floor (Sec. 4.1 compares the 3D code with periodic sides
against such a reduced 1D computation).

TEST INFRASTRUCTURE ONLY: used by tests/ to check the 3D oracle's periodic
layer against the 1D reduction. Plain FP64 numpy, written independently of the
3D oracle (lp_oracle.cpp) and of the CUDA library.

With u = (0, 0, w(z)) and V = V(z), every quantity of Sec. 2.2-2.3 reduces to
z-derivatives: div u = w', gdot = diag(-w'/3, -w'/3, 2w'/3), |gdot| =
sqrt(gdot:gdot / 2) = |w'| / sqrt 3, and (1/2) Lap u + (1/6) grad div u has the
z-component (2/3) w''. The step is the paper's explicit step (Sec. 3.1 items
8 and 10) with the time levels the 3D oracle takes: V first,
V^{n+1} = V^n + dt V^n w'^n; the momentum right-hand side with V^{n+1} and
the time-n velocity quantities; w^{n+1} = w^n + dt a; z^{n+1} = z^n + dt
(w^n + w^{n+1}) / 2. Derivatives come from 1D least-squares fits (Sec. 3.1
item 7) with rows [dz/h, (dz/h)^2 / 2] over the particles within the stencil
radius, floor mirrors (Sec. 3.1 item 9: mirror at -z with w* = -w, the same
V, |gdot| = 0) and, at the free top, ghost particles with the free-boundary
rule the 3D code uses (a stencil is one-sided when its weighted mean offset,
weights r^2 - d^2, exceeds 0.22 h; its entries at least h/2 on the inner side
are reflected through the particle unless an entry lies within h/2 of the
reflection or it falls below the floor), here on real offsets: a ghost
carries the particle's velocity, solid fraction
phi_G = phi_min (1 - 1e-3) and |gdot|_G = |gdot| (phi_c - phi_G)/(phi_c - phi)
in the inertial regime.
"""
from __future__ import annotations

import numpy as np


def closure(phi, mui, eos):
    """M, N, S, R of Sec. 2.3 (R = dN/dphi) at solid fraction phi."""
    a = eos["phi_c"] - eos["phi_min"]
    c = eos["phi_c"] - phi
    k = 4.0 * a * a * mui["d"] ** 2
    M = -k / c ** 2
    S = -2.0 * k / c ** 3
    den = a * mui["I0"] + c
    mu = (a * mui["mu_s"] * mui["I0"] + mui["mu_2"] * c) / den
    dmu = -a * mui["I0"] * (mui["mu_2"] - mui["mu_s"]) / den ** 2
    return M, -M * mu, S, -S * mu - M * dmu


def stencils(z, r, h, floor_z=0.0):
    """Per particle: offsets of its entries (real particles j != i with
    |z_j - z_i| <= r, then floor mirrors j* at 2 floor_z - z_j passing the
    same test), their source index and mirror flag, and the ghost offsets of
    the free-boundary rule (module docstring) on real 1D offsets."""
    n = z.size
    out = []
    for i in range(n):
        off, src, mir = [], [], []
        for j in range(n):
            d = z[j] - z[i]
            if j != i and d * d <= r * r:
                off.append(d); src.append(j); mir.append(False)
        for j in range(n):
            d = (2.0 * floor_z - z[j]) - z[i]
            if d * d <= r * r:
                off.append(d); src.append(j); mir.append(True)
        off = np.array(off)
        w = np.maximum(0.0, r * r - off * off)
        S = (w * off).sum()
        ghosts = []
        if abs(S) > 0.22 * h * w.sum():
            for k, o in enumerate(off):
                if o * S >= 0.5 * h * abs(S) and (2.0 * z[i] - (z[i] + o)) >= floor_z:
                    if np.all(np.abs(off + o) >= 0.5 * h):
                        ghosts.append(-o)
        out.append((off, np.array(src, dtype=int), np.array(mir), np.array(ghosts)))
    return out


def fit(off, b, h):
    """Least-squares [s', s''] from rows [dz/h, (dz/h)^2/2] and right-hand
    sides b (Sec. 3.1 item 7), scaled back by h."""
    d = off / h
    A = np.stack([d, 0.5 * d * d], 1)
    c = np.linalg.lstsq(A, b, rcond=None)[0]
    return c[0] / h, c[1] / (h * h)


def step(z, w, V, mui, eos, h, r, dt, g=-9.81, floor_z=0.0):
    """One explicit LP step of the 1D layer. Returns (z, w, V) at n+1 and the
    regime of each particle (0 gas, 1 inertial, 2 quasi-static)."""
    n = z.size
    st = stencils(z, r, h, floor_z)
    dw = np.zeros(n)
    d2w = np.zeros(n)
    for i, (off, src, mir, gh) in enumerate(st):
        wj = np.where(mir, -w[src], w[src])
        o = np.concatenate([off, gh])
        b = np.concatenate([wj - w[i], np.zeros(gh.size)])  # a ghost carries w_i
        dw[i], d2w[i] = fit(o, b, h)
    gn = np.abs(dw) / np.sqrt(3.0)
    gzz = 2.0 * dw / 3.0
    lapdiv = 2.0 * d2w / 3.0
    Vn = V + dt * (V * dw)
    phi_g = eos["phi_min"] * (1.0 - 1e-3)
    a = np.zeros(n)
    reg = np.zeros(n, dtype=int)
    for i, (off, src, mir, gh) in enumerate(st):
        phi = 1.0 / Vn[i]
        inertial = eos["phi_min"] < phi <= eos["phi_max"]
        gn_g = gn[i] * (eos["phi_c"] - phi_g) / (eos["phi_c"] - phi) if inertial else gn[i]
        o = np.concatenate([off, gh])
        bg = np.concatenate([np.where(mir, 0.0, gn[src]) - gn[i], np.full(gh.size, gn_g - gn[i])])
        bv = np.concatenate([Vn[src] - Vn[i], np.full(gh.size, 1.0 / phi_g - Vn[i])])
        dgn, _ = fit(o, bg, h)
        dV, _ = fit(o, bv, h)
        if phi <= eos["phi_min"]:
            a[i] = g
        elif phi <= eos["phi_max"]:
            reg[i] = 1
            M, N, S, R = closure(phi, mui, eos)
            Vi, G = Vn[i], gn[i]
            t1 = -(G / (Vi * Vi)) * (S * G * dV + R * gzz[i] * dV)
            t2 = 2.0 * M * G * dgn
            t3 = N * gzz[i] * dgn
            t4 = N * G * lapdiv[i]
            a[i] = Vi * (((t1 + t2) + t3) + t4) + g
        else:
            reg[i] = 2
            a[i] = eos["beta"] * dV / Vn[i] + g
    w1 = w + dt * a
    z1 = z + 0.5 * dt * (w + w1)
    return z1, w1, Vn, reg
