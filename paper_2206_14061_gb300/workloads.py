"""Seeded synthetic inputs shaped like the paper's column-collapse workloads.

This module only draws inputs: lattices with jitter, cylinders, batches of
columns, smooth test fields and the material/EOS parameter sets. It holds none
of the method's arithmetic, and both the CUDA path and the CPU oracle read the
same arrays from it.

Geometry follows Sec. 4.2 (axisymmetric column on a floor, lattice initial
distribution as in Sec. 3.1 item 2). Material values follow the benchmark
parameter set (mu_s 0.38, mu_2 0.64, I0 0.28, d 5e-4 m, rho 2500 kg/m^3);
phi_c = 0.60 and phi_min = 0.35 are the paper's (Sec. 4). The paper gives no
phi_max, alpha, beta or initial solid fraction; the values below are this
project's readings: phi_max 0.59, beta 400 m^2/s^2, alpha = -beta phi_max,
phi_0 = 0.585.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20220628

# material and EOS parameters (see module docstring)
MUI = dict(mu_s=0.38, mu_2=0.64, I0=0.28, d=5e-4, rho_s=2500.0)
EOS = dict(phi_c=0.60, phi_min=0.35, phi_max=0.59, beta=400.0)
EOS["alpha"] = -EOS["beta"] * EOS["phi_max"]
PHI0 = 0.585
GRAVITY = (0.0, 0.0, -9.81)
# the paper's own parameter set (Sec. 4), used only for context checks
PAPER_MUI = dict(mu_s=math.tan(math.radians(30.0)), mu_2=math.tan(math.radians(50.0)), I0=2.65,
                 d=0.32e-3, rho_s=2600.0)


@dataclass
class Workload:
    name: str
    h: float
    radius: float
    dt: float
    state: dict                      # x, y, z, u, v, w, V  (float64, length n)
    column_offsets: np.ndarray | None = None   # int32 [ncolumns + 1]
    mu_s_col: np.ndarray | None = None         # per-column mu_s
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.state["x"].size)


def _rng(index: int, salt: int = 0) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + index + 1000 * salt)


def _rest_state(x, y, z, phi0=PHI0) -> dict:
    n = x.size
    return dict(x=x, y=y, z=z, u=np.zeros(n), v=np.zeros(n), w=np.zeros(n),
                V=np.full(n, 1.0 / phi0))


def _jitter(rng, pts, h, frac):
    return [p + rng.uniform(-frac * h, frac * h, size=p.size) for p in pts]


def lattice_box(nx, ny, nz, h, jitter, rng):
    """Cell-centred lattice (i + 1/2) h, uniform jitter of +-jitter*h per axis."""
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    pts = [((a.ravel(order="F") + 0.5) * h) for a in (ix, iy, iz)]
    return _jitter(rng, pts, h, jitter)


def lattice_cylinder(R, H, h, jitter, rng, x0=0.0, y0=0.0):
    """Lattice centres inside the cylinder x^2 + y^2 <= R^2, 0 < z < H."""
    nr = int(math.ceil(R / h))
    nz = int(round(H / h))
    c = (np.arange(-nr, nr) + 0.5) * h
    X, Y = np.meshgrid(c, c, indexing="xy")
    keep = (X * X + Y * Y) <= R * R
    X, Y = X[keep], Y[keep]
    Z = (np.arange(nz) + 0.5) * h
    x = np.tile(X, nz) + x0
    y = np.tile(Y, nz) + y0
    z = np.repeat(Z, X.size)
    return _jitter(rng, [x, y, z], h, jitter)


def cube(n_side=20, h=1e-3, jitter=0.05, index=0) -> Workload:
    """Column at rest on a no-slip floor: n_side^3 lattice, r = 2.2h, dt = 1e-5."""
    rng = _rng(index)
    x, y, z = lattice_box(n_side, n_side, n_side, h, jitter, rng)
    return Workload(f"cube{n_side}", h, 2.2 * h, 1e-5, _rest_state(x, y, z))


def cylinder(R=0.02, aspect=2.0, spacing_div=50, jitter=0.05, index=2) -> Workload:
    """Cylindrical column of radius R, height aspect*R, lattice spacing R/spacing_div."""
    rng = _rng(index)
    h = R / spacing_div
    x, y, z = lattice_cylinder(R, aspect * R, h, jitter, rng)
    return Workload(f"cylinder_R{R}_a{aspect}_h{h:.2e}", h, 2.2 * h, 1e-5, _rest_state(x, y, z),
                    extra=dict(R=R, H=aspect * R))


def columns(ncol=256, n_lo=2000, n_hi=64000, h=1e-3, index=3, only=None) -> Workload:
    """Batch of independent columns: N_c log-uniform in [n_lo, n_hi], aspect
    U(0.5, 6), mu_s U(0.3, 0.45), R_c = h (N_c / (pi a_c))^(1/3). Each column
    lives in its own frame (centred at the origin); `only` selects a subset."""
    rng = _rng(index)
    Nc = np.round(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=ncol))).astype(np.int64)
    ac = rng.uniform(0.5, 6.0, size=ncol)
    mus = rng.uniform(0.30, 0.45, size=ncol)
    sel = range(ncol) if only is None else only
    parts, offs, R_all, mu_sel = [], [0], [], []
    for c in sel:
        R = h * (Nc[c] / (math.pi * ac[c])) ** (1.0 / 3.0)
        crng = _rng(index, salt=1 + int(c))
        x, y, z = lattice_cylinder(R, ac[c] * R, h, 0.05, crng)
        parts.append((x, y, z))
        offs.append(offs[-1] + x.size)
        R_all.append(R)
        mu_sel.append(mus[c])
    x = np.concatenate([p[0] for p in parts])
    y = np.concatenate([p[1] for p in parts])
    z = np.concatenate([p[2] for p in parts])
    return Workload(f"columns{len(offs) - 1}", h, 2.2 * h, 1e-5, _rest_state(x, y, z),
                    column_offsets=np.asarray(offs, dtype=np.int32),
                    mu_s_col=np.asarray(mu_sel, dtype=np.float64),
                    extra=dict(N_target=Nc[list(sel)], aspect=ac[list(sel)], R=np.asarray(R_all)))


def periodic_layer(n_xy=16, H=0.03, h=1e-3, jitter=0.05, phi_bot=0.50, phi_top=0.48,
                   index=5) -> Workload:
    """Granular layer of height H on the floor, periodic along x and y with
    period L = n_xy h (the 3D run of the paper's 1D/3D compaction check,
    Sec. 4): at rest, solid fraction falling linearly from phi_bot at the
    floor to phi_top at the top (the paper shows the initial profile only in a
    figure; a slight linear decrease is this project's reading),
    positions in [0, L)."""
    rng = _rng(index)
    nz = int(round(H / h))
    x, y, z = lattice_box(n_xy, n_xy, nz, h, jitter, rng)
    L = n_xy * h
    x, y = np.mod(x, L), np.mod(y, L)
    st = _rest_state(x, y, z)
    st["V"] = 1.0 / (phi_bot + (phi_top - phi_bot) * (z / H))
    return Workload(f"periodic_layer{n_xy}x{n_xy}x{nz}", h, 2.2 * h, 1e-5, st,
                    extra=dict(L=L, H=H))


def sweep_lattice(n_side=126, h=1e-3, jitter=0.2, index=1, nfields=4, nterms=8):
    """Derivative-operator sweep: jittered lattice, per-particle radius
    U(1.8h, 2.6h), and nfields smooth fields s(x) = sum_k a_k sin(kvec_k . x + p_k)
    with a_k ~ N(0,1), p_k ~ U(0, 2 pi), kvec_k = k (2 pi / L) e_k, e_k a random
    unit vector, k = 1..nterms, L the lattice edge. Returns (x, y, z, radius,
    fields [nfields, n], spec) where spec holds (a, kvec, phase) per field."""
    rng = _rng(index)
    x, y, z = lattice_box(n_side, n_side, n_side, h, jitter, rng)
    radius = rng.uniform(1.8 * h, 2.6 * h, size=x.size)
    L = n_side * h
    spec = []
    fields = np.zeros((nfields, x.size))
    for f in range(nfields):
        a = rng.standard_normal(nterms)
        ph = rng.uniform(0.0, 2.0 * math.pi, size=nterms)
        e = rng.standard_normal((nterms, 3))
        e /= np.linalg.norm(e, axis=1, keepdims=True)
        kv = (np.arange(1, nterms + 1)[:, None] * (2.0 * math.pi / L)) * e
        spec.append((a, kv, ph))
        for k in range(nterms):
            fields[f] += a[k] * np.sin(kv[k, 0] * x + kv[k, 1] * y + kv[k, 2] * z + ph[k])
    return x, y, z, radius, fields, spec


def param_dict(wl: Workload, mirror_mode: int = 1) -> dict:
    """Flat parameter dictionary for one column (material, EOS, numerics)."""
    d = dict(MUI)
    d.update(EOS)
    d.update(h=wl.h, radius=wl.radius, gx=GRAVITY[0], gy=GRAVITY[1], gz=GRAVITY[2],
             floor_z=0.0, dt=wl.dt, mirror_mode=mirror_mode)
    return d
