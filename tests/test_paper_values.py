"""The paper's printed validation values against its own fits and against the
readings built on them (tests/golden/validation_values.txt, each value cited).

- Sec. 4.2.1 prints, for the a = 0.6 column, the fits' final height 0.03 m and
  radius 0.087 m at t = 0.17 s. The fits of Sec. 4.2 (h_inf = a r_i,
  r_inf = r_i (1 + 1.24 a), t_inf = 3 (h_i/g)^(1/2)) give all three from one
  initial radius, r_i = 0.05 m.
- Sec. 4.1 expects the 0.03 m layer to settle at 0.025 m. Compaction to the
  critical solid fraction phi_c = 0.60 (Sec. 4) then fixes the layer's
  initial mean solid fraction at 0.5, the start of the runs at the stated
  lengths. The initial profile the layer workload takes (0.50 at the floor
  to 0.48 at the top; the paper shows it only in a figure) averages 0.49 and
  settles 2 % lower, at 0.0245 m.
"""
import math
import os

import numpy as np

from paper_2206_14061_gb300 import workloads as W


def _golden():
    path = os.path.join(os.path.dirname(__file__), "golden", "validation_values.txt")
    out = {}
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            name, value = line.split()[:2]
            out[name] = float(value)
    return out


def test_column_fits_reproduce_the_printed_expectations():
    g = _golden()
    a = g["column_aspect"]
    r_i = g["column_expected_h"] / a            # h_inf = a r_i = h_i for a < 1.7
    assert abs(r_i - 0.05) < 1e-12
    r_inf = r_i * (1.0 + g["fit_r_small"] * a)
    assert abs(r_inf - g["column_expected_r"]) <= 0.0005   # printed to 1 mm
    t_inf = g["fit_t"] * math.sqrt(a * r_i / 9.81)
    assert abs(t_inf - g["column_time"]) <= 0.005           # printed to 0.01 s
    # the two radius fits meet at a = 1.7 to within 1 % (the height fits, as
    # printed, do not: a r_i against 0.88 r_i a^(1/6))
    a1 = 1.7
    assert abs((1 + g["fit_r_small"] * a1) / (1 + g["fit_r_large"] * math.sqrt(a1)) - 1) < 0.01
    # the simulated column is within 10 % (height) and 5 % (radius) of the fits
    assert abs(g["column_simulated_h"] / g["column_expected_h"] - 1) <= 0.1
    assert abs(g["column_simulated_r"] / g["column_expected_r"] - 1) <= 0.05


def test_layer_expectation_fixes_the_initial_solid_fraction():
    g = _golden()
    phi_c = W.EOS["phi_c"]
    phi0 = phi_c * g["layer_expected_height"] / g["layer_initial_height"]
    assert abs(phi0 - 0.5) < 1e-12
    wl = W.periodic_layer(n_xy=8, jitter=0.0)
    phi = 1.0 / wl.state["V"]
    assert abs(wl.extra["H"] - g["layer_initial_height"]) < 1e-15
    assert 0.48 <= phi.min() and phi.max() <= 0.50 and abs(phi.mean() - 0.49) < 1e-3
    settled = g["layer_initial_height"] * phi.mean() / phi_c
    assert abs(settled / g["layer_expected_height"] - 1) < 0.025
