"""Host logic of binary-bank sizing (App. A, Eq. (N_binary); Sec. IV.B box policy):

* the closed-form template count equals the integral of the density k f0^5 a_p^2 Omega^3 over
  the region (numerical quadrature, angles in radians);
* the per-dimension cell counts (resolutions at the centre) multiply to about it;
* plans give at least the requested boxes, no box above the cap, at least o N templates, and
  never more divisions of a dimension than it has cells.
"""
import math

import numpy as np
from scipy import integrate

from paper_2411_18370_b300 import binary_bank as BB

T, TOBS, VC = 1024.0, 183 * 86400.0, 1e-4
LO = (100.0, 0.1, -0.3, 5.0, 2 * math.pi / (15 * 86400), 0.2)
HI = (100.125, 0.4, 0.5, 15.0, 2 * math.pi / (7 * 86400), 0.9)


def test_count_is_the_density_integral():
    k = T ** 6 * TOBS * VC ** 2
    i_f = integrate.quad(lambda f: f ** 5, LO[0], HI[0])[0]
    i_a = integrate.quad(lambda a: a ** 2, LO[3], HI[3])[0]
    i_o = integrate.quad(lambda o: o ** 3, LO[4], HI[4])[0]
    sky = 2 * math.pi * (HI[1] - LO[1]) * (HI[2] - LO[2])
    want = k * i_f * sky * i_a * i_o * 2 * math.pi * (HI[5] - LO[5])
    assert math.isclose(BB.n_templates(LO, HI, T, TOBS, VC), want, rel_tol=1e-10)
    # the per-dimension cells (resolutions at the centre) multiply to about the same count
    assert 0.5 < np.prod(BB.cells_per_dim(LO, HI, T, TOBS, VC)) / want < 2.0


def test_plans_respect_the_box_policy():
    full_lo = (100.0, 0.0, -1.0, 5.0, 2 * math.pi / (15 * 86400), 0.0)
    full_hi = (100.125, 1.0, 1.0, 15.0, 2 * math.pi / (7 * 86400), 1.0)
    for o, min_boxes, max_box in [(3.44, 10_000, 1e8), (1.0, 100, 1e6), (8.0, 1, 1e9)]:
        n_div, n_per_box = BB.plan(full_lo, full_hi, o, T, TOBS, VC, min_boxes, max_box)
        total = o * BB.n_templates(full_lo, full_hi, T, TOBS, VC)
        nb = int(np.prod(n_div))
        assert nb >= min_boxes
        assert n_per_box <= max(max_box, math.ceil(total / nb))
        assert nb * n_per_box >= total
        cells = BB.cells_per_dim(full_lo, full_hi, T, TOBS, VC)
        assert all(d >= 1 for d in n_div)
        assert all(d <= max(1, math.ceil(c)) or d == 1 for d, c in zip(n_div, cells))
    # the paper's band (0.125 Hz at 100 Hz, o = 3.44): boxes of far fewer than 1e8 templates
    n_div, n_per_box = BB.plan(full_lo, full_hi, 3.44, T, TOBS, VC)
    assert np.prod(n_div) >= 10_000 and 1e6 < n_per_box < 1e8
    assert n_div[0] <= 128  # no more f0 divisions than the band's 128 bins
    # a region with fewer cells than boxes wanted: every dimension capped at its cell count
    tiny_hi = (100.002, 0.1001, -0.2999, 5.01, LO[4] * 1.001, 0.2001)
    n_div, n_per_box = BB.plan(LO, tiny_hi, 1.0, T, TOBS, VC, 10_000, 1e8)
    assert n_per_box >= 1 and np.prod(n_div) >= 10_000


def test_signal_bins_zero_orbit_zero_doppler():
    t = np.array([1000.0, 5000.0, 9000.0])
    v = np.zeros((3, 3))
    b = BB.signal_bins((100.0003, 0.3, 0.1, 0.0, 1e-5, 0.4), t, v, 0.0, 1800.0, 179_990)
    assert np.all(b == int(math.floor(100.0003 * 1800 + 0.5)) - 179_990)
