"""The mismatch distribution p(m | o) of a random binary bank (Sec. IV.A): signals on
noise-free data, banks of oversampling o over a region of +-1.5 resolution cells around each
(App. A resolutions), the best template's mismatch.  It lies in [0, 1] and falls as the
oversampling grows; with the region's expected number of cells the best of o N random
templates at o = 8 is usually close (median below 0.35)."""
import math

import numpy as np
import pytest

import ftsynth
import paper_2411_18370_b300 as ft
from paper_2411_18370_b300 import binary_bank as BB

pytestmark = pytest.mark.gpu


def test_mismatch_falls_with_oversampling():
    ctx = ft.create(0)
    T = 1024.0
    n_slots = int(30 * 86400 / T)
    starts = ftsynth.timeline(2, n_slots, T, 0.7, ftsynth.rng(77, 1))
    t_mid = np.concatenate([st + 0.5 * T for st in starts])
    v = np.concatenate([ftsynth.detector_velocity(st + 0.5 * T, X) for X, st in enumerate(starts)])
    n_sft = [len(st) for st in starts]
    g = np.random.default_rng(5)
    n_sig = 16
    sig = np.column_stack([
        g.uniform(100.0, 100.1, n_sig), g.uniform(0.1, 0.9, n_sig), g.uniform(-0.8, 0.8, n_sig),
        g.uniform(6.0, 14.0, n_sig), 2 * math.pi / (86400.0 * g.uniform(7.5, 14.5, n_sig)),
        g.uniform(0.1, 0.9, n_sig)])
    m = {o: BB.sample_mismatch(ctx, t_mid, v, n_sft, 0.0, T, sig, 1.5, o, seed=100 + 10 * o)
         for o in (1, 8)}
    for o, mm in m.items():
        assert np.all((mm >= 0) & (mm <= 1)), o
    assert np.mean(m[8]) < np.mean(m[1])
    assert np.median(m[8]) < 0.35
    print("mean mismatch o=1:", np.mean(m[1]), "o=8:", np.mean(m[8]))
    ctx.close()
