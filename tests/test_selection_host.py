"""Host logic of the follow-up selection over boxes (Sec. VI.A), on hand-made numbers:

* the detection rule's truth table (rejected / followed-up / other boxes);
* with every box followed up and nothing rejected, a signal is detected exactly when it
  beats its box's candidate;
* a population whose z grows linearly in c: the amplitude at p_det = 0.95 is the closed form
  z_last / (5 % quantile of the slopes) when no draw falls in a followed-up box;
* with a few contaminated (very loud) boxes, rejecting exactly those gives the lowest
  amplitude at a fixed follow-up budget (fewer waste follow-up slots, more discard clean
  boxes).
"""
import math

import numpy as np
import pytest

from paper_2411_18370_b300 import selection as S


class _Linear:
    """z(c) = slope * c per draw."""

    def __init__(self, slope):
        self.slope = np.asarray(slope, np.float64)

    def z(self, c):
        return self.slope * c


def test_truth_table():
    T = np.array([9.0, 3.0, 5.0, 4.0, 1.0])      # ranks: box0 0, box2 1, box3 2, box1 3, box4 4
    # reject 1 (box 0), follow up 2 (boxes 2 and 3): z_last = T[3] = 4
    box = np.array([0, 2, 2, 3, 1, 1, 4])
    z = np.array([100.0, 5.5, 4.5, 4.5, 4.5, 3.5, 4.1])
    got = S.detected(z, box, T, 1, 2)
    assert got.tolist() == [False, True, False, True, True, False, True]
    with pytest.raises(ValueError):
        S.detected(z, box, T, 4, 2)
    with pytest.raises(ValueError):
        S.detected(z, box, T, 0, 0)


def test_all_followed_up():
    g = np.random.default_rng(1)
    T = g.normal(3, 1, 40)
    box = g.integers(0, 40, 1000)
    z = g.normal(3, 2, 1000)
    assert np.array_equal(S.detected(z, box, T, 0, 40), z > T[box])


def test_linear_population_closed_form():
    g = np.random.default_rng(2)
    n_box = 200
    T = g.normal(4.0, 0.5, n_box)
    order, _ = S.box_ranks(T)
    n_cand = 10
    followed = set(order[:n_cand].tolist())
    others = np.array([b for b in range(n_box) if b not in followed])
    slope = g.uniform(0.5, 2.0, 5000)
    box = g.choice(others, 5000)
    sel = S.Selection(_Linear(slope), box, T)
    x = sel.log10_c_at(0.95, 0, n_cand)
    z_last = T[order[n_cand - 1]]
    # detected iff slope > z_last / c: p = 0.95 at c = z_last / (5 % quantile of the slopes)
    q = np.sort(slope)[int(math.floor(0.05 * len(slope)))]
    assert abs(10 ** x - z_last / q) < 1e-6 * z_last / q
    assert sel.pdet(10 ** x, 0, n_cand) >= 0.95


def test_rejecting_contaminated_boxes_helps():
    g = np.random.default_rng(3)
    n_box = 300
    T = g.normal(4.0, 0.4, n_box)
    bad = [7, 120, 255]
    T[bad] = [80.0, 60.0, 40.0]      # instrumental lines: far louder than noise
    slope = g.uniform(0.5, 2.0, 20000)
    box = g.integers(0, n_box, 20000)
    sel = S.Selection(_Linear(slope), box, T)
    best, x_best, xs = sel.optimise(n_cand=15, max_reject=8)
    # kept, the lines' boxes take follow-up slots that no signal in them can win; rejecting
    # more than them discards clean boxes
    assert best == 3
    assert xs[3] < xs[0] and xs[3] < xs[8]
    assert np.isfinite(xs).all()
