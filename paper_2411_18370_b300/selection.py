"""Follow-up selection over ahead-of-time boxes and its sensitivity (Sec. VI.A).

After the search every box b has its loudest candidate, with critical ratio T[b] (the
candidate list ft_topk_per_band / ft_binary_topk_per_box returns, k = 1).  A follow-up
budget of N_cand boxes is spent on the boxes ranked N_reject .. N_reject + N_cand - 1 by T
(descending): the N_reject loudest boxes are rejected as contaminated, the next N_cand are
followed up.  A signal of critical ratio z falling in box b is then detected when
  - b is rejected: never;
  - b is followed up: z > T[b] (the signal, not the noise candidate, is the box's loudest);
  - otherwise: z > T of the last followed-up box (the signal would have entered the list).
The population's detection probability at amplitude c uses the semi-analytic draws of
Sec. V (semianalytic.Estimate: one z per draw and amplitude), and the amplitude at which it
reaches p (the paper quotes the 95 % depth) is found by bisection.  For a fixed budget the
number of rejected boxes that minimises that amplitude (maximises the depth) is found by
scanning N_reject.  Everything here is host bookkeeping over per-box and per-draw numbers
that the library's kernels produced.
"""
from __future__ import annotations

import math

import numpy as np


def box_ranks(T):
    """Rank of every box by T descending (ties by the smaller box index)."""
    T = np.asarray(T, np.float64)
    order = np.lexsort((np.arange(len(T)), -T))
    rank = np.empty(len(T), np.int64)
    rank[order] = np.arange(len(T))
    return order, rank


def detected(z, box, T, n_reject, n_cand, order=None, rank=None):
    """Detection of signals with critical ratios z in boxes `box` under the rule above."""
    T = np.asarray(T, np.float64)
    if n_cand < 1 or n_reject < 0 or n_reject + n_cand > len(T):
        raise ValueError("need n_cand >= 1, n_reject >= 0 and n_reject + n_cand <= n_boxes")
    if order is None or rank is None:
        order, rank = box_ranks(T)
    z = np.asarray(z, np.float64)
    r = rank[np.asarray(box)]
    rejected = r < n_reject
    followed = (r >= n_reject) & (r < n_reject + n_cand)
    z_last = T[order[n_reject + n_cand - 1]]
    return ~rejected & np.where(followed, z > T[box], z > z_last)


class Selection:
    """p_det of a population under one (N_reject, N_cand) choice.  `estimate` gives z(c) per
    draw (semianalytic.Estimate or any object with a z(c) method); `box` the box of each
    draw; T the loudest critical ratio of each box."""

    def __init__(self, estimate, box, T):
        self.est = estimate
        self.box = np.asarray(box, np.int64)
        self.T = np.asarray(T, np.float64)
        self.order, self.rank = box_ranks(self.T)

    def pdet(self, c, n_reject, n_cand):
        return float(np.mean(detected(self.est.z(c), self.box, self.T, n_reject, n_cand,
                                      self.order, self.rank)))

    def log10_c_at(self, p, n_reject, n_cand, lo=-1.5, hi=3.0, iters=60):
        """Smallest log10 c with p_det >= p, to 2^-60 of [lo, hi] (nan when p is not
        reached within [lo, hi])."""
        a, b = lo, hi
        if self.pdet(10 ** a, n_reject, n_cand) >= p or self.pdet(10 ** b, n_reject, n_cand) < p:
            return math.nan
        for _ in range(iters):
            mid = 0.5 * (a + b)
            if self.pdet(10 ** mid, n_reject, n_cand) >= p:
                b = mid
            else:
                a = mid
        return b  # the upper end: p_det(10^b) >= p

    def optimise(self, n_cand, max_reject, p=0.95):
        """Scan N_reject = 0 .. max_reject at a fixed budget; returns (best N_reject,
        log10 c_p at the best, log10 c_p per N_reject)."""
        max_reject = min(max_reject, len(self.T) - n_cand)
        x = np.array([self.log10_c_at(p, r, n_cand) for r in range(max_reject + 1)])
        ok = np.isfinite(x)
        if not ok.any():
            return -1, math.nan, x
        best = int(np.nanargmin(x))
        return best, float(x[best]), x
