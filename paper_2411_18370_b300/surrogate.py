"""Learned p_det surrogate: features, training on campaign outcomes, h0 at a target p_det.

The network (ft_mlp, trained and evaluated by the library's CUDA kernels) maps
    [log10 c, log10 S_ref, duty cycle, n_x, n_y, n_z, f0 position in the band, f1 / 1e-9]
to the probability that the search detects the signal (Sec. V's p_det), where
c = h0 / sqrt(S_ref / T_SFT).  The amplitude at which a band reaches p_det = p is the root
in log10 c of the network's p_det averaged over the population's other parameters
(sky, f0, f1, and implicitly the orientation the network marginalises), found by
bisection with BF16 inference.
"""
from __future__ import annotations

import math

import numpy as np

from . import MLP

N_FEATURES = 8


def features(log10_c, log10_s, duty, n, f0_frac, f1):
    """Feature matrix [n_samples, 8] (FP32)."""
    m = len(log10_c)
    F = np.empty((m, N_FEATURES), np.float64)
    F[:, 0] = log10_c
    F[:, 1] = log10_s
    F[:, 2] = duty
    F[:, 3:6] = n
    F[:, 6] = f0_frac
    F[:, 7] = np.asarray(f1, np.float64) / 1e-9
    return F


class Surrogate:
    def __init__(self, ctx, width=128, seed=0):
        self.net = MLP(ctx, N_FEATURES, width, seed=seed)
        self.mu = None
        self.sd = None

    def _std(self, F):
        return ((F - self.mu) / self.sd).astype(np.float32)

    def fit(self, F, y, epochs=200, batch=1024, lr=2e-3, seed=0, val_frac=0.1, patience=12):
        """Train on the GPU one pass at a time, keeping the parameters of the pass with the
        lowest binary cross entropy on a seeded validation split (early stopping: the
        outcomes are noisy, so a long run memorises noise and over-states p_det).
        Returns (training losses, validation losses, best pass)."""
        y = np.asarray(y, np.float32)
        g = np.random.default_rng(seed)
        perm = g.permutation(len(y))
        n_val = max(1, int(round(val_frac * len(y))))
        vi, ti = perm[:n_val], perm[n_val:]
        self.mu = F[ti].mean(0)
        self.sd = F[ti].std(0) + 1e-12
        Xt, yt = self._std(F[ti]), y[ti]
        Xv, yv = self._std(F[vi]), y[vi].astype(np.float64)
        best, best_ep, best_theta = np.inf, -1, None
        tr, va = [], []
        for ep in range(epochs):
            tr.append(float(self.net.train(Xt, yt, batch=batch, epochs=1, lr=lr,
                                           seed=seed * 1000003 + ep)[0]))
            p = np.clip(self.net.predict(Xv, bf16=False).astype(np.float64), 1e-7, 1 - 1e-7)
            v = float(-np.mean(yv * np.log(p) + (1 - yv) * np.log(1 - p)))
            va.append(v)
            if v < best:
                best, best_ep, best_theta = v, ep, self.net.get_params()
            elif ep - best_ep >= patience:
                break
        self.net.set_params(best_theta)
        return np.array(tr), np.array(va), best_ep

    def p(self, F, bf16=True):
        return self.net.predict(self._std(F), bf16=bf16)

    def log10_c_at(self, p, log10_s, duty, pop, lo=-1.5, hi=2.5, bf16=True, iters=40):
        """Root in log10 c of mean_pop p_det = p; pop = dict(n [m,3], f0_frac [m], f1 [m])."""
        m = len(pop["f0_frac"])

        def mean_p(lc):
            F = features(np.full(m, lc), np.full(m, log10_s), np.full(m, duty), pop["n"],
                         pop["f0_frac"], pop["f1"])
            return float(np.mean(self.p(F, bf16=bf16)))

        a, b = lo, hi
        fa, fb = mean_p(a) - p, mean_p(b) - p
        if fa * fb > 0:
            return math.nan
        for _ in range(iters):
            mid = 0.5 * (a + b)
            fm = mean_p(mid) - p
            if (fm > 0) == (fb > 0):
                b, fb = mid, fm
            else:
                a, fa = mid, fm
        return 0.5 * (a + b)

    def close(self):
        self.net.close()
