"""Semi-analytic sensitivity estimate (Sec. V.A-V.C): p_det by sampling s instead of
simulating data.

For a population draw i the statistic of the best-matching template is Gaussian in the
many-SFT limit (Eq. (s_gauss)) with
    mean  mu_G + (1 - m_i) rho1_i h0^2,   variance  sigma_G^2 + (1 - m_i) rho2_i h0^2,
where rho1_i = sum w rho^2(h0 = 1) and rho2_i = sum w^2 rho^2(h0 = 1) depend only on the
draw's sky direction and orientation (computed once per band by ft_pdet_q), and m_i is the
mismatch of the closest template of the bank (Eq. (mismatch)).  Detection is z > tau
(Sec. V.B) with z = (s - mu_G) / sigma_G, and p_det at an amplitude is the fraction of draws
detected (Sec. V.C); the amplitude at which it reaches p is found by bisection.

The mismatch distribution p(m|o) comes from the same draws searched by the local bank of the
injection runs on noise-free data (ft_run_injections with noise_scale = 0): the loudest
template then recovers s' = z sigma_G + mu_G of the full signal power rho1 h0^2, and
m = 1 - s' / (rho1 h0^2).  Every step that touches per-SFT data runs in the library's CUDA
kernels; this module only combines the per-draw numbers.

The mean of s under noise uses mu_G without the running-median PSD bias factor of Sec. V.A
(1.012): the synthetic bands are normalised by their true S_n.  Amplitudes are in units of
sqrt(S_ref / T_SFT) as in the injection campaign (c = h0 / sqrt(S_ref / T_SFT)).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import pdet_q, run_injections


@dataclasses.dataclass
class Estimate:
    rho1: np.ndarray   # per draw, sum w rho^2 at h0 = 1
    rho2: np.ndarray   # per draw, sum w^2 rho^2 at h0 = 1
    m: np.ndarray      # per draw, mismatch of the best local template
    xi: np.ndarray     # per draw, a standard normal deviate (the noise of s), common to all c
    mu: float          # mu_G of the band
    sigma: float       # sigma_G of the band
    h2_per_c2: float   # h0^2 per c^2 = S_ref / T_SFT
    tau: float         # detection threshold on z

    def z(self, c):
        """z of every draw at amplitude c."""
        h2 = (np.asarray(c, np.float64) ** 2) * self.h2_per_c2
        keep = 1.0 - self.m
        mean = keep * self.rho1 * h2
        sd = np.sqrt(self.sigma ** 2 + keep * self.rho2 * h2)
        return (mean + self.xi * sd) / self.sigma

    def pdet(self, c):
        return float(np.mean(self.z(c) > self.tau))

    def log10_c_at(self, p, lo=-1.5, hi=2.5, iters=60):
        """Root in log10 c of p_det = p (p_det is monotone in c draw by draw)."""
        a, b = lo, hi
        if self.pdet(10 ** a) >= p or self.pdet(10 ** b) < p:
            return math.nan
        for _ in range(iters):
            mid = 0.5 * (a + b)
            if self.pdet(10 ** mid) >= p:
                b = mid
            else:
                a = mid
        return 0.5 * (a + b)


def build(ctx, band, bank, det_tensor, pop, tau, s_ref, t_sft, seed, first_run_id, probe_c=10.0,
          **kw):
    """The semi-analytic estimate for population draws `pop` (INJECTION_DTYPE; h0 ignored) of
    one band: q numbers on the GPU, mismatches from noise-free local-bank runs at amplitude
    probe_c (any amplitude gives the same mismatch), and seeded normal deviates."""
    rho1, rho2 = pdet_q(ctx, band, det_tensor, pop)
    h2_per_c2 = s_ref / t_sft
    probe = np.array(pop, copy=True)
    probe["h0"] = probe_c * math.sqrt(h2_per_c2)
    res = run_injections(ctx, band, bank, det_tensor, probe, seed=seed, first_run_id=first_run_id,
                         noise_scale=0.0, **kw)
    if np.any(res["n_out_of_window"] != 0):
        raise RuntimeError("local bank reads outside the generated window; widen half_window")
    recovered = res["max_z"] * band.sigma_g + band.mu_g
    m = np.clip(1.0 - recovered / (rho1 * probe_c ** 2 * h2_per_c2), 0.0, 1.0)
    xi = np.random.default_rng(seed).standard_normal(len(pop))
    return Estimate(rho1=rho1, rho2=rho2, m=m, xi=xi, mu=band.mu_g, sigma=band.sigma_g,
                    h2_per_c2=h2_per_c2, tau=tau)
