"""Injection campaigns: detection threshold, p_det(h0) and the amplitude at a target p_det.

Sec. V: the sensitivity of a search is the amplitude h0 (or depth sqrt(S_n)/h0) at which a
fraction p of a signal population is detected; p_det is estimated by Monte Carlo over
software-simulated signals (Eq. (sampling)) scored by the threshold rule R(z; tau) = 1[z >
tau] (Sec. V.B).  The per-run work (simulating the data and searching the local bank) runs
in the library's CUDA kernels (ft_run_injections); this module draws the population, sets
tau from noise-only runs, and fits the detection curve with a sigmoid in log10 h0 whose
uncertainty comes from the fit covariance (Sec. VI).

Amplitudes are handled in noise units: c = h0 / sqrt(S_ref / T_SFT) with S_ref the band's
mean PSD level.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import INJECTION_DTYPE, run_injections


def draw_population(n, f_lo, f_hi, g, log10_c=None, c_range=(0.3, 30.0), f1_range=(-1e-9, 0.0),
                    s_ref=1.0, t_sft=1800.0):
    """Isotropic sky, cos(iota) ~ U[-1, 1], psi ~ U[0, pi], f0 ~ U[f_lo, f_hi],
    f1 ~ U[f1_range], and log10 c ~ U[log10 c_range] unless given.  Returns the injection
    records and the log10 c of each."""
    inj = np.zeros(n, INJECTION_DTYPE)
    if log10_c is None:
        log10_c = g.uniform(math.log10(c_range[0]), math.log10(c_range[1]), n)
    log10_c = np.broadcast_to(np.asarray(log10_c, np.float64), (n,)).copy()
    inj["h0"] = 10.0 ** log10_c * math.sqrt(s_ref / t_sft)
    inj["cosi"] = g.uniform(-1.0, 1.0, n)
    inj["psi"] = g.uniform(0.0, math.pi, n)
    inj["f0"] = g.uniform(f_lo, f_hi, n)
    inj["f1"] = g.uniform(f1_range[0], f1_range[1], n)
    m = g.standard_normal((n, 3))
    inj["n"] = m / np.linalg.norm(m, axis=1)[:, None]
    return inj, log10_c


def noise_threshold(ctx, band, bank, det_tensor, n_runs, seed, first_run_id, f_lo, f_hi,
                    false_alarm=0.01, g=None, **kw):
    """tau = the (1 - false_alarm) quantile of the loudest z over noise-only local searches
    with the same bank shape.  Returns tau and the noise-only max z values."""
    g = np.random.default_rng(seed) if g is None else g
    inj, _ = draw_population(n_runs, f_lo, f_hi, g, log10_c=np.full(n_runs, -np.inf))
    inj["h0"] = 0.0
    res = run_injections(ctx, band, bank, det_tensor, inj, seed=seed, first_run_id=first_run_id,
                         **kw)
    if np.any(res["n_out_of_window"] != 0):
        raise RuntimeError("local bank reads outside the generated window; widen half_window")
    z = res["max_z"]
    return float(np.quantile(z, 1.0 - false_alarm, method="higher")), z


class CampaignInterrupted(RuntimeError):
    """Raised by run_campaign(stop_after=...) once its batch budget is spent."""


def run_campaign(ctx, band, bank, det_tensor, n, tau, seed, first_run_id, f_lo, f_hi, s_ref,
                 t_sft, c_range=(0.3, 30.0), g=None, checkpoint_dir=None, batch_runs=4096,
                 stop_after=None, **kw):
    """n injections with log-uniform amplitude; returns log10 c, detected (0/1), max z and the
    injection records.

    checkpoint_dir: the runs go in batches of batch_runs (run ids first_run_id + index, so a
    batch's outcomes equal the same slice of one launch); each finished batch is written to
    batch_<seed>_<first_run_id>_<b>.npz there and skipped by a later call with the same
    arguments.  stop_after: stop (raising CampaignInterrupted) after that many batches were
    run by this call."""
    g = np.random.default_rng(seed) if g is None else g
    inj, lc = draw_population(n, f_lo, f_hi, g, c_range=c_range, s_ref=s_ref, t_sft=t_sft)
    if checkpoint_dir is None:
        res = run_injections(ctx, band, bank, det_tensor, inj, seed=seed, first_run_id=first_run_id,
                             **kw)
        max_z, oob = res["max_z"], res["n_out_of_window"]
    else:
        import os

        os.makedirs(checkpoint_dir, exist_ok=True)
        max_z = np.empty(n, np.float64)
        oob = np.empty(n, np.int64)
        ran = 0
        for b, lo in enumerate(range(0, n, batch_runs)):
            hi = min(n, lo + batch_runs)
            path = os.path.join(checkpoint_dir, f"batch_{seed}_{first_run_id}_{b}.npz")
            if os.path.exists(path):
                with np.load(path) as z:
                    max_z[lo:hi], oob[lo:hi] = z["max_z"], z["n_out_of_window"]
                continue
            if stop_after is not None and ran >= stop_after:
                raise CampaignInterrupted(f"stopped after {ran} batches")
            res = run_injections(ctx, band, bank, det_tensor, inj[lo:hi], seed=seed,
                                 first_run_id=first_run_id + lo, **kw)
            max_z[lo:hi], oob[lo:hi] = res["max_z"], res["n_out_of_window"]
            tmp = path + ".tmp.npz"
            np.savez(tmp, max_z=res["max_z"], n_out_of_window=res["n_out_of_window"])
            os.replace(tmp, path)
            ran += 1
    if np.any(oob != 0):
        raise RuntimeError("local bank reads outside the generated window; widen half_window")
    det = (max_z > tau).astype(np.float64)
    return lc, det, max_z, inj


@dataclasses.dataclass
class Sigmoid:
    """p(x) = 1 / (1 + exp(-k (x - x0))), x = log10 of the amplitude."""

    x0: float
    k: float
    cov: np.ndarray  # covariance of (b0, b1) with p = sigmoid(b0 + b1 x)
    b: np.ndarray

    def p(self, x):
        return 1.0 / (1.0 + np.exp(-(self.b[0] + self.b[1] * np.asarray(x, np.float64))))

    def x_at(self, p):
        return (math.log(p / (1.0 - p)) - self.b[0]) / self.b[1]

    def x_at_sigma(self, p):
        """Standard error of x_at(p) from the fit covariance (delta method)."""
        b0, b1 = self.b
        L = math.log(p / (1.0 - p))
        grad = np.array([-1.0 / b1, -(L - b0) / (b1 * b1)])
        return float(math.sqrt(grad @ self.cov @ grad))


def local_x_at(x, det, p, x0, half=0.05, iters=5):
    """Amplitude x at which the detection fraction is p, from sigmoid fits restricted to the
    samples with |x - x_p| < half, re-centred on each fit's estimate (starting from x0).

    Far above the transition the detection curve rises more slowly than a logistic (the
    least favourable orientations keep p_det below 1), so one sigmoid over a wide range
    places the 90% point too low; within a narrow window the curve is a sigmoid.  Returns
    (x_p, its standard error, samples used)."""
    x = np.asarray(x, np.float64)
    det = np.asarray(det, np.float64)
    xp, f, m = x0, None, None
    for _ in range(iters):
        m = np.abs(x - xp) < half
        if m.sum() < 20:
            raise ValueError("local_x_at: fewer than 20 samples in the window")
        f = fit_sigmoid(x[m], det[m])
        xp = f.x_at(p)
    return xp, f.x_at_sigma(p), int(m.sum())


def fit_sigmoid(x, det, iters=100):
    """Maximum-likelihood logistic fit of detections against x (Newton's method on the
    binomial log-likelihood); the covariance is the inverse observed information."""
    x = np.asarray(x, np.float64)
    y = np.asarray(det, np.float64)
    A = np.stack([np.ones_like(x), x], axis=1)
    b = np.array([-np.mean(x) * 3.0, 3.0])
    for _ in range(iters):
        p = 1.0 / (1.0 + np.exp(-(A @ b)))
        wv = np.clip(p * (1 - p), 1e-12, None)
        H = A.T @ (A * wv[:, None])
        grad = A.T @ (y - p)
        step = np.linalg.solve(H + 1e-12 * np.eye(2), grad)
        b = b + step
        if np.max(np.abs(step)) < 1e-12:
            break
    p = 1.0 / (1.0 + np.exp(-(A @ b)))
    H = A.T @ (A * np.clip(p * (1 - p), 1e-12, None)[:, None])
    cov = np.linalg.inv(H)
    return Sigmoid(x0=-b[0] / b[1], k=b[1], cov=cov, b=b)
