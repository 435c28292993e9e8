"""Pins of the oracle's number count (Eq. (number_count): nc = 1[P > 3.2] per SFT, summed
with the statistic's weights) and of the gated selection of Sec. VI.B.

* brute force on a tiny band: per template, the count of SFTs whose power at the track bin
  (the independently pinned canonical bins) exceeds the threshold;
* a track whose every bin is above the threshold counts sum w (N unweighted, 1 under the
  all-sky weights, whose rows sum to 1); a threshold below every power gives sum w too;
* in Gaussian noise P is exponential with mean 2: the count over templates with disjoint
  tracks has mean exp(-1.6) N = 0.2019 N and variance p (1 - p) N (closed forms);
* the gated selection with no effective gate is the plain selection; with a gate nobody
  passes every slot is empty; otherwise only passing templates appear.
"""
import math

import numpy as np

import ftsynth
import oracle


def _tiny(seed=4, n_sft=23, W=70, n_f0=20, n_f1=3, n_sky=4, sub=6):
    g = np.random.default_rng(seed)
    k_band = 150_000
    t_mid = np.sort(g.uniform(0, 2e7, n_sft)) + 900
    v = ftsynth.detector_velocity(t_mid, 0)
    P = g.integers(0, 10, (n_sft, W)).astype(np.float64)
    sfts = ftsynth.SFTSet(power=P, t_mid=t_mid, v=v, s_n=np.ones(n_sft), n_sft=[n_sft],
                          k_lo=k_band - 25, t_sft=1800.0, t0=0.0)
    bank = ftsynth.Bank(k0=k_band, n_f0=n_f0, f1=np.linspace(-2e-10, 0, n_f1),
                        sky=ftsynth.fibonacci_sky(n_sky), subband_bins=sub)
    return sfts, bank


def test_brute_force_tiny():
    sfts, bank = _tiny()
    t = np.arange(bank.n_templates)
    b = oracle.bins(sfts, bank, t)  # columns of the band (bin - k_lo)
    W = sfts.power.shape[1]
    for thr in (0.0, 3.2, 4.5, 8.5):
        nc, oob = oracle.number_count(sfts, bank, threshold=thr)
        for ti in range(0, bank.n_templates, 7):
            want = 0
            for a in range(sfts.n_total):
                k = b[ti, a]
                if 0 <= k < W and sfts.power[a, k] > thr:
                    want += 1
            assert nc[ti] == want
            assert oob[ti] == np.sum((b[ti] < 0) | (b[ti] >= W))


def test_saturated_track_counts_the_weights():
    sfts, bank = _tiny(seed=5)
    t0 = 2 * bank.n_f0 * bank.n_f1 + bank.n_f0 + 7
    b = oracle.bins(sfts, bank, [t0])[0]
    P = np.zeros_like(sfts.power)
    P[np.arange(sfts.n_total), b] = 6.0
    sx = ftsynth.SFTSet(**{**sfts.__dict__, "power": P})
    nc, _ = oracle.number_count(sx, bank, [t0])
    assert nc[0] == sfts.n_total
    w = np.random.default_rng(1).uniform(0.2, 2.0, sfts.n_total)
    nc_w, _ = oracle.number_count(sx, bank, [t0], w=w)
    assert math.isclose(nc_w[0], w.sum(), rel_tol=1e-14)
    D = ftsynth.detector_tensor(sfts.t_mid, 0)
    wsky = oracle.sky_weights(D, sfts.s_n, bank.sky)
    nc_s, _ = oracle.number_count(sx, bank, [t0], wsky=wsky)
    assert math.isclose(nc_s[0], 1.0, rel_tol=1e-13)
    # every power above a negative threshold: the count is sum w for every template
    nc_all, oob = oracle.number_count(sfts, bank, threshold=-1.0, w=w)
    assert np.all(oob == 0)
    assert np.allclose(nc_all, w.sum(), rtol=1e-14, atol=0)


def test_noise_moments_closed_form():
    p = math.exp(-1.6)
    assert abs(p - 0.20189651799) < 1e-11
    mu, sd = oracle.nc_moments(3.2, n_sft=1000)
    assert math.isclose(mu, 1000 * p) and math.isclose(sd, math.sqrt(1000 * p * (1 - p)))
    assert oracle.nc_moments(0.0, n_sft=10) == (10.0, 0.0)
    # Gaussian noise: exponential power with mean 2.  Templates of one sky point and f1 at
    # f0 bins 4 apart never share a bin, so their counts are independent Binomial(N, p).
    g = np.random.default_rng(11)
    N, W = 400, 4200
    t_mid = np.sort(g.uniform(0, 3e7, N)) + 900
    sfts = ftsynth.SFTSet(power=g.exponential(2.0, (N, W)), t_mid=t_mid,
                          v=ftsynth.detector_velocity(t_mid, 0), s_n=np.ones(N), n_sft=[N],
                          k_lo=300_000 - 50, t_sft=1800.0, t0=0.0)
    bank = ftsynth.Bank(k0=300_000, n_f0=4000, f1=np.array([0.0]), sky=np.array([[0.0, 0.0, 1.0]]),
                        subband_bins=4000)
    t = np.arange(0, 4000, 4)
    b = oracle.bins(sfts, bank, t)
    assert np.all(b[1:] - b[:-1] > 0)  # disjoint tracks
    nc, oob = oracle.number_count(sfts, bank, t)
    assert np.all(oob == 0)
    n = len(t)
    mu, sd = oracle.nc_moments(3.2, n_sft=N)
    assert abs(nc.mean() - mu) < 5 * sd / math.sqrt(n)
    # the sample variance of n = 1000 draws: relative standard error ~ sqrt(2 / n) = 4.5 %
    assert abs(nc.std(ddof=1) / sd - 1.0) < 0.15


def test_gated_selection():
    sfts, bank = _tiny(seed=6)
    s, _ = oracle.statistic(sfts, bank)
    nc, _ = oracle.number_count(sfts, bank)
    i0, v0 = oracle.topk_per_subband(s, bank, 4)
    i1, v1 = oracle.topk_gated(s, nc, -np.inf, bank, 4)
    assert np.array_equal(i0, i1) and np.array_equal(v0, v1)
    i2, v2 = oracle.topk_gated(s, nc, nc.max() + 1, bank, 4)
    assert np.all(i2 == -1) and np.all(v2 == -np.inf)
    gmin = np.median(nc)
    i3, v3 = oracle.topk_gated(s, nc, gmin, bank, 4)
    ok = i3 >= 0
    assert np.all(nc[i3[ok]] >= gmin)
    # each chosen value beats every passing template of its sub-band left out
    sub = (np.arange(bank.n_templates) % bank.n_f0) // bank.subband_bins
    for b in range(bank.n_subbands):
        chosen = set(i3[b][i3[b] >= 0].tolist())
        rest = [t for t in np.nonzero((sub == b) & (nc >= gmin))[0] if t not in chosen]
        if len(chosen) == 4 and rest:
            assert max(s[rest]) <= v3[b, 3]
