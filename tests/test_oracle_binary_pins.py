"""Pins of the oracle's binary-orbit track (Eq. (track)) and random hyperbox bank
(Eq. (xi_of_lambda), App. A Eq. (unif_transform), Sec. IV.B):

* every template lies in its own box and is uniform in the uniform coordinates
  xi = {f0^6, alpha, sin(delta), a_p^3, Omega^4, phi_b} there (mean 1/2, variance 1/12 of the
  position within the box along each axis);
* the orbit term in closed form: with the detectors at rest, SFTs placed where the orbit phase
  Omega t - phi_b is 0, pi/2, pi and 3 pi/2 put the track at f0 T_SFT (1 - a_p Omega),
  f0 T_SFT, f0 T_SFT (1 + a_p Omega) and f0 T_SFT (a source receding at the ascending node
  is redshifted by a_p Omega);
* the Doppler term in closed form: an isolated source (a_p = 0) at n = x, y or z sits at
  f0 T_SFT (1 + v_x), (1 + v_y) or (1 + v_z);
* with a_p = 0 and no detector motion every SFT reads the same bin, round(f0 T_SFT)
  (zero-Doppler tracks collapse to fixed bins);
* on random templates and SFTs of a moving detector the oracle's FP64 position equals a
  40-digit evaluation (mpmath) of Eq. (track) to 1e-9 bins, so its bins are those of the
  exact track except within 1e-9 bins of a rounding boundary;
* the statistic equals a Python sum over SFTs along the bins, and a noise-free track of unit
  power recovers N_SFT;
* the per-box selection returns each box's loudest templates.
"""
import math

import mpmath
import numpy as np

import ftsynth
import oracle

DAY = 86400.0


def _bank(n_div=(2, 2, 2, 2, 2, 2), n_per_box=40, seed=11, f0=(100.0, 100.05), ap=(5.0, 15.0),
          alpha=(0.0, 1.0), sind=(-1.0, 1.0), om=None):
    om = om or (2 * math.pi / (15 * DAY), 2 * math.pi / (7 * DAY))
    return ftsynth.BinaryBank(lo=(f0[0], alpha[0], sind[0], ap[0], om[0], 0.0),
                              hi=(f0[1], alpha[1], sind[1], ap[1], om[1], 1.0),
                              n_div=n_div, n_per_box=n_per_box, seed=seed)


def _sfts(n_sft=(70, 60), W=200, wings=55, seed=3, k_band=180_000, moving=True, t0=0.0):
    g = np.random.default_rng(seed)
    t_mid, v = [], []
    for X, n in enumerate(n_sft):
        t = np.sort(g.uniform(0, ftsynth.YEAR_S, n)) + 900 + t0
        t_mid.append(t)
        v.append(ftsynth.detector_velocity(t, X) if moving else np.zeros((n, 3)))
    t_mid = np.concatenate(t_mid)
    N = len(t_mid)
    return ftsynth.SFTSet(power=g.exponential(2.0, (N, W)), t_mid=t_mid, v=np.concatenate(v),
                          s_n=np.ones(N), n_sft=list(n_sft), k_lo=k_band - wings, t_sft=1800.0,
                          t0=t0)


def _xi(lam):
    return np.column_stack([lam[:, 0] ** 6, lam[:, 1], lam[:, 2], lam[:, 3] ** 3, lam[:, 4] ** 4,
                            lam[:, 5]])


def test_templates_fill_their_boxes_uniformly():
    bank = _bank(n_per_box=200)
    lam = oracle.binary_templates(bank)
    xi = _xi(lam)
    lo = _xi(np.array([bank.lo]))[0]
    hi = _xi(np.array([bank.hi]))[0]
    box = np.arange(bank.n_templates) // bank.n_per_box
    bk = np.zeros((bank.n_templates, 6), np.int64)
    b = box.copy()
    for d in range(5, -1, -1):
        bk[:, d] = b % bank.n_div[d]
        b //= bank.n_div[d]
    pos = (xi - lo) / ((hi - lo) / np.array(bank.n_div)) - bk
    assert np.all(pos > -1e-9) and np.all(pos < 1 + 1e-9)
    n = bank.n_templates
    for d in range(6):
        assert abs(pos[:, d].mean() - 0.5) < 4 * math.sqrt(1 / 12 / n)
        assert abs(pos[:, d].var() - 1 / 12) < 0.006
    # lambda inside the physical range
    assert np.all(lam >= np.array(bank.lo) - 1e-12) and np.all(lam <= np.array(bank.hi) + 1e-12)
    # a different seed draws different templates; the same seed the same ones
    assert np.array_equal(lam, oracle.binary_templates(bank))
    lam3 = oracle.binary_templates(ftsynth.BinaryBank(**{**bank.__dict__, "seed": 12}))
    assert not np.any(lam3[:, 0] == lam[:, 0])


def test_orbit_term_closed_form():
    """Detectors at rest; for each template, SFTs at the times where Omega t - 2 pi phi_b is
    0, pi/2, pi, 3 pi/2 (+ whole orbits), counted from an observation start t0 != 0."""
    bank = _bank(n_div=(1, 1, 1, 2, 2, 3), n_per_box=4)
    lam = oracle.binary_templates(bank)
    t0, T, k_lo = 5.0e5, 1800.0, 180_000 - 60
    for i in range(bank.n_templates):
        f0, _, _, ap, om, pb = lam[i]
        theta = np.array([0.0, 0.5, 1.0, 1.5, 2.0, 2.5, 3.0, 3.5]) * math.pi + 2 * math.pi * 7
        t_rel = (theta + 2 * math.pi * pb) / om
        sf = ftsynth.SFTSet(power=np.ones((len(t_rel), 10)), t_mid=t0 + t_rel,
                            v=np.zeros((len(t_rel), 3)), s_n=np.ones(len(t_rel)), n_sft=[len(t_rel)],
                            k_lo=k_lo, t_sft=T, t0=t0)
        b, dist = oracle.binary_bins(sf, bank, [i], with_dist=True)
        F = f0 * T
        want = F * (1.0 - ap * om * np.round(np.cos(theta))) - k_lo
        kb = np.floor(want + 0.5)
        d = np.minimum(want - (kb - 0.5), kb + 0.5 - want)
        ok = d > 1e-6
        assert np.array_equal(b[0][ok], kb[ok].astype(np.int64)), i
        assert np.all(np.abs(dist[0] - d) < 1e-6)


def test_doppler_term_closed_form():
    """An isolated source (a_p = 0) at n = x (alpha = 0, sin(delta) = 0), n = y (alpha = 1/4
    turn) and n = z (sin(delta) = 1): the track is f0 T_SFT (1 + v.n)."""
    sfts = _sfts(n_sft=(40, 30), moving=True, t0=1234.5)
    for axis, (alpha, sind) in enumerate([(0.0, 0.0), (0.25, 0.0), (0.0, 1.0)]):
        bank = _bank(n_div=(2, 1, 1, 1, 1, 1), n_per_box=5, ap=(0.0, 0.0), alpha=(alpha, alpha),
                     sind=(sind, sind))
        lam = oracle.binary_templates(bank)
        b, dist = oracle.binary_bins(sfts, bank, np.arange(bank.n_templates), with_dist=True)
        for i in range(bank.n_templates):
            X = lam[i, 0] * sfts.t_sft * (1.0 + sfts.v[:, axis]) - sfts.k_lo
            kb = np.floor(X + 0.5)
            ok = np.abs(X - kb - 0.5) > 1e-6
            ok &= np.abs(X - kb + 0.5) > 1e-6
            assert np.array_equal(b[i][ok], kb[ok].astype(np.int64)), (axis, i)
        # the Doppler really moves the track (about +-10 bins over the year at 100 Hz)
        assert np.ptp(b) > 10


def test_zero_doppler_isolated_limit():
    bank = _bank(n_per_box=30, ap=(0.0, 0.0))
    sfts = _sfts(moving=False)
    lam = oracle.binary_templates(bank)
    b = oracle.binary_bins(sfts, bank, np.arange(bank.n_templates))
    F = lam[:, 0] * sfts.t_sft
    want = np.floor(F + 0.5).astype(np.int64) - sfts.k_lo
    frac = F - np.floor(F)
    ok = np.abs(frac - 0.5) > 1e-6
    assert np.all(b[ok] == want[ok, None])
    assert np.all(b == b[:, :1])


def _mp_position(lam, v, t_mid, t0, t_sft, k_lo):
    """Eq. (track) times T_SFT minus k_lo at 40 significant digits from the FP64 inputs."""
    with mpmath.workdps(40):
        f0, al, sd, ap, om, pb = (mpmath.mpf(float(x)) for x in lam)
        cd = mpmath.sqrt(1 - sd * sd)
        n = (cd * mpmath.cos(2 * mpmath.pi * al), cd * mpmath.sin(2 * mpmath.pi * al), sd)
        vn = sum(mpmath.mpf(float(v[i])) * n[i] for i in range(3))
        t = mpmath.mpf(float(t_mid)) - mpmath.mpf(float(t0))
        f = f0 * (1 + vn - ap * om * mpmath.cos(om * t - 2 * mpmath.pi * pb))
        X = f * mpmath.mpf(float(t_sft)) - int(k_lo)
        k = mpmath.floor(X + mpmath.mpf(1) / 2)
        d = min(X - (k - mpmath.mpf(1) / 2), (k + mpmath.mpf(1) / 2) - X)
        return int(k), float(d)


def test_bins_equal_high_precision_track():
    bank = _bank(n_per_box=25, f0=(100.0, 100.125))
    sfts = _sfts(t0=321.0)
    g = np.random.default_rng(5)
    tmpl = g.choice(bank.n_templates, 60, replace=False)
    b, dist = oracle.binary_bins(sfts, bank, tmpl, with_dist=True)
    lam = oracle.binary_templates(bank, tmpl)
    checked = 0
    for r, i in enumerate(tmpl):
        for a in g.choice(sfts.n_total, 40, replace=False):
            k, d = _mp_position(lam[r], sfts.v[a], sfts.t_mid[a], sfts.t0, sfts.t_sft, sfts.k_lo)
            assert abs(dist[r, a] - d) < 1e-9, (i, a)
            if d > 1e-9:
                assert b[r, a] == k, (i, a)
                checked += 1
    assert checked > 2000
    # the orbit really moves the track: several bins of spread within each template
    assert np.median(b.max(axis=1) - b.min(axis=1)) > 20


def test_statistic_brute_force_and_noise_free_track():
    bank = _bank(n_div=(1, 1, 1, 1, 1, 2), n_per_box=6)
    sfts = _sfts(W=200)
    w = np.random.default_rng(4).uniform(0.5, 1.5, sfts.n_total)
    t = np.arange(bank.n_templates)
    s, oob = oracle.binary_statistic(sfts, bank, w=w)
    b = oracle.binary_bins(sfts, bank, t)
    W = sfts.power.shape[1]
    for i in t:
        acc, out = 0.0, 0
        for a in range(sfts.n_total):
            k = b[i, a]
            if 0 <= k < W:
                acc += w[a] * sfts.power[a, k]
            else:
                out += 1
        assert s[i] == acc and oob[i] == out
    # unit power on the track of template 3 only: it recovers every SFT, exactly
    P = np.zeros_like(sfts.power)
    assert np.all((b[3] >= 0) & (b[3] < W))
    P[np.arange(sfts.n_total), b[3]] = 1.0
    sx = ftsynth.SFTSet(**{**sfts.__dict__, "power": P})
    s3, o3 = oracle.binary_statistic(sx, bank, [3])
    assert o3[0] == 0 and s3[0] == sfts.n_total


def test_topk_per_box():
    bank = _bank(n_div=(1, 1, 1, 1, 1, 3), n_per_box=10)
    s = np.random.default_rng(8).permutation(bank.n_templates).astype(np.float64)
    idx, val = oracle.topk_per_box(s, bank.n_per_box, bank.n_boxes, 3)
    for b in range(bank.n_boxes):
        seg = s[b * 10:(b + 1) * 10]
        order = np.argsort(-seg)[:3]
        assert np.array_equal(idx[b], b * 10 + order)
        assert np.array_equal(val[b], seg[order])
    idx, val = oracle.topk_per_box(s, bank.n_per_box, bank.n_boxes, 12)
    assert np.all(idx[:, 10:] == -1) and np.all(val[:, 10:] == -np.inf)


def test_all_sky_weighted_statistic():
    """Sec. II.B weights on the binary bank: with one detector tensor and one S_n for every
    SFT the weights are 1/N (s = the plain sum / N, sigma_G = 2 / sqrt(N)); in general s is
    the sum along the track's bins with the normalised weights of the template's sky
    direction (sky_weights of its unit vector)."""
    bank = _bank(n_div=(1, 1, 1, 1, 2, 2), n_per_box=4)
    sfts = _sfts(n_sft=(40, 33))
    N = sfts.n_total
    D1 = np.tile(ftsynth.detector_tensor(np.array([5000.0]), 0), (N, 1))
    s_sky, sig, oob = oracle.binary_statistic_sky(sfts, bank, D1)
    s_plain, oob2 = oracle.binary_statistic(sfts, bank)
    assert np.array_equal(oob, oob2)
    assert np.allclose(s_sky, s_plain / N, rtol=1e-12, atol=0)
    assert np.allclose(sig, 2 / math.sqrt(N), rtol=1e-12, atol=0)
    g = np.random.default_rng(9)
    sx = ftsynth.SFTSet(**{**sfts.__dict__, "s_n": g.uniform(0.5, 2.0, N)})
    D = np.concatenate([ftsynth.detector_tensor(sx.t_mid[:40], 0), ftsynth.detector_tensor(sx.t_mid[40:], 1)])
    s_sky, sig, _ = oracle.binary_statistic_sky(sx, bank, D)
    lam = oracle.binary_templates(bank)
    b = oracle.binary_bins(sx, bank, np.arange(bank.n_templates))
    W = sx.power.shape[1]
    for i in range(bank.n_templates):
        cd = math.sqrt(1 - lam[i, 2] ** 2)
        n = np.array([[cd * math.cos(2 * math.pi * lam[i, 1]), cd * math.sin(2 * math.pi * lam[i, 1]),
                       lam[i, 2]]])
        w = oracle.sky_weights(D, sx.s_n, n)[0]
        ok = (b[i] >= 0) & (b[i] < W)
        want = np.sum(w[ok] * sx.power[np.arange(N)[ok], b[i][ok]])
        assert abs(s_sky[i] - want) <= 1e-12 * want
        assert abs(sig[i] - 2 * math.sqrt(np.sum(w * w))) <= 1e-12 * sig[i]
