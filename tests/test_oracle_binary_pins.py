"""Pins of the oracle's binary-orbit track (Eq. (track)) and random hyperbox bank
(Eq. (xi_of_lambda), App. A Eq. (unif_transform), Sec. IV.B):

* the canonical cosine of a 32-bit phase (linear interpolation in a full-turn table of 1024
  intervals) is within the interpolation bound (2 pi/1024)^2 / 8 = 4.7e-6 plus FP32 rounding
  of libm's cos, and exact at the table's nodes;
* every template lies in its own box and is uniform in the uniform coordinates
  xi = {f0^6, alpha, sin(delta), a_p^3, Omega^4, phi_b} there (mean 1/2, variance 1/12 of the
  position within the box along each axis);
* the fixed-point orbit phase equals (Omega t - phi_b) / 2 pi mod 1 to 1e-8 turns;
* the canonical FP32 bin equals the FP64 bin of Eq. (track) (libm cos) wherever the track is
  more than 5e-4 bins from the rounding boundary, and such cases are rare (the cosine's
  error, under 4.9e-6, times the orbit amplitude, under 28 bins here, and times F (|v_x| +
  |v_y|) in the sky vector, under 27 bins, plus FP32 rounding: about 2.8e-4 at most);
* with a_p = 0 and no detector motion the bin is round(f0 T_SFT) (zero-Doppler tracks collapse
  to fixed bins);
* the statistic equals a Python sum over SFTs along the canonical bins, and a noise-free track
  of unit power recovers N_SFT;
* the per-box selection returns each box's loudest templates.
"""
import math

import numpy as np

import ftsynth
import oracle

DAY = 86400.0


def _bank(n_div=(2, 2, 2, 2, 2, 2), n_per_box=40, seed=11, f0=(100.0, 100.05), ap=(5.0, 15.0)):
    om = (2 * math.pi / (15 * DAY), 2 * math.pi / (7 * DAY))
    return ftsynth.BinaryBank(lo=(f0[0], 0.0, -1.0, ap[0], om[0], 0.0),
                              hi=(f0[1], 1.0, 1.0, ap[1], om[1], 1.0),
                              n_div=n_div, n_per_box=n_per_box, seed=seed)


def _sfts(n_sft=(70, 60), W=200, wings=55, seed=3, k_band=180_000, moving=True):
    g = np.random.default_rng(seed)
    t_mid, v = [], []
    for X, n in enumerate(n_sft):
        t = np.sort(g.uniform(0, ftsynth.YEAR_S, n)) + 900
        t_mid.append(t)
        v.append(ftsynth.detector_velocity(t, X) if moving else np.zeros((n, 3)))
    t_mid = np.concatenate(t_mid)
    N = len(t_mid)
    return ftsynth.SFTSet(power=g.exponential(2.0, (N, W)), t_mid=t_mid, v=np.concatenate(v),
                          s_n=np.ones(N), n_sft=list(n_sft), k_lo=k_band - wings, t_sft=1800.0,
                          t0=0.0)


def test_canonical_cosine():
    g = np.random.default_rng(1)
    th = np.concatenate([g.integers(0, 2 ** 32, 20000, dtype=np.uint64),
                         np.array([0, 1 << 29, (1 << 29) - 1, 1 << 30, 1 << 31, 3 << 30, 2 ** 32 - 1],
                                  np.uint64)])
    c = oracle.cos_q32(th).astype(np.float64)
    ref = np.cos(2 * np.pi * th.astype(np.float64) / 2 ** 32)
    bound = (2 * np.pi / 1024) ** 2 / 8 + 1.2e-7
    assert np.max(np.abs(c - ref)) < bound
    s = oracle.cos_q32((th - (1 << 30)) % 2 ** 32).astype(np.float64)
    assert np.max(np.abs(s - np.sin(2 * np.pi * th.astype(np.float64) / 2 ** 32))) < bound
    assert oracle.cos_q32([0])[0] == 1.0
    # nodes: the FP32 rounding of cos at multiples of 2 pi / 1024, exactly
    nodes = np.arange(0, 1024, dtype=np.uint64) << np.uint64(22)
    want = np.cos(np.arange(1024) * (2 * np.pi / 1024)).astype(np.float32)
    got = oracle.cos_q32(nodes)
    assert np.max(np.abs(got.astype(np.float64) - want.astype(np.float64))) < 1.2e-7


def _xi(lam):
    return np.column_stack([lam[:, 0] ** 6, lam[:, 1], lam[:, 2], lam[:, 3] ** 3, lam[:, 4] ** 4,
                            lam[:, 5]])


def test_templates_fill_their_boxes_uniformly():
    bank = _bank(n_per_box=200)
    lam, _ = oracle.binary_templates(bank)
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
    lam2, _ = oracle.binary_templates(bank)
    assert np.array_equal(lam, lam2)
    lam3, _ = oracle.binary_templates(ftsynth.BinaryBank(**{**bank.__dict__, "seed": 12}))
    assert not np.any(lam3[:, 0] == lam[:, 0])


def test_orbit_phase_fixed_point():
    bank = _bank(n_per_box=10)
    sfts = _sfts()
    lam, der = oracle.binary_templates(bank, None, sfts.t_sft, sfts.k_lo)
    tq = oracle.binary_tq(sfts.t_mid, sfts.t0).astype(np.uint64)
    for i in range(0, bank.n_templates, 37):
        ph = (der["nu_q"][i] * tq - der["psi_q"][i]).astype(np.float64) / 2 ** 64
        want = ((lam[i, 4] * (sfts.t_mid - sfts.t0) - 2 * np.pi * lam[i, 5]) / (2 * np.pi)) % 1.0
        d = np.abs(ph - want)
        assert np.all(np.minimum(d, 1 - d) < 1e-8)


def test_canonical_bins_match_the_fp64_track():
    bank = _bank(n_per_box=25)
    sfts = _sfts()
    b, b64, dist = oracle.binary_bins(sfts, bank, np.arange(bank.n_templates), with_fp64=True)
    differ = b != b64
    assert np.all(dist[differ] < 5e-4)
    assert differ.mean() < 1e-3
    # the orbit really moves the track: several bins of spread within each template
    assert np.median(b.max(axis=1) - b.min(axis=1)) > 20


def test_zero_doppler_isolated_limit():
    bank = _bank(n_per_box=30, ap=(0.0, 0.0))
    sfts = _sfts(moving=False)
    lam, _ = oracle.binary_templates(bank, None, sfts.t_sft, sfts.k_lo)
    b = oracle.binary_bins(sfts, bank, np.arange(bank.n_templates))
    F = lam[:, 0] * sfts.t_sft
    want = np.floor(F + 0.5).astype(np.int64) - sfts.k_lo
    frac = F - np.floor(F)
    ok = np.abs(frac - 0.5) > 1e-6
    assert np.all(b[ok] == want[ok, None])
    assert np.all(b == b[:, :1])


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
    # unit power on the FP64 track of template 3 only
    _, b64, dist = oracle.binary_bins(sfts, bank, [3], with_fp64=True)
    P = np.zeros_like(sfts.power)
    P[np.arange(sfts.n_total), b64[0]] = 1.0
    sx = ftsynth.SFTSet(**{**sfts.__dict__, "power": P})
    s3, o3 = oracle.binary_statistic(sx, bank, [3])
    assert o3[0] == 0
    assert s3[0] >= sfts.n_total - np.sum(dist[0] < 5e-4)


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
    the sum along the canonical bins with the normalised weights of the template's sky
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
    lam, _ = oracle.binary_templates(bank)
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
