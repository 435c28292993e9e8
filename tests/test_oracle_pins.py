"""Pins of the CPU oracle against what arXiv 2411.18370 and plain mathematics fix.

None of these re-types the oracle's own formula: bins are checked against exact rational
arithmetic (tests/exact.py) and against closed forms of special cases; the statistic
against exact distributions (chi^2, Gamma, non-central chi^2) and against hand-placed
noise-free power; the candidate reduction against brute force with Python's sort.
"""
import math
from fractions import Fraction as F

import numpy as np
import pytest
import scipy.stats as st

import ftsynth
import oracle
from tests import exact


def _tiny_problem(n_sft=40, W=64, v_scale=1.0, f1=(0.0,), sky=None, k_band=360000, n_f0=16,
                  wing=24, seed=5, t_span=3e7):
    """A small hand-made problem (1 detector) with random times/velocities."""
    g = np.random.default_rng(seed)
    t_mid = np.sort(g.uniform(0, t_span, n_sft)) + 900.0
    v = ftsynth.detector_velocity(t_mid, 0) * v_scale
    P = g.exponential(2.0, (n_sft, W))
    sfts = ftsynth.SFTSet(power=P, t_mid=t_mid, v=v, s_n=np.ones(n_sft), n_sft=[n_sft],
                          k_lo=k_band - wing, t_sft=1800.0, t0=0.0)
    bank = ftsynth.Bank(k0=k_band, n_f0=n_f0, f1=np.array(f1, float),
                        sky=ftsynth.fibonacci_sky(8) if sky is None else np.asarray(sky, float),
                        subband_bins=4)
    return sfts, bank


# ----------------------------------------------------------------------------- inputs


def test_generator_noise_is_chi2_2():
    """Sec. II.B.1: Re, Im ~ N(0, sqrt S_n) each => P = |x|^2/S_n ~ chi^2_2 (mean 2, var 4)."""
    g = ftsynth.rng(99, 1)
    s_n = g.uniform(0.8, 1.2, 4000)
    P = ftsynth.power_of(ftsynth.complex_noise(4000, 64, s_n, g), s_n).ravel()
    n = P.size
    assert abs(P.mean() - 2.0) < 5 * 2.0 / math.sqrt(n)
    assert abs(P.var() - 4.0) < 5 * math.sqrt(80.0 / n)  # Var(s^2-ish) bound for Exp(2)
    for x in (1.0, 3.2, 6.0):
        assert abs((P > x).mean() - math.exp(-x / 2)) < 5 * math.sqrt(0.25 / n)


# ----------------------------------------------------------------------------- track bins


def test_zero_doppler_fixed_bins():
    """Eq. (track) with v = 0 and f1 = 0: f(t) = f0, so k = K0 + j - k_lo for every SFT."""
    sfts, bank = _tiny_problem(v_scale=0.0, f1=(0.0,))
    t = np.arange(bank.n_templates)
    b, bf, _ = oracle.bins(sfts, bank, t, with_fp64=True)
    want = (bank.k0 + t % bank.n_f0 - sfts.k_lo)[:, None]
    assert np.array_equal(b, np.broadcast_to(want, b.shape))
    assert np.array_equal(bf, b)


def test_zero_doppler_spindown_closed_form():
    """v = 0, f1 != 0: k = K0 + j - k_lo + round_half_up(f1 (t - t0) T_SFT), by hand."""
    f1s = (-1e-9, -3.3e-10, 2.7e-10)
    sfts, bank = _tiny_problem(v_scale=0.0, f1=f1s)
    t = np.arange(bank.n_templates)
    b = oracle.bins(sfts, bank, t)
    isky, if1, j = bank.split(t)
    for row in range(0, len(t), 7):
        f1 = f1s[if1[row]]
        for a in range(sfts.n_total):
            drift = F(f1) * (F(sfts.t_mid[a]) - F(sfts.t0)) * F(sfts.t_sft)
            want = bank.k0 + j[row] - sfts.k_lo + math.floor(drift + F(1, 2))
            assert b[row, a] == want


def test_f0_neighbours_one_bin_apart():
    """App. A: delta f0 = 1/T_SFT; with v = 0, f1 = 0 neighbouring f0 differ by one bin."""
    sfts, bank = _tiny_problem(v_scale=0.0)
    b = oracle.bins(sfts, bank, np.arange(bank.n_f0))
    assert np.all(np.diff(b, axis=0) == 1)


def test_q32_bins_equal_exact_rational():
    """The canonical Q32 bin equals the exact real-valued round-half-up of Eq. (track)
    except where the exact position lies within 1e-6 bin of a half-integer."""
    sfts, bank = _tiny_problem(f1=(-1e-9, -4e-10, 0.0), n_sft=30)
    g = np.random.default_rng(1)
    tmpl = g.choice(bank.n_templates, 60, replace=False)
    b, bf, _ = oracle.bins(sfts, bank, tmpl, with_fp64=True)
    isky, if1, j = bank.split(tmpl)
    n_near = 0
    for r in range(len(tmpl)):
        for a in range(sfts.n_total):
            x = exact.position(bank.k0, sfts.k_lo, j[r], bank.f1[if1[r]], sfts.t_mid[a], sfts.t0,
                               sfts.t_sft, sfts.v[a], bank.sky[isky[r]])
            k, d = exact.bin_and_tie_distance(x)
            if d < 1e-6:
                n_near += 1
                continue
            assert b[r, a] == k, (r, a)
            assert bf[r, a] == k, (r, a)
    assert n_near <= 2


def test_q32_bins_large_spindown_exact_rational():
    """Same as above with |f1 (t - t0) T_SFT| up to ~500 bins, so the f1 tau eps cross term
    of Eq. (track) (up to ~0.05 bin) decides many roundings."""
    sfts, bank = _tiny_problem(f1=(-1e-8, -6e-9, 4e-9), n_sft=40, seed=11)
    g = np.random.default_rng(12)
    tmpl = g.choice(bank.n_templates, 80, replace=False)
    b = oracle.bins(sfts, bank, tmpl)
    isky, if1, j = bank.split(tmpl)
    for r in range(len(tmpl)):
        for a in range(sfts.n_total):
            x = exact.position(bank.k0, sfts.k_lo, j[r], bank.f1[if1[r]], sfts.t_mid[a], sfts.t0,
                               sfts.t_sft, sfts.v[a], bank.sky[isky[r]])
            k, d = exact.bin_and_tie_distance(x)
            if d > 1e-6:
                assert b[r, a] == k, (r, a)


def test_q32_bins_tiny_workload_full_exact():
    """All 207,360 (template, SFT) pairs of the tiny workload: Q32 == exact rational."""
    sfts, bank, _ = ftsynth.tiny_workload("literal")
    t = np.arange(bank.n_templates)
    b, bf, d = oracle.bins(sfts, bank, t, with_fp64=True)
    # the direct FP64 form agrees everywhere it is not within 1e-7 of a tie
    assert np.all((b == bf) | (np.abs(d) < 1e-7))
    isky, if1, j = bank.split(t)
    g = np.random.default_rng(2)
    for r in g.choice(len(t), 40, replace=False):
        for a in range(sfts.n_total):
            x = exact.position(bank.k0, sfts.k_lo, j[r], bank.f1[if1[r]], sfts.t_mid[a], sfts.t0,
                               sfts.t_sft, sfts.v[a], bank.sky[isky[r]])
            k, dd = exact.bin_and_tie_distance(x)
            if dd > 1e-7:
                assert b[r, a] == k


def test_doppler_direction_and_size():
    """Eq. (track): a source along +v is blue-shifted by (K0+j)|v| bins, along -v red-shifted."""
    sfts, bank = _tiny_problem(n_sft=12, v_scale=1.0, f1=(0.0,))
    for a in range(sfts.n_total):
        v = sfts.v[a]
        u = v / np.linalg.norm(v)
        for sgn in (+1, -1):
            one = ftsynth.Bank(k0=bank.k0, n_f0=bank.n_f0, f1=np.zeros(1), sky=(sgn * u)[None, :],
                               subband_bins=4)
            row = ftsynth.SFTSet(power=sfts.power[a:a + 1], t_mid=sfts.t_mid[a:a + 1],
                                 v=sfts.v[a:a + 1], s_n=np.ones(1), n_sft=[1], k_lo=sfts.k_lo,
                                 t_sft=1800.0, t0=0.0)
            b = oracle.bins(row, one, np.arange(one.n_f0))[:, 0]
            for jj in range(one.n_f0):
                shift = sgn * (bank.k0 + jj) * np.linalg.norm(v)
                want = bank.k0 + jj - sfts.k_lo + math.floor(shift + 0.5)
                assert b[jj] == want


# ----------------------------------------------------------------------------- statistic


def test_noise_free_injection_recovers_summed_power():
    """Eq. (short_coh_general): with P = 4 on the injected track (placed by exact rational
    arithmetic) and 0 elsewhere, s(lambda_inj) = 4 * N_SFT exactly and no template exceeds it."""
    sfts, bank, inj = ftsynth.tiny_workload("auto")
    P = np.zeros_like(sfts.power)
    n = bank.sky[inj["i_sky"]]
    f1 = bank.f1[inj["i_f1"]]
    for a in range(sfts.n_total):
        x = exact.position(bank.k0, sfts.k_lo, inj["j"], f1, sfts.t_mid[a], sfts.t0, sfts.t_sft,
                           sfts.v[a], n)
        k, d = exact.bin_and_tie_distance(x)
        assert d > 1e-6
        P[a, k] = 4.0
    sfts.power = P
    s, oob = oracle.statistic(sfts, bank)
    t_inj = (inj["i_sky"] * bank.n_f1 + inj["i_f1"]) * bank.n_f0 + inj["j"]
    assert s[t_inj] == 4.0 * sfts.n_total == 192.0
    assert s.max() == 192.0 and oob.sum() == 0


def test_noise_statistic_is_gamma():
    """Sec. II.B.1: with w = 1, s is a sum of N_SFT independent chi^2_2 = Gamma(N, 2);
    mean 2N, variance 4N.  Zero-Doppler templates at distinct f0 read disjoint bins."""
    N, W = 100, 3000
    g = ftsynth.rng(98, 1)
    sfts, _ = _tiny_problem(n_sft=N, W=W, v_scale=0.0, wing=0)
    sfts.power = ftsynth.power_of(ftsynth.complex_noise(N, W, np.ones(N), g), np.ones(N))
    bank = ftsynth.Bank(k0=sfts.k_lo, n_f0=W, f1=np.zeros(1), sky=ftsynth.fibonacci_sky(1),
                        subband_bins=W)
    s, _ = oracle.statistic(sfts, bank)
    assert abs(s.mean() - 2 * N) < 5 * math.sqrt(4 * N / W)
    assert abs(s.var() / (4 * N) - 1) < 0.15
    assert st.kstest(s, st.gamma(a=N, scale=2.0).cdf).pvalue > 1e-3
    z = oracle.zscore(s, N)
    assert abs(z.mean()) < 0.1 and abs(z.std() - 1) < 0.08


def test_signal_statistic_is_noncentral_chi2():
    """Sec. II.B.2: a deterministic amplitude h in the track bin makes each P non-central
    chi^2_2(rho^2) with rho^2 = |h|^2 / S_n; s ~ chi^2_{2N}(N rho^2), mean 2N + N rho^2."""
    N, W = 60, 2000
    g = ftsynth.rng(98, 2)
    s_n = np.full(N, 1.5)
    x = ftsynth.complex_noise(N, W, s_n, g)
    h = 0.9 * np.exp(1j * g.uniform(0, 2 * np.pi, (N, W)))
    rho2 = 0.81 / 1.5
    sfts, _ = _tiny_problem(n_sft=N, W=W, v_scale=0.0, wing=0)
    sfts.power = ftsynth.power_of(x + h, s_n)
    bank = ftsynth.Bank(k0=sfts.k_lo, n_f0=W, f1=np.zeros(1), sky=ftsynth.fibonacci_sky(1),
                        subband_bins=W)
    s, _ = oracle.statistic(sfts, bank)
    assert abs(s.mean() - (2 * N + N * rho2)) < 5 * math.sqrt((4 * N + 4 * N * rho2) / W)
    assert st.kstest(s, st.ncx2(df=2 * N, nc=N * rho2).cdf).pvalue > 1e-3


def test_weights_scale_and_z_invariance():
    """Weights are defined up to a constant (Sec. II.B, normalisation sum w = 1):
    s(c w) = c s(w) and z(c w) = z(w); mu_G = 2 sum w, sigma_G^2 = 4 sum w^2."""
    sfts, bank = _tiny_problem(n_sft=25)
    w = np.random.default_rng(3).uniform(0.5, 2.0, sfts.n_total)
    s1, _ = oracle.statistic(sfts, bank, w=w)
    s2, _ = oracle.statistic(sfts, bank, w=4.0 * w)
    assert np.array_equal(s2, 4.0 * s1)
    np.testing.assert_allclose(oracle.zscore(s2, sfts.n_total, 4.0 * w),
                               oracle.zscore(s1, sfts.n_total, w), rtol=0, atol=1e-12)
    mu, sig = oracle.mu_sigma(sfts.n_total, w / w.sum())
    assert abs(mu - 2.0) < 1e-12  # normalised weights: mu_G = 2
    assert abs(sig ** 2 - 4 * np.sum((w / w.sum()) ** 2)) < 1e-15


def test_weighted_statistic_bruteforce():
    """s = sum_alpha w_alpha P[alpha][k_alpha] with bins from exact rational arithmetic."""
    sfts, bank = _tiny_problem(n_sft=20, f1=(-1e-8, 4e-9), W=1300, wing=650)
    w = np.random.default_rng(4).uniform(0.5, 2.0, sfts.n_total)
    tmpl = np.arange(0, bank.n_templates, 5)
    s, oob = oracle.statistic(sfts, bank, tmpl, w=w)
    isky, if1, j = bank.split(tmpl)
    for r in range(len(tmpl)):
        acc, nb = 0.0, 0
        for a in range(sfts.n_total):
            x = exact.position(bank.k0, sfts.k_lo, j[r], bank.f1[if1[r]], sfts.t_mid[a], sfts.t0,
                               sfts.t_sft, sfts.v[a], bank.sky[isky[r]])
            k, d = exact.bin_and_tie_distance(x)
            assert d > 1e-7
            if 0 <= k < sfts.n_bins:
                acc += w[a] * sfts.power[a, k]
            else:
                nb += 1
        assert abs(s[r] - acc) <= 1e-12 * abs(acc)
        assert oob[r] == nb


def test_out_of_window_counts_literal_wings(tiny_literal):
    """Tracks leaving the 10-bin literal wings contribute 0 and are counted."""
    sfts, bank, _ = tiny_literal
    s, oob = oracle.statistic(sfts, bank)
    assert oob.sum() > 0
    tmpl = np.nonzero(oob)[0][:12]
    isky, if1, j = bank.split(tmpl)
    for r, t in enumerate(tmpl):
        nb = 0
        for a in range(sfts.n_total):
            x = exact.position(bank.k0, sfts.k_lo, j[r], bank.f1[if1[r]], sfts.t_mid[a], sfts.t0,
                               sfts.t_sft, sfts.v[a], bank.sky[isky[r]])
            k, _ = exact.bin_and_tie_distance(x)
            nb += not (0 <= k < sfts.n_bins)
        assert oob[t] == nb


# ----------------------------------------------------------------------------- candidates


def test_topk_bruteforce_with_ties():
    """Sec. IV.B: the loudest per disjoint box; ties broken by the smaller template index."""
    bank = ftsynth.Bank(k0=0, n_f0=23, f1=np.zeros(3), sky=np.zeros((5, 3)), subband_bins=5)
    g = np.random.default_rng(7)
    s = g.integers(0, 6, bank.n_templates).astype(float)  # many exact ties
    for k in (1, 3, 10, 40):
        idx, val = oracle.topk_per_subband(s, bank, k)
        for b in range(bank.n_subbands):
            members = [t for t in range(bank.n_templates) if (t % bank.n_f0) // 5 == b]
            want = sorted(members, key=lambda t: (-s[t], t))[:k]
            got = [int(t) for t in idx[b] if t >= 0]
            assert got == want
            assert np.array_equal(val[b, : len(want)], s[want])
            assert np.all(idx[b, len(want):] == -1)


def test_topk_is_an_upper_set():
    """Every template outside the selection ranks below the k-th selected one."""
    bank = ftsynth.Bank(k0=0, n_f0=40, f1=np.zeros(2), sky=np.zeros((30, 3)), subband_bins=7)
    s = np.random.default_rng(8).standard_normal(bank.n_templates)
    idx, val = oracle.topk_per_subband(s, bank, 4)
    j = np.arange(bank.n_templates) % bank.n_f0
    for b in range(bank.n_subbands):
        sel = set(idx[b].tolist())
        kth = val[b, -1]
        rest = [t for t in np.nonzero(j // 7 == b)[0] if t not in sel]
        assert all(s[t] <= kth for t in rest)
        assert np.all(np.diff(val[b]) <= 0)
