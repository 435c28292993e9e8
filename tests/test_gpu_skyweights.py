"""All-sky weights on the GPU (Sec. II.B): w_alpha(n) = r_alpha(n) / sum r(n) with
r = (a^2 + b^2) / S_n, computed per (SFT, sky point) inside the evaluation kernels, against
the oracle's statistic with its own FP64 weights:

* unchecked (grouped sky points, ragged groups) and checked kernels, FP32 and FP16 storage;
* s per template within the FP32 tolerance, z with each sky point's own mu_G and sigma_G;
* the candidate sets of the per-band top-k, and of the persistent batch;
* turning the weights off again gives the per-SFT-weighted results back; a bank made before
  the weights were set is refused.
"""
import numpy as np
import pytest

import ftsynth
import oracle
import paper_2411_18370_b300 as ft
from tests import helpers as H
from tests.test_gpu_parity import assert_topk

pytestmark = pytest.mark.gpu

REL = 1e-6


@pytest.fixture(scope="module")
def ctx():
    c = ft.create(0)
    yield c
    c.close()


def _det_tensor(sfts):
    parts, off = [], 0
    for X, n in enumerate(sfts.n_sft):
        parts.append(ftsynth.detector_tensor(sfts.t_mid[off:off + n], X))
        off += n
    return np.concatenate(parts)


def _two_detector_band(n_sft=(50, 41), W=140, n_f0=60, n_f1=5, n_sky=7, sub=11, wings=40, seed=21):
    g = np.random.default_rng(seed)
    k_band = 250_000
    t_mid, v = [], []
    for X, n in enumerate(n_sft):
        t = np.sort(g.uniform(0, 2.5e7, n)) + 900
        t_mid.append(t)
        v.append(ftsynth.detector_velocity(t, X))
    t_mid = np.concatenate(t_mid)
    v = np.concatenate(v)
    N = len(t_mid)
    s_n = g.uniform(0.5, 2.0, N)
    P = g.exponential(2.0, (N, W))
    sfts = ftsynth.SFTSet(power=P, t_mid=t_mid, v=v, s_n=s_n, n_sft=list(n_sft),
                          k_lo=k_band - wings, t_sft=1800.0, t0=0.0)
    bank = ftsynth.Bank(k0=k_band, n_f0=n_f0, f1=np.linspace(-3e-10, 0, n_f1),
                        sky=ftsynth.fibonacci_sky(n_sky), subband_bins=sub)
    return sfts, bank


def _as_stored(sfts, dtype):
    if dtype == "f32":
        return sfts
    P = sfts.power.astype(np.float16).astype(np.float64)
    return ftsynth.SFTSet(power=P, t_mid=sfts.t_mid, v=sfts.v, s_n=sfts.s_n, n_sft=sfts.n_sft,
                          k_lo=sfts.k_lo, t_sft=sfts.t_sft, t0=sfts.t0)


def _check_against_oracle(ctx, sfts, bank, dtype, expect_safe):
    D = _det_tensor(sfts)
    band = H.band_from(ctx, sfts, dtype=dtype)
    ft.band_set_sky_weights(band, D)
    bk = H.bank_from(ctx, band, bank)
    assert bk.window_safe == expect_safe
    s, z, o = H.eval_host(ctx, band, bk, bank.n_templates)
    ref = _as_stored(sfts, dtype)
    wsky = oracle.sky_weights(D, sfts.s_n, bank.sky)
    s_or, o_or = oracle.statistic(ref, bank, wsky=wsky)
    assert np.array_equal(o, o_or)
    err = np.abs(s.astype(np.float64) - s_or)
    assert np.all(err <= REL * np.abs(s_or)), f"worst rel {np.max(err / np.abs(s_or))}"
    mu, sig = oracle.mu_sigma_sky(wsky)
    i_sky = np.arange(bank.n_templates) // (bank.n_f1 * bank.n_f0)
    z_or = (s_or - mu[i_sky]) / sig[i_sky]
    assert np.all(np.abs(z.astype(np.float64) - z_or) <= REL * np.abs(s_or) / sig[i_sky] + 1e-6)
    for k in (1, 6):
        idx, val, zc = H.topk_host(ctx, band, bk, bank.n_subbands, k)
        assert_topk(idx, val, s_or, bank, k, s_gpu=s)
        ok = idx >= 0
        assert np.array_equal(zc[ok], z[idx[ok]])
    return band, bk, s


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_unchecked_kernel_grouped_sky(ctx, dtype):
    sfts, bank = _two_detector_band()
    _check_against_oracle(ctx, sfts, bank, dtype, expect_safe=True)


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_checked_kernel_narrow_wings(ctx, dtype):
    sfts, bank = _two_detector_band(W=64, n_f0=60, wings=2, n_sky=5, seed=22)
    _check_against_oracle(ctx, sfts, bank, dtype, expect_safe=False)


def test_weights_off_again_and_stale_bank_refused(ctx):
    sfts, bank = _two_detector_band(n_sky=4, seed=23)
    w = np.random.default_rng(5).uniform(0.5, 2.0, sfts.n_total)
    band = H.band_from(ctx, sfts, w=w)
    stale = H.bank_from(ctx, band, bank)
    ft.band_set_sky_weights(band, _det_tensor(sfts))
    with pytest.raises(ft.FtError):
        H.eval_host(ctx, band, stale, bank.n_templates)
    ft.band_set_sky_weights(band, None)
    s, _, _ = H.eval_host(ctx, band, stale, bank.n_templates)
    s_or, _ = oracle.statistic(sfts, bank, w=w.astype(np.float32).astype(np.float64))
    assert np.all(np.abs(s - s_or) <= REL * np.abs(s_or))


def test_band_without_psd_refused(ctx):
    sfts, bank = _two_detector_band(n_sky=2, seed=24)
    band = ft.load_sfts(ctx, sfts.power, sfts.t_mid, sfts.v, sfts.n_sft, sfts.k_lo, sfts.t_sft,
                        sfts.t0)
    with pytest.raises(ft.FtError):
        ft.band_set_sky_weights(band, _det_tensor(sfts))


def test_batch_with_sky_weights(ctx):
    data = ftsynth.batch_workload(n_bands=64, n_slots=1200, max_sky=40, bands=[3, 30, 60])
    K = 8
    bands, banks = [], []
    for sfts, bank in data:
        band = H.band_from(ctx, sfts, dtype="f16")
        ft.band_set_sky_weights(band, _det_tensor(sfts))
        bands.append(band)
        banks.append(H.bank_from(ctx, band, bank))
    n_sub = sum(b.n_subbands for b in banks)
    out = np.zeros((n_sub, K), dtype=ft.CANDIDATE_DTYPE)
    ft.Batch(ctx, bands, banks, K).run(out)
    ctx.check_status()
    off = 0
    for (sfts, bank), band, bk in zip(data, bands, banks):
        got = out[off:off + bk.n_subbands]
        off += bk.n_subbands
        single = np.zeros((bk.n_subbands, K), dtype=ft.CANDIDATE_DTYPE)
        ft.topk_per_band(ctx, band, bk, K, single)
        assert np.array_equal(got["template_idx"], single["template_idx"])
        assert np.array_equal(got["s"], single["s"])
        wsky = oracle.sky_weights(_det_tensor(sfts), sfts.s_n, bank.sky)
        s_or, _ = oracle.statistic(_as_stored(sfts, "f16"), bank, wsky=wsky)
        assert_topk(got["template_idx"], got["s"], s_or, bank, K)
