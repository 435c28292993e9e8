"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Tolerances: the FP32 statistic within 1e-6 relative of the oracle; track bins, out-of-
window counts and candidate sets bit-exact (candidate sets up to the near-tie exemption:
a sub-band whose oracle k-th and (k+1)-th values differ by < 2e-6 relative).  z is
compared with the absolute tolerance that the s tolerance implies, 1e-6 s / sigma_G + 1e-6.
"""
import numpy as np
import pytest

import ftsynth
import oracle
import paper_2411_18370_b300 as ft
from tests import helpers as H

pytestmark = pytest.mark.gpu

REL = 1e-6


@pytest.fixture(scope="module")
def ctx():
    c = ft.create(0)
    yield c
    c.close()


def _with_power(sfts, P):
    return ftsynth.SFTSet(power=P, t_mid=sfts.t_mid, v=sfts.v, s_n=sfts.s_n, n_sft=sfts.n_sft,
                          k_lo=sfts.k_lo, t_sft=sfts.t_sft, t0=sfts.t0)


def _injected_tiny(cfg):
    sfts, bank, inj = cfg
    t_inj = (inj["i_sky"] * bank.n_f1 + inj["i_f1"]) * bank.n_f0 + inj["j"]
    b = oracle.bins(sfts, bank, [t_inj])[0]
    x = H.inject(sfts, b, inj["amp"], inj["phase_seed"])
    return _with_power(sfts, ftsynth.power_of(x, sfts.s_n)), bank, t_inj


def assert_s_close(s_gpu, s_or, rel=REL):
    s_gpu = np.asarray(s_gpu, np.float64)
    err = np.abs(s_gpu - s_or)
    tol = rel * np.maximum(np.abs(s_or), 1.0)
    bad = np.nonzero(err > tol)[0]
    assert bad.size == 0, f"{bad.size} values off; worst rel {np.max(err / np.maximum(np.abs(s_or), 1))}"


def assert_z_close(z_gpu, s_or, n_sft, w=None):
    z_or = oracle.zscore(s_or, n_sft, w)
    _, sig = oracle.mu_sigma(n_sft, w)
    tol = REL * np.abs(s_or) / sig + 1e-6
    assert np.all(np.abs(np.asarray(z_gpu, np.float64) - z_or) <= tol)


def assert_topk(idx, val, s_or, bank, k, s_gpu=None, templates=None, margin=2e-6):
    """Candidate sets equal the oracle's (near-tie exemption: the oracle's k-th and (k+1)-th
    values closer than `margin` relative) and, when the GPU's own values are given, exactly
    the CPU selection over them.  Returns the number of exempt sub-bands."""
    o_idx, o_val = oracle.topk_per_subband(s_or, bank, k + 1, templates)
    exempt = 0
    for b in range(bank.n_subbands):
        got = set(int(t) for t in idx[b] if t >= 0)
        want = set(int(t) for t in o_idx[b, :k] if t >= 0)
        if got == want:
            continue
        kth, nxt = o_val[b, k - 1], o_val[b, k]
        assert np.isfinite(nxt) and abs(kth - nxt) < margin * abs(kth), f"sub-band {b} differs"
        exempt += 1
    if s_gpu is not None:
        c_idx, c_val = oracle.topk_per_subband(np.asarray(s_gpu, np.float64), bank, k, templates)
        assert np.array_equal(idx, c_idx)
        ok = c_idx >= 0
        assert np.array_equal(val[ok].astype(np.float64), c_val[ok])
    return exempt


# ----------------------------------------------------------------------------- tiny workload


def test_tiny_literal_wings_checked_kernel(ctx, tiny_literal):
    """4320 templates x 48 SFTs, 10-bin wings: edge tracks leave the window (checked kernel)."""
    sfts, bank, t_inj = _injected_tiny(tiny_literal)
    band = H.band_from(ctx, sfts)
    bk = H.bank_from(ctx, band, bank)
    assert not bk.window_safe
    s, z, o = H.eval_host(ctx, band, bk, bank.n_templates)
    s_or, o_or = oracle.statistic(sfts, bank)
    assert np.array_equal(o, o_or) and o_or.sum() > 0
    assert_s_close(s, s_or)
    assert_z_close(z, s_or, sfts.n_total)
    for k in (1, 10, 32):
        idx, val, zc = H.topk_host(ctx, band, bk, bank.n_subbands, k)
        assert_topk(idx, val, s_or, bank, k, s_gpu=s)


def test_tiny_auto_wings_fast_kernel_and_injection(ctx, tiny_auto):
    sfts, bank, t_inj = _injected_tiny(tiny_auto)
    band = H.band_from(ctx, sfts)
    bk = H.bank_from(ctx, band, bank)
    assert bk.window_safe
    s, z, o = H.eval_host(ctx, band, bk, bank.n_templates)
    s_or, o_or = oracle.statistic(sfts, bank)
    assert o_or.sum() == 0 and np.all(o == 0)
    assert_s_close(s, s_or)
    assert_z_close(z, s_or, sfts.n_total)
    idx, val, _ = H.topk_host(ctx, band, bk, bank.n_subbands, 10)
    assert_topk(idx, val, s_or, bank, 10, s_gpu=s)
    # the injected template is the loudest of its sub-band
    b = (t_inj % bank.n_f0) // bank.subband_bins
    assert idx[b, 0] == t_inj


def test_noise_free_injection_exact(ctx, tiny_auto):
    """P = 4 on the injected track and 0 elsewhere: s(lambda_inj) = 192 exactly in FP32."""
    sfts, bank, inj = tiny_auto
    t_inj = (inj["i_sky"] * bank.n_f1 + inj["i_f1"]) * bank.n_f0 + inj["j"]
    b = oracle.bins(sfts, bank, [t_inj])[0]
    P = np.zeros_like(sfts.power)
    P[np.arange(sfts.n_total), b] = 4.0
    band = H.band_from(ctx, _with_power(sfts, P))
    bk = H.bank_from(ctx, band, bank)
    s, _, _ = H.eval_host(ctx, band, bk, bank.n_templates)
    assert s[t_inj] == 192.0 and s.max() == 192.0


@pytest.mark.parametrize("wings", ["literal", "auto"])
@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_integer_power_bins_exact(ctx, wings, dtype):
    """Integer powers 0..255 are exact in every storage type and their sums < 2^24 are exact
    in FP32, so s must equal the oracle bit for bit: any wrong bin shows."""
    sfts, bank, _ = ftsynth.tiny_workload(wings)
    g = np.random.default_rng(31)
    P = g.integers(0, 256, sfts.power.shape).astype(np.float64)
    sx = _with_power(sfts, P)
    band = H.band_from(ctx, sx, dtype=dtype)
    bk = H.bank_from(ctx, band, bank)
    s, _, o = H.eval_host(ctx, band, bk, bank.n_templates)
    s_or, o_or = oracle.statistic(sx, bank)
    assert np.array_equal(s.astype(np.float64), s_or)
    assert np.array_equal(o, o_or)


def test_track_bins_tiny_all_pairs(ctx, tiny_literal):
    sfts, bank, _ = tiny_literal
    band = H.band_from(ctx, sfts)
    bk = H.bank_from(ctx, band, bank)
    t = np.arange(bank.n_templates, dtype=np.int64)
    out = np.empty((len(t), sfts.n_total), np.int32)
    ft.track_bins(ctx, band, bk, t, out)
    assert np.array_equal(out.astype(np.int64), oracle.bins(sfts, bank, t))


# ----------------------------------------------------------------------------- search-shaped


@pytest.fixture(scope="module")
def search_slice(search_cfg):
    """Search-shaped data (2 detectors, 1 yr, ~24.4k SFTs) with a 3-sky slice of the bank."""
    sfts, bank = search_cfg
    sub = ftsynth.Bank(k0=bank.k0, n_f0=bank.n_f0, f1=bank.f1, sky=bank.sky[[0, 4321, 9999]],
                       subband_bins=bank.subband_bins)
    s_or, o_or = oracle.statistic(sfts, sub)
    return sfts, sub, s_or, o_or


def test_search_shaped_slice_elementwise(ctx, search_slice):
    sfts, bank, s_or, o_or = search_slice
    band = H.band_from(ctx, sfts, power_f32=True)
    bk = H.bank_from(ctx, band, bank)
    assert bk.window_safe and o_or.sum() == 0
    s, z, o = H.eval_host(ctx, band, bk, bank.n_templates)
    assert_s_close(s, s_or)
    assert_z_close(z, s_or, sfts.n_total)
    idx, val, _ = H.topk_host(ctx, band, bk, bank.n_subbands, 10)
    assert_topk(idx, val, s_or, bank, 10, s_gpu=s)


@pytest.mark.parametrize("dtype,max_rel,rms_rel", [("f16", 2e-5, 5e-6), ("bf16", 1.5e-4, 4e-5)])
def test_search_shaped_reduced_precision_error(ctx, search_slice, dtype, max_rel, rms_rel):
    """FP16/BF16 storage, FP32 accumulation: error against the FP64 oracle within the bound
    set by one rounding per stored value (2^-11, 2^-8), averaged over ~24k SFTs."""
    sfts, bank, s_or, _ = search_slice
    band = H.band_from(ctx, sfts, dtype=dtype)
    bk = H.bank_from(ctx, band, bank)
    s, _, _ = H.eval_host(ctx, band, bk, bank.n_templates)
    rel = np.abs(s.astype(np.float64) - s_or) / s_or
    assert rel.max() < max_rel and np.sqrt(np.mean(rel ** 2)) < rms_rel


@pytest.fixture(scope="module")
def search_subbank(search_cfg):
    """Search-shaped data with every f0 and f1 of the bank and one sky point in 250 (40 sky
    points, 144 000 templates): ten whole sub-bands of 14 400 templates each."""
    sfts, bank = search_cfg
    sub = ftsynth.Bank(k0=bank.k0, n_f0=bank.n_f0, f1=bank.f1, sky=bank.sky[::250],
                       subband_bins=bank.subband_bins)
    s_or, _ = oracle.statistic(sfts, sub)
    return sfts, sub, s_or


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_search_shaped_candidate_sets(ctx, search_subbank, dtype):
    """The precision comparison's candidate sets: the top-10 of every sub-band from FP32,
    FP16 and BF16 storage (FP32 accumulation) equal the FP64 oracle's, except in sub-bands
    whose oracle 10th and 11th values nearly tie.  The margin is twice the storage type's
    6-sigma error of s: one rounding per stored value with unit roundoff u (2^-11 for FP16,
    2^-8 for BF16), independent across SFTs, gives sigma(s)/s = u sqrt(2 / (3 N)) for
    exponential power (E[P^2] = 2 E[P]^2); FP32 keeps the 2e-6 of the FP32 tolerance.  The
    sets also equal the CPU selection over the GPU's own values exactly."""
    import math

    sfts, bank, s_or = search_subbank
    u = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}
    margin = 2 * 6 * u[dtype] * math.sqrt(2.0 / (3.0 * sfts.n_total)) if dtype in u else 2e-6
    band = H.band_from(ctx, sfts, dtype=dtype, power_f32=True)
    bk = H.bank_from(ctx, band, bank)
    s, _, _ = H.eval_host(ctx, band, bk, bank.n_templates, with_z=False, with_oob=False)
    idx, val, _ = H.topk_host(ctx, band, bk, bank.n_subbands, 10)
    exempt = assert_topk(idx, val, s_or, bank, 10, s_gpu=s, margin=margin)
    assert exempt <= 2
    # the statistic itself stays within the same 6-sigma bound per template
    if dtype in u:
        rel = np.abs(s.astype(np.float64) - s_or) / s_or
        assert rel.max() < margin


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_search_shaped_integer_power_exact(ctx, search_slice, dtype):
    """Integer powers on the search-shaped data: every bin of the shifted-row kernel, its
    per-row carry corrections and the 16-bit pair layout must reproduce the oracle's sum
    exactly (sums < 2^24 are exact in FP32)."""
    sfts, bank, _, _ = search_slice
    P = np.random.default_rng(77).integers(0, 256, sfts.power.shape).astype(np.float64)
    sx = _with_power(sfts, P)
    band = H.band_from(ctx, sx, dtype=dtype)
    bk = H.bank_from(ctx, band, bank)
    assert bk.window_safe
    s, _, _ = H.eval_host(ctx, band, bk, bank.n_templates)
    s_or, _ = oracle.statistic(sx, bank)
    assert np.array_equal(s.astype(np.float64), s_or)


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_weighted_integer_power_exact(ctx, tiny_auto, dtype):
    """Power-of-two weights and integer powers: the weighted kernels are exact too."""
    sfts, bank, _ = tiny_auto
    g = np.random.default_rng(78)
    P = g.integers(0, 256, sfts.power.shape).astype(np.float64)
    w = 2.0 ** g.integers(-2, 3, sfts.n_total)
    sx = _with_power(sfts, P)
    band = H.band_from(ctx, sx, dtype=dtype, w=w)
    bk = H.bank_from(ctx, band, bank)
    s, z, _ = H.eval_host(ctx, band, bk, bank.n_templates)
    s_or, _ = oracle.statistic(sx, bank, w=w)
    assert np.array_equal(s.astype(np.float64), s_or)
    assert_z_close(z, s_or, sfts.n_total, w)


def test_track_bins_search_shaped_sample(ctx, search_cfg):
    sfts, bank = search_cfg
    band = H.band_from(ctx, sfts, power_f32=True)
    bk = H.bank_from(ctx, band, bank)
    t = np.random.default_rng(5).choice(bank.n_templates, 64, replace=False).astype(np.int64)
    out = np.empty((len(t), sfts.n_total), np.int32)
    ft.track_bins(ctx, band, bk, t, out)
    assert np.array_equal(out.astype(np.int64), oracle.bins(sfts, bank, t))


def test_search_shaped_full_bank_sampled(ctx, search_cfg):
    """The full 3.6e7-template bank in the launch configuration the benchmark times, with
    device outputs: sampled templates against the oracle; candidates against the CPU
    selection over the GPU's own values, and each candidate's s against the oracle."""
    import torch

    sfts, bank = search_cfg
    band = H.band_from(ctx, sfts, power_f32=True)
    bk = H.bank_from(ctx, band, bank)
    n = bank.n_templates
    s_d = torch.empty(n, dtype=torch.float32, device="cuda")
    z_d = torch.empty(n, dtype=torch.float32, device="cuda")
    ft.eval_statistic(ctx, band, bk, s_d, z_d)
    cand = torch.empty(bank.n_subbands * 10 * 16, dtype=torch.uint8, device="cuda")
    ft.topk_per_band(ctx, band, bk, 10, cand)
    torch.cuda.synchronize()
    ctx.check_status()
    s = s_d.cpu().numpy()
    z = z_d.cpu().numpy()
    idx, val, zc = ft.decode_candidates(cand, bank.n_subbands, 10)
    samp = np.random.default_rng(6).choice(n, 1500, replace=False)
    s_or, _ = oracle.statistic(sfts, bank, samp)
    assert_s_close(s[samp], s_or)
    assert_z_close(z[samp], s_or, sfts.n_total)
    c_idx, c_val = oracle.topk_per_subband(s.astype(np.float64), bank, 10)
    assert np.array_equal(idx, c_idx) and np.array_equal(val.astype(np.float64), c_val)
    flat = idx.ravel()
    s_or_c, _ = oracle.statistic(sfts, bank, flat)
    assert_s_close(val.ravel(), s_or_c)
    assert_z_close(zc.ravel(), s_or_c, sfts.n_total)


# ----------------------------------------------------------------------------- edge cases


def _small(n_sft=37, W=96, n_f0=33, n_f1=3, n_sky=5, sub=7, seed=3, wings=30):
    g = np.random.default_rng(seed)
    k_band = 200_000
    t_mid = np.sort(g.uniform(0, 2e7, n_sft)) + 900
    v = ftsynth.detector_velocity(t_mid, 1)
    P = g.exponential(2.0, (n_sft, W))
    sfts = ftsynth.SFTSet(power=P, t_mid=t_mid, v=v, s_n=np.ones(n_sft), n_sft=[n_sft],
                          k_lo=k_band - wings, t_sft=1800.0, t0=0.0)
    bank = ftsynth.Bank(k0=k_band, n_f0=n_f0, f1=np.linspace(-2e-10, 0, n_f1),
                        sky=ftsynth.fibonacci_sky(n_sky), subband_bins=sub)
    return sfts, bank


@pytest.mark.parametrize("shape", [
    dict(n_sft=1, n_f0=1, n_f1=1, n_sky=1, sub=1),
    dict(n_sft=37, n_f0=33, n_f1=3, n_sky=5, sub=7),
    dict(n_sft=65, n_f0=257, n_f1=33, n_sky=2, sub=18, W=360),
    dict(n_sft=130, n_f0=5, n_f1=40, n_sky=3, sub=100),
    dict(n_sft=9, n_f0=64, n_f1=2, n_sky=4, sub=64, wings=2),
])
def test_edge_shapes(ctx, shape):
    """Ragged f0 tiles, several and ragged f1 groups, one SFT, one template, a sub-band wider
    than the band, k larger than a sub-band's population, windows too narrow."""
    sfts, bank = _small(**shape)
    band = H.band_from(ctx, sfts)
    bk = H.bank_from(ctx, band, bank)
    s, z, o = H.eval_host(ctx, band, bk, bank.n_templates)
    s_or, o_or = oracle.statistic(sfts, bank)
    assert np.array_equal(o, o_or)
    assert_s_close(s, s_or)
    for k in (1, 5, 32):
        idx, val, _ = H.topk_host(ctx, band, bk, bank.n_subbands, k)
        assert_topk(idx, val, s_or, bank, k, s_gpu=s)


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_wide_band_windowed_rows_exact(ctx, dtype):
    """A band ~4x wider than one f0 tile plus the f1 spread: each CTA copies only the
    window of every row that its tracks can reach (two f1 groups, so two windows per
    row), and integer powers keep the comparison with the oracle bit-exact."""
    sfts, bank = _small(n_sft=150, W=1160, n_f0=1000, n_f1=25, n_sky=3, sub=40, wings=40)
    g = np.random.default_rng(77)
    P = g.integers(0, 256, sfts.power.shape).astype(np.float64)
    sx = _with_power(sfts, P)
    # precondition: the window (tile + spread + margin) is under 3/4 of the padded row
    spread = (bank.f1.max() - bank.f1.min()) * (sfts.t_mid.max() + 900.0) * sfts.t_sft
    assert 256 + spread + 72 < 0.75 * 1152
    band = H.band_from(ctx, sx, dtype=dtype)
    bk = H.bank_from(ctx, band, bank)
    assert bk.window_safe
    s, _, o = H.eval_host(ctx, band, bk, bank.n_templates)
    s_or, o_or = oracle.statistic(sx, bank)
    assert np.array_equal(o, o_or) and o_or.sum() == 0
    assert np.array_equal(s.astype(np.float64), s_or)
    idx, val, _ = H.topk_host(ctx, band, bk, bank.n_subbands, 8)
    assert_topk(idx, val, s_or, bank, 8, s_gpu=s)


def test_weighted_statistic(ctx):
    sfts, bank = _small(n_sft=80, n_f0=40, n_f1=4, n_sky=6)
    w = np.random.default_rng(9).uniform(0.2, 3.0, sfts.n_total)
    band = H.band_from(ctx, sfts, w=w)
    bk = H.bank_from(ctx, band, bank)
    s, z, _ = H.eval_host(ctx, band, bk, bank.n_templates)
    w32 = w.astype(np.float32).astype(np.float64)  # the ABI takes FP32 weights
    s_or, _ = oracle.statistic(sfts, bank, w=w32)
    assert_s_close(s, s_or)
    assert_z_close(z, s_or, sfts.n_total, w32)


def test_device_and_host_outputs_agree_and_are_deterministic(ctx):
    import torch

    sfts, bank = _small(n_sft=300, n_f0=70, n_f1=5, n_sky=20)
    band = H.band_from(ctx, sfts, on_device=True)
    bk = H.bank_from(ctx, band, bank)
    s_h, _, _ = H.eval_host(ctx, band, bk, bank.n_templates)
    s_d = torch.empty(bank.n_templates, dtype=torch.float32, device="cuda")
    ft.eval_statistic(ctx, band, bk, s_d)
    torch.cuda.synchronize()
    assert np.array_equal(s_d.cpu().numpy(), s_h)
    s_h2, _, _ = H.eval_host(ctx, band, bk, bank.n_templates)
    assert np.array_equal(s_h, s_h2)


def test_error_paths(ctx):
    sfts, bank = _small()
    band = H.band_from(ctx, sfts)
    bk = H.bank_from(ctx, band, bank)
    out = np.zeros((bank.n_subbands, 33), dtype=ft.CANDIDATE_DTYPE)
    for k in (0, 33):
        with pytest.raises(ft.FtError) as e:
            ft.topk_per_band(ctx, band, bk, k, out)
        assert e.value.code == -5
    other = H.band_from(ctx, sfts)
    with pytest.raises(ft.FtError) as e:
        ft.eval_statistic(ctx, other, bk, np.empty(bank.n_templates, np.float32))
    assert e.value.code == -1
    bad = sfts.power.copy()
    bad[3, 5] = np.nan
    with pytest.raises(ft.FtError) as e:
        H.band_from(ctx, _with_power(sfts, bad))
    assert e.value.code == -1
    fast = ftsynth.SFTSet(power=sfts.power, t_mid=sfts.t_mid, v=sfts.v * 20, s_n=sfts.s_n,
                          n_sft=sfts.n_sft, k_lo=sfts.k_lo, t_sft=1800.0, t0=0.0)
    with pytest.raises(ft.FtError) as e:
        H.band_from(ctx, fast)
    assert e.value.code == -5
    # the context stays usable after errors
    s, _, _ = H.eval_host(ctx, band, bk, bank.n_templates)
    assert np.all(np.isfinite(s))


def test_gather_roof_microbenchmark(ctx):
    """The measured ceiling of the inner loop runs and is plausible: positive, 16-bit pairs
    above FP32 per evaluation, and below the shared-memory bandwidth bound (128 B per clock
    per SM = 32 FP32 or 64 16-bit evaluations)."""
    e32, c32 = ft.gather_roof(ctx, "f32")
    e16, c16 = ft.gather_roof(ctx, "f16")
    assert 0 < c32 <= 32.5 and 0 < c16 <= 64.5
    assert e16 > e32 > 0
