"""The binary-orbit track over a random hyperbox bank on the GPU, against the oracle:

* the screen's cosine step is within the bound its delta assumes, over all 2^32 phases;
* the templates the kernels derive from their Philox counters equal the oracle's, bit for bit;
* the bins of every (template, SFT) pair are the FP64 bins of Eq. (track): equal to the
  oracle's except where the oracle's FP64 position lies within TIE = 1e-9 bins of a rounding
  boundary (the two FP64 evaluations' own rounding); such pairs are counted and listed;
* a bank whose every evaluation falls inside the FP32 screen's bound (the FP64 decision path
  for all of them) gets the oracle's bins and statistic too, and the kernels report one FP64
  decision per evaluation;
* s per template within the FP32 tolerance (FP32, FP16 and BF16 storage; the oracle reads the
  same stored values); where a bin differs at a tie, s differs by exactly the power difference
  at those pairs; z and the out-of-window counts;
* the loudest templates of every hyperbox: the oracle's sets (near-tie exemption) and exactly
  the CPU selection over the GPU's own values;
* ragged shapes: boxes that are not a multiple of the CTA, SFT counts that are not a multiple
  of a stage, a single template, isolated sources (a_p = 0), k above the box population;
* the number count along binary tracks (exact) and the count-gated per-box selection;
* the benchmark's full-size workload in its timed launch, on sampled templates, with the
  fraction of FP64 decisions near its expected 2 delta.
"""
import math

import numpy as np
import pytest

import ftsynth
import oracle
import paper_2411_18370_b300 as ft
from tests import helpers as H

pytestmark = pytest.mark.gpu

REL = 1e-6
DAY = 86400.0


@pytest.fixture(scope="module")
def ctx():
    c = ft.create(0)
    yield c
    c.close()


def _bank(n_div=(2, 2, 2, 2, 1, 2), n_per_box=300, seed=5, f0=(100.0, 100.05), ap=(5.0, 15.0)):
    om = (2 * math.pi / (15 * DAY), 2 * math.pi / (7 * DAY))
    return ftsynth.BinaryBank(lo=(f0[0], 0.0, -1.0, ap[0], om[0], 0.0),
                              hi=(f0[1], 1.0, 1.0, ap[1], om[1], 1.0),
                              n_div=n_div, n_per_box=n_per_box, seed=seed)


def _sfts(n_sft=(150, 123), W=200, wings=55, seed=3, k_band=180_000):
    g = np.random.default_rng(seed)
    t_mid, v = [], []
    for X, n in enumerate(n_sft):
        t = np.sort(g.uniform(0, ftsynth.YEAR_S, n)) + 900
        t_mid.append(t)
        v.append(ftsynth.detector_velocity(t, X))
    t_mid = np.concatenate(t_mid)
    N = len(t_mid)
    return ftsynth.SFTSet(power=g.exponential(2.0, (N, W)), t_mid=t_mid, v=np.concatenate(v),
                          s_n=np.ones(N), n_sft=list(n_sft), k_lo=k_band - wings, t_sft=1800.0,
                          t0=0.0)


def _stored(sfts, dtype):
    import torch

    t = torch.from_numpy(sfts.power).to(torch.float32)
    if dtype != "f32":
        t = t.to(torch.float16 if dtype == "f16" else torch.bfloat16)
    return ftsynth.SFTSet(**{**sfts.__dict__, "power": t.to(torch.float64).numpy()})


def _gpu_bank(ctx, band, bank):
    return ft.make_binary_bank(ctx, band, bank.lo, bank.hi, bank.n_div, bank.n_per_box, bank.seed)


TIE = 1e-9


def _check_bins_and_s(ctx, band, gb, stored, bank, tmpl, s_gpu, w=None, rel=REL):
    """GPU bins of templates tmpl equal the oracle's FP64 bins except within TIE of a rounding
    boundary; s within rel of the oracle where no bin differs, and shifted by exactly the
    power difference at the differing pairs where one does.  Returns the differing pairs."""
    tmpl = np.asarray(tmpl, np.int64)
    N = stored.n_total
    W = stored.power.shape[1]
    gbins = np.empty((len(tmpl), N), np.int32)
    ft.binary_track_bins(ctx, band, gb, tmpl, gbins)
    b_or, dist = oracle.binary_bins(stored, bank, tmpl, with_dist=True)
    diff = gbins.astype(np.int64) != b_or
    assert np.all(dist[diff] < TIE), f"bins differ away from a tie: {np.sum(dist[diff] >= TIE)} pairs"
    s_or, _ = oracle.binary_statistic(stored, bank, tmpl, w=w)
    wv = np.ones(N) if w is None else np.asarray(w, np.float64)
    rows = np.arange(N)
    for r in range(len(tmpl)):
        want = s_or[r]
        if diff[r].any():
            a = rows[diff[r]]
            pg = np.where((gbins[r, a] >= 0) & (gbins[r, a] < W), stored.power[a, np.clip(gbins[r, a], 0, W - 1)], 0.0)
            po = np.where((b_or[r, a] >= 0) & (b_or[r, a] < W), stored.power[a, np.clip(b_or[r, a], 0, W - 1)], 0.0)
            want = want + np.sum(wv[a] * (pg - po))
        assert abs(float(s_gpu[r]) - want) <= rel * max(abs(want), 1.0), (int(tmpl[r]), float(s_gpu[r]), want)
    return int(diff.sum())


def test_cos_screen_within_its_bound(ctx):
    """The screen's cosine step (integer orbit phase -> FP32 angle -> the special-function
    unit's cosine), over every one of the 2^32 phases, stays within the bound the screen's
    delta assumes for it; that bound is what makes every bin the FP64 bin."""
    m, bound = ft.binary_cos_screen_check(ctx)
    assert 0.0 < m <= bound, (m, bound)
    assert bound < 2e-6


def test_templates_and_bins_equal_the_fp64_track(ctx):
    sfts = _sfts()
    bank = _bank()
    band = H.band_from(ctx, sfts, power_f32=True)
    gb = _gpu_bank(ctx, band, bank)
    assert gb.n_templates == bank.n_templates and gb.n_boxes == bank.n_boxes
    lam = ft.binary_templates(ctx, gb, 0, gb.n_templates)
    assert np.array_equal(lam, oracle.binary_templates(bank))
    t = np.random.default_rng(1).choice(bank.n_templates, 400, replace=False).astype(np.int64)
    out = np.empty((len(t), sfts.n_total), np.int32)
    ft.binary_track_bins(ctx, band, gb, t, out)
    b_or, dist = oracle.binary_bins(sfts, bank, t, with_dist=True)
    differ = out.astype(np.int64) != b_or
    assert np.all(dist[differ] < TIE)
    assert differ.sum() <= 2
    # the orbit and the Doppler really move the tracks
    assert np.median(out.max(axis=1) - out.min(axis=1)) > 20


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_every_evaluation_through_the_fp64_decision(ctx, dtype):
    """Tracks that hover within the screen's bound of a rounding boundary: f0 T_SFT within
    5e-8 of a half-integer, detector velocities scaled to |v| ~ 5e-13 and an orbit of 4e-8
    bins (a_p = 2e-8 lt-s), so that F v.n and the orbit term move X by ~1e-7 bins around it.
    Every evaluation takes the FP64 decision; the bins are the oracle's (ties within TIE
    excepted) and so is s."""
    import dataclasses

    sfts = _sfts(seed=22, n_sft=(90, 77))
    sfts = dataclasses.replace(sfts, v=sfts.v * 5e-9)
    T = sfts.t_sft
    K = 180_020
    om = (2 * math.pi / (15 * DAY), 2 * math.pi / (7 * DAY))
    bank = ftsynth.BinaryBank(lo=((K + 0.5 - 5e-8) / T, 0.0, -1.0, 2e-8, om[0], 0.0),
                              hi=((K + 0.5 + 5e-8) / T, 1.0, 1.0, 2e-8, om[1], 1.0),
                              n_div=(1, 2, 1, 1, 1, 2), n_per_box=300, seed=23)
    band = H.band_from(ctx, sfts, dtype=dtype, power_f32=True)
    gb = _gpu_bank(ctx, band, bank)
    ft.binary_decisions(gb)
    n = bank.n_templates
    s = np.empty(n, np.float32)
    ft.binary_eval(ctx, band, gb, 0, n, s)
    n64, delta = ft.binary_decisions(gb)
    assert delta < 1e-6
    assert n64 == n * sfts.n_total
    b_or, dist = oracle.binary_bins(sfts, bank, np.arange(n), with_dist=True)
    assert np.all(dist < delta / 2)
    # both roundings happen: the tracks really straddle the boundary
    assert np.all(np.isin(b_or, [K - sfts.k_lo, K + 1 - sfts.k_lo])) and len(np.unique(b_or)) == 2
    ndiff = _check_bins_and_s(ctx, band, gb, _stored(sfts, dtype), bank, np.arange(n), s)
    assert ndiff <= 0.002 * n * sfts.n_total


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_statistic_and_z(ctx, dtype):
    sfts = _sfts(seed=4)
    bank = _bank(seed=6)
    band = H.band_from(ctx, sfts, dtype=dtype, power_f32=True)
    gb = _gpu_bank(ctx, band, bank)
    n = bank.n_templates
    s = np.empty(n, np.float32)
    z = np.empty(n, np.float32)
    o = np.empty(n, np.int32)
    ft.binary_eval(ctx, band, gb, 0, n, s, z, o)
    s_or, o_or = oracle.binary_statistic(_stored(sfts, dtype), bank)
    assert np.array_equal(o, o_or)
    _check_bins_and_s(ctx, band, gb, _stored(sfts, dtype), bank, np.arange(n), s)
    mu, sig = oracle.mu_sigma(sfts.n_total)
    assert np.all(np.abs(z - (s.astype(np.float64) - mu) / sig) <= REL * np.abs(s_or) / sig + 1e-6)
    # a sub-range equals the same slice of the full evaluation
    s2 = np.empty(777, np.float32)
    ft.binary_eval(ctx, band, gb, 1001, 777, s2)
    assert np.array_equal(s2, s[1001:1778])


def test_weighted_statistic(ctx):
    sfts = _sfts(seed=7, n_sft=(100, 77))
    bank = _bank(seed=8, n_per_box=100)
    w = np.random.default_rng(3).uniform(0.3, 2.0, sfts.n_total)
    band = H.band_from(ctx, sfts, w=w, power_f32=True)
    gb = _gpu_bank(ctx, band, bank)
    s = np.empty(bank.n_templates, np.float32)
    ft.binary_eval(ctx, band, gb, 0, bank.n_templates, s)
    _check_bins_and_s(ctx, band, gb, _stored(sfts, "f32"), bank, np.arange(bank.n_templates), s,
                      w=w.astype(np.float32).astype(np.float64))


def _check_topk(ctx, band, gb, sfts_stored, bank, k):
    out = np.zeros((bank.n_boxes, k), dtype=ft.CANDIDATE_DTYPE)
    ft.binary_topk_per_box(ctx, band, gb, k, out)
    s = np.empty(bank.n_templates, np.float32)
    ft.binary_eval(ctx, band, gb, 0, bank.n_templates, s)
    s_or, _ = oracle.binary_statistic(sfts_stored, bank)
    idx, val = out["template_idx"], out["s"]
    # exactly the CPU selection over the GPU's own values
    c_idx, c_val = oracle.topk_per_box(s.astype(np.float64), bank.n_per_box, bank.n_boxes, k)
    assert np.array_equal(idx, c_idx)
    ok = idx >= 0
    assert np.array_equal(val[ok].astype(np.float64), c_val[ok])
    assert np.all(val[~ok] == -np.inf)
    # the oracle's sets, except where its k-th and (k+1)-th values nearly tie
    o_idx, o_val = oracle.topk_per_box(s_or, bank.n_per_box, bank.n_boxes, k + 1)
    for b in range(bank.n_boxes):
        got = set(int(x) for x in idx[b] if x >= 0)
        want = set(int(x) for x in o_idx[b, :k] if x >= 0)
        if got != want:
            kth, nxt = o_val[b, k - 1], o_val[b, k]
            assert np.isfinite(nxt) and abs(kth - nxt) < 2e-6 * abs(kth), f"box {b}"
    mu, sig = oracle.mu_sigma(sfts_stored.n_total)
    assert np.all(np.abs(out["z"][ok] - (val[ok] - mu) / sig) <= 1e-5)


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_topk_per_box(ctx, dtype):
    sfts = _sfts(seed=9)
    bank = _bank(seed=10, n_per_box=700)   # 2 tiles of 512 per box, the second ragged
    band = H.band_from(ctx, sfts, dtype=dtype, power_f32=True)
    gb = _gpu_bank(ctx, band, bank)
    for k in (1, 5):
        _check_topk(ctx, band, gb, _stored(sfts, dtype), bank, k)


@pytest.mark.parametrize("shape", [
    dict(n_sft=(5,), n_div=(1, 1, 1, 1, 1, 1), n_per_box=1, k=3),
    dict(n_sft=(70, 1), n_div=(1, 2, 1, 1, 1, 3), n_per_box=257, k=2),
    dict(n_sft=(40, 9), n_div=(1, 1, 1, 1, 1, 2), n_per_box=1537, k=4),
    dict(n_sft=(33, 31), n_div=(3, 1, 1, 1, 1, 1), n_per_box=20, k=32, ap=(0.0, 0.0)),
])
def test_edge_shapes(ctx, shape):
    sfts = _sfts(n_sft=shape["n_sft"], seed=11)
    bank = _bank(n_div=shape["n_div"], n_per_box=shape["n_per_box"], seed=12,
                 ap=shape.get("ap", (5.0, 15.0)))
    band = H.band_from(ctx, sfts, power_f32=True)
    gb = _gpu_bank(ctx, band, bank)
    s = np.empty(bank.n_templates, np.float32)
    o = np.empty(bank.n_templates, np.int32)
    ft.binary_eval(ctx, band, gb, 0, bank.n_templates, s, None, o)
    s_or, o_or = oracle.binary_statistic(_stored(sfts, "f32"), bank)
    assert np.array_equal(o, o_or)
    _check_bins_and_s(ctx, band, gb, _stored(sfts, "f32"), bank, np.arange(bank.n_templates), s)
    _check_topk(ctx, band, gb, _stored(sfts, "f32"), bank, shape["k"])


def test_bins_leaving_the_window_are_counted(ctx):
    sfts = _sfts(W=80, wings=5, seed=13)   # narrow wings: many tracks leave the band
    bank = _bank(seed=14, n_per_box=50)
    band = H.band_from(ctx, sfts, power_f32=True)
    gb = _gpu_bank(ctx, band, bank)
    s = np.empty(bank.n_templates, np.float32)
    o = np.empty(bank.n_templates, np.int32)
    ft.binary_eval(ctx, band, gb, 0, bank.n_templates, s, None, o)
    s_or, o_or = oracle.binary_statistic(_stored(sfts, "f32"), bank)
    assert o_or.sum() > 0
    assert np.array_equal(o, o_or)
    _check_bins_and_s(ctx, band, gb, _stored(sfts, "f32"), bank, np.arange(bank.n_templates), s)


def test_errors(ctx):
    sfts = _sfts(n_sft=(20,), seed=15)
    band = H.band_from(ctx, sfts)
    b = _bank()
    bad = [dict(lo=(100.0, 0, -1, 5, 1e-5, 0), hi=(99.0, 1, 1, 15, 2e-5, 1)),      # lo > hi
           dict(lo=(100.0, 0, -1, 1, 1e-5, 0), hi=(100.1, 1, 1, 17, 2e-5, 1)),     # a_p ratio > 16
           dict(lo=(100.0, 0, -2, 5, 1e-5, 0), hi=(100.1, 1, 1, 15, 2e-5, 1)),     # sin(delta) < -1
           dict(lo=(100.0, 0, -1, 5, 1e-5, 0), hi=(100.1, 1.5, 1, 15, 2e-5, 1))]   # alpha > 1 turn
    for d in bad:
        with pytest.raises(ft.FtError):
            ft.make_binary_bank(ctx, band, d["lo"], d["hi"], b.n_div, 10, 1)
    with pytest.raises(ft.FtError):
        ft.make_binary_bank(ctx, band, b.lo, b.hi, (1, 1, 1, 0, 1, 1), 10, 1)
    gb = _gpu_bank(ctx, band, b)
    out = np.zeros((gb.n_boxes, 40), dtype=ft.CANDIDATE_DTYPE)
    with pytest.raises(ft.FtError):
        ft.binary_topk_per_box(ctx, band, gb, 40, out)
    with pytest.raises(ft.FtError):
        ft.binary_eval(ctx, band, gb, gb.n_templates - 1, 5, np.empty(5, np.float32))


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_number_count_gated_boxes(ctx, dtype):
    """Sec. VI.B on the binary bank: the loudest s per box among templates whose number
    count reaches its noise mean + sigma (a gate that keeps a few templates per box)."""
    import dataclasses

    import torch

    sfts = _sfts(seed=16)
    bank = _bank(seed=17, n_per_box=300)
    band = H.band_from(ctx, sfts, dtype=dtype, power_f32=True)
    gb = _gpu_bank(ctx, band, bank)
    ncb = ft.number_count_band(ctx, band, 3.2)
    gnc = _gpu_bank(ctx, ncb, bank)
    n = bank.n_templates
    gate = torch.empty(n, dtype=torch.float32, device="cuda")
    ft.binary_eval(ctx, ncb, gnc, 0, n, gate)
    torch.cuda.synchronize()
    stored = _stored(sfts, dtype)
    nc_or, _ = oracle.binary_statistic(dataclasses.replace(stored, power=(stored.power > 3.2) * 1.0), bank)
    assert np.array_equal(gate.cpu().numpy().astype(np.float64), nc_or)
    s = np.empty(n, np.float32)
    ft.binary_eval(ctx, band, gb, 0, n, s)
    for gmin in (ncb.mu_g + ncb.sigma_g, ncb.mu_g + 3 * ncb.sigma_g):
        keep = nc_or >= np.float32(gmin)
        k = 3
        out = np.zeros((bank.n_boxes, k), dtype=ft.CANDIDATE_DTYPE)
        ft.binary_topk_per_box_gated(ctx, band, gb, k, gate, gmin, out)
        t = np.arange(n)[keep]
        c_idx, c_val = oracle.topk_per_box(s[keep].astype(np.float64), bank.n_per_box, bank.n_boxes, k, t)
        assert np.array_equal(out["template_idx"], c_idx)
        ok = c_idx >= 0
        assert np.array_equal(out["s"][ok].astype(np.float64), c_val[ok])
        assert np.all(out["s"][~ok] == -np.inf)


def _det_tensor(sfts):
    parts, off = [], 0
    for X, n in enumerate(sfts.n_sft):
        parts.append(ftsynth.detector_tensor(sfts.t_mid[off:off + n], X))
        off += n
    return np.concatenate(parts)


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_all_sky_weights(ctx, dtype):
    """Sec. II.B weights on the binary bank: per (template, SFT) r = (a^2 + b^2)/S_n of the
    template's own sky direction, computed in the kernel (FP32, frame-free form), s = sum r P /
    sum r and z with sigma_G = 2 sqrt(sum r^2) / sum r.  Tolerance 2e-6 relative: the FP32
    weights (error ~ 1e-7 of the largest r) enter every term."""
    import dataclasses

    sfts = _sfts(seed=18)
    sfts = dataclasses.replace(sfts, s_n=np.random.default_rng(4).uniform(0.5, 2.0, sfts.n_total))
    bank = _bank(seed=19, n_per_box=200)
    band = H.band_from(ctx, sfts, dtype=dtype, power_f32=True)
    stale = _gpu_bank(ctx, band, bank)
    D = _det_tensor(sfts)
    ft.band_set_sky_weights(band, D)
    with pytest.raises(ft.FtError):
        ft.binary_eval(ctx, band, stale, 0, 10, np.empty(10, np.float32))
    gb = _gpu_bank(ctx, band, bank)
    n = bank.n_templates
    s = np.empty(n, np.float32)
    z = np.empty(n, np.float32)
    o = np.empty(n, np.int32)
    ft.binary_eval(ctx, band, gb, 0, n, s, z, o)
    s_or, sig_or, o_or = oracle.binary_statistic_sky(_stored(sfts, dtype), bank, D)
    assert np.array_equal(o, o_or)
    assert np.all(np.abs(s - s_or) <= 2e-6 * s_or)
    z_or = (s_or - 2.0) / sig_or
    assert np.all(np.abs(z - z_or) <= 2e-6 * s_or / sig_or + 1e-5)
    k = 4
    out = np.zeros((bank.n_boxes, k), dtype=ft.CANDIDATE_DTYPE)
    ft.binary_topk_per_box(ctx, band, gb, k, out)
    c_idx, c_val = oracle.topk_per_box(s.astype(np.float64), bank.n_per_box, bank.n_boxes, k)
    assert np.array_equal(out["template_idx"], c_idx)
    assert np.array_equal(out["s"].astype(np.float64), c_val)


def test_sky_weighted_number_count(ctx):
    """A number-count band inherits the all-sky weights: its binary statistic is the weighted
    count with per-template weights, and z uses the count's noise moments (mu = p, sigma =
    sqrt(p (1 - p) sum w^2))."""
    import dataclasses
    import math

    sfts = _sfts(seed=20)
    sfts = dataclasses.replace(sfts, s_n=np.random.default_rng(6).uniform(0.5, 2.0, sfts.n_total))
    bank = _bank(seed=21, n_per_box=100)
    band = H.band_from(ctx, sfts, power_f32=True)
    D = _det_tensor(sfts)
    ft.band_set_sky_weights(band, D)
    ncb = ft.number_count_band(ctx, band, 3.2)
    gb = _gpu_bank(ctx, ncb, bank)
    n = bank.n_templates
    s = np.empty(n, np.float32)
    z = np.empty(n, np.float32)
    ft.binary_eval(ctx, ncb, gb, 0, n, s, z)
    stored = _stored(sfts, "f32")
    bin_ = dataclasses.replace(stored, power=(stored.power > 3.2) * 1.0)
    s_or, sig_pow, _ = oracle.binary_statistic_sky(bin_, bank, D)
    assert np.all(np.abs(s - s_or) <= 2e-6 * np.maximum(s_or, 1e-3))
    p = math.exp(-1.6)
    sig = sig_pow / 2.0 * math.sqrt(p * (1 - p))  # sig_pow = 2 sqrt(sum w^2)
    z_or = (s_or - p) / sig
    assert np.all(np.abs(z - z_or) <= 2e-6 * np.maximum(s_or, 1e-3) / sig + 1e-5)


def test_full_workload_sampled(ctx):
    """The benchmark's binary workload (2^20 templates in 32 boxes, 21 657 SFTs, FP16
    storage) in the launch it times (loudest per box, k = 1): the selection is exactly the CPU
    selection over the GPU's s of every template; bins, s and the out-of-window counts of 192
    sampled templates and of every box winner match the oracle; the launch took FP64
    decisions for a fraction of its evaluations near 2 delta (the screen's error is uniform
    across the bin, so about 2 delta of the positions fall within delta of a boundary)."""
    sfts, bank = ftsynth.binary_workload()
    band = H.band_from(ctx, sfts, dtype="f16", power_f32=True, on_device=True)
    gb = _gpu_bank(ctx, band, bank)
    ft.binary_decisions(gb)
    out = np.zeros((bank.n_boxes, 1), dtype=ft.CANDIDATE_DTYPE)
    ft.binary_topk_per_box(ctx, band, gb, 1, out)
    n64, delta = ft.binary_decisions(gb)
    evals = bank.n_templates * sfts.n_total
    assert 0.8 * 2 * delta < n64 / evals < 1.2 * 2 * delta, (n64, evals, delta)
    n = bank.n_templates
    s = np.empty(n, np.float32)
    o = np.empty(n, np.int32)
    ft.binary_eval(ctx, band, gb, 0, n, s, None, o)
    c_idx, c_val = oracle.topk_per_box(s.astype(np.float64), bank.n_per_box, bank.n_boxes, 1)
    assert np.array_equal(out["template_idx"], c_idx)
    assert np.array_equal(out["s"].astype(np.float64), c_val)
    samp = np.concatenate([np.random.default_rng(12).choice(n, 192, replace=False),
                           out["template_idx"][:, 0]]).astype(np.int64)
    s_or, o_or = oracle.binary_statistic(_stored(sfts, "f16"), bank, samp)
    assert np.array_equal(o[samp], o_or)
    _check_bins_and_s(ctx, band, gb, _stored(sfts, "f16"), bank, samp, s[samp])
