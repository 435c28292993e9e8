"""Number count on the GPU (Eq. (number_count)) and the gated selection of Sec. VI.B,
against the oracle:

* the number-count band's weighted count per template: exact for unit weights (integer sums)
  with FP32, FP16 and BF16 storage (the oracle binarises the same stored values), in both the
  unchecked and the checked kernel; FP32 tolerance for per-SFT and all-sky weights;
* the band's mu_G / sigma_G are the count's noise moments, and z uses them;
* the loudest s per sub-band among templates whose count reaches a minimum: equal to the
  oracle's gated selection (near-tie exemption) and exactly the CPU selection over the GPU's
  own s and counts.
"""
import math

import numpy as np
import pytest

import ftsynth
import oracle
import paper_2411_18370_b300 as ft
from tests import helpers as H
from tests.test_gpu_parity import assert_topk

pytestmark = pytest.mark.gpu

REL = 1e-6
THR = 3.2


@pytest.fixture(scope="module")
def ctx():
    c = ft.create(0)
    yield c
    c.close()


def _band(n_sft=(60, 45), W=150, n_f0=64, n_f1=4, n_sky=6, sub=16, wings=40, seed=31):
    g = np.random.default_rng(seed)
    k_band = 220_000
    t_mid, v = [], []
    for X, n in enumerate(n_sft):
        t = np.sort(g.uniform(0, 2.5e7, n)) + 900
        t_mid.append(t)
        v.append(ftsynth.detector_velocity(t, X))
    t_mid = np.concatenate(t_mid)
    N = len(t_mid)
    sfts = ftsynth.SFTSet(power=g.exponential(2.0, (N, W)), t_mid=t_mid, v=np.concatenate(v),
                          s_n=g.uniform(0.5, 2.0, N), n_sft=list(n_sft), k_lo=k_band - wings,
                          t_sft=1800.0, t0=0.0)
    bank = ftsynth.Bank(k0=k_band, n_f0=n_f0, f1=np.linspace(-3e-10, 0, n_f1),
                        sky=ftsynth.fibonacci_sky(n_sky), subband_bins=sub)
    return sfts, bank


def _stored(sfts, dtype):
    import torch

    # the bands are loaded from FP32 rows: FP64 -> FP32 -> storage type, each round to nearest even
    t = torch.from_numpy(sfts.power).to(torch.float32)
    if dtype != "f32":
        t = t.to(torch.float16 if dtype == "f16" else torch.bfloat16)
    P = t.to(torch.float64).numpy()
    return ftsynth.SFTSet(**{**sfts.__dict__, "power": P})


def _det_tensor(sfts):
    parts, off = [], 0
    for X, n in enumerate(sfts.n_sft):
        parts.append(ftsynth.detector_tensor(sfts.t_mid[off:off + n], X))
        off += n
    return np.concatenate(parts)


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("wings", [40, 2])
def test_unit_weight_count_exact(ctx, dtype, wings):
    sfts, bank = _band(wings=wings, W=150 if wings == 40 else 70, seed=32 + wings)
    band = H.band_from(ctx, sfts, dtype=dtype, power_f32=True)
    ncb = ft.number_count_band(ctx, band, THR)
    bk = H.bank_from(ctx, ncb, bank)
    assert bk.window_safe == (wings == 40)
    nc, z, o = H.eval_host(ctx, ncb, bk, bank.n_templates)
    want, o_or = oracle.number_count(_stored(sfts, dtype), bank, threshold=THR)
    assert np.array_equal(o, o_or)
    assert np.array_equal(nc.astype(np.float64), want)
    mu, sd = oracle.nc_moments(THR, n_sft=sfts.n_total)
    assert math.isclose(ncb.mu_g, mu, rel_tol=1e-12) and math.isclose(ncb.sigma_g, sd, rel_tol=1e-12)
    assert np.all(np.abs(z - (want - mu) / sd) <= 1e-5)


def test_weighted_counts(ctx):
    sfts, bank = _band(seed=40)
    w = np.random.default_rng(2).uniform(0.3, 2.0, sfts.n_total)
    w32 = w.astype(np.float32).astype(np.float64)
    band = H.band_from(ctx, sfts, w=w, power_f32=True)
    ncb = ft.number_count_band(ctx, band, THR)
    bk = H.bank_from(ctx, ncb, bank)
    nc, z, _ = H.eval_host(ctx, ncb, bk, bank.n_templates)
    ref = _stored(sfts, "f32")
    want, _ = oracle.number_count(ref, bank, threshold=THR, w=w32)
    assert np.all(np.abs(nc - want) <= REL * np.maximum(want, 1.0))
    mu, sd = oracle.nc_moments(THR, w=w32)
    assert math.isclose(ncb.mu_g, mu, rel_tol=1e-7) and math.isclose(ncb.sigma_g, sd, rel_tol=1e-7)
    # all-sky weights: copied from the source band to the count
    ft.band_set_sky_weights(band, _det_tensor(sfts))
    ncs = ft.number_count_band(ctx, band, THR)
    bks = H.bank_from(ctx, ncs, bank)
    nc_s, z_s, _ = H.eval_host(ctx, ncs, bks, bank.n_templates)
    wsky = oracle.sky_weights(_det_tensor(sfts), sfts.s_n, bank.sky)
    want_s, _ = oracle.number_count(ref, bank, threshold=THR, wsky=wsky)
    assert np.all(np.abs(nc_s - want_s) <= REL * np.maximum(want_s, 1e-3))
    p = math.exp(-0.5 * THR)
    sig = np.sqrt(p * (1 - p) * (wsky * wsky).sum(axis=1))
    i_sky = np.arange(bank.n_templates) // (bank.n_f1 * bank.n_f0)
    z_or = (want_s - p) / sig[i_sky]
    assert np.all(np.abs(z_s - z_or) <= REL * np.maximum(want_s, 1e-3) / sig[i_sky] + 1e-5)


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_gated_selection(ctx, dtype):
    import torch

    sfts, bank = _band(n_f0=200, W=290, n_sky=5, sub=25, seed=50)
    band = H.band_from(ctx, sfts, dtype=dtype, power_f32=True)
    bk = H.bank_from(ctx, band, bank)
    ncb = ft.number_count_band(ctx, band, THR)
    bkn = H.bank_from(ctx, ncb, bank)
    n = bank.n_templates
    gate = torch.empty(n, dtype=torch.float32, device="cuda")
    ft.eval_statistic(ctx, ncb, bkn, gate)
    torch.cuda.synchronize()
    nc = gate.cpu().numpy().astype(np.float64)
    s, _, _ = H.eval_host(ctx, band, bk, n)
    ref = _stored(sfts, dtype)
    s_or, _ = oracle.statistic(ref, bank)
    nc_or, _ = oracle.number_count(ref, bank, threshold=THR)
    assert np.array_equal(nc, nc_or)
    t_all = np.arange(n)
    K = 5
    for gmin in (ncb.mu_g, ncb.mu_g + ncb.sigma_g, ncb.mu_g + 3 * ncb.sigma_g):
        out = np.zeros((bk.n_subbands, K), dtype=ft.CANDIDATE_DTYPE)
        ft.topk_per_band_gated(ctx, band, bk, K, gate, gmin, out)
        idx, val = out["template_idx"], out["s"]
        keep = nc_or >= np.float32(gmin)
        assert keep.any()
        assert_topk(idx, val, s_or[keep], bank, K, s_gpu=s[keep], templates=t_all[keep])
        ok = idx >= 0
        assert np.all(nc[idx[ok]] >= np.float32(gmin))
        assert np.all(out["s"][~ok] == -np.inf)


def test_number_count_errors(ctx):
    import torch

    sfts, bank = _band(n_sky=2, seed=60)
    band = H.band_from(ctx, sfts)
    with pytest.raises(ft.FtError):
        ft.number_count_band(ctx, band, -1.0)
    ncb = ft.number_count_band(ctx, band, THR)
    with pytest.raises(ft.FtError):
        ft.number_count_band(ctx, ncb, THR)
    bk = H.bank_from(ctx, band, bank)
    out = np.zeros((bk.n_subbands, 2), dtype=ft.CANDIDATE_DTYPE)
    with pytest.raises(ValueError):
        ft.topk_per_band_gated(ctx, band, bk, 2, np.zeros(bank.n_templates, np.float32), 0.0, out)
    gate = torch.zeros(bank.n_templates, dtype=torch.float32, device="cuda")
    with pytest.raises(ft.FtError):
        ft.topk_per_band_gated(ctx, band, bk, 2, gate, float("nan"), out)
