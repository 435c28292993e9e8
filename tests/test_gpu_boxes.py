"""Ahead-of-time boxes over all three dimensions of the regular bank (Sec. IV.B): box
(x, y, b) = the templates of sub-band b whose sky point sits at positions x sky_box ..
(x + 1) sky_box - 1 of the bank's sky order and whose f1 index is in y f1_box ..
(y + 1) f1_box - 1; the loudest per box, plain or count-gated (Sec. VI.B).  Checked exactly
against the CPU selection over the GPU's own values and, with the near-tie exemption, against
the oracle's values, for box sizes that do and do not divide the CTA's f1 and sky groups, both
kernels and FP32 / FP16 storage; boxes spanning a whole dimension reduce to the per-sky-box
and per-sub-band selections."""
import numpy as np
import pytest
import torch

import oracle
import paper_2411_18370_b300 as ft
from tests import helpers as H
from tests.test_gpu_parity import _small

pytestmark = pytest.mark.gpu

K = 3


@pytest.fixture(scope="module")
def ctx():
    c = ft.create(0)
    yield c
    c.close()


def _keys(bank, order, sky_box, f1_box):
    pos = np.empty(bank.n_sky, np.int64)
    pos[order] = np.arange(bank.n_sky)
    t = np.arange(bank.n_templates)
    i_sky = t // (bank.n_f1 * bank.n_f0)
    i_f1 = (t // bank.n_f0) % bank.n_f1
    j = t % bank.n_f0
    n_f1b = -(-bank.n_f1 // f1_box)
    return ((pos[i_sky] // sky_box) * n_f1b + i_f1 // f1_box) * bank.n_subbands + j // bank.subband_bins


def _check(out, s_gpu, s_or, key, n_keys, keep):
    idx = out["template_idx"].reshape(n_keys, K)
    val = out["s"].reshape(n_keys, K)
    t = np.nonzero(keep)[0]
    c_idx, c_val = oracle.topk_per_key(s_gpu[t].astype(np.float64), key[t], n_keys, K, t)
    assert np.array_equal(idx, c_idx)
    ok = idx >= 0
    assert np.array_equal(val[ok].astype(np.float64), c_val[ok])
    o_idx, o_val = oracle.topk_per_key(s_or[t], key[t], n_keys, K + 1, t)
    for b in range(n_keys):
        got = set(int(x) for x in idx[b] if x >= 0)
        want = set(int(x) for x in o_idx[b, :K] if x >= 0)
        if got != want:
            kth, nxt = o_val[b, K - 1], o_val[b, K]
            assert np.isfinite(nxt) and abs(kth - nxt) < 2e-6 * abs(kth)


@pytest.mark.parametrize("dtype", ["f32", "f16"])
@pytest.mark.parametrize("wings", [30, 2])
def test_sky_f1_boxes(ctx, dtype, wings):
    sfts, bank = _small(n_sft=60, n_f0=50, n_f1=23, n_sky=11, sub=9, W=120 if wings == 30 else 64,
                        wings=wings, seed=9)
    band = H.band_from(ctx, sfts, dtype=dtype)
    bk = H.bank_from(ctx, band, bank)
    assert bk.window_safe == (wings == 30)
    order = ft.bank_sky_order(bk, bank.n_sky)
    s, _, _ = H.eval_host(ctx, band, bk, bank.n_templates)
    p = sfts.power if dtype == "f32" else sfts.power.astype(np.float16).astype(np.float64)
    s_or, _ = oracle.statistic(type(sfts)(**{**sfts.__dict__, "power": p}), bank)
    gate = np.random.default_rng(3).uniform(0, 1, bank.n_templates).astype(np.float32)
    gate_d = torch.from_numpy(gate).cuda()
    all_in = np.ones(bank.n_templates, bool)
    for sky_box, f1_box in ((1, 1), (3, 5), (6, 7), (4, 12), (11, 4), (100, 3), (2, 23), (5, 40)):
        n_skyb = -(-bank.n_sky // sky_box)
        n_f1b = -(-bank.n_f1 // f1_box)
        n_keys = n_skyb * n_f1b * bank.n_subbands
        key = _keys(bank, order, sky_box, f1_box)
        out = np.zeros((n_skyb, n_f1b, bank.n_subbands, K), dtype=ft.CANDIDATE_DTYPE)
        ft.topk_per_box(ctx, band, bk, sky_box, f1_box, K, out)
        _check(out, s, s_or, key, n_keys, all_in)
        gout = np.zeros_like(out)
        ft.topk_per_box(ctx, band, bk, sky_box, f1_box, K, gout, gate=gate_d, gate_min=0.6)
        _check(gout, s, s_or, key, n_keys, gate >= np.float32(0.6))
        if f1_box >= bank.n_f1:
            ref = np.zeros((n_skyb, bank.n_subbands, K), dtype=ft.CANDIDATE_DTYPE)
            ft.topk_per_skybox(ctx, band, bk, sky_box, K, ref)
            assert np.array_equal(out["template_idx"][:, 0], ref["template_idx"])
        if f1_box >= bank.n_f1 and sky_box >= bank.n_sky:
            ref = np.zeros((bank.n_subbands, K), dtype=ft.CANDIDATE_DTYPE)
            ft.topk_per_band(ctx, band, bk, K, ref)
            assert np.array_equal(out["template_idx"][0, 0], ref["template_idx"])


def test_box_arguments(ctx):
    sfts, bank = _small(n_sft=20, n_f0=20, n_f1=3, n_sky=4, sub=10, seed=10)
    band = H.band_from(ctx, sfts)
    bk = H.bank_from(ctx, band, bank)
    out = np.zeros((4, 3, bank.n_subbands, K), dtype=ft.CANDIDATE_DTYPE)
    for sb, fb in ((0, 1), (1, 0), (-1, 2)):
        with pytest.raises(ft.FtError):
            ft.topk_per_box(ctx, band, bk, sb, fb, K, out)
    with pytest.raises(ft.FtError):
        ft.topk_per_box(ctx, band, bk, 1, 1, 0, out)
    gate = torch.zeros(bank.n_templates, dtype=torch.float32, device="cuda")
    with pytest.raises(ft.FtError):
        ft.topk_per_box(ctx, band, bk, 1, 1, K, out, gate=gate, gate_min=float("nan"))
    # a gate nobody passes leaves every slot empty
    ft.topk_per_box(ctx, band, bk, 1, 1, K, out, gate=gate, gate_min=1.0)
    assert np.all(out["template_idx"] == -1) and np.all(np.isneginf(out["s"]))


def test_full_bank_boxes(ctx, search_cfg):
    """The full search-shaped bank (3.6e7 templates, 24 419 SFTs) in boxes of 100 sky points x
    5 f1 values x one 0.01 Hz sub-band, plain and gated: the CPU selection over the GPU's s of
    every template (from the default launch shape, whose stage lengths may differ from the
    box launch's, so sets may differ only at near-ties and values by FP32 rounding), every
    candidate's s against the oracle, and, on 8 sampled boxes, the sets against the oracle's
    selection over its own s of every template in the box (same near-tie rule)."""
    from tests.test_gpu_parity import assert_s_close

    sfts, bank = search_cfg
    band = H.band_from(ctx, sfts, power_f32=True)
    bk = H.bank_from(ctx, band, bank)
    n = bank.n_templates
    s_d = torch.empty(n, dtype=torch.float32, device="cuda")
    ft.eval_statistic(ctx, band, bk, s_d)
    s = s_d.cpu().numpy().astype(np.float64)
    del s_d
    order = ft.bank_sky_order(bk, bank.n_sky)
    sky_box, f1_box = 100, 5
    n_skyb, n_f1b = -(-bank.n_sky // sky_box), -(-bank.n_f1 // f1_box)
    n_keys = n_skyb * n_f1b * bank.n_subbands
    key = _keys(bank, order, sky_box, f1_box)
    gate = np.random.default_rng(5).uniform(0, 1, n).astype(np.float32)
    gate_d = torch.from_numpy(gate).cuda()
    for g in (None, gate_d):
        out = np.zeros((n_skyb, n_f1b, bank.n_subbands, K), dtype=ft.CANDIDATE_DTYPE)
        ft.topk_per_box(ctx, band, bk, sky_box, f1_box, K, out, gate=g, gate_min=0.5)
        idx = out["template_idx"].reshape(n_keys, K)
        val = out["s"].reshape(n_keys, K)
        t = np.arange(n) if g is None else np.nonzero(gate >= np.float32(0.5))[0]
        c_idx, c_val = oracle.topk_per_key(s[t], key[t], n_keys, K + 1, t)
        for bx in range(n_keys):
            if set(idx[bx].tolist()) != set(c_idx[bx, :K].tolist()):
                kth, nxt = c_val[bx, K - 1], c_val[bx, K]
                assert abs(kth - nxt) < 2e-6 * abs(kth), f"box {bx}"
        flat = idx.ravel()
        assert np.all(flat >= 0)
        assert np.all(np.abs(val.ravel() - s[flat]) <= 2e-6 * np.abs(s[flat]))
        s_or, _ = oracle.statistic(sfts, bank, flat)
        assert_s_close(val.ravel(), s_or)
        # sampled boxes: every template of the box through the oracle
        boxes = np.random.default_rng(9).choice(n_keys, 8, replace=False)
        ts = t[np.isin(key[t], boxes)]
        s_box, _ = oracle.statistic(sfts, bank, ts)
        o_idx, o_val = oracle.topk_per_key(s_box, key[ts], n_keys, K + 1, ts)
        for bx in boxes:
            if set(idx[bx].tolist()) != set(o_idx[bx, :K].tolist()):
                kth, nxt = o_val[bx, K - 1], o_val[bx, K]
                assert abs(kth - nxt) < 2e-6 * abs(kth), f"box {bx} against the oracle"
