"""Ahead-of-time boxes across the sky for the regular bank (Sec. IV.B): box (x, b) = the
templates of sub-band b whose sky point sits at positions x sky_box .. (x + 1) sky_box - 1 of
the bank's sky order, every f1.  Checked against the CPU selection over the GPU's own values
(exact) and the oracle's values (near-tie exemption), for ragged sky counts, box sizes that
do and do not divide the CTA's sky group, both kernels and FP32 / FP16 storage; one box
holding the whole sky equals the per-sub-band selection; the boxes are compact on the sky."""
import numpy as np
import pytest

import oracle
import paper_2411_18370_b300 as ft
from tests import helpers as H
from tests.test_gpu_parity import _small

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = ft.create(0)
    yield c
    c.close()


def _keys(bank, order, sky_box):
    pos = np.empty(bank.n_sky, np.int64)
    pos[order] = np.arange(bank.n_sky)
    t = np.arange(bank.n_templates)
    i_sky = t // (bank.n_f1 * bank.n_f0)
    j = t % bank.n_f0
    return (pos[i_sky] // sky_box) * bank.n_subbands + j // bank.subband_bins


@pytest.mark.parametrize("dtype", ["f32", "f16"])
@pytest.mark.parametrize("wings", [30, 2])
def test_sky_boxes(ctx, dtype, wings):
    sfts, bank = _small(n_sft=90, n_f0=60, n_f1=5, n_sky=37, sub=11, W=120 if wings == 30 else 64,
                        wings=wings, seed=7)
    band = H.band_from(ctx, sfts, dtype=dtype)
    bk = H.bank_from(ctx, band, bank)
    assert bk.window_safe == (wings == 30)
    order = ft.bank_sky_order(bk, bank.n_sky)
    assert np.array_equal(np.sort(order), np.arange(bank.n_sky))
    s, _, _ = H.eval_host(ctx, band, bk, bank.n_templates)
    s_or, _ = oracle.statistic(sfts if dtype == "f32" else
                               type(sfts)(**{**sfts.__dict__, "power": sfts.power.astype(np.float16).astype(np.float64)}),
                               bank)
    k = 3
    for sky_box in (1, 6, 8, 37, 100):
        n_box = -(-bank.n_sky // sky_box)
        out = np.zeros((n_box, bank.n_subbands, k), dtype=ft.CANDIDATE_DTYPE)
        ft.topk_per_skybox(ctx, band, bk, sky_box, k, out)
        key = _keys(bank, order, sky_box)
        n_keys = n_box * bank.n_subbands
        idx = out["template_idx"].reshape(n_keys, k)
        val = out["s"].reshape(n_keys, k)
        c_idx, c_val = oracle.topk_per_key(s.astype(np.float64), key, n_keys, k)
        assert np.array_equal(idx, c_idx), f"sky_box {sky_box}"
        ok = idx >= 0
        assert np.array_equal(val[ok].astype(np.float64), c_val[ok])
        o_idx, o_val = oracle.topk_per_key(s_or, key, n_keys, k + 1)
        for b in range(n_keys):
            got = set(int(x) for x in idx[b] if x >= 0)
            want = set(int(x) for x in o_idx[b, :k] if x >= 0)
            if got != want:
                kth, nxt = o_val[b, k - 1], o_val[b, k]
                assert np.isfinite(nxt) and abs(kth - nxt) < 2e-6 * abs(kth)
        if sky_box >= bank.n_sky:
            ref = np.zeros((bank.n_subbands, k), dtype=ft.CANDIDATE_DTYPE)
            ft.topk_per_band(ctx, band, bk, k, ref)
            assert np.array_equal(out["template_idx"][0], ref["template_idx"])


def test_sky_boxes_are_compact(ctx):
    sfts, bank = _small(n_sft=20, n_f0=10, n_f1=2, n_sky=400, sub=10, seed=8)
    band = H.band_from(ctx, sfts)
    bk = H.bank_from(ctx, band, bank)
    order = ft.bank_sky_order(bk, bank.n_sky)
    sky = bank.sky[order]
    box = 8

    def spread(pts):
        return np.mean([np.max(np.linalg.norm(g[:, None] - g[None], axis=2))
                        for g in np.split(pts[: len(pts) // box * box], len(pts) // box)])

    # the order follows a Hilbert curve over the equal-area map of the sphere: runs of 8
    # points are patches well under half as wide as random groups of 8 (0.37 of them here)
    rnd = bank.sky[np.random.default_rng(1).permutation(bank.n_sky)]
    assert spread(sky) < 0.45 * spread(rnd)
