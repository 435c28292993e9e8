"""The batching pattern: many uneven bands in one persistent, graph-captured launch.

Per band, the candidates must equal the oracle's (near-tie exemption) and those of the
single-band path; graph replays must be bit-identical; the autotuned and the explicit
launch shapes must agree on the candidate sets.
"""
import numpy as np
import pytest

import ftsynth
import oracle
import paper_2411_18370_b300 as ft
from tests import helpers as H
from tests.test_gpu_parity import assert_topk

pytestmark = pytest.mark.gpu

K = 10


@pytest.fixture(scope="module")
def ctx():
    c = ft.create(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def bands_small():
    """Six bands of the batching workload (widths 90..900 bins, 100..500 Hz), a short
    timeline (1200 slots) and at most 60 sky points each, so the oracle finishes."""
    return ftsynth.batch_workload(n_bands=64, n_slots=1200, max_sky=60, bands=[0, 5, 17, 29, 42, 63])


def _split(cand, banks):
    out, off = [], 0
    for bk in banks:
        out.append(cand[off:off + bk.n_subbands])
        off += bk.n_subbands
    return out


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_batch_matches_oracle_and_single_band_path(ctx, bands_small, dtype):
    bands = [H.band_from(ctx, s, dtype=dtype) for s, _ in bands_small]
    banks = [H.bank_from(ctx, b, bk) for b, (_, bk) in zip(bands, bands_small)]
    assert all(b.window_safe for b in banks)
    batch = ft.Batch(ctx, bands, banks, K)
    n_sub = sum(b.n_subbands for b in banks)
    out = np.zeros((n_sub, K), dtype=ft.CANDIDATE_DTYPE)
    batch.run(out)
    again = np.zeros_like(out)
    batch.run(again)
    assert np.array_equal(out.view(np.uint8), again.view(np.uint8))  # graph replay is deterministic
    for (sfts, bank), got, band, bk in zip(bands_small, _split(out, banks), bands, banks):
        s_or, _ = oracle.statistic(sfts, bank)
        assert_topk(got["template_idx"], got["s"], s_or, bank, K)
        single = np.zeros((bank.n_subbands, K), dtype=ft.CANDIDATE_DTYPE)
        ft.topk_per_band(ctx, band, bk, K, single)
        # same candidates up to near-ties, same values within FP32 accumulation-order noise
        ok = got["template_idx"] >= 0
        same = got["template_idx"] == single["template_idx"]
        rel = np.abs(got["s"].astype(np.float64) - single["s"]) / np.abs(single["s"])
        assert np.all(rel[ok & same] < 1e-6)
        if dtype == "f32":
            np.testing.assert_allclose(got["s"][ok], s_or[got["template_idx"][ok]], rtol=1e-6)
    batch.close()


def test_batch_explicit_shapes_agree(ctx, bands_small):
    bands = [H.band_from(ctx, s, dtype="f16") for s, _ in bands_small[:3]]
    banks = [H.bank_from(ctx, b, bk) for b, (_, bk) in zip(bands, bands_small[:3])]
    n_sub = sum(b.n_subbands for b in banks)
    res = []
    for tile, stages in ((128, 2), (192, 3), (256, 2)):
        batch = ft.Batch(ctx, bands, banks, K, tile_f0=tile, stages=stages)
        assert batch.tile_f0 == tile and batch.stages == stages
        out = np.zeros((n_sub, K), dtype=ft.CANDIDATE_DTYPE)
        batch.run(out)
        res.append(out)
        batch.close()
    for (sfts, bank), *outs in zip(bands_small[:3], *[_split(r, banks) for r in res]):
        s_or, _ = oracle.statistic(sfts, bank)
        for got in outs:
            assert_topk(got["template_idx"], got["s"], s_or, bank, K)


def test_batch_integer_power_exact(ctx, bands_small):
    """Integer powers: every band's candidate values are exact sums in the batch too."""
    subset = bands_small[:4]
    g = np.random.default_rng(5)
    data = []
    for sfts, bank in subset:
        P = g.integers(0, 64, sfts.power.shape).astype(np.float64)
        sx = ftsynth.SFTSet(power=P, t_mid=sfts.t_mid, v=sfts.v, s_n=sfts.s_n, n_sft=sfts.n_sft,
                            k_lo=sfts.k_lo, t_sft=sfts.t_sft, t0=sfts.t0)
        data.append((sx, bank))
    bands = [H.band_from(ctx, s, dtype="bf16") for s, _ in data]
    banks = [H.bank_from(ctx, b, bk) for b, (_, bk) in zip(bands, data)]
    n_sub = sum(b.n_subbands for b in banks)
    out = np.zeros((n_sub, K), dtype=ft.CANDIDATE_DTYPE)
    ft.Batch(ctx, bands, banks, K).run(out)
    for (sfts, bank), got in zip(data, _split(out, banks)):
        s_or, _ = oracle.statistic(sfts, bank)
        ok = got["template_idx"] >= 0
        assert np.array_equal(got["s"][ok].astype(np.float64), s_or[got["template_idx"][ok]])
        assert_topk(got["template_idx"], got["s"], s_or, bank, K)


def test_batch_rejects_mixed_inputs(ctx, bands_small):
    (s0, b0), (s1, b1) = bands_small[:2]
    band0 = H.band_from(ctx, s0, dtype="f32")
    band1 = H.band_from(ctx, s1, dtype="f16")
    bk0 = H.bank_from(ctx, band0, b0)
    bk1 = H.bank_from(ctx, band1, b1)
    with pytest.raises(ft.FtError) as e:
        ft.Batch(ctx, [band0, band1], [bk0, bk1], K)
    assert e.value.code == -1
    with pytest.raises(ft.FtError) as e:
        ft.Batch(ctx, [band0, band0], [bk0, bk1], K)
    assert e.value.code == -1
