"""ft_topk_per_band_noalloc against ft_topk_per_band.

The no-allocation entry point serves callers that cannot let the library allocate device
memory during a call (device memory owned by another allocator or fixed at start-up,
latency-critical loops).  It must return the same candidates as the allocating entry point,
call after call, although its fixed scratch array keeps the previous call's contents.
"""
import numpy as np
import pytest

import ftsynth
import paper_2411_18370_b300 as ft

pytestmark = pytest.mark.gpu

REL = 1e-6


@pytest.fixture(scope="module")
def search():
    ctx = ft.create(0)
    sfts, bank = ftsynth.search_workload()
    band = ft.load_sfts(ctx, sfts.power.astype(np.float32), sfts.t_mid, sfts.v, sfts.n_sft,
                        sfts.k_lo, sfts.t_sft, sfts.t0, dtype="f32")
    bk = ft.make_bank(ctx, band, bank.k0, bank.n_f0, bank.f1, bank.sky, bank.subband_bins)
    yield ctx, band, bk, bank
    bk.close()
    band.close()
    ctx.close()


def _same(a, b):
    assert np.array_equal(a["template_idx"], b["template_idx"])
    ok = a["template_idx"] >= 0
    sa, sb = a["s"][ok].astype(np.float64), b["s"][ok].astype(np.float64)
    assert np.all(np.abs(sa - sb) <= REL * np.abs(sb))
    za, zb = a["z"][ok].astype(np.float64), b["z"][ok].astype(np.float64)
    assert np.all(np.abs(za - zb) <= REL * np.abs(sb) + 1e-6)


def test_noalloc_matches_allocating_entry_point_twice(search):
    import torch

    ctx, band, bk, bank = search
    k = 10
    ref = np.zeros((bank.n_subbands, k), dtype=ft.CANDIDATE_DTYPE)
    ft.topk_per_band(ctx, band, bk, k, ref)
    assert np.all(ref["template_idx"] >= 0)
    # two calls in a row with host output, then two with device output
    for _ in range(2):
        got = np.zeros_like(ref)
        ft.topk_per_band_noalloc(ctx, band, bk, k, got)
        _same(got, ref)
    for _ in range(2):
        dev = torch.zeros(bank.n_subbands * k * 16, dtype=torch.uint8, device="cuda")
        ft.topk_per_band_noalloc(ctx, band, bk, k, dev)
        torch.cuda.synchronize()
        ctx.check_status()
        got = np.frombuffer(dev.cpu().numpy().tobytes(), dtype=ft.CANDIDATE_DTYPE).reshape(ref.shape)
        _same(got, ref)


def test_noalloc_allocates_nothing():
    """On a context whose search scratch was never grown, two no-allocation searches (host
    output, then device output) leave its scratch at zero bytes and its staging buffer as it
    was: the candidate lists live in the library's fixed array, not in memory allocated during
    the call."""
    import torch

    ctx = ft.create(0)
    try:
        sfts, bank, _ = ftsynth.tiny_workload("auto")
        band = ft.load_sfts(ctx, sfts.power.astype(np.float32), sfts.t_mid, sfts.v, sfts.n_sft,
                            sfts.k_lo, sfts.t_sft, sfts.t0, dtype="f32")
        bk = ft.make_bank(ctx, band, bank.k0, bank.n_f0, bank.f1, bank.sky, bank.subband_bins)
        before = ctx.memory()
        assert before[0] == 0, before
        got = np.zeros((bank.n_subbands, 5), dtype=ft.CANDIDATE_DTYPE)
        ft.topk_per_band_noalloc(ctx, band, bk, 5, got)
        dev = torch.zeros(bank.n_subbands * 5 * 16, dtype=torch.uint8, device="cuda")
        ft.topk_per_band_noalloc(ctx, band, bk, 5, dev)
        torch.cuda.synchronize()
        assert ctx.memory() == before
        # the allocating entry point, for contrast, grows the context's scratch
        ref = np.zeros_like(got)
        ft.topk_per_band(ctx, band, bk, 5, ref)
        assert ctx.memory()[0] > 0
        _same(got, ref)
        bk.close()
        band.close()
    finally:
        ctx.close()


def test_noalloc_rejects_requests_beyond_its_scratch(search):
    ctx, band, bk, bank = search
    out = np.zeros((bank.n_subbands, 32), dtype=ft.CANDIDATE_DTYPE)
    with pytest.raises(ft.FtError) as e:
        ft.topk_per_band_noalloc(ctx, band, bk, 32, out)
    assert e.value.code == -5 and "bytes" in str(e.value)
