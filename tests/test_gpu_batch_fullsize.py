"""The persistent batch at the batching workload's full size (64 bands, 1-year 2-detector
timeline, sky scale 0.1, FP16 storage, the autotuned launch shape the bench times), checked
on outputs the oracle can compute one by one:

* every candidate's s and z equal the oracle's for that template (oracle run on the same
  FP16-rounded power, so storage rounding is common to both; FP32 accumulation tolerance);
* in every sub-band of the checked bands, no sampled template beats the sub-band's k-th
  candidate (a sampled check that the selection kept the loudest);
* candidates sit in their own sub-band, are distinct and sorted by (s desc, index asc).
"""
import math

import numpy as np
import pytest

import ftsynth
import oracle
import paper_2411_18370_b300 as ft

pytestmark = pytest.mark.gpu

K = 10
REL = 2e-6
SKY_SCALE = 0.1
SAMPLES_PER_SUBBAND = 48


@pytest.fixture(scope="module")
def fullsize():
    import torch

    ctx = ft.create(0)
    T = ftsynth.T_SFT
    n_slots = int(round(ftsynth.YEAR_S / T))
    starts = ftsynth.timeline(2, n_slots, T, 0.7, ftsynth.rng(3, 1))
    t_mid = np.concatenate([st + 0.5 * T for st in starts])
    v = np.concatenate([ftsynth.detector_velocity(st + 0.5 * T, X) for X, st in enumerate(starts)])
    n_sft = [len(st) for st in starts]
    N = len(t_mid)
    specs = ftsynth.batch_bands(64, SKY_SCALE)
    # checked bands: the narrowest, the widest and the one with the most sky points
    widths = [sp["n_bins"] for sp in specs]
    skies = [sp["n_sky"] for sp in specs]
    check = sorted({int(np.argmin(widths)), int(np.argmax(widths)), int(np.argmax(skies))})
    bands, banks, host = [], [], {}
    for b, sp in enumerate(specs):
        wl, wh = ftsynth.wings_for(sp["f_hi"], -1e-9, n_slots * T, T)
        W = sp["n_bins"] + wl + wh
        g = torch.Generator(device="cuda")
        g.manual_seed(ftsynth.derive_seed(3, 1000 + b) & ((1 << 63) - 1))
        P = torch.empty((N, W), dtype=torch.float32, device="cuda").exponential_(0.5, generator=g)
        band = ft.load_sfts(ctx, P, t_mid, v, n_sft, sp["k_band"] - wl, T, 0.0, dtype="f16")
        bank_d = ftsynth.Bank(k0=sp["k_band"], n_f0=sp["n_bins"], f1=ftsynth.f1_grid(10, -1e-9, 0.0),
                              sky=ftsynth.fibonacci_sky(sp["n_sky"]), subband_bins=18)
        bank = ft.make_bank(ctx, band, bank_d.k0, bank_d.n_f0, bank_d.f1, bank_d.sky,
                            bank_d.subband_bins)
        if b in check:
            # the power as stored (FP16, round to nearest even), for the oracle
            P16 = P.to(torch.float16).to(torch.float64).cpu().numpy()
            host[b] = (ftsynth.SFTSet(power=P16, t_mid=t_mid, v=v, s_n=np.ones(N), n_sft=n_sft,
                                      k_lo=sp["k_band"] - wl, t_sft=T, t0=0.0), bank_d)
        del P
        bands.append(band)
        banks.append(bank)
    batch = ft.Batch(ctx, bands, banks, K)
    n_sub = sum(b.n_subbands for b in banks)
    out = np.zeros((n_sub, K), dtype=ft.CANDIDATE_DTYPE)
    batch.run(out)
    ctx.check_status()
    offs = np.cumsum([0] + [b.n_subbands for b in banks])
    yield {b: (host[b], out[offs[b]:offs[b + 1]]) for b in check}
    batch.close()
    ctx.close()


def test_candidates_equal_oracle_values(fullsize):
    for b, ((sfts, bank), cand) in fullsize.items():
        t = cand["template_idx"].ravel()
        assert np.all(t >= 0), f"band {b}: empty candidate slot"
        s_or, o_or = oracle.statistic(sfts, bank, t)
        assert np.all(o_or == 0)
        s = cand["s"].ravel().astype(np.float64)
        assert np.all(np.abs(s - s_or) <= REL * np.abs(s_or)), f"band {b}"
        z_or = oracle.zscore(s_or, sfts.n_total)
        _, sig = oracle.mu_sigma(sfts.n_total)
        assert np.all(np.abs(cand["z"].ravel() - z_or) <= REL * np.abs(s_or) / sig + 1e-5)


def test_candidates_are_valid_sorted_lists(fullsize):
    for b, ((sfts, bank), cand) in fullsize.items():
        t = cand["template_idx"]
        sub = (t % bank.n_f0) // bank.subband_bins
        assert np.array_equal(sub, np.repeat(np.arange(bank.n_subbands)[:, None], K, axis=1))
        for row in cand:
            assert len(set(row["template_idx"].tolist())) == K
            key = list(zip((-row["s"]).tolist(), row["template_idx"].tolist()))
            assert key == sorted(key)


def test_no_sampled_template_beats_the_kth(fullsize):
    g = np.random.default_rng(2024)
    for b, ((sfts, bank), cand) in fullsize.items():
        n_per_f0 = bank.n_sky * bank.n_f1
        samp, owner = [], []
        for sb in range(bank.n_subbands):
            j0, j1 = sb * bank.subband_bins, min((sb + 1) * bank.subband_bins, bank.n_f0)
            j = g.integers(j0, j1, SAMPLES_PER_SUBBAND)
            q = g.integers(0, n_per_f0, SAMPLES_PER_SUBBAND)
            samp.append(q * bank.n_f0 + j)
            owner.append(np.full(SAMPLES_PER_SUBBAND, sb))
        samp = np.concatenate(samp)
        owner = np.concatenate(owner)
        s_or, _ = oracle.statistic(sfts, bank, samp)
        kth = cand["s"][:, K - 1].astype(np.float64)
        chosen = set(cand["template_idx"].ravel().tolist())
        for tt, so, sb in zip(samp.tolist(), s_or.tolist(), owner.tolist()):
            if tt in chosen:
                continue
            assert so <= kth[sb] * (1 + REL), f"band {b} sub-band {sb}: template {tt} ({so}) > k-th"
