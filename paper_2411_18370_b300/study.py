"""The sensitivity study across many bands: per-band thresholds, a pooled injection campaign,
the p_det surrogate trained on it, and h0 at 90% p_det on held-out bands from (a) the
surrogate, (b) per-band sigmoid fits with the same per-band injection budget and (c) a
high-statistics campaign of the held-out band itself (the reference).

Sec. V defines the sensitivity as the amplitude at which a fraction p of the signal
population is detected above a threshold set by noise-only searches; Sec. VI estimates it
band by band from sigmoid fits to injection outcomes.  The surrogate replaces the per-band
campaign by one network that takes the band's noise level and duty cycle as inputs, so a
new band costs a query instead of a campaign.  Everything that touches data (the simulated
SFT bins, the local searches, the network's training and inference) runs in the library's
CUDA kernels; this module is the bookkeeping around them.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import campaign as C
from . import semianalytic as SA
from . import surrogate as SG

# amplitudes of the training and per-band campaigns: log-uniform c = h0 / sqrt(S_ref/T_SFT)
C_RANGE = (0.3, 30.0)


def _load(ctx, bands, T):
    import ftsynth
    from . import load_sfts, make_bank

    objs = []
    for bd in bands:
        sp = bd["spec"]
        N = len(bd["t_mid"])
        band = load_sfts(ctx, np.zeros((N, 1), np.float32), bd["t_mid"], bd["v"], bd["n_sft"],
                         sp["k_band"], T, 0.0, dtype="f32", s_n=bd["s_n"])
        bank = make_bank(ctx, band, sp["k_band"], sp["n_bins"], ftsynth.f1_grid(10, -1e-9, 0.0),
                         ftsynth.fibonacci_sky(sp["n_sky"]), 18)
        objs.append((band, bank))
    return objs


def run_study(ctx, n_bands=64, sky_scale=0.1, n_held=4, n_noise=2000, n_train=20000,
              n_ref=8000, members=5, epochs=200, k_sky=64, n_semi=4000):
    import ftsynth

    T = ftsynth.T_SFT
    bands = ftsynth.surrogate_bands(n_bands, sky_scale)
    held = list(range(0, n_bands, max(1, n_bands // n_held)))[:n_held]
    train_bands = [b for b in range(n_bands) if b not in held]
    kw = dict(k_sky=k_sky, half_f0=2, half_window=160)
    t0 = time.perf_counter()
    objs = _load(ctx, bands, T)
    timing = {"setup_s": time.perf_counter() - t0}
    run_id = 0

    def frange(b):
        sp = bands[b]["spec"]
        return sp["k_band"] / T, (sp["k_band"] + sp["n_bins"] - 1) / T

    def campaign(b, n, seed, c_range):
        nonlocal run_id
        band, bank = objs[b]
        lo, hi = frange(b)
        lc, det, _, inj = C.run_campaign(ctx, band, bank, bands[b]["D"], n, taus[b], seed, run_id,
                                         lo, hi, bands[b]["s_ref"], T, c_range=c_range, **kw)
        run_id += n
        return lc, det, inj

    # 1. thresholds: 1% false alarm from noise-only local searches, per band
    t0 = time.perf_counter()
    taus = []
    for b, (band, bank) in enumerate(objs):
        lo, hi = frange(b)
        tau, _ = C.noise_threshold(ctx, band, bank, bands[b]["D"], n_noise, 1 + b, run_id, lo, hi,
                                   **kw)
        run_id += n_noise
        taus.append(tau)
    timing["thresholds_s"] = time.perf_counter() - t0

    # 2. pooled training campaign over the training bands: n_train injections in all, the
    # same number per band
    t0 = time.perf_counter()
    per_band = max(1, n_train // len(train_bands))
    feats, labels = [], []
    for b in train_bands:
        lo, hi = frange(b)
        lc, det, inj = campaign(b, per_band, 5000 + b, C_RANGE)
        feats.append(SG.features(lc, np.full(per_band, math.log10(bands[b]["s_ref"])),
                                 np.full(per_band, bands[b]["duty"]), inj["n"],
                                 (inj["f0"] - lo) / (hi - lo), inj["f1"], inj["cosi"], inj["psi"],
                                 np.full(per_band, taus[b])))
        labels.append(det)
    F = np.concatenate(feats)
    y = np.concatenate(labels)
    timing["training_campaign_s"] = time.perf_counter() - t0

    # 3. surrogate training on the GPU
    t0 = time.perf_counter()
    sur = SG.Surrogate(ctx, width=128, seed=7, members=members)
    hist = sur.fit(F, y, epochs=epochs, batch=1024, lr=2e-3, seed=3)
    timing["surrogate_training_s"] = time.perf_counter() - t0

    # 4. held-out bands
    rows = []
    g = np.random.default_rng(99)
    g_sa = np.random.default_rng(199)  # the semi-analytic draws, apart from the others
    for b in held:
        lo, hi = frange(b)
        # reference: a rough fit over a wide range, then 3/4 of the budget within +-0.12 dex
        # of its 90% point, and the 90% point from local fits over all of them
        t0 = time.perf_counter()
        n1 = n_ref // 4
        lc1, det1, _ = campaign(b, n1, 7000 + b, (0.2, 5.0))
        x_rough = C.fit_sigmoid(lc1, det1).x_at(0.9)
        lc2, det2, _ = campaign(b, n_ref - n1, 7500 + b,
                                (10 ** (x_rough - 0.12), 10 ** (x_rough + 0.12)))
        x_ref, s_ref, n_used = C.local_x_at(np.concatenate([lc1, lc2]),
                                            np.concatenate([det1, det2]), 0.9, x_rough)
        t_ref = time.perf_counter() - t0
        # per-band fit: as many injections as a training band contributes, fitted alone
        lc, det, _ = campaign(b, per_band, 8000 + b, C_RANGE)
        x_b = C.fit_sigmoid(lc, det).x_at(0.9)
        inj_pop, _ = C.draw_population(2000, lo, hi, g)
        pop = dict(n=inj_pop["n"], f0_frac=(inj_pop["f0"] - lo) / (hi - lo), f1=inj_pop["f1"],
                   cosi=inj_pop["cosi"], psi=inj_pop["psi"])
        t0 = time.perf_counter()
        x_sur = sur.log10_c_at(0.9, math.log10(bands[b]["s_ref"]), bands[b]["duty"], taus[b],
                               pop)
        t_sur = time.perf_counter() - t0
        # semi-analytic estimate (Sec. V.A-C) from its own population draws
        t0 = time.perf_counter()
        band, bank = objs[b]
        sa_pop, _ = C.draw_population(n_semi, lo, hi, g_sa)
        # (noise-free runs: their run ids draw no noise; kept apart from the campaigns' ids)
        est = SA.build(ctx, band, bank, bands[b]["D"], sa_pop, taus[b], bands[b]["s_ref"], T,
                       seed=9000 + b, first_run_id=(1 << 40) + b * n_semi, **kw)
        x_sa = est.log10_c_at(0.9)
        t_sa = time.perf_counter() - t0
        rows.append({"band": b, "f_start_hz": bands[b]["spec"]["k_band"] / T,
                     "duty": bands[b]["duty"], "log10_S": math.log10(bands[b]["s_ref"]),
                     "tau": taus[b], "ref_c90": 10 ** x_ref,
                     "ref_c90_rel_sigma": math.log(10) * s_ref, "ref_local_samples": n_used,
                     "surrogate_c90": 10 ** x_sur, "per_band_fit_c90": 10 ** x_b,
                     "surrogate_err": 10 ** (x_sur - x_ref) - 1,
                     "per_band_fit_err": 10 ** (x_b - x_ref) - 1,
                     "semi_analytic_c90": 10 ** x_sa, "semi_analytic_err": 10 ** (x_sa - x_ref) - 1,
                     "semi_analytic_mean_mismatch": float(np.mean(est.m)),
                     "ref_campaign_s": t_ref, "surrogate_query_s": t_sur, "semi_analytic_s": t_sa})
    sur.close()
    return {
        "bands": n_bands, "held_out": held, "n_noise_per_band": n_noise,
        "n_train": int(len(y)), "n_ref_per_heldout": n_ref,
        "per_band_budget": per_band, "members": members,
        "train_detected_frac": float(y.mean()),
        "best_epochs": [int(h[2]) for h in hist],
        "val_loss_at_best": [float(h[1][h[2]]) for h in hist],
        "timing": timing, "held_out_results": rows,
        "max_abs_surrogate_err": max(abs(r["surrogate_err"]) for r in rows),
        "rms_surrogate_err": math.sqrt(np.mean([r["surrogate_err"] ** 2 for r in rows])),
        "max_abs_per_band_fit_err": max(abs(r["per_band_fit_err"]) for r in rows),
        "rms_per_band_fit_err": math.sqrt(np.mean([r["per_band_fit_err"] ** 2 for r in rows])),
        "max_abs_semi_analytic_err": max(abs(r["semi_analytic_err"]) for r in rows),
        "rms_semi_analytic_err": math.sqrt(np.mean([r["semi_analytic_err"] ** 2 for r in rows])),
        "n_semi_analytic_draws": n_semi,
        "h0_unit": "sqrt(S_ref / T_SFT)",
    }
