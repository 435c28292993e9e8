"""The surrogate's sensitivity estimate across the 64-band workload (Sec. V p_det, Sec. VI
sigmoid fits), end to end on the GPU: thresholds, a pooled 2e4-injection campaign, the
ensemble trained by the library's kernels, and h0 at 90% p_det on held-out bands.

The surrogate must agree with a high-statistics campaign of each held-out band within 5%,
and beat sigmoid fits that get the same per-band budget (the pooled runs / training bands).
"""
import pytest

import paper_2411_18370_b300 as ft
from paper_2411_18370_b300 import study

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def result():
    ctx = ft.create(0)
    try:
        yield study.run_study(ctx, n_bands=64, sky_scale=0.1, n_held=4, n_noise=2000,
                              n_train=20000, n_ref=8000, members=5)
    finally:
        ctx.close()


def test_surrogate_within_5_percent_of_campaign(result):
    for r in result["held_out_results"]:
        assert abs(r["surrogate_err"]) <= 0.05, r
        # the reference itself is pinned to about 1%
        assert r["ref_c90_rel_sigma"] < 0.015, r


def test_surrogate_beats_equal_budget_per_band_fits(result):
    assert result["per_band_budget"] == 20000 // 60
    assert result["rms_surrogate_err"] < result["rms_per_band_fit_err"]


def test_surrogate_query_is_cheaper_than_a_campaign(result):
    for r in result["held_out_results"]:
        assert r["surrogate_query_s"] < r["ref_campaign_s"]


def test_semi_analytic_estimate_is_a_conservative_comparator(result):
    """Sec. V.A-C: sampling s of the best local template (mismatch from noise-free runs)
    instead of simulating data.  It ignores that the loudest of many partially matching
    templates in noise sits above the best one's mean, so it places the 90 % point a little
    high: within 15 % above the campaign, and the band-to-band pattern is kept (the ratio to
    the campaign varies by less than 5 % across the held-out bands)."""
    errs = [r["semi_analytic_err"] for r in result["held_out_results"]]
    assert all(0.0 < e < 0.15 for e in errs), errs
    assert max(errs) - min(errs) < 0.05, errs
    for r in result["held_out_results"]:
        assert r["semi_analytic_s"] < r["ref_campaign_s"]
