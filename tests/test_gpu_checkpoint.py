"""Checkpoint / resume of the long-running host loops, with results identical to an
uninterrupted run:

* an injection campaign written in batches: interrupted twice, resumed, and finally read back
  from its batch files alone;
* surrogate training: the whole optimiser state (parameters, Adam moments and step count)
  saved every few passes; interrupted in the first member and again in the second, resumed.
"""
import numpy as np
import pytest

import paper_2411_18370_b300 as ft
from paper_2411_18370_b300 import campaign as C
from paper_2411_18370_b300 import surrogate as SG
from tests import helpers as H
from tests.test_oracle_injection_pins import _short_band

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = ft.create(0)
    yield c
    c.close()


def test_campaign_resumes_from_batches(ctx, tmp_path):
    sfts, bank, D = _short_band(n_slots=300, n_sky=120)
    band = H.band_from(ctx, sfts)
    bk = H.bank_from(ctx, band, bank)
    f_lo = bank.k0 / sfts.t_sft
    f_hi = (bank.k0 + bank.n_f0 - 1) / sfts.t_sft
    args = (ctx, band, bk, D, 300, 4.0, 17, 5000, f_lo, f_hi, 1.0, sfts.t_sft)
    kw = dict(k_sky=16)
    ref = C.run_campaign(*args, **kw)
    ck = str(tmp_path / "campaign")
    with pytest.raises(C.CampaignInterrupted):
        C.run_campaign(*args, checkpoint_dir=ck, batch_runs=64, stop_after=2, **kw)
    with pytest.raises(C.CampaignInterrupted):
        C.run_campaign(*args, checkpoint_dir=ck, batch_runs=64, stop_after=1, **kw)
    got = C.run_campaign(*args, checkpoint_dir=ck, batch_runs=64, **kw)
    for a, b in zip(ref[:3], got[:3]):
        assert np.array_equal(a, b)
    # everything on disk now: nothing left to run
    again = C.run_campaign(*args, checkpoint_dir=ck, batch_runs=64, stop_after=0, **kw)
    assert np.array_equal(again[2], ref[2])


def test_surrogate_training_resumes(ctx, tmp_path):
    g = np.random.default_rng(3)
    F = g.standard_normal((3000, SG.N_FEATURES))
    y = (F[:, 0] + 0.5 * g.standard_normal(3000) > 0).astype(np.float32)
    kw = dict(epochs=12, batch=256, lr=2e-3, seed=5, patience=100)
    ref = SG.Surrogate(ctx, width=32, seed=4, members=2)
    h_ref = ref.fit(F, y, **kw)
    ck = str(tmp_path / "sur.npz")
    s1 = SG.Surrogate(ctx, width=32, seed=4, members=2)
    with pytest.raises(SG.TrainingInterrupted):
        s1.fit(F, y, checkpoint=ck, every=5, stop_after=7, **kw)
    s2 = SG.Surrogate(ctx, width=32, seed=4, members=2)
    with pytest.raises(SG.TrainingInterrupted):
        s2.fit(F, y, checkpoint=ck, every=5, stop_after=13, **kw)
    s3 = SG.Surrogate(ctx, width=32, seed=4, members=2)
    h = s3.fit(F, y, checkpoint=ck, every=5, **kw)
    for a, b in zip(ref.nets, s3.nets):
        assert np.array_equal(a.get_params(), b.get_params())
    for (tr0, va0, be0), (tr1, va1, be1) in zip(h_ref, h):
        assert np.array_equal(tr0, tr1) and np.array_equal(va0, va1) and be0 == be1
    for s in (ref, s1, s2, s3):
        s.close()
