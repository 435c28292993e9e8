"""Failure detection without a GPU fault: a bounded wait that nothing completes gives up
after about a second, the kernel records the timeout in the context's status word and
returns; the host reports FT_ERR_TIMEOUT, the status is cleared, and the same context then
runs a search correctly."""
import numpy as np
import pytest

import ftsynth
import oracle
import paper_2411_18370_b300 as ft
from tests import helpers as H

pytestmark = pytest.mark.gpu

FT_ERR_TIMEOUT = -4


def test_bounded_wait_times_out_and_context_survives():
    ctx = ft.create(0)
    rc, waited = ft.selftest_bounded_wait(ctx)
    assert rc == FT_ERR_TIMEOUT
    assert 0.9 < waited < 5.0
    ctx.check_status()  # the status word was cleared by the report
    sfts, bank, _ = ftsynth.tiny_workload("auto")
    band = H.band_from(ctx, sfts)
    bk = H.bank_from(ctx, band, bank)
    s, _, _ = H.eval_host(ctx, band, bk, bank.n_templates)
    s_or, _ = oracle.statistic(sfts, bank)
    assert np.all(np.abs(s - s_or) <= 1e-6 * s_or)
    bk.close()
    band.close()
    ctx.close()
