"""Host-side fault injection: corrupt or inconsistent inputs come back as error codes (never a
GPU fault), and the context keeps working afterwards."""
import dataclasses

import numpy as np
import pytest

import ftsynth
import oracle
import paper_2411_18370_b300 as ft
from tests import helpers as H

pytestmark = pytest.mark.gpu

ARG, RANGE = -1, -5


@pytest.fixture(scope="module")
def ctx():
    c = ft.create(0)
    yield c
    c.close()


def _code(fn):
    with pytest.raises(ft.FtError) as e:
        fn()
    return e.value.code


def test_corrupt_sft_inputs(ctx):
    sfts, bank, _ = ftsynth.tiny_workload("auto")

    def load(**kw):
        s = dataclasses.replace(sfts, **{k: v for k, v in kw.items() if k in ("power", "t_mid", "v", "s_n")})
        return lambda: ft.load_sfts(ctx, s.power, s.t_mid, s.v, kw.get("n_sft", s.n_sft), s.k_lo,
                                    kw.get("t_sft", s.t_sft), s.t0, s_n=s.s_n)

    zero_sn = sfts.s_n.copy()
    zero_sn[7] = 0.0
    assert _code(load(s_n=zero_sn)) == ARG
    neg_sn = sfts.s_n.copy()
    neg_sn[0] = -1.0
    assert _code(load(s_n=neg_sn)) == ARG
    nan_t = sfts.t_mid.copy()
    nan_t[3] = np.nan
    assert _code(load(t_mid=nan_t)) == ARG
    inf_p = sfts.power.copy()
    inf_p[2, 4] = np.inf
    assert _code(load(power=inf_p)) == ARG
    assert _code(load(t_sft=0.0)) == ARG
    assert _code(load(t_sft=-1800.0)) == ARG
    assert _code(load(v=sfts.v * 50)) == RANGE          # |v/c| far beyond any detector
    with pytest.raises((ft.FtError, ValueError)):
        load(n_sft=[sfts.n_total + 5])()                 # counts that do not match the rows


def test_corrupt_bank_inputs(ctx):
    sfts, bank, _ = ftsynth.tiny_workload("auto")
    band = H.band_from(ctx, sfts)

    def mk(**kw):
        d = dict(k0=bank.k0, n_f0=bank.n_f0, f1=bank.f1, sky=bank.sky, subband_bins=bank.subband_bins)
        d.update(kw)
        return lambda: ft.make_bank(ctx, band, d["k0"], d["n_f0"], d["f1"], d["sky"], d["subband_bins"])

    assert _code(mk(n_f0=0)) == RANGE
    assert _code(mk(subband_bins=0)) == ARG
    assert _code(mk(f1=np.array([np.nan]))) == ARG
    assert _code(mk(sky=bank.sky * 1.01)) == ARG        # not unit vectors
    assert _code(mk(sky=np.zeros((0, 3)))) == ARG
    # the context still evaluates correctly
    bk = H.bank_from(ctx, band, bank)
    s, _, _ = H.eval_host(ctx, band, bk, bank.n_templates)
    s_or, _ = oracle.statistic(sfts, bank)
    assert np.all(np.abs(s - s_or) <= 1e-6 * s_or)


def test_binding_refuses_bad_gates_and_short_device_buffers(ctx):
    """A gate must be a float32 CUDA tensor of one value per template, and a device output
    buffer must hold what the call writes; the binding refuses both before the library runs,
    and the context still searches correctly afterwards."""
    import torch

    sfts, bank, _ = ftsynth.tiny_workload("auto")
    band = H.band_from(ctx, sfts)
    bk = H.bank_from(ctx, band, bank)
    n = bank.n_templates
    out = torch.empty(bank.n_subbands * 5 * 16, dtype=torch.uint8, device="cuda")
    for bad in (torch.zeros(n, dtype=torch.float64, device="cuda"),
                torch.zeros(n - 1, dtype=torch.float32, device="cuda")):
        with pytest.raises(ValueError):
            ft.topk_per_band_gated(ctx, band, bk, 5, bad, 0.0, out)
        with pytest.raises(ValueError):
            ft.topk_per_box(ctx, band, bk, 4, 1, 5, torch.empty(10 ** 6, dtype=torch.uint8, device="cuda"),
                            gate=bad)
    with pytest.raises(ValueError):
        ft.topk_per_band(ctx, band, bk, 5, out[:-1])
    with pytest.raises(ValueError):
        ft.eval_statistic(ctx, band, bk, torch.empty(n - 1, dtype=torch.float32, device="cuda"))
    ft.topk_per_band(ctx, band, bk, 5, out)
    torch.cuda.synchronize()
    idx, _, _ = ft.decode_candidates(out, bank.n_subbands, 5)
    s, _, _ = H.eval_host(ctx, band, bk, n)
    s_or, _ = oracle.statistic(sfts, bank)
    assert np.all(np.abs(s - s_or) <= 1e-6 * s_or)
    c_idx, _ = oracle.topk_per_subband(s.astype(np.float64), bank, 5)
    assert np.array_equal(idx, c_idx)
