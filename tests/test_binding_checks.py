"""The binding refuses, before calling the library, any output buffer smaller than what the
call writes (the kernels would write past it on the device, and a host copy past the end of
a host array), a gate of the wrong kind, and a sky count that is not the bank's.  No GPU is
needed: the checks fire before the first library call, so stand-in handles do."""
import types

import numpy as np
import pytest

import paper_2411_18370_b300 as ft

CTX = types.SimpleNamespace(handle=None)
BAND = types.SimpleNamespace(handle=None, n_sft=50)
BANK = types.SimpleNamespace(handle=None, n_templates=1000, n_subbands=4, n_f0=10, n_f1=5, n_sky=20)
BBANK = types.SimpleNamespace(handle=None, n_templates=600, n_boxes=3)


def _cands(n):
    return np.zeros(n, dtype=ft.CANDIDATE_DTYPE)


@pytest.mark.parametrize("call,n_cand", [
    (lambda out: ft.topk_per_band(CTX, BAND, BANK, 5, out), 4 * 5),
    (lambda out: ft.topk_per_band_noalloc(CTX, BAND, BANK, 5, out), 4 * 5),
    (lambda out: ft.topk_per_skybox(CTX, BAND, BANK, 7, 5, out), 3 * 4 * 5),
    (lambda out: ft.topk_per_box(CTX, BAND, BANK, 7, 2, 5, out), 3 * 3 * 4 * 5),
    (lambda out: ft.binary_topk_per_box(CTX, BAND, BBANK, 5, out), 3 * 5),
])
def test_undersized_candidate_buffers(call, n_cand):
    with pytest.raises(ValueError, match="buffer of"):
        call(_cands(3))
    # one byte short of the size the call writes
    with pytest.raises(ValueError, match="buffer of"):
        call(np.zeros(16 * n_cand - 1, np.uint8))


def test_box_sizes_count_ceil_boxes():
    # 20 sky points in boxes of 7 -> 3 sky boxes; 5 f1 in boxes of 2 -> 3 f1 boxes
    need = 3 * 3 * BANK.n_subbands * 5
    with pytest.raises(ValueError):
        ft.topk_per_box(CTX, BAND, BANK, 7, 2, 5, _cands(need - 1))
    need = 3 * BANK.n_subbands * 5
    with pytest.raises(ValueError):
        ft.topk_per_skybox(CTX, BAND, BANK, 7, 5, _cands(need - 1))


def test_undersized_statistic_and_bin_buffers():
    with pytest.raises(ValueError, match="s_out"):
        ft.eval_statistic(CTX, BAND, BANK, np.empty(999, np.float32))
    with pytest.raises(ValueError, match="z_out"):
        ft.eval_statistic(CTX, BAND, BANK, np.empty(1000, np.float32), np.empty(10, np.float32))
    with pytest.raises(ValueError, match="n_oob_out"):
        ft.binary_eval(CTX, BAND, BBANK, 0, 100, np.empty(100, np.float32), None, np.empty(99, np.int32))
    t = np.arange(4, dtype=np.int64)
    with pytest.raises(ValueError, match="track_bins out"):
        ft.track_bins(CTX, BAND, BANK, t, np.empty((4, 49), np.int32))
    with pytest.raises(ValueError, match="binary_track_bins out"):
        ft.binary_track_bins(CTX, BAND, BBANK, t, np.empty((3, 50), np.int32))
    with pytest.raises(ValueError, match="int64"):
        ft.track_bins(CTX, BAND, BANK, t.astype(np.int32), np.empty((4, 50), np.int32))


def test_gate_must_be_a_device_float_tensor_and_sky_count_the_banks():
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError, match="CUDA tensor"):
        ft.topk_per_band_gated(CTX, BAND, BANK, 5, torch.zeros(1000), 0.0, _cands(20))
    with pytest.raises(ValueError, match="CUDA tensor"):
        ft.binary_topk_per_box_gated(CTX, BAND, BBANK, 5, np.zeros(600, np.float32), 0.0, _cands(15))
    with pytest.raises(ValueError, match="sky points"):
        ft.bank_sky_order(BANK, 21)
