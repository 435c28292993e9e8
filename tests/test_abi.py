"""CPU-side checks of the C ABI: the library loads, exports every declared entry point,
and its host-only logic behaves (no kernel is launched here)."""
import ctypes
import os
import re

import numpy as np
import pytest

import ftsynth
import paper_2411_18370_b300 as ft
from paper_2411_18370_b300 import build as ftbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"FT_API\s+[\w\s\*]*?\b(ft_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def built():
    return ftbuild.build()


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("ft_load_sfts", "ft_make_bank", "ft_eval_statistic", "ft_topk_per_band",
                 "ft_required_wings", "ft_track_bins", "ft_create", "ft_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(built):
    L = ctypes.CDLL(built)
    for name in sorted(declared_symbols()):
        assert hasattr(L, name), name


def test_abi_version(built):
    assert ft.abi_version() == 1


def test_create_without_device_is_an_error_not_a_crash(built):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(ft.FtError):
        ft.create(0)
    assert ft.lib().ft_last_error().decode() != ""


def test_required_wings_cover_search_tracks(built):
    """Host-only conservative extent: the config-1 wings sized from |v| <= v_max are enough."""
    sfts, bank = ftsynth.search_workload(n_sky=16)
    lo, hi = ft.required_wings(sfts.n_sft, sfts.t_mid, sfts.v, sfts.t_sft, sfts.t0, bank.k0,
                               bank.n_f0, bank.f1, bank.sky, bank.subband_bins)
    wl = bank.k0 - sfts.k_lo
    wh = sfts.k_lo + sfts.n_bins - 1 - (bank.k0 + bank.n_f0 - 1)
    assert 0 < lo <= wl and 0 < hi <= wh
    # the literal 10-bin wings of the tiny workload are NOT enough
    s0, b0, _ = ftsynth.tiny_workload("literal")
    lo0, hi0 = ft.required_wings(s0.n_sft, s0.t_mid, s0.v, s0.t_sft, s0.t0, b0.k0, b0.n_f0, b0.f1,
                                 b0.sky, b0.subband_bins)
    assert lo0 > 10 and hi0 > 10


def test_required_wings_rejects_bad_bank(built):
    sfts, bank = ftsynth.search_workload(n_sky=4)
    with pytest.raises(ft.FtError) as e:
        ft.required_wings(sfts.n_sft, sfts.t_mid, sfts.v, sfts.t_sft, sfts.t0, bank.k0, bank.n_f0,
                          bank.f1, bank.sky * 2.0, bank.subband_bins)
    assert e.value.code == -1
    with pytest.raises(ft.FtError) as e:
        ft.required_wings(sfts.n_sft, sfts.t_mid, sfts.v, sfts.t_sft, sfts.t0, bank.k0, 0,
                          bank.f1, bank.sky, bank.subband_bins)
    assert e.value.code == -5


def test_candidate_dtype_is_16_bytes():
    assert ft.CANDIDATE_DTYPE.itemsize == 16


def test_cos_screen_check_refuses_null_arguments(built):
    """The cosine-step check rejects a null context or output before touching a device."""
    L = ft.lib()
    m = ctypes.c_double(0.0)
    assert L.ft_binary_cos_screen_check(None, ctypes.byref(m), None) == -1  # FT_ERR_ARG
    assert "null" in L.ft_last_error().decode()
