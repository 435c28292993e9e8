"""Planted mistakes: each plausible error in the oracle must make at least one pin fail.

Each mutation edits a temporary copy of one oracle source (the oracle itself is never
touched), compiles it with the same flags, swaps it in for the duration of the check and
runs that source's pins against it: tests/test_oracle_pins.py for ft_oracle.c,
tests/test_oracle_binary_pins.py for ft_oracle_bin.c, and the injection and all-sky weight
pins for ft_oracle_inj.c.
"""
import os
import subprocess
import tempfile

import pytest

import oracle
from oracle import build as obuild
from tests import test_oracle_pins as pins

MUTATIONS = {
    "eps_sign": ("return fma(v[2], n[2], fma(v[1], n[1], v[0] * n[0]));",
                 "return -fma(v[2], n[2], fma(v[1], n[1], v[0] * n[0]));"),
    "eps_drop_z": ("return fma(v[2], n[2], fma(v[1], n[1], v[0] * n[0]));",
                   "return fma(v[1], n[1], v[0] * n[0]);"),
    "drop_f1_doppler_cross_term": ("int64_t X0 = C + G + floor_div_2_32((__int128)G * (__int128)E);",
                                   "int64_t X0 = C + G;"),
    "drop_j_eps": ("(__int128)X0 + (__int128)j * (__int128)E + ((__int128)1 << 31);",
                   "(__int128)X0 + ((__int128)1 << 31);"),
    "floor_not_round": ("(__int128)X0 + (__int128)j * (__int128)E + ((__int128)1 << 31);",
                        "(__int128)X0 + (__int128)j * (__int128)E;"),
    "k_lo_sign": ("llrint(fma((double)K0, eps, (double)(K0 - k_lo)) * TWO32);",
                  "llrint(fma((double)K0, eps, (double)(K0 + k_lo)) * TWO32);"),
    "start_time_not_mid": ("return (p->t_mid[a] - p->t0) * p->t_sft;",
                           "return (p->t_mid[a] - 0.5 * p->t_sft - p->t0) * p->t_sft;"),
    "weight_dropped": ("s += w * p->power[a * p->W + k];", "s += p->power[a * p->W + k];"),
    "mirrored_column": ("s += w * p->power[a * p->W + k];", "s += w * p->power[a * p->W + (p->W - 1 - k)];"),
    "f1_sign": ("int64_t G = llrint((f1 * tau) * TWO32);", "int64_t G = llrint((-f1 * tau) * TWO32);"),
}

PINS = [
    pins.test_zero_doppler_fixed_bins,
    pins.test_zero_doppler_spindown_closed_form,
    pins.test_f0_neighbours_one_bin_apart,
    pins.test_q32_bins_equal_exact_rational,
    pins.test_q32_bins_large_spindown_exact_rational,
    pins.test_doppler_direction_and_size,
    pins.test_noise_free_injection_recovers_summed_power,
    pins.test_weights_scale_and_z_invariance,
    pins.test_weighted_statistic_bruteforce,
]


# the binary-orbit track and random bank (oracle/ft_oracle_bin.c), against its own pins
BIN_SRC = os.path.join(os.path.dirname(obuild.SRC), "ft_oracle_bin.c")
MUTATIONS_BIN = {
    "orbit_sign": ("double f = lam[0] * (1.0 + vn - orbit);", "double f = lam[0] * (1.0 + vn + orbit);"),
    "doppler_dropped": ("double f = lam[0] * (1.0 + vn - orbit);", "double f = lam[0] * (1.0 - orbit);"),
    "doppler_sign": ("double f = lam[0] * (1.0 + vn - orbit);", "double f = lam[0] * (1.0 - vn - orbit);"),
    "orbit_phase_sign": ("cos(lam[4] * t - TWO_PI * lam[5])", "cos(lam[4] * t + TWO_PI * lam[5])"),
    "orbit_phase_in_radians": ("cos(lam[4] * t - TWO_PI * lam[5])", "cos(lam[4] * t - lam[5])"),
    "orbit_sin_not_cos": ("cos(lam[4] * t - TWO_PI * lam[5])", "sin(lam[4] * t - TWO_PI * lam[5])"),
    "amplitude_without_omega": ("double orbit = lam[3] * lam[4] * cos(", "double orbit = lam[3] * cos("),
    "alpha_in_radians": ("n[0] = cd * cos(TWO_PI * lam[1]);", "n[0] = cd * cos(lam[1]);"),
    "sky_z_dropped": ("n[2] = lam[2];", "n[2] = 0.0;"),
    "time_from_zero": ("return t_mid[a] - t0;", "return t_mid[a];"),
    "start_time_not_mid": ("return t_mid[a] - t0;", "return t_mid[a] - 900.0 - t0;"),
    "floor_not_round": ("double k = floor(X + 0.5);", "double k = floor(X);"),
    "k_lo_sign": ("return f * t_sft - (double)k_lo;", "return f * t_sft + (double)k_lo;"),
    "weight_dropped": ("acc += (w ? w[a] : 1.0) * power[a * W + k];", "acc += power[a * W + k];"),
    "box_order_reversed": ("for (int d = 5; d >= 0; d--) {", "for (int d = 0; d < 6; d++) {"),
    "ap_root_wrong": ("case 3: return cbrt_newton(xi, b->hi[3]);", "case 3: return sqrt(xi);"),
    "sky_weight_times_psd": ("double r = (aa * aa + bb * bb) / s_n[a];",
                             "double r = (aa * aa + bb * bb) * s_n[a];"),
}


# injections, antenna patterns and all-sky weights (oracle/ft_oracle_inj.c)
INJ_SRC = os.path.join(os.path.dirname(obuild.SRC), "ft_oracle_inj.c")
MUTATIONS_INJ = {
    "sky_weight_times_psd": ("wi[a] = (aa * aa + bb * bb) / s_n[a];",
                             "wi[a] = (aa * aa + bb * bb) * s_n[a];"),
    "sky_weight_not_normalised": ("wi[a] /= tot;", "wi[a] /= 1.0;"),
    "antenna_cross_sign": ("sx += M[i][j] * (X[i] * Y[j] + Y[i] * X[j]);",
                           "sx += M[i][j] * (X[i] * Y[j] - Y[i] * X[j]);"),
    "polarisations_in_phase": ("double q2 = fp * fp * ap * ap + fx * fx * ax * ax;",
                               "double q2 = (fp * ap + fx * ax) * (fp * ap + fx * ax);"),
}


def _inj_pins():
    import inspect

    from tests import test_oracle_injection_pins as ip
    from tests import test_oracle_skyweights_pins as sp

    out = []
    for mod in (ip, sp):
        for n in sorted(dir(mod)):
            f = getattr(mod, n)
            if n.startswith("test_") and callable(f) and not inspect.signature(f).parameters:
                out.append(f)
    return out


def _bin_pins():
    from tests import test_oracle_binary_pins as bp

    return [getattr(bp, n) for n in sorted(dir(bp)) if n.startswith("test_")]


def _compile(src: str, out: str, which=None):
    which = obuild.SRC if which is None else which
    cfile = os.path.join(os.path.dirname(out), os.path.basename(which))
    with open(cfile, "w") as f:
        f.write(src)
    others = [s for s in obuild.SRCS if s != which]
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                           "-std=gnu11", cfile] + others + ["-o", out, "-lm"])


def _runs_clean(lib, pins_=None):
    saved = oracle._lib
    oracle._lib = lib
    try:
        failed = []
        for p in (PINS if pins_ is None else pins_):
            try:
                p()
            except Exception:  # an assertion, or a mutated value breaking the pin outright
                failed.append(p.__name__)
        return failed
    finally:
        oracle._lib = saved


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    src = open(obuild.SRC).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    with tempfile.TemporaryDirectory() as d:
        so = os.path.join(d, f"mut_{name}.so")
        _compile(src.replace(old, new), so)
        failed = _runs_clean(oracle.load_library(so))
    assert failed, f"no pin caught mutation {name}"


def test_unmutated_oracle_passes_all_pins():
    with tempfile.TemporaryDirectory() as d:
        so = os.path.join(d, "clean.so")
        _compile(open(obuild.SRC).read(), so)
        assert _runs_clean(oracle.load_library(so)) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS_BIN))
def test_planted_mistake_in_binary_oracle_is_caught(name):
    src = open(BIN_SRC).read()
    old, new = MUTATIONS_BIN[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    with tempfile.TemporaryDirectory() as d:
        so = os.path.join(d, f"mut_{name}.so")
        _compile(src.replace(old, new), so, BIN_SRC)
        failed = _runs_clean(oracle.load_library(so), _bin_pins())
    assert failed, f"no pin caught mutation {name}"


def test_unmutated_binary_oracle_passes_its_pins():
    with tempfile.TemporaryDirectory() as d:
        so = os.path.join(d, "clean_bin.so")
        _compile(open(BIN_SRC).read(), so, BIN_SRC)
        assert _runs_clean(oracle.load_library(so), _bin_pins()) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS_INJ))
def test_planted_mistake_in_injection_oracle_is_caught(name):
    src = open(INJ_SRC).read()
    old, new = MUTATIONS_INJ[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    with tempfile.TemporaryDirectory() as d:
        so = os.path.join(d, f"mut_{name}.so")
        _compile(src.replace(old, new), so, INJ_SRC)
        failed = _runs_clean(oracle.load_library(so), _inj_pins())
    assert failed, f"no pin caught mutation {name}"


def test_unmutated_injection_oracle_passes_its_pins():
    with tempfile.TemporaryDirectory() as d:
        so = os.path.join(d, "clean_inj.so")
        _compile(open(INJ_SRC).read(), so, INJ_SRC)
        assert _runs_clean(oracle.load_library(so), _inj_pins()) == []
