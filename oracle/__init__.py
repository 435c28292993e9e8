"""CPU FP64 oracle for the short-coherence statistic and its candidate reduction.

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
leg may import this package.  It shares no code with the CUDA path
(paper_2411_18370_b300/); the only module both sides import is ftsynth (seeded inputs).

Functions and the passages of arXiv 2411.18370 they follow:

* statistic()        Eq. (short_coh_general) with Eq. (track), a_p = 0, plus an f1 term;
                     bins by the canonical Q32 rule (C source ft_oracle.c).  FP64.
* bins(), bins_fp64() the canonical Q32 track bins and the direct FP64 rounding of
                     f(t) T_SFT, Eq. (track).
* mu_sigma(), zscore() Sec. II.B.1: mu_G = 2 sum w, sigma_G^2 = 4 sum w^2, and the critical
                     ratio z = (s - mu_G)/sigma_G, Eq. (critical_ratio).
* topk_per_subband() Sec. IV.B (ahead-of-time clustering): the loudest templates of each
                     disjoint box, here the 1-D boxes "f0 bin j // subband_bins", ordered by
                     s descending, then template index ascending.
* number_count()     Eq. (number_count) summed like Eq. (short_coh_general): the weighted
                     count of SFTs whose normalised power on the track exceeds a threshold.
* nc_moments()       its mean and deviation in Gaussian noise (P exponential with mean 2,
                     so P(P > x) = exp(-x / 2); Bernoulli per SFT).
* topk_gated()       Sec. VI.B: the loudest per box among templates whose second statistic
                     (the weighted number count) reaches a minimum.
* binary_*()         Eq. (track) with the binary-orbit term, evaluated as written in FP64
                     with libm's cos / sin and rounded half up to a bin; the random bank in
                     the uniform coordinates of Eq. (xi_of_lambda) / App. A and its
                     hyperboxes (Sec. IV.B); the statistic along those tracks (C source
                     ft_oracle_bin.c).
* topk_per_box()     the loudest templates of each hyperbox.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math

import numpy as np

from . import build as _build

_lib = None


class _Problem(ctypes.Structure):
    _fields_ = [
        ("power", ctypes.c_void_p),
        ("n_sft", ctypes.c_int64),
        ("W", ctypes.c_int64),
        ("k_lo", ctypes.c_int64),
        ("t_mid", ctypes.c_void_p),
        ("v", ctypes.c_void_p),
        ("w", ctypes.c_void_p),
        ("t0", ctypes.c_double),
        ("t_sft", ctypes.c_double),
        ("K0", ctypes.c_int64),
        ("n_f0", ctypes.c_int64),
        ("n_f1", ctypes.c_int64),
        ("f1", ctypes.c_void_p),
        ("n_sky", ctypes.c_int64),
        ("sky", ctypes.c_void_p),
        ("wsky", ctypes.c_void_p),
    ]


class _InjProblem(ctypes.Structure):
    _fields_ = [
        ("n_sft", ctypes.c_int64),
        ("k_lo", ctypes.c_int64),
        ("t_mid", ctypes.c_void_p),
        ("v", ctypes.c_void_p),
        ("w", ctypes.c_void_p),
        ("s_n", ctypes.c_void_p),
        ("D", ctypes.c_void_p),
        ("t0", ctypes.c_double),
        ("t_sft", ctypes.c_double),
        ("K0", ctypes.c_int64),
        ("n_f0", ctypes.c_int64),
        ("n_f1", ctypes.c_int64),
        ("f1", ctypes.c_void_p),
        ("n_sky", ctypes.c_int64),
        ("sky", ctypes.c_void_p),
    ]


INJ_DTYPE = np.dtype([("h0", "<f8"), ("cosi", "<f8"), ("psi", "<f8"), ("f0", "<f8"),
                      ("f1", "<f8"), ("n", "<f8", (3,))])


def load_library(path):
    """Open an oracle shared library and declare its signatures."""
    L = ctypes.CDLL(path)
    L.or_bin_q32.restype = ctypes.c_int64
    L.or_bin_q32.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                             ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
    L.or_bin_fp64.restype = ctypes.c_int64
    L.or_bin_fp64.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                              ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.or_statistic.restype = None
    L.or_statistic.argtypes = [ctypes.POINTER(_Problem), ctypes.c_void_p, ctypes.c_int64,
                               ctypes.c_void_p, ctypes.c_void_p]
    L.or_bins.restype = None
    L.or_bins.argtypes = [ctypes.POINTER(_Problem), ctypes.c_void_p, ctypes.c_int64,
                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.or_num_threads.restype = ctypes.c_int
    L.or_philox4x32_10.restype = None
    L.or_philox4x32_10.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.or_uniform24.restype = ctypes.c_double
    L.or_uniform24.argtypes = [ctypes.c_uint32]
    L.or_antenna_ab.restype = None
    L.or_antenna_ab.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.or_rho2.restype = ctypes.c_double
    L.or_rho2.argtypes = [ctypes.c_void_p, ctypes.c_void_p] + [ctypes.c_double] * 5
    L.or_inj_power.restype = ctypes.c_double
    L.or_inj_power.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64,
                               ctypes.c_double, ctypes.c_double]
    L.or_sky_weights.restype = None
    L.or_sky_weights.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                 ctypes.c_void_p, ctypes.c_void_p]
    L.or_pdet_q.restype = None
    L.or_pdet_q.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                            ctypes.c_void_p]
    L.or_bt_templates.restype = None
    L.or_bt_templates.argtypes = [ctypes.POINTER(_BDesc), ctypes.c_void_p, ctypes.c_int64,
                                  ctypes.c_void_p]
    L.or_bt_sky.restype = None
    L.or_bt_sky.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.or_bt_position.restype = ctypes.c_double
    L.or_bt_position.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_int64]
    L.or_bt_bins.restype = None
    L.or_bt_bins.argtypes = [ctypes.POINTER(_BDesc), ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                             ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    L.or_bt_statistic_sky.restype = None
    L.or_bt_statistic_sky.argtypes = [ctypes.POINTER(_BDesc), ctypes.c_void_p, ctypes.c_int64,
                                      ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]
    L.or_bt_statistic.restype = None
    L.or_bt_statistic.argtypes = [ctypes.POINTER(_BDesc), ctypes.c_void_p, ctypes.c_int64,
                                  ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    L.or_injections.restype = None
    L.or_injections.argtypes = [ctypes.POINTER(_InjProblem), ctypes.c_void_p, ctypes.c_int64,
                                ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_void_p]
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load_library(_build.build())
    return _lib


def num_threads() -> int:
    return int(lib().or_num_threads())


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class _Keep:
    """Holds the numpy arrays a _Problem points into."""

    def __init__(self, sfts, bank, w, wsky=None):
        self.wsky = None if wsky is None else _c(wsky, np.float64)
        self.power = _c(sfts.power, np.float64)
        self.t_mid = _c(sfts.t_mid, np.float64)
        self.v = _c(sfts.v, np.float64)
        self.w = None if w is None else _c(w, np.float64)
        self.f1 = _c(bank.f1, np.float64)
        self.sky = _c(bank.sky, np.float64)
        p = _Problem()
        p.power = self.power.ctypes.data
        p.n_sft = self.power.shape[0]
        p.W = self.power.shape[1]
        p.k_lo = int(sfts.k_lo)
        p.t_mid = self.t_mid.ctypes.data
        p.v = self.v.ctypes.data
        p.w = None if self.w is None else self.w.ctypes.data
        p.t0 = float(sfts.t0)
        p.t_sft = float(sfts.t_sft)
        p.K0 = int(bank.k0)
        p.n_f0 = int(bank.n_f0)
        p.n_f1 = len(self.f1)
        p.f1 = self.f1.ctypes.data
        p.n_sky = len(self.sky)
        p.sky = self.sky.ctypes.data
        p.wsky = None if self.wsky is None else self.wsky.ctypes.data
        self.p = p


def statistic(sfts, bank, templates=None, w=None, wsky=None):
    """FP64 s for the given template indices (all when None) and out-of-window counts.
    wsky [n_sky][n_sft] (sky-dependent weights) replaces w when given."""
    k = _Keep(sfts, bank, w, wsky)
    if templates is None:
        n = bank.n_templates
        tp = None
        tarr = None
    else:
        tarr = _c(templates, np.int64)
        n = len(tarr)
        tp = tarr.ctypes.data
    s = np.empty(n, np.float64)
    oob = np.empty(n, np.int32)
    lib().or_statistic(ctypes.byref(k.p), tp, n, s.ctypes.data, oob.ctypes.data)
    return s, oob


def bins(sfts, bank, templates, with_fp64=False):
    """Canonical Q32 bins [n, N_SFT]; with_fp64 also returns direct FP64 bins and the
    distance of the real-valued track from the rounding boundary."""
    k = _Keep(sfts, bank, None)
    tarr = _c(templates, np.int64)
    n = len(tarr)
    N = k.power.shape[0]
    b = np.empty((n, N), np.int64)
    if not with_fp64:
        lib().or_bins(ctypes.byref(k.p), tarr.ctypes.data, n, b.ctypes.data, None, None)
        return b
    bf = np.empty((n, N), np.int64)
    d = np.empty((n, N), np.float64)
    lib().or_bins(ctypes.byref(k.p), tarr.ctypes.data, n, b.ctypes.data, bf.ctypes.data,
                  d.ctypes.data)
    return b, bf, d


def mu_sigma(n_sft: int, w=None):
    """mu_G = 2 sum w, sigma_G = sqrt(4 sum w^2) (Sec. II.B.1, Gaussian limit)."""
    if w is None:
        return 2.0 * n_sft, math.sqrt(4.0 * n_sft)
    w = np.asarray(w, np.float64)
    return 2.0 * float(w.sum()), math.sqrt(4.0 * float((w * w).sum()))


def zscore(s, n_sft: int, w=None):
    """Critical ratio z = (s - mu_G) / sigma_G, Eq. (critical_ratio)."""
    mu, sig = mu_sigma(n_sft, w)
    return (np.asarray(s, np.float64) - mu) / sig


def topk_per_subband(s, bank, k: int, templates=None):
    """Per sub-band b (templates whose f0 index j has j // subband_bins == b), the k largest
    s, ties broken by the smaller template index.  Returns (idx[n_sub, k], val[n_sub, k]);
    slots beyond the sub-band's population hold idx -1 and val -inf."""
    s = np.asarray(s, np.float64)
    t = np.arange(len(s), dtype=np.int64) if templates is None else np.asarray(templates, np.int64)
    j = t % bank.n_f0
    sub = j // bank.subband_bins
    nsub = bank.n_subbands
    idx = np.full((nsub, k), -1, np.int64)
    val = np.full((nsub, k), -np.inf)
    for b in range(nsub):
        m = sub == b
        tb, sb = t[m], s[m]
        order = np.lexsort((tb, -sb))[:k]
        idx[b, : len(order)] = tb[order]
        val[b, : len(order)] = sb[order]
    return idx, val


# ----------------------------------------------------------------------------- injections


def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al., SC'11) of counter ctr[4], key key[2]."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.empty(4, np.uint32)
    lib().or_philox4x32_10(c.ctypes.data, k.ctypes.data, o.ctypes.data)
    return o


def uniform24(x):
    return lib().or_uniform24(int(x))


def antenna_ab(D, n):
    """a = D : e+, b = D : ex for detector tensor D (6 components) and source direction n."""
    Dv = _c(D, np.float64)
    nv = _c(n, np.float64)
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().or_antenna_ab(Dv.ctypes.data, nv.ctypes.data, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def rho2(D, n, h0, cosi, psi, t_sft, s_n):
    """Normalised signal power of one SFT (Sec. II.B.2 signal model)."""
    Dv = _c(D, np.float64)
    nv = _c(n, np.float64)
    return lib().or_rho2(Dv.ctypes.data, nv.ctypes.data, h0, cosi, psi, t_sft, s_n)


def inj_power(kabs, alpha, run_id, seed, amp, noise_scale=1.0):
    return lib().or_inj_power(int(kabs), int(alpha), int(run_id), int(seed), float(amp),
                              float(noise_scale))


def injections(sfts, bank, D, inj, first_id, seed, K=64, half_f0=2, H=160, noise_scale=1.0,
               w=None, with_second=False):
    """Independent injection-recovery runs (run r uses run id first_id + r): max z over the
    local bank, argmax template and out-of-window reads (and, with_second, the second largest
    z of the local bank).  inj: structured INJ_DTYPE array."""
    keep = dict(t_mid=_c(sfts.t_mid, np.float64), v=_c(sfts.v, np.float64),
                s_n=_c(sfts.s_n, np.float64), D=_c(D, np.float64), f1=_c(bank.f1, np.float64),
                sky=_c(bank.sky, np.float64),
                w=None if w is None else _c(w, np.float64))
    p = _InjProblem()
    p.n_sft = len(keep["t_mid"])
    p.k_lo = int(sfts.k_lo)
    p.t_mid = keep["t_mid"].ctypes.data
    p.v = keep["v"].ctypes.data
    p.w = None if keep["w"] is None else keep["w"].ctypes.data
    p.s_n = keep["s_n"].ctypes.data
    p.D = keep["D"].ctypes.data
    p.t0 = float(sfts.t0)
    p.t_sft = float(sfts.t_sft)
    p.K0 = int(bank.k0)
    p.n_f0 = int(bank.n_f0)
    p.n_f1 = len(keep["f1"])
    p.f1 = keep["f1"].ctypes.data
    p.n_sky = len(keep["sky"])
    p.sky = keep["sky"].ctypes.data
    arr = np.ascontiguousarray(inj, dtype=INJ_DTYPE)
    n = len(arr)
    mz = np.empty(n, np.float64)
    am = np.empty(n, np.int64)
    oob = np.empty(n, np.int64)
    z2 = np.empty(n, np.float64)
    lib().or_injections(ctypes.byref(p), arr.ctypes.data, n, int(first_id), int(seed), int(K),
                        int(half_f0), int(H), float(noise_scale), mz.ctypes.data, am.ctypes.data,
                        oob.ctypes.data, z2.ctypes.data)
    return (mz, am, oob, z2) if with_second else (mz, am, oob)


def pdet_q(s_n, t_sft, D, inj, w=None):
    """Sec. V.A q numbers per population draw: (sum w rho^2, sum w^2 rho^2) at h0 = 1."""
    sn = _c(s_n, np.float64)
    Dv = _c(D, np.float64)
    wv = None if w is None else _c(w, np.float64)
    draws = np.ascontiguousarray(np.column_stack([inj["cosi"], inj["psi"], inj["n"]]), np.float64)
    n = len(draws)
    r1 = np.empty(n, np.float64)
    r2 = np.empty(n, np.float64)
    lib().or_pdet_q(len(sn), float(t_sft), sn.ctypes.data, Dv.ctypes.data,
                    None if wv is None else wv.ctypes.data, n, draws.ctypes.data,
                    r1.ctypes.data, r2.ctypes.data)
    return r1, r2


def sky_weights(D, s_n, sky):
    """Sec. II.B all-sky weights w[i_sky][alpha] ~ (a^2 + b^2) / S_n, each row summing to 1."""
    Dv = _c(D, np.float64)
    sn = _c(s_n, np.float64)
    sk = _c(sky, np.float64)
    out = np.empty((len(sk), len(sn)), np.float64)
    lib().or_sky_weights(len(sn), Dv.ctypes.data, sn.ctypes.data, len(sk), sk.ctypes.data,
                         out.ctypes.data)
    return out


def mu_sigma_sky(wsky):
    """Per sky point mu_G = 2 sum_alpha w and sigma_G = sqrt(4 sum_alpha w^2)."""
    w = np.asarray(wsky, np.float64)
    return 2.0 * w.sum(axis=1), np.sqrt(4.0 * (w * w).sum(axis=1))


# ----------------------------------------------------------------------------- number count


def number_count(sfts, bank, templates=None, threshold=3.2, w=None, wsky=None):
    """Weighted number count sum_alpha w_alpha 1[P_alpha(track bin) > threshold] per template
    (Eq. (number_count)): the statistic of the binarised spectrogram.  Out-of-window reads
    count 0, as in statistic()."""
    binar = (np.asarray(sfts.power, np.float64) > threshold).astype(np.float64)
    return statistic(dataclasses.replace(sfts, power=binar), bank, templates, w=w, wsky=wsky)


def nc_moments(threshold, n_sft=None, w=None):
    """Gaussian-noise mean and deviation of the weighted number count: p sum w and
    sqrt(p (1 - p) sum w^2) with p = exp(-threshold / 2)."""
    p = math.exp(-0.5 * threshold)
    if w is None:
        return p * n_sft, math.sqrt(p * (1.0 - p) * n_sft)
    w = np.asarray(w, np.float64)
    return p * float(w.sum()), math.sqrt(p * (1.0 - p) * float((w * w).sum()))


def topk_gated(s, gate, gate_min, bank, k, templates=None):
    """topk_per_subband over the templates with gate >= gate_min only."""
    s = np.asarray(s, np.float64)
    t = np.arange(len(s), dtype=np.int64) if templates is None else np.asarray(templates, np.int64)
    keep = np.asarray(gate) >= gate_min
    return topk_per_subband(s[keep], bank, k, t[keep])


# ----------------------------------------------------------------------------- binary track


class _BDesc(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 6), ("hi", ctypes.c_double * 6), ("n_div", ctypes.c_int32 * 6),
                ("n_per_box", ctypes.c_int64), ("seed", ctypes.c_uint64)]


def _bdesc(bank):
    d = _BDesc()
    for k in range(6):
        d.lo[k] = float(bank.lo[k])
        d.hi[k] = float(bank.hi[k])
        d.n_div[k] = int(bank.n_div[k])
    d.n_per_box = int(bank.n_per_box)
    d.seed = int(bank.seed) & ((1 << 64) - 1)
    return d


def _tmpl(bank, templates):
    return _c(np.arange(bank.n_templates) if templates is None else templates, np.int64)


def binary_templates(bank, templates=None):
    """lambda [n][6] (BINARY_DIMS order: f0, alpha in turns, sin(delta), a_p, Omega, phi_b in
    turns) of the given templates (default: all)."""
    t = _tmpl(bank, templates)
    n = len(t)
    lam = np.empty((n, 6), np.float64)
    d = _bdesc(bank)
    lib().or_bt_templates(ctypes.byref(d), t.ctypes.data, n, lam.ctypes.data)
    return lam


def binary_sky(lam):
    """The unit sky vectors [n][3] of lambda rows (FP64, libm cos / sin of 2 pi alpha)."""
    lam = _c(np.atleast_2d(lam), np.float64)
    out = np.empty((len(lam), 3), np.float64)
    for i in range(len(lam)):
        lib().or_bt_sky(lam[i].ctypes.data, out[i].ctypes.data)
    return out


def binary_position(lam, v, t, t_sft, k_lo):
    """Eq. (track) times T_SFT as a band column, X = f(t) T_SFT - k_lo, for one template
    (lambda row) and one SFT (v/c [3], t = t_mid - t0)."""
    lam = _c(lam, np.float64)
    n = binary_sky(lam)[0]
    vv = _c(v, np.float64)
    return float(lib().or_bt_position(lam.ctypes.data, n.ctypes.data, vv.ctypes.data, float(t),
                                      float(t_sft), int(k_lo)))


def binary_bins(sfts, bank, templates, with_dist=False):
    """Bins [n, N_SFT] (band columns) of Eq. (track), FP64, rounded half up; with_dist also the
    distance of each real-valued position from its rounding boundary."""
    t = _tmpl(bank, templates)
    n = len(t)
    tm = _c(sfts.t_mid, np.float64)
    v = _c(sfts.v, np.float64)
    N = len(tm)
    b = np.empty((n, N), np.int64)
    dist = np.empty((n, N), np.float64) if with_dist else None
    d = _bdesc(bank)
    lib().or_bt_bins(ctypes.byref(d), t.ctypes.data, n, N, tm.ctypes.data, v.ctypes.data,
                     float(sfts.t0), float(sfts.t_sft), int(sfts.k_lo), b.ctypes.data,
                     None if dist is None else dist.ctypes.data)
    return (b, dist) if with_dist else b


def binary_statistic(sfts, bank, templates=None, w=None):
    """FP64 s along the binary tracks of Eq. (track) and the out-of-window counts."""
    t = None if templates is None else _c(templates, np.int64)
    n = bank.n_templates if t is None else len(t)
    P = _c(sfts.power, np.float64)
    tm = _c(sfts.t_mid, np.float64)
    v = _c(sfts.v, np.float64)
    wv = None if w is None else _c(w, np.float64)
    s = np.empty(n, np.float64)
    oob = np.empty(n, np.int32)
    d = _bdesc(bank)
    lib().or_bt_statistic(ctypes.byref(d), None if t is None else t.ctypes.data, n, P.shape[0],
                           P.shape[1], P.ctypes.data, None if wv is None else wv.ctypes.data,
                           tm.ctypes.data, v.ctypes.data, float(sfts.t0), float(sfts.t_sft),
                           int(sfts.k_lo), s.ctypes.data, oob.ctypes.data)
    return s, oob


def binary_statistic_sky(sfts, bank, D, templates=None):
    """s along the binary tracks of Eq. (track) under the all-sky weights (a^2 + b^2)/S_n of each
    template's sky direction (Sec. II.B), normalised per template; returns (s, sigma_G, oob)
    with mu_G = 2."""
    t = None if templates is None else _c(templates, np.int64)
    n = bank.n_templates if t is None else len(t)
    P = _c(sfts.power, np.float64)
    Dv = _c(D, np.float64)
    sn = _c(sfts.s_n, np.float64)
    tm = _c(sfts.t_mid, np.float64)
    v = _c(sfts.v, np.float64)
    s = np.empty(n, np.float64)
    sig = np.empty(n, np.float64)
    oob = np.empty(n, np.int32)
    d = _bdesc(bank)
    lib().or_bt_statistic_sky(ctypes.byref(d), None if t is None else t.ctypes.data, n, P.shape[0],
                              P.shape[1], P.ctypes.data, Dv.ctypes.data, sn.ctypes.data, tm.ctypes.data,
                              v.ctypes.data, float(sfts.t0), float(sfts.t_sft), int(sfts.k_lo),
                              s.ctypes.data, sig.ctypes.data, oob.ctypes.data)
    return s, sig, oob


def topk_per_key(s, key, n_keys, k, templates=None):
    """Per box id in 0 .. n_keys - 1 (key[i] is the box of template templates[i]), the k largest
    s, ties by the smaller template index; idx -1 / val -inf beyond the box's population."""
    s = np.asarray(s, np.float64)
    key = np.asarray(key, np.int64)
    t = np.arange(len(s), dtype=np.int64) if templates is None else np.asarray(templates, np.int64)
    idx = np.full((n_keys, k), -1, np.int64)
    val = np.full((n_keys, k), -np.inf)
    order = np.lexsort((t, -s, key))
    bounds = np.searchsorted(key[order], np.arange(n_keys + 1))
    for b in range(n_keys):
        sel = order[bounds[b]:bounds[b + 1]][:k]
        idx[b, : len(sel)] = t[sel]
        val[b, : len(sel)] = s[sel]
    return idx, val


def topk_per_box(s, n_per_box, n_boxes, k, templates=None):
    """Per box b (templates i with i // n_per_box == b), the k largest s, ties by the smaller
    index; idx -1 / val -inf beyond the box's population."""
    s = np.asarray(s, np.float64)
    t = np.arange(len(s), dtype=np.int64) if templates is None else np.asarray(templates, np.int64)
    box = t // n_per_box
    idx = np.full((n_boxes, k), -1, np.int64)
    val = np.full((n_boxes, k), -np.inf)
    for b in range(n_boxes):
        m = box == b
        tb, sb = t[m], s[m]
        order = np.lexsort((tb, -sb))[:k]
        idx[b, : len(order)] = tb[order]
        val[b, : len(order)] = sb[order]
    return idx, val
