"""Pins of the oracle's injection-recovery pieces against closed forms and exact results.

* Philox4x32-10 output: uniform bits, uniform 24-bit variates, avalanche on the counter.
* Noise power: chi^2_2 (Sec. II.B.1); signal-bin power: non-central chi^2_2(rho^2) with
  mean 2 + rho^2 (Sec. II.B.2).
* Antenna patterns: the zenith case of an L-shaped detector, psi-invariance of F+^2 + Fx^2,
  and its isotropic average 2/5 for a 90-degree interferometer.
* rho^2 closed form for a face-on source at the zenith.
* A noise-free injection on a grid template recovers exactly sum_alpha w_alpha rho^2_alpha;
  the reported runner-up z equals a brute-force pass over the local bank.
"""
import math
from fractions import Fraction as F

import numpy as np
import pytest
import scipy.stats as st

import ftsynth
import oracle
from tests import exact


def test_philox_bits_are_uniform():
    outs = np.array([oracle.philox4x32_10([i, 7, 3, 0], [11, 13]) for i in range(20000)],
                    dtype=np.uint64)
    bits = ((outs[:, :, None] >> np.arange(32, dtype=np.uint64)) & 1).reshape(-1, 32)
    frac = bits.mean(axis=0)
    n = bits.shape[0]
    assert np.all(np.abs(frac - 0.5) < 5 * 0.5 / math.sqrt(n))
    u = np.array([oracle.uniform24(int(x)) for x in outs[:, 0]])
    assert u.min() > 0 and u.max() <= 1
    assert st.kstest(u, "uniform").pvalue > 1e-3


def test_philox_avalanche():
    g = np.random.default_rng(1)
    flips = []
    for _ in range(300):
        c = [int(x) for x in g.integers(0, 2 ** 32, 4)]
        k = [int(x) for x in g.integers(0, 2 ** 32, 2)]
        b = int(g.integers(0, 128))
        c2 = list(c)
        c2[b // 32] ^= 1 << (b % 32)
        o1 = oracle.philox4x32_10(c, k).astype(np.uint64)
        o2 = oracle.philox4x32_10(c2, k).astype(np.uint64)
        flips.append(sum(bin(int(x ^ y)).count("1") for x, y in zip(o1, o2)))
    assert abs(np.mean(flips) - 64) < 2.5


def test_noise_power_is_chi2_2():
    P = np.array([oracle.inj_power(k, a, 5, 77, 0.0) for k in range(200) for a in range(100)])
    assert abs(P.mean() - 2) < 5 * 2 / math.sqrt(len(P))
    assert st.kstest(P, st.chi2(2).cdf).pvalue > 1e-3


@pytest.mark.parametrize("rho2", [0.5, 4.0])
def test_signal_bin_power_is_noncentral_chi2(rho2):
    a = math.sqrt(rho2)
    P = np.array([oracle.inj_power(1000, alpha, run, 99, a) for run in range(100)
                  for alpha in range(100)])
    assert abs(P.mean() - (2 + rho2)) < 5 * math.sqrt((4 + 4 * rho2) / len(P))
    assert st.kstest(P, st.ncx2(df=2, nc=rho2).cdf).pvalue > 1e-3


def _L_tensor():
    """Arms along x and y: D = (xx - yy)/2."""
    return np.array([0.5, 0.0, 0.0, -0.5, 0.0, 0.0])


def test_antenna_zenith_of_L_detector():
    a, b = oracle.antenna_ab(_L_tensor(), [0.0, 0.0, 1.0])
    assert a == 1.0 and b == 0.0


def test_antenna_psi_invariance_and_isotropic_average():
    g = np.random.default_rng(3)
    D = ftsynth.detector_tensor(np.array([12345.0]), 1)[0]
    n = g.standard_normal((20000, 3))
    n /= np.linalg.norm(n, axis=1)[:, None]
    ab = np.array([oracle.antenna_ab(D, m) for m in n])
    # F+^2 + Fx^2 = a^2 + b^2 averages to 2/5 over an isotropic sky (90-degree arms)
    assert abs(np.mean(ab[:, 0] ** 2 + ab[:, 1] ** 2) - 0.4) < 0.006
    # F+^2 + Fx^2 does not depend on psi: rho^2 of a face-on source is psi-independent
    for m in n[:20]:
        r = [oracle.rho2(D, m, 1.0, 1.0, psi, 1800.0, 1.0) for psi in (0.0, 0.3, 1.1, 2.9)]
        assert max(r) - min(r) < 1e-12 * max(r)


def test_rho2_closed_form_face_on_zenith():
    T, h0, sn = 1800.0, 2.5e-2, 1.7
    r = oracle.rho2(_L_tensor(), [0.0, 0.0, 1.0], h0, 1.0, 0.0, T, sn)
    assert abs(r - 0.7737 ** 2 * T * h0 * h0 / sn) < 1e-14 * r


def _short_band(n_slots=300, n_sky=40):
    starts = ftsynth.timeline(2, n_slots, ftsynth.T_SFT, 0.7, ftsynth.rng(41, 1))
    k_band = 360000
    wl, wh = ftsynth.wings_for(200.1, -1e-9, n_slots * 1800.0, 1800.0)
    sfts = ftsynth.make_sfts(41, 2, n_slots, 1800.0, 0.7, k_band, 180, wl, wh,
                             psd_range=(0.8, 1.2), slot_starts=starts)
    D = np.concatenate([ftsynth.detector_tensor(st + 900.0, X) for X, st in enumerate(starts)])
    bank = ftsynth.Bank(k0=k_band, n_f0=180, f1=ftsynth.f1_grid(10, -1e-9, 0.0),
                        sky=ftsynth.fibonacci_sky(n_sky), subband_bins=18)
    return sfts, bank, D


def test_noise_free_injection_on_grid_template_is_exact():
    """With noise_scale 0 and the source on a grid template, s(true) = sum w rho^2 exactly
    and it is the loudest template; z = (s - mu_G)/sigma_G."""
    sfts, bank, D = _short_band()
    j, f1i, ski = 77, 3, 9
    inj = np.zeros(1, oracle.INJ_DTYPE)
    inj["h0"] = 0.05
    inj["cosi"] = 0.3
    inj["psi"] = 0.7
    inj["f0"] = (bank.k0 + j) / sfts.t_sft
    inj["f1"] = bank.f1[f1i]
    inj["n"] = bank.sky[ski]
    # the signal bin (nearest bin to f T) equals the template's track bin in every SFT
    for a in range(sfts.n_total):
        x = exact.position(bank.k0, sfts.k_lo, j, bank.f1[f1i], sfts.t_mid[a], sfts.t0,
                           sfts.t_sft, sfts.v[a], bank.sky[ski])
        assert exact.bin_and_tie_distance(x)[1] > 1e-6
    mz, am, oob, z2 = oracle.injections(sfts, bank, D, inj, 0, 123, K=8, noise_scale=0.0,
                                        with_second=True)
    rho2 = np.array([oracle.rho2(D[a], bank.sky[ski], 0.05, 0.3, 0.7, 1800.0, sfts.s_n[a])
                     for a in range(sfts.n_total)])
    mu, sig = oracle.mu_sigma(sfts.n_total)
    t_inj = (ski * bank.n_f1 + f1i) * bank.n_f0 + j
    assert am[0] == t_inj
    assert abs(mz[0] - (rho2.sum() - mu) / sig) < 1e-9 * abs(mz[0])
    assert oob[0] == 0
    # brute force over the local bank (f0 within 2 bins, every f1, the 8 sky points nearest
    # the source): noise-free, a template collects rho^2 in the SFTs where its bin is the
    # signal's; the second largest z is the runner-up's
    near = np.argsort(-(bank.sky @ bank.sky[ski]), kind="stable")[:8]
    loc = np.array([(sk * bank.n_f1 + f) * bank.n_f0 + jj for sk in near for f in range(bank.n_f1)
                    for jj in range(j - 2, j + 3)])
    b = oracle.bins(sfts, bank, loc)
    b_sig = oracle.bins(sfts, bank, [t_inj])[0]
    z = np.sort(((b == b_sig[None, :]) * rho2[None, :]).sum(axis=1) - mu) / sig
    assert abs(z[-1] - mz[0]) < 1e-9 * abs(mz[0])
    assert abs(z[-2] - z2[0]) < 1e-9 * abs(z2[0]) and z2[0] < mz[0]
    # with no signal every template has z = -mu/sigma: the runner-up ties the loudest
    inj["h0"] = 0.0
    mz0, _, _, z20 = oracle.injections(sfts, bank, D, inj, 0, 123, K=8, noise_scale=0.0,
                                       with_second=True)
    assert z20[0] == mz0[0] == -mu / sig


def test_window_too_narrow_is_counted():
    sfts, bank, D = _short_band(n_slots=200)
    inj = np.zeros(2, oracle.INJ_DTYPE)
    inj["h0"] = 0.0
    inj["f0"] = (bank.k0 + 90.3) / 1800.0
    inj["f1"] = -3e-10
    inj["n"] = bank.sky[[4, 17]]
    _, _, oob_wide = oracle.injections(sfts, bank, D, inj, 0, 5, K=16, H=160)
    _, _, oob_narrow = oracle.injections(sfts, bank, D, inj, 0, 5, K=16, H=1)
    assert np.all(oob_wide == 0) and np.all(oob_narrow > 0)


def test_pdet_q_isotropic_average():
    """Sec. V.A q numbers: over an isotropic population (n uniform on the sphere,
    cos iota ~ U[-1, 1], psi ~ U[0, pi]), E|Q|^2 = <F+^2> <A+^2> + <Fx^2> <Ax^2>
    = 0.2 (7/15) + 0.2 (1/3) = 0.16 (with <a^2 + b^2> = 0.4 for a detector of unit
    orthogonal arms), so E[rho1] = 0.7737^2 T 0.16 sum w / S_n and E[rho2] the same with w^2.
    Checked against Monte Carlo within 4 standard errors."""
    g = np.random.default_rng(11)
    t = np.sort(g.uniform(0, 3e7, 40)) + 900.0
    D = np.concatenate([ftsynth.detector_tensor(t[:20], 0), ftsynth.detector_tensor(t[20:], 1)])
    s_n = g.uniform(0.5, 2.0, 40)
    w = g.uniform(0.2, 3.0, 40)
    n = 40000
    inj = np.zeros(n, oracle.INJ_DTYPE)
    m = g.standard_normal((n, 3))
    inj["n"] = m / np.linalg.norm(m, axis=1)[:, None]
    inj["cosi"] = g.uniform(-1, 1, n)
    inj["psi"] = g.uniform(0, math.pi, n)
    r1, r2 = oracle.pdet_q(s_n, 1800.0, D, inj, w)
    k = 0.7737 ** 2 * 1800.0 * 0.16
    for r, want in ((r1, k * np.sum(w / s_n)), (r2, k * np.sum(w * w / s_n))):
        se = r.std() / math.sqrt(n)
        assert abs(r.mean() - want) < 4 * se, (r.mean(), want, se)
    # unit weights: the two sums coincide
    r1u, r2u = oracle.pdet_q(s_n, 1800.0, D, inj[:100])
    assert np.allclose(r1u, r2u, rtol=1e-15, atol=0)
