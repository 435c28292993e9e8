"""Pins of the oracle's all-sky weights (Sec. II.B: w_alpha(n) proportional to
(a^2 + b^2) / S_n, normalised to sum 1 per sky point) and of the statistic they weight.

* a^2 + b^2 = 2 |TT(D)|^2 (Frobenius), TT(D) = P D P - (1/2) P tr(P D P), P = I - n n^T:
  e+ / sqrt 2 and ex / sqrt 2 are an orthonormal basis of the transverse-traceless tensors,
  so a^2 + b^2 is twice the squared norm of D's projection on them (a frame-free formula,
  independent of the oracle's choice of wave-frame axes);
* rows are non-negative and sum to 1; a common factor on S_n cancels; doubling one SFT's S_n
  halves its weight relative to the others;
* with the same detector tensor and S_n in every SFT, w = 1/N and the weighted statistic is
  the unweighted one divided by N.
"""
import numpy as np

import ftsynth
import oracle


def _frame_free(D6, n):
    D = np.array([[D6[0], D6[1], D6[2]], [D6[1], D6[3], D6[4]], [D6[2], D6[4], D6[5]]])
    P = np.eye(3) - np.outer(n, n)
    M = P @ D @ P
    TT = M - 0.5 * P * np.trace(M)
    return 2.0 * np.sum(TT * TT)


def test_response_numerator_is_frame_free():
    g = np.random.default_rng(1)
    t = g.uniform(0, 3e7, 12)
    D = np.concatenate([ftsynth.detector_tensor(t[:6], 0), ftsynth.detector_tensor(t[6:], 1)])
    m = g.standard_normal((25, 3))
    sky = m / np.linalg.norm(m, axis=1)[:, None]
    sky[0] = [0.0, 0.0, 1.0]  # a pole: the oracle picks its own frame there
    for Dk in D:
        for n in sky:
            a, b = oracle.antenna_ab(Dk, n)
            assert abs(a * a + b * b - _frame_free(Dk, n)) < 1e-13


def test_weights_normalise_and_scale_with_psd():
    g = np.random.default_rng(2)
    t = np.sort(g.uniform(0, 3e7, 30))
    D = ftsynth.detector_tensor(t, 1)
    s_n = g.uniform(0.5, 2.0, 30)
    sky = ftsynth.fibonacci_sky(17)
    w = oracle.sky_weights(D, s_n, sky)
    assert np.all(w >= 0) and np.allclose(w.sum(axis=1), 1.0, rtol=0, atol=1e-14)
    assert np.allclose(oracle.sky_weights(D, 3.7 * s_n, sky), w, rtol=1e-14, atol=0)
    s2 = s_n.copy()
    s2[5] *= 2.0
    w2 = oracle.sky_weights(D, s2, sky)
    ratio = (w2[:, 5] / w2[:, 6]) / (w[:, 5] / w[:, 6])
    assert np.allclose(ratio, 0.5, rtol=1e-13)


def test_constant_response_reduces_to_plain_mean():
    sfts, bank, _ = ftsynth.tiny_workload("auto")
    N = sfts.n_total
    D = np.tile(ftsynth.detector_tensor(np.array([1234.5]), 0), (N, 1))
    wsky = oracle.sky_weights(D, np.ones(N), bank.sky)
    assert np.allclose(wsky, 1.0 / N, rtol=1e-13)
    tpl = np.arange(0, bank.n_templates, 7)
    s_w, _ = oracle.statistic(sfts, bank, tpl, wsky=wsky)
    s_u, _ = oracle.statistic(sfts, bank, tpl)
    assert np.allclose(s_w, s_u / N, rtol=1e-13)
    mu, sig = oracle.mu_sigma_sky(wsky)
    assert np.allclose(mu, 2.0, rtol=1e-13) and np.allclose(sig, 2.0 / np.sqrt(N), rtol=1e-12)
