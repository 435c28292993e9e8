"""Host-side campaign logic: the sigmoid fit recovers a known detection curve and its
quoted uncertainty is calibrated; population draws follow their priors."""
import math

import numpy as np

from paper_2411_18370_b300 import campaign as C


def test_sigmoid_fit_recovers_known_curve():
    g = np.random.default_rng(0)
    x0, k = 0.1, 6.0
    xs90, sig = [], []
    for rep in range(200):
        x = g.uniform(-1, 1.5, 600)
        det = (g.random(600) < 1 / (1 + np.exp(-k * (x - x0)))).astype(float)
        f = C.fit_sigmoid(x, det)
        xs90.append(f.x_at(0.9))
        sig.append(f.x_at_sigma(0.9))
    truth = x0 + math.log(9) / k
    xs90 = np.array(xs90)
    assert abs(xs90.mean() - truth) < 3 * xs90.std() / math.sqrt(len(xs90)) + 0.01
    # the delta-method error matches the spread of repeated fits within 25%
    assert abs(np.mean(sig) / xs90.std() - 1) < 0.25


def test_population_priors():
    g = np.random.default_rng(1)
    inj, lc = C.draw_population(20000, 100.0, 100.5, g, s_ref=2.0)
    assert np.allclose(np.linalg.norm(inj["n"], axis=1), 1)
    assert abs(np.mean(inj["n"][:, 2])) < 0.02 and abs(np.mean(inj["cosi"])) < 0.02
    assert inj["f0"].min() >= 100.0 and inj["f0"].max() <= 100.5
    assert lc.min() >= math.log10(0.3) and lc.max() <= math.log10(30)
    assert np.allclose(inj["h0"], 10 ** lc * math.sqrt(2.0 / 1800.0))


def test_local_fit_recovers_90_percent_point_of_a_long_tailed_curve():
    """A mixture of two logistics (a slow upper tail, as orientation averaging produces):
    one sigmoid over a wide range misplaces the 90% point, local re-centred fits find it."""
    g = np.random.default_rng(5)

    def p_true(x):
        return 0.8 / (1 + np.exp(-12 * x)) + 0.2 / (1 + np.exp(-4 * (x - 0.3)))

    # the 90% point by bisection on the known curve
    a, b = -1.0, 2.0
    for _ in range(60):
        m = 0.5 * (a + b)
        a, b = (m, b) if p_true(m) < 0.9 else (a, m)
    x90 = 0.5 * (a + b)
    x = g.uniform(-1.0, 1.5, 400_000)
    det = (g.uniform(size=x.size) < p_true(x)).astype(float)
    wide = C.fit_sigmoid(x, det).x_at(0.9)
    loc, sig, n = C.local_x_at(x, det, 0.9, wide, half=0.05)
    assert abs(wide - x90) > 0.02
    assert abs(loc - x90) < max(4 * sig, 0.01) and n > 1000


def test_semi_analytic_closed_form_limit():
    """With no mismatch and rho2 = 0 every draw's z is c^2 h rho1 / sigma_G + xi, so p_det(c)
    = P(xi > tau - c^2 h rho1 / sigma_G) and the 90 % point is
    c = sqrt((tau - Phi^-1(0.1)) sigma_G / (h rho1)); the bisection over 2e5 normal draws
    must land on it within the sampling error of the 10 % quantile."""
    import scipy.stats as st

    from paper_2411_18370_b300 import semianalytic as SA

    n = 200_000
    g = np.random.default_rng(3)
    est = SA.Estimate(rho1=np.full(n, 2.0), rho2=np.zeros(n), m=np.zeros(n),
                      xi=g.standard_normal(n), mu=100.0, sigma=10.0, h2_per_c2=0.5, tau=4.5)
    x = est.log10_c_at(0.9)
    want = math.sqrt((4.5 - st.norm.ppf(0.1)) * 10.0 / (0.5 * 2.0))
    assert abs(10 ** x / want - 1) < 2e-3
    # monotone in c, 0 far below and 1 far above
    ps = [est.pdet(c) for c in (0.1, 1.0, 3.0, 10.0, 100.0)]
    assert ps == sorted(ps) and ps[0] == 0.0 and ps[-1] == 1.0
    # mismatch m scales the signal power by (1 - m): the 90 % point moves by 1/sqrt(1 - m)
    est.m = np.full(n, 0.36)
    assert abs(10 ** (est.log10_c_at(0.9) - x) - 1 / 0.8) < 3e-3
