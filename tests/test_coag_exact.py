"""Pins of the Smoluchowski solutions that the coagulation tests compare against
(Appendix A), each against something other than its own formula:

* constant kernel: the closed-form partial sums against direct sums of the paper's number
  distribution, its mean against 1 + t~, and its large-t~ limit (the mass-weighted
  gamma(2) of scale t~/2);
* linear kernel: the density integrates to the total mass, its mean follows the moment
  equation (2 exp(2 t~)), and at t~ -> 0 it is the gamma(2) start;
* product kernel: normalised and with mean 1 / (1 - t~) before gelation.
"""
import math

import numpy as np

import coag_exact as X


def test_constant_closed_form_against_direct_sum():
    for t in (0.5, 3.0, 40.0):
        k = np.arange(1, 40001, dtype=float)
        # the paper's (t/2)^(k-1) / (1 + t/2)^(k+1), through logarithms
        n = np.exp((k - 1) * math.log(t / 2.0) - (k + 1) * math.log1p(t / 2.0))
        w = k * n
        assert abs(w.sum() - 1.0) < 1e-12                  # mass conservation
        assert abs((k * w).sum() / X.mean_constant(t) - 1.0) < 1e-12
        F = X.cdf_constant(t)
        ks = np.array([1, 2, 5, 17, 100, 1000], dtype=float)
        ks = ks[ks < 20 * (1 + t)]
        got = F(np.log10(ks))
        want = np.cumsum(w)[ks.astype(int) - 1]
        assert np.abs(got - want).max() < 1e-12, (t, got, want)
        # below one unit grain there is no mass; non-integer masses read the integer below
        assert F(np.array([-0.5]))[0] == 0.0
        assert F(np.array([math.log10(2.5)]))[0] == F(np.array([math.log10(2.0)]))[0]


def test_constant_large_time_limit():
    t = 1e8
    F = X.cdf_constant(t)
    for u in (0.1, 0.5, 1.0, 3.0):                     # k = u t~/2
        k = u * t / 2.0
        assert abs((1.0 - F(np.array([math.log10(k)]))[0]) - math.exp(-u) * (1.0 + u)) < 1e-6


def test_linear_normalisation_mean_and_start():
    for t in (0.25, 1.0, 2.0, 4.0):
        lx = X.linear_grid(t)
        w = X.linear_density(t, lx) * 10.0 ** lx * math.log(10.0)
        wx = w * 10.0 ** lx
        tot = np.sum(0.5 * (w[1:] + w[:-1]) * np.diff(lx))
        mean = np.sum(0.5 * (wx[1:] + wx[:-1]) * np.diff(lx))
        assert abs(tot - 1.0) < 1e-9, (t, tot)
        assert abs(mean / X.mean_linear(t) - 1.0) < 1e-9, (t, mean)
    # t~ -> 0: the mass-weighted gamma(2) start, 1 - exp(-m)(1 + m)
    F = X.cdf_linear(1e-7)
    m = np.array([0.1, 0.5, 1.0, 2.0, 5.0])
    assert np.abs(F(np.log10(m)) - (1.0 - np.exp(-m) * (1.0 + m))).max() < 1e-5


def test_product_normalisation_and_mean():
    from scipy.special import gammaln
    for t in (0.1, 0.5, 0.9):
        k = np.arange(1, 4000, dtype=float)
        p = np.exp((k - 1) * np.log(k * t) - gammaln(k + 1) - k * t)
        assert abs(p.sum() - 1.0) < 1e-8, (t, p.sum())
        assert abs((k * p).sum() / X.mean_product(t) - 1.0) < 1e-6
        F = X.cdf_product(t)
        assert abs(F(np.array([0.0]))[0] - math.exp(-t)) < 1e-9   # mass in unit grains
