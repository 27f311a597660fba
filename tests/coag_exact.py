"""Smoluchowski solutions of the coagulation tests (Appendix A) and the W1 distance of
Appendix B, for the tests of the linear and product kernels.

All masses are dimensionless (m~ = m / m0) and the distributions are mass-weighted:
F(m~) is the fraction of the total dust mass in grains of mass below m~.

* Linear kernel K = (m_i + m_j)/m0 from the gamma(2) start: the mass-weighted density is
  g/sqrt(1-g) exp(-m~(2-g)) I1(2 m~ sqrt(1-g)) with g = exp(-t~) (Appendix A, Eq. for the
  linear kernel); I1 is evaluated through the exponentially scaled e^-x I1(x).
* Product kernel K = m_i m_j / m0^2 from monodisperse grains, before gelation (t~ < 1):
  the mass-weighted probability of k unit grains is (k t~)^(k-1) exp(-k t~) / k!
  (Appendix A, Trubnikov's solution).
* Moments: the mass-weighted mean grain mass follows 2 exp(2 t~) (linear; dM2/dt = 2 M1 M2)
  and 1 / (1 - t~) (product; dM2/dt = M2^2), with M1 = 1.
"""
import math

import numpy as np
from scipy.special import gammaln, i1e


def cdf_linear(t):
    g = math.exp(-t)
    x = np.linspace(1e-6, 400.0, 400001)
    a = 2.0 * math.sqrt(1.0 - g)
    dens = g / math.sqrt(1.0 - g) * np.exp(-x * (2.0 - g) + a * x) * i1e(a * x)
    cdf = np.cumsum(dens)
    cdf /= cdf[-1]
    lx = np.log10(x)
    return lambda lg: np.interp(lg, lx, cdf)


def cdf_product(t):
    assert 0.0 < t < 1.0
    k = np.arange(1, 4000)
    p = np.exp((k - 1) * np.log(k * t) - gammaln(k + 1) - k * t)
    cdf = np.cumsum(p)
    cdf /= cdf[-1]
    lk = np.log10(k)
    return lambda lg: np.where(lg < 0.0, 0.0,
                               cdf[np.clip(np.searchsorted(lk, lg, side="right") - 1, 0, len(k) - 1)])


def mean_linear(t):
    return 2.0 * math.exp(2.0 * t)


def mean_product(t):
    return 1.0 / (1.0 - t)


def w1(m, M, cdf, lo, hi, n=4001):
    """Appendix B: integral of |F_sim - F_exact| d log10 m~ over [lo, hi] (dex)."""
    lg = np.linspace(lo, hi, n)
    order = np.argsort(m)
    cm = np.cumsum(M[order]) / M.sum()
    idx = np.searchsorted(np.log10(m[order]), lg, side="right")
    fs = np.where(idx > 0, cm[np.maximum(idx - 1, 0)], 0.0)
    return float(np.sum(np.abs(fs - cdf(lg))[:-1] * np.diff(lg)))
