"""Smoluchowski solutions of the coagulation tests (Appendix A) and the W1 distance of
Appendix B, for the tests of the constant, linear and product kernels.

All masses are dimensionless (m~ = m / m0) and the distributions are mass-weighted:
F(m~) is the fraction of the total dust mass in grains of mass below m~.

* Constant kernel K = 1 from monodisperse grains: the number of grains of mass k m0 is
  (t~/2)^(k-1) / (1 + t~/2)^(k+1) (Appendix A).  With q = t~/(2 + t~) the mass-weighted
  probability of k is k (1-q)^2 q^(k-1), whose partial sums have the closed form
  F(k) = 1 - q^k (1 + k (1-q)); that form reaches the t~ = 1e8 of the survey (Appendix B),
  where a direct sum would need ~1e9 terms.
* Linear kernel K = (m_i + m_j)/m0 from the gamma(2) start: the mass-weighted density is
  g/sqrt(1-g) exp(-m~(2-g)) I1(2 m~ sqrt(1-g)) with g = exp(-t~) (Appendix A, Eq. for the
  linear kernel), evaluated in the paper's overflow-free form
  exp(-m~ (g/(1+sqrt(1-g)))^2) I1e(2 m~ sqrt(1-g)) with I1e(x) = e^-x I1(x), on a grid
  logarithmic in m~ that reaches 60 decay lengths of the exponential (m~ ~ 7e5 at t~ = 4).
* Product kernel K = m_i m_j / m0^2 from monodisperse grains, before gelation (t~ < 1):
  the mass-weighted probability of k unit grains is (k t~)^(k-1) exp(-k t~) / k!
  (Appendix A, Trubnikov's solution).
* Moments: the mass-weighted mean grain mass follows 1 + t~ (constant; dM2/dt = M1^2),
  2 exp(2 t~) (linear; dM2/dt = 2 M1 M2) and 1 / (1 - t~) (product; dM2/dt = M2^2), with
  M1 = 1.
"""
import math

import numpy as np
from scipy.special import gammaln, i1e


def cdf_constant(t):
    lq = -math.log1p(2.0 / t)            # ln q, q = t/(2 + t)
    omq = -math.expm1(lq)                # 1 - q

    def F(lg):
        k = np.floor(10.0 ** np.asarray(lg, dtype=float) + 1e-9)
        tail = np.exp(k * lq) * (1.0 + k * omq)
        return np.where(k < 1.0, 0.0, 1.0 - tail)
    return F


def linear_density(t, lx):
    """Mass-weighted density of the linear-kernel solution per unit m~ at m~ = 10^lx."""
    g = math.exp(-t)
    r = math.sqrt(1.0 - g)
    a = g / (1.0 + r)
    x = 10.0 ** lx
    return g / r * np.exp(-x * a * a) * i1e(2.0 * x * r)


def linear_grid(t, n=400001):
    g = math.exp(-t)
    a = g / (1.0 + math.sqrt(1.0 - g))
    return np.linspace(-8.0, math.log10(60.0 / (a * a) + 60.0), n)


def cdf_linear(t):
    lx = linear_grid(t)
    w = linear_density(t, lx) * 10.0 ** lx * math.log(10.0)      # per unit log10 m~
    cdf = np.concatenate(([0.0], np.cumsum(0.5 * (w[1:] + w[:-1]) * np.diff(lx))))
    cdf /= cdf[-1]
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


def mean_constant(t):
    return 1.0 + t


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
