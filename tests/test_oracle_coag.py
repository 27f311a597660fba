"""Pins of the oracle's Monte Carlo on the linear and product coagulation kernels
(Appendix A), against the Smoluchowski solutions through the W1 distance of Appendix B
and the mass-weighted mean grain mass.

The representative-particle method matches these solutions only statistically (finite
neighbourhoods, frozen intervals), so the thresholds sit above the spread of the oracle's
own runs (W1 0.025-0.032 dex for the linear kernel at t~ = 1, 0.007-0.017 dex for the
product kernel at t~ = 0.5, N = 1024, N_K = 16) and well below the distance of a wrong
answer (the same runs against the solution at 0.7 t~: 0.20-0.24 and 0.05-0.08 dex).  The
product-kernel runs permute the particle positions before every neighbour build: the
paper reshuffles the neighbour lists there (Appendix B) so that the population stays well
mixed; with static positions a permutation of the positions does the same.
"""
import math

import numpy as np

from paper_2609_35967_gb300 import workloads as W

import coag_exact as X

W1_LINEAR = 0.06
W1_PRODUCT = 0.035


def _run(oracle, mode, seed, t_end, n=1024, K=16, shuffle=False):
    ins = W.coag_instance(n, K=K, mode=mode, seed=seed)
    P = oracle.params(ins["params"])
    st = oracle.new_state(P)
    s = ins["s"].copy()
    x, y, z = ins["x"].copy(), ins["y"].copy(), ins["z"].copy()
    rng = np.random.default_rng(1000 + seed)
    t = 0.0
    while t < t_end - 1e-12:
        if shuffle:
            p = rng.permutation(n)
            x, y, z = x[p].copy(), y[p].copy(), z[p].copy()
        oracle.interval_step(P, st, x, y, z, s, ins["M"], want=())
        t += st.dt_exe
        assert st.status == 0
    m = math.pi * P.rho_s * s ** 3 / 6.0
    return m, ins["M"], t


def test_linear_kernel_solution(oracle):
    ratios = []
    for seed in (11, 12, 13):
        m, M, t = _run(oracle, W.LINEAR, seed, 1.0)
        assert X.w1(m, M, X.cdf_linear(t), -3.0, 3.0) < W1_LINEAR
        ratios.append(m.mean() / X.mean_linear(t))
    # per-seed spread about 6%: the mean of three within 15%
    assert abs(np.mean(ratios) - 1.0) < 0.15, ratios


def test_product_kernel_solution(oracle):
    ratios = []
    for seed in (11, 12, 13):
        m, M, t = _run(oracle, W.PRODUCT, seed, 0.5, shuffle=True)
        # unit grains coagulate into integer multiples of m0
        assert np.abs(m - np.rint(m)).max() < 1e-9
        assert X.w1(m, M, X.cdf_product(t), 0.0, 3.0) < W1_PRODUCT
        ratios.append(m.mean() / X.mean_product(t))
    assert abs(np.mean(ratios) - 1.0) < 0.10, ratios


def test_wrong_kernel_is_rejected(oracle):
    """The pins separate the kernels: a constant-kernel run misses the linear-kernel
    solution (its mean mass grows as 1 + t~, not 2 exp(2 t~))."""
    ins = W.coag_instance(1024, K=16, mode=W.LINEAR, seed=11)   # gamma(2) start
    P = oracle.params(dict(ins["params"], kernel_mode=W.CONSTANT))
    s = ins["s"].copy()
    st = oracle.new_state(P)
    t = 0.0
    while t < 1.0 - 1e-12:
        oracle.interval_step(P, st, ins["x"], ins["y"], ins["z"], s, ins["M"], want=())
        t += st.dt_exe
    m = math.pi * P.rho_s * s ** 3 / 6.0
    assert X.w1(m, ins["M"], X.cdf_linear(t), -3.0, 3.0) > 2 * W1_LINEAR
