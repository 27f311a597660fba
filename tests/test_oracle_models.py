"""Pins of the oracle's reduced collision models (Sect. 2.5.1): the 2D radial-polar model
(neighbours in the meridional plane, the sampled area times 2 pi R), the vertically
integrated radial-azimuthal model (neighbours in the midplane, the area of a disk of
radius d) and the 1D radial model (an annulus), the last two with the Gaussian vertical
average lambda_ij = N_j K_ij / (V_i sqrt(2 pi (H_i^2 + H_j^2))).

* The measures against quadrature: areas of a disk cut by a straight radial edge and of a
  clipped annulus, and the vertical length against the integral of the product of the
  two Gaussians.
* The neighbour lists against an independent numpy brute force on the model's coordinates.
* The vertically integrated models see the midplane gas; with every particle in the
  midplane the rate of a particle scales exactly as V_3D / V_model between the models.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_2609_35967_gb300 import workloads as W

MODELS = {"3d": 0, "rz": 1, "rphi": 2, "r": 3}


def _disk(oracle, model, **kw):
    ins = W.disk_instance(8, seed=1)
    return oracle.params(dict(ins["params"], model=model, **kw))


def _area_numeric(R, d, R_in, R_out):
    # chords of the disk of radius d around (R, 0), kept where R + u lies inside the disk
    def chord(u):
        return 2.0 * math.sqrt(max(d * d - u * u, 0.0))
    lo, hi = max(-d, R_in - R), min(d, R_out - R)
    return integrate.quad(chord, lo, hi, epsabs=0.0, epsrel=1e-13, limit=200)[0]


def test_measures_against_quadrature(oracle):
    AU = W.AU
    for model in (1, 2, 3):
        P = _disk(oracle, model)
        for R, d in ((5.3 * AU, 0.5 * AU), (20 * AU, 0.7 * AU), (99.8 * AU, 0.4 * AU), (5.05 * AU, 0.2 * AU)):
            V = oracle.volume(P, d, R)
            H = oracle.gas(P, R, 0.0, 0.0)["H"]
            if model == 3:
                lo, hi = max(R - d, P.R_in), min(R + d, P.R_out)
                A = integrate.quad(lambda r: 2 * math.pi * r, lo, hi, epsrel=1e-14)[0]
            else:
                A = _area_numeric(R, d, P.R_in, P.R_out)
            if model == 1:
                want = A * 2 * math.pi * R
            else:
                # 1 / integral of N(Z; 0, H^2) N(Z; 0, H^2) dZ, with Z = H u
                phi2 = integrate.quad(lambda u: math.exp(-u * u) / (2 * math.pi), -12.0, 12.0,
                                      epsabs=0.0, epsrel=1e-13)[0]
                want = A / (phi2 / H)
            assert abs(V / want - 1.0) < 1e-9, (model, R / AU, d / AU, V, want)
    # a vertically integrated patch is periodic: the full disk of radius d
    Pp = oracle.params(dict(W.patch_instance(8, seed=2)["params"], model=2))
    d = 1e11
    H = oracle.gas(Pp, 0.0, 0.0, 0.0)["H"]
    assert abs(oracle.volume(Pp, d, Pp.r0) / (math.pi * d * d * 2 * math.sqrt(math.pi) * H) - 1.0) < 1e-14


def _brute(X, Y, Z, K):
    n = len(X)
    nbr = np.zeros((n, K), dtype=np.int32)
    dist = np.zeros(n)
    for i in range(n):
        d2 = (X - X[i]) ** 2 + (Y - Y[i]) ** 2 + (Z - Z[i]) ** 2
        d2[i] = np.inf
        order = np.lexsort((np.arange(n), d2))[:K - 1]
        dist[i] = math.sqrt(d2[order[-1]])
        nbr[i, 0] = i
        nbr[i, 1:] = np.sort(order)
    return nbr, dist


@pytest.mark.parametrize("model", [1, 2, 3])
def test_knn_in_model_coordinates(oracle, model):
    ins = W.disk_instance(700, seed=7, sizes=("lognormal", 10.0, 1.0))
    P = oracle.params(dict(ins["params"], model=model, K=16))
    x, y, z = ins["x"], ins["y"], ins["z"]
    R = np.sqrt(x * x + y * y)
    X, Y, Z = {1: (R, z, 0 * z), 2: (x, y, 0 * z), 3: (R, 0 * z, 0 * z)}[model]
    nbr, dist = _brute(X, Y, Z, 16)
    q = np.arange(0, 700, 7)
    onbr, od = oracle.knn(P, x, y, z, q)
    assert np.array_equal(onbr, nbr[q])
    assert np.array_equal(od, dist[q])


def test_vertically_integrated_rates(oracle):
    ins = W.disk_instance(600, seed=8, sizes=("lognormal", 10.0, 1.0))
    z0 = np.zeros(600)
    x, y, s, M = ins["x"], ins["y"], ins["s"], ins["M"]
    # midplane gas in the integrated models
    Pr = oracle.params(dict(ins["params"], model=2))
    g = oracle.gas(Pr, x[3], y[3], 1e12)
    g0 = oracle.gas(oracle.params(ins["params"]), x[3], y[3], 0.0)
    assert g["Z"] == 0.0 and g["H"] == g0["H"] and g["rho_g"] == g0["rho_g"]
    # every particle in the midplane: the 3D and the radial-azimuthal models find the same
    # neighbours and the same gas, so the rates differ only by the measure
    q = np.arange(0, 600, 11)
    out = {}
    for model in (0, 2):
        P = oracle.params(dict(ins["params"], model=model))
        nbr, d = oracle.knn(P, x, y, z0, q)
        r = oracle.rates_subset(P, x, y, z0, s, M, q, nbr, d)
        out[model] = (r["lam"], d, nbr)
    assert np.array_equal(out[0][2], out[2][2])
    d = out[0][1]
    R = np.hypot(x[q], y[q])
    P3, P2 = (oracle.params(dict(ins["params"], model=m)) for m in (0, 2))
    ratio = np.array([oracle.volume(P3, d[t], R[t]) / oracle.volume(P2, d[t], R[t]) for t in range(len(q))])
    assert np.all(np.abs(out[2][0] / out[0][0] / ratio - 1.0) < 1e-13)
