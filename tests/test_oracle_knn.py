"""Pins of the oracle's brute-force K-NN (Sect. 2.5.1).

* hand-built lattices with exact equal distances fix the lowest-index tie rule;
* exhaustive enumeration (numpy lexsort over all pairs) on small random sets;
* invariance under a permutation of the input order;
* the minimum image across the periodic x and y edges of a patch.
"""
import numpy as np

from paper_2609_35967_gb300 import workloads as W


def _P(oracle, K, geometry=W.DISK, box=1.0):
    d = dict(geometry=geometry, K=K, box_x=box, box_y=box, r0=W.AU, sigma0=1.0, T0=100.0,
             M_star=W.MSUN, rho_s=1.0)
    return oracle.params(d)


def test_lattice_ties_lowest_index(oracle):
    # points on a line at integer spacing: from the origin, x = +-1 tie, then +-2
    xs = np.array([0.0, 2.0, -1.0, 1.0, -2.0, 3.0])
    z = np.zeros_like(xs)
    P = _P(oracle, K=4)
    nbr, d = oracle.knn(P, xs, z, z, [0])
    # self, then the three nearest others: idx2 (-1), idx3 (+1) and, of the tie
    # at distance 2 between idx1 (+2) and idx4 (-2), the lower index 1
    assert list(nbr[0]) == [0, 1, 2, 3]
    assert d[0] == 2.0
    P3 = _P(oracle, K=3)
    nbr, d = oracle.knn(P3, xs, z, z, [0])
    assert list(nbr[0]) == [0, 2, 3] and d[0] == 1.0
    # query from idx 3 (x=+1): distances 1 (idx0, idx1), 2 (idx2, idx5), 3 (idx4)
    nbr, d = oracle.knn(P3, xs, z, z, [3])
    assert list(nbr[0]) == [3, 0, 1] and d[0] == 1.0
    P5 = _P(oracle, K=5)
    nbr, d = oracle.knn(P5, xs, z, z, [3])
    assert list(nbr[0]) == [3, 0, 1, 2, 5] and d[0] == 2.0


def test_cubic_lattice_ties(oracle):
    g = np.arange(4.0)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    x, y, z = X.ravel(), Y.ravel(), Z.ravel()
    P = _P(oracle, K=7)
    # an interior point has 6 face neighbours at distance 1: the list is all of them
    i = 1 * 16 + 1 * 4 + 1
    nbr, d = oracle.knn(P, x, y, z, [i])
    face = sorted([i - 16, i + 16, i - 4, i + 4, i - 1, i + 1])
    assert list(nbr[0]) == [i] + face and d[0] == 1.0
    # K = 9 takes the two lowest-index edge neighbours at sqrt(2)
    P9 = _P(oracle, K=9)
    nbr, d = oracle.knn(P9, x, y, z, [i])
    d2 = (x - x[i]) ** 2 + (y - y[i]) ** 2 + (z - z[i]) ** 2
    edge = sorted(np.nonzero(d2 == 2.0)[0])[:2]
    assert list(nbr[0]) == [i] + sorted(face + list(edge))
    assert d[0] == np.sqrt(2.0)


def _exhaustive(x, y, z, i, K, box=None):
    dx, dy, dz = x - x[i], y - y[i], z - z[i]
    if box is not None:
        dx = np.where(dx > 0.5 * box, dx - box, np.where(dx < -0.5 * box, dx + box, dx))
        dy = np.where(dy > 0.5 * box, dy - box, np.where(dy < -0.5 * box, dy + box, dy))
    d2 = (dx * dx + dy * dy) + dz * dz
    idx = np.arange(len(x))
    mask = idx != i
    order = np.lexsort((idx[mask], d2[mask]))
    sel = idx[mask][order[:K - 1]]
    return [i] + sorted(sel.tolist()), np.sqrt(d2[mask][order[K - 2]])


def test_exhaustive_random(oracle):
    rng = np.random.default_rng(3)
    for geometry, box in ((W.DISK, None), (W.PATCH, 1.0)):
        n, K = 200, 12
        x, y, z = rng.uniform(-0.5, 0.5, (3, n))
        P = _P(oracle, K, geometry, box or 1.0)
        q = list(range(0, n, 7))
        nbr, d = oracle.knn(P, x, y, z, q)
        for t, i in enumerate(q):
            want, dk = _exhaustive(x, y, z, i, K, box)
            assert list(nbr[t]) == want
            assert d[t] == dk


def test_permutation_invariance(oracle):
    rng = np.random.default_rng(5)
    n, K = 150, 9
    x, y, z = rng.normal(size=(3, n))
    P = _P(oracle, K)
    nbr, d = oracle.knn(P, x, y, z, range(n))
    perm = rng.permutation(n)
    inv = np.argsort(perm)
    nbr2, d2 = oracle.knn(P, x[perm], y[perm], z[perm], range(n))
    for i in range(n):
        t = inv[i]
        assert sorted(perm[nbr2[t]].tolist()) == sorted(nbr[i].tolist())
        assert d2[t] == d[i]


def test_periodic_minimum_image(oracle):
    # two clusters on opposite x edges are neighbours through the periodic edge
    x = np.array([-0.49, 0.49, 0.0, 0.1, -0.1])
    y = np.zeros(5)
    z = np.zeros(5)
    P = _P(oracle, K=2, geometry=W.PATCH, box=1.0)
    nbr, d = oracle.knn(P, x, y, z, [0])
    assert list(nbr[0]) == [0, 1]
    assert abs(d[0] - 0.02) < 1e-15
    Pd = _P(oracle, K=2, geometry=W.DISK)
    nbr, d = oracle.knn(Pd, x, y, z, [0])
    assert list(nbr[0]) == [0, 4]
