"""gd_neighbors_fixed: the neighbour search without device allocation.

Some callers cannot allocate device memory while they run (their program has
already reserved the GPU's memory for its own pool, or a latency-bound loop
cannot take cudaMalloc's implicit synchronisation).  gd_neighbors_fixed serves
them from a fixed array inside libgd.so.  This test calls it through the C ABI
twice in a row and checks both results bit-exactly against the oracle's brute
force and against gd_build_neighbors (the bar of every neighbour test), on a
patch, a disk, an instance of K coincident particles and a cell size far below
the extent (both served by the grid's bounded fallback), plus its size limit.
The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2609_35967_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _fixed(gd, ins, K, stream=0, params=None):
    n = len(ins["x"])
    dev = torch.device("cuda:0")
    xs = [torch.as_tensor(np.ascontiguousarray(ins[k], dtype=np.float64), device=dev) for k in ("x", "y", "z")]
    params = params or gd.instance_params(ins["params"])
    out = []
    for _ in range(2):
        nbr = torch.full((n, K), -7, dtype=torch.int32, device=dev)
        d = torch.full((n,), -7.0, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        gd.gd_neighbors_fixed(xs[0].data_ptr(), xs[1].data_ptr(), xs[2].data_ptr(), n, K, params,
                              nbr.data_ptr(), d.data_ptr(), stream)
        torch.cuda.synchronize()
        out.append((nbr.cpu().numpy(), d.cpu().numpy()))
    return out


def _check(gd, oracle, ins, K, params=None):
    n = len(ins["x"])
    P = oracle.params(dict(ins["params"], K=K))
    onbr, od = oracle.knn(P, ins["x"], ins["y"], ins["z"], np.arange(n))
    for call, (nbr, d) in enumerate(_fixed(gd, ins, K, params=params)):
        assert np.array_equal(nbr, onbr), f"call {call}: lists differ from the oracle's"
        assert np.array_equal(d, od), f"call {call}: distances differ from the oracle's"
    sess = gd.Session([ins], K=K, precision=gd.GD_FP64)
    nbr_ref, d_ref = sess.build_neighbors(want=True)
    assert np.array_equal(nbr_ref.cpu().numpy(), onbr)
    assert np.array_equal(d_ref.cpu().numpy(), od)
    sess.close()


def test_fixed_scratch_patch_matches_oracle(gd, oracle):
    _check(gd, oracle, W.patch_instance(3000, K=32, seed=12), 32)


def test_fixed_scratch_disk_matches_oracle(gd, oracle):
    _check(gd, oracle, W.disk_instance(20000, seed=13, K=48, sizes=("lognormal", 1.0, 0.5)), 48)


def test_fixed_scratch_coincident_particles(gd, oracle):
    """K particles of a disk at one position: the zero-volume grid falls back to one cell;
    every distance is zero and ties go to the lowest index."""
    ins = W.disk_instance(16, seed=14, K=16)
    for k in ("x", "y", "z"):
        ins[k] = np.full(16, ins[k][3])
    _check(gd, oracle, ins, 16)


def test_fixed_scratch_tiny_cell_size(gd, oracle):
    """A cell size far below the extent cannot fit the fixed grid: the bounded fallback
    keeps every cell index inside the scratch and the lists stay exact."""
    ins = W.patch_instance(2000, K=16, seed=15)
    params = gd.instance_params(dict(ins["params"], cell_size=1e-30))
    _check(gd, oracle, ins, 16, params=params)


def test_fixed_scratch_rejects_oversize(gd):
    lim = 65536
    params = gd.instance_params(W.patch_instance(64, K=16, seed=1)["params"])
    code = gd.load().gd_neighbors_fixed(ctypes.c_void_p(1), ctypes.c_void_p(1), ctypes.c_void_p(1),
                                        lim + 1, 16, ctypes.byref(params), ctypes.c_void_p(1), None, None)
    assert code == gd.GD_ERR_CAPACITY
