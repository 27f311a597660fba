"""gd_neighbors_fixed: the neighbour search without device allocation.

Some callers cannot allocate device memory while they run (their program has
already reserved the GPU's memory for its own pool, or a latency-bound loop
cannot take cudaMalloc's implicit synchronisation).  gd_neighbors_fixed serves
them from a fixed array inside libgd.so.  This test calls it through the C ABI
twice in a row and checks both results against gd_build_neighbors (bit-exact
lists and distances, the bar of every neighbour test), plus its size limit.
The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2609_35967_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _check_against_context(gd, ins, K):
    sess = gd.Session([ins], precision=gd.GD_FP64)
    nbr_ref, d_ref = sess.build_neighbors(want=True)
    nbr_ref, d_ref = nbr_ref.cpu().numpy(), d_ref.cpu().numpy()
    n = len(ins["x"])
    params = gd.instance_params(ins["params"])
    for call in range(2):
        nbr = torch.full((n, K), -7, dtype=torch.int32, device=sess.device)
        d = torch.full((n,), -7.0, dtype=torch.float64, device=sess.device)
        torch.cuda.synchronize()
        gd.gd_neighbors_fixed(sess.t["x"].data_ptr(), sess.t["y"].data_ptr(), sess.t["z"].data_ptr(),
                              n, K, params, nbr.data_ptr(), d.data_ptr(), sess.stream.cuda_stream)
        sess.stream.synchronize()
        assert np.array_equal(nbr.cpu().numpy(), nbr_ref), f"call {call}: lists differ"
        assert np.array_equal(d.cpu().numpy(), d_ref), f"call {call}: distances differ"
    sess.close()


def test_fixed_scratch_patch_matches_build_neighbors(gd):
    _check_against_context(gd, W.patch_instance(3000, K=32, seed=12), 32)


def test_fixed_scratch_disk_matches_build_neighbors(gd):
    _check_against_context(gd, W.disk_instance(20000, seed=13, K=48, sizes=("lognormal", 1.0, 0.5)), 48)


def test_fixed_scratch_rejects_oversize(gd):
    lim = 65536
    params = gd.instance_params(W.patch_instance(64, K=16, seed=1)["params"])
    code = gd.load().gd_neighbors_fixed(ctypes.c_void_p(1), ctypes.c_void_p(1), ctypes.c_void_p(1),
                                        lim + 1, 16, ctypes.byref(params), ctypes.c_void_p(1), None, None)
    assert code == gd.GD_ERR_CAPACITY
