"""Failure detection with faults made on the host (no GPU fault, no trap, no hang).

* a NaN diameter written into the caller's array: its rates are non-finite, the rate kernel
  sets GD_ST_NONFINITE and gd_stats returns GD_ERR_NONFINITE (both forms);
* gd_collide bounded to one interval on a collision step that needs many: GD_ERR_TIMEOUT;
* a cell size far below the extent that no grid of the context's capacity can take: the
  grid falls back to one cell per instance, GD_ST_CAPACITY is set and gd_stats returns
  GD_ERR_CAPACITY, while the lists stay exact.
"""
import math

import numpy as np
import pytest
import torch

from paper_2609_35967_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_nan_diameter_reports_nonfinite(gd, precision):
    ins = W.patch_instance(1500, K=16, seed=41)
    sess = gd.Session([ins], precision=precision)
    s = sess.t["s"]
    s[123] = float("nan")
    torch.cuda.synchronize()
    sess.build_neighbors()
    sess.collision_rates()
    sess.sample_collisions()
    st = sess.stats(check=False)
    assert st["code"] == gd.GD_ERR_NONFINITE
    assert st["status"] & gd.ST_NONFINITE
    # M is never written, whatever the state
    assert np.array_equal(sess.t["M"].cpu().numpy(), ins["M"])
    sess.close()


def test_collide_bounded_intervals_times_out(gd):
    ins = W.coag_instance(2048, K=16, mode=W.CONSTANT, seed=42)
    sess = gd.Session([ins], precision=gd.GD_FP64)
    with pytest.raises(gd.GDError) as e:
        sess.collide(10.0, max_intervals=1)
    assert e.value.code == gd.GD_ERR_TIMEOUT
    # the context stays usable: a whole bounded step afterwards
    n = sess.collide(0.5)
    assert n >= 1
    assert sess.stats()["status"] == 0
    sess.close()


def test_capacity_fallback_keeps_lists_exact(gd, oracle):
    ins = W.patch_instance(2000, K=16, seed=43)
    ins["params"] = dict(ins["params"], cell_size=1e-300)
    sess = gd.Session([ins], precision=gd.GD_MIXED)
    nbr, d = sess.build_neighbors(want=True)
    st = sess.stats(check=False)
    assert st["code"] == gd.GD_ERR_CAPACITY
    assert st["status"] & gd.ST_CAPACITY
    P = oracle.params(ins["params"])
    q = np.arange(0, 2000, 37)
    onbr, od = oracle.knn(P, ins["x"], ins["y"], ins["z"], q)
    assert np.array_equal(nbr.cpu().numpy()[q], onbr)
    assert np.array_equal(d.cpu().numpy()[q], od)
    sess.close()
