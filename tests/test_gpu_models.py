"""GPU parity of the reduced collision models of Sect. 2.5.1 against the oracle.

The 2D radial-polar model (neighbours in the meridional plane, V = A 2 pi R), the
vertically integrated radial-azimuthal model (neighbours in the midplane, V = A times the
Gaussian vertical length) on a disk and on a periodic patch, and the 1D radial model
(the clipped annulus, in a context of its own), the 2D models in one context with a 3D
disk: lists and d_i bit-exact,
lambda*_i within 1e-12 (FP64 form) or 1e-4 (mixed form), first-interval event sequences
identical except flagged near ties, in both forms; then a few whole intervals of each
model against the oracle's interval step.  The argument checks refuse the radial models
on a patch and a 1D instance beside others.
"""
import numpy as np
import pytest

from paper_2609_35967_gb300 import workloads as W

from test_gpu_edge import _lists_rates

pytestmark = pytest.mark.gpu


def _model_insts(models):
    insts = []
    for b, model in enumerate(models):
        ins = W.disk_instance(1500 + 300 * b, seed=90 + b + 5 * model, sizes=("lognormal", 10.0, 1.0), alpha=1e-2)
        ins["params"] = dict(ins["params"], model=model)
        insts.append(ins)
    return insts


@pytest.mark.parametrize("precision", [0, 1])
def test_models_lists_rates_events(gd, oracle, precision):
    # the 2D models and a 3D disk in one context, with a vertically integrated patch
    insts = _model_insts((1, 2, 0))
    pat = W.patch_instance(1200, seed=94, alpha=3e-3)
    pat["params"] = dict(pat["params"], model=2)
    _lists_rates(gd, oracle, insts + [pat], precision)
    # the 1D model takes a context of its own
    _lists_rates(gd, oracle, _model_insts((3, 3)), precision)


@pytest.mark.parametrize("model", [1, 2, 3])
def test_model_intervals(gd, oracle, model):
    ins = W.disk_instance(2500, seed=96 + model, sizes=("lognormal", 10.0, 1.0), alpha=1e-2)
    ins["params"] = dict(ins["params"], model=model)
    sess = gd.Session([ins], precision=gd.GD_FP64)
    P = oracle.params(ins["params"])
    st = oracle.new_state(P)
    s = ins["s"].copy()
    near = 0
    for _ in range(5):
        oracle.interval_step(P, st, ins["x"], ins["y"], ins["z"], s, ins["M"], want=())
        near += st.near_draw + st.near_dt + st.near_audit
        sess.build_neighbors()
        sess.collision_rates()
        sess.sample_collisions()
    g = sess.stats()
    got = sess.t["s"].cpu().numpy()
    sess.close()
    assert g["status"] == 0
    if near + g["near_draw"] + g["near_dt"] + g["near_audit"] == 0:
        assert np.abs(got / s - 1.0).max() < 1e-12
        assert g["instances"][0]["C"] == st.C
    assert np.abs(got / ins["s"] - 1.0).max() > 1e-6      # the sizes did evolve


def test_radial_models_need_a_disk(gd):
    for model in (1, 3):
        pat = W.patch_instance(200, seed=97)
        pat["params"] = dict(pat["params"], model=model)
        with pytest.raises(gd.GDError) as e:
            gd.Session([pat], precision=1)
        assert e.value.code == gd.GD_ERR_ARG
    ins = W.disk_instance(200, seed=98)
    ins["params"] = dict(ins["params"], model=4)
    with pytest.raises(gd.GDError):
        gd.Session([ins], precision=1)
    # 1D instances cannot share a context with the others
    with pytest.raises(gd.GDError) as e:
        gd.Session(_model_insts((3, 0)), precision=1)
    assert e.value.code == gd.GD_ERR_ARG
