"""The mixed form's error against the FP64 form after many intervals (the precision split:
FP32 distances, pair rates and waiting times; FP64 prefix, time sums and masses).

The same 2^16-particle disk (log-normal sizes, the bench disk's parameters) runs 40
intervals in each form with the same Philox streams.  The mixed form certifies every FP32
decision against its error bound and settles the rest in FP64, so unless a near tie was
flagged the two runs take the same events: the event counts are equal, every diameter
agrees to 1e-12, and the size spectra of gd_stats (M per fine log-size bin) agree to 1e-12
per bin.  The mass-weighted size spectrum's W1 distance (log10 s, the Appendix B measure
applied to sizes) and mean mass are stated either way.  M is never written in either form.
"""
import numpy as np
import pytest

from paper_2609_35967_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _w1_log(a, b, M):
    """W1 between two mass-weighted size distributions over log10 s (dex)."""
    la, lb = np.sort(np.log10(a)), np.sort(np.log10(b))
    wa = M[np.argsort(np.log10(a))] / M.sum()
    wb = M[np.argsort(np.log10(b))] / M.sum()
    grid = np.union1d(la, lb)
    Fa = np.cumsum(wa)[np.searchsorted(la, grid, side="right") - 1]
    Fb = np.cumsum(wb)[np.searchsorted(lb, grid, side="right") - 1]
    return float(np.sum(np.abs(Fa - Fb)[:-1] * np.diff(grid)))


def _run(gd, ins, precision, n):
    sess = gd.Session([ins], precision=precision)
    for _ in range(n):
        sess.build_neighbors()
        sess.collision_rates()
        sess.sample_collisions()
    st = sess.stats()
    s = sess.t["s"].cpu().numpy()
    M = sess.t["M"].cpu().numpy()
    sess.close()
    return s, M, st


def test_mixed_form_aggregates_match_fp64(gd):
    ins = W.disk_instance(1 << 16, seed=3, sizes=("lognormal", 10.0, 1.0))
    s64, M64, st64 = _run(gd, ins, gd.GD_FP64, 40)
    s32, M32, st32 = _run(gd, ins, gd.GD_MIXED, 40)
    assert st64["status"] == 0 and st32["status"] == 0
    assert np.array_equal(M64, ins["M"]) and np.array_equal(M32, ins["M"])
    w_forms = _w1_log(s64, s32, ins["M"])
    w_start = _w1_log(s64, ins["s"], ins["M"])
    m64 = np.sum(ins["M"] * s64 ** 3) / ins["M"].sum()
    m32 = np.sum(ins["M"] * s32 ** 3) / ins["M"].sum()
    ev64, ev32 = st64["events"], st32["events"]
    sp64 = np.array(st64["instances"][0]["spectrum"])
    sp32 = np.array(st32["instances"][0]["spectrum"])
    nz = (sp64 > 0) | (sp32 > 0)
    sp_err = float(np.abs(sp32[nz] / np.maximum(sp64[nz], 1e-300) - 1.0).max())
    print(f"W1 FP64 vs mixed {w_forms:.2e} dex (evolution since the start {w_start:.2e} dex); "
          f"mass-weighted <s^3> relative difference {m32 / m64 - 1:.2e}; events {ev64} / {ev32}; "
          f"spectrum max bin difference {sp_err:.2e}; mixed FP64 redo {st32['rate_redo']} rates, "
          f"{st32['sample_redo']} samplings")
    assert w_start > 0.0
    near = (st64["near_draw"] + st64["near_dt"] + st64["near_audit"] + st32["near_draw"] + st32["near_dt"]
            + st32["near_audit"])
    if near == 0:
        # certified: the same events, diameters and spectrum
        assert ev32 == ev64
        assert np.abs(s32 / s64 - 1.0).max() < 1e-12
        assert sp_err < 1e-12
    # either way the two forms evolve the spectrum alike, far inside the evolution itself
    assert w_forms < 0.02 * w_start + 1e-4
    assert abs(m32 / m64 - 1.0) < 1e-3
    assert abs(ev32 / ev64 - 1.0) < 1e-3
