"""Thin ctypes binding of the C ABI in include/gd.h (argument marshalling only).

Every function keeps the ABI's name and takes the same arguments; device
buffers are passed as integer addresses (torch.Tensor.data_ptr()).  All work
runs in libgd.so: if the library has not been built, load() raises instead of
falling back to anything else.

`Session` is a convenience wrapper used by the tests and bench.py: it copies a
workload (see workloads.py) into torch device tensors, creates a context on a
torch stream, and forwards each call.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgd.so")

GD_OK, GD_ERR_ARG, GD_ERR_CUDA, GD_ERR_OOM, GD_ERR_CAPACITY = 0, -1, -2, -3, -4
GD_ERR_NONFINITE, GD_ERR_EVENT_CAP, GD_ERR_TIMEOUT, GD_ERR_STATE = -5, -6, -7, -8
GD_FP64, GD_MIXED = 0, 1
GD_GEOM_PATCH, GD_GEOM_DISK = 0, 1
GD_FLAG_TIMING, GD_FLAG_NO_AUDIT = 1, 2
GD_TAU_3D, GD_TAU_2D = 0, 1
ST_EVENT_CAP, ST_DT_FLOOR, ST_NONFINITE, ST_KNN, ST_CAPACITY, ST_TIMEOUT = 1, 2, 4, 8, 16, 32
TIMING_SLOTS = ("cells", "knn", "rates", "interval", "sample", "push", "stats", "diffuse")


class InstanceParams(C.Structure):
    _fields_ = [("geometry", C.c_int32), ("kernel_mode", C.c_int32), ("audit", C.c_int32),
                ("model", C.c_int32), ("r0", C.c_double), ("sigma0", C.c_double),
                ("p", C.c_double), ("T0", C.c_double), ("q", C.c_double), ("alpha", C.c_double),
                ("M_star", C.c_double), ("rho_s", C.c_double), ("s_min", C.c_double),
                ("v_frag", C.c_double), ("eps", C.c_double), ("dt_coll", C.c_double),
                ("dt_fn_max", C.c_double), ("R_in", C.c_double), ("R_out", C.c_double),
                ("box_x", C.c_double), ("box_y", C.c_double), ("t0", C.c_double),
                ("m0", C.c_double), ("cell_size", C.c_double), ("seed", C.c_uint64),
                ("diff_mode", C.c_int32), ("diff_chi", C.c_int32), ("Sc_R", C.c_double),
                ("Sc_Z", C.c_double), ("Sc_phi", C.c_double), ("D0", C.c_double),
                ("spatial_groups", C.c_int32), ("pad_sg", C.c_int32),
                ("beta0", C.c_double), ("kappa0", C.c_double), ("rad_s0", C.c_double),
                ("t_beta", C.c_double), ("rad_pr", C.c_int32), ("tau_geom", C.c_int32),
                ("tau_nr", C.c_int32), ("tau_nmu", C.c_int32), ("tau_nphi", C.c_int32),
                ("pad_tau", C.c_int32), ("tau_rmin", C.c_double), ("tau_rmax", C.c_double),
                ("tau_mu", C.c_double), ("t_start", C.c_double)]


class Config(C.Structure):
    _fields_ = [("n_instances", C.c_int32), ("K", C.c_int32), ("precision", C.c_int32),
                ("flags", C.c_int32), ("offsets", C.c_void_p), ("params", C.c_void_p),
                ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p), ("s", C.c_void_p),
                ("M", C.c_void_p), ("vr", C.c_void_p), ("lth", C.c_void_p), ("lph", C.c_void_p),
                ("stream", C.c_void_p), ("max_events_per_interval", C.c_int64),
                ("cell_factor", C.c_double), ("cell_xsplit", C.c_int32), ("pad1", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("intervals", C.c_int64), ("events", C.c_int64), ("near_draw", C.c_int64),
                ("near_dt", C.c_int64), ("near_audit", C.c_int64), ("launches", C.c_int64),
                ("status", C.c_uint32), ("n_instances", C.c_int32),
                ("kernel_ms", C.c_double * 8), ("kernel_calls", C.c_int64 * 8), ("knn_redo", C.c_int64),
                ("rate_redo", C.c_int64), ("sample_redo", C.c_int64), ("sample_deferred", C.c_int64)]


class InstanceStats(C.Structure):
    _fields_ = [("C", C.c_double), ("dt_exe", C.c_double), ("dt_req", C.c_double),
                ("dt_remain", C.c_double), ("sum_M", C.c_double), ("sum_Mm", C.c_double),
                ("sum_Ms", C.c_double), ("interval", C.c_int64), ("events", C.c_int64),
                ("events_total", C.c_int64), ("near_draw", C.c_int64), ("near_dt", C.c_int64),
                ("near_audit", C.c_int64), ("status", C.c_uint32), ("n_groups", C.c_int32),
                ("spectrum", C.c_double * 96), ("t_rad", C.c_double)]


class GroupStats(C.Structure):
    """gd_group_stats_t: one spatial group of one instance."""
    _fields_ = [("C", C.c_double), ("dt_exe", C.c_double), ("dt_req", C.c_double),
                ("clock", C.c_int64), ("members", C.c_int64), ("intervals", C.c_int64),
                ("events_total", C.c_int64), ("near_dt", C.c_int64), ("near_draw", C.c_int64),
                ("interacts", C.c_uint64), ("level", C.c_int32), ("k_req", C.c_int32),
                ("active", C.c_int32), ("n_groups", C.c_int32), ("status", C.c_uint32),
                ("pad", C.c_int32), ("rounds", C.c_int64), ("delayed", C.c_int64),
                ("breaks", C.c_int64), ("round_clock", C.c_int64)]


class DtRule(C.Structure):
    """gd_dt_rule: the common transport timestep's bounds and local limits."""
    _fields_ = [("dt_max", C.c_double), ("dt_out", C.c_double), ("f_orb", C.c_double),
                ("dx_H", C.c_double), ("c_adv", C.c_double), ("c_diff", C.c_double)]


# every function declared in include/gd.h, with ctypes signatures
SIGNATURES = {
    "gd_create": ([C.c_void_p, C.c_void_p], C.c_int),
    "gd_destroy": ([C.c_void_p], C.c_int),
    "gd_build_neighbors": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "gd_collision_rates": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "gd_sample_collisions": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "gd_push_staggered": ([C.c_void_p, C.c_double], C.c_int),
    "gd_diffuse": ([C.c_void_p, C.c_double], C.c_int),
    "gd_optical_depth": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "gd_collide": ([C.c_void_p, C.c_double, C.c_int32, C.c_int32, C.c_void_p], C.c_int),
    "gd_step": ([C.c_void_p, C.c_double, C.c_int32, C.c_void_p], C.c_int),
    "gd_timestep": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "gd_stats": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "gd_run_intervals": ([C.c_void_p, C.c_int32, C.c_int32], C.c_int),
    "gd_status_string": ([C.c_int], C.c_char_p),
    "gd_autotune": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "gd_controller_bins": ([C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "gd_group_stats": ([C.c_void_p, C.c_int32, C.c_int32, C.c_void_p], C.c_int),
    "gd_neighbors_fixed": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p,
                            C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
}

_lib = None
_lock = threading.Lock()


class GDError(RuntimeError):
    def __init__(self, fn, code):
        msg = load().gd_status_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{fn} failed: {code} ({msg})")
        self.code = code


def load():
    """Loads libgd.so (built by __graft_entry__.build()); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    "libgd.so is not built; run: python -c 'import __graft_entry__ as g; g.build()'")
            L = C.CDLL(LIB_PATH)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def _check(fn, code):
    if code != GD_OK:
        raise GDError(fn, code)
    return code


# ------------------------------------------------------------------ the ABI calls
def gd_create(cfg: Config):
    h = C.c_void_p()
    _check("gd_create", load().gd_create(C.byref(h), C.byref(cfg)))
    return h


def gd_destroy(ctx):
    return _check("gd_destroy", load().gd_destroy(ctx))


def gd_build_neighbors(ctx, nbr_out=0, d_out=0):
    return _check("gd_build_neighbors", load().gd_build_neighbors(ctx, nbr_out or None, d_out or None))


def gd_collision_rates(ctx, lambda_out=0, chan_out=0):
    return _check("gd_collision_rates",
                  load().gd_collision_rates(ctx, lambda_out or None, chan_out or None))


def gd_sample_collisions(ctx, ev_count_out=0, ev_hash_out=0, near_out=0):
    return _check("gd_sample_collisions",
                  load().gd_sample_collisions(ctx, ev_count_out or None, ev_hash_out or None,
                                              near_out or None))


def gd_push_staggered(ctx, dt):
    return _check("gd_push_staggered", load().gd_push_staggered(ctx, float(dt)))


def gd_diffuse(ctx, dt):
    return _check("gd_diffuse", load().gd_diffuse(ctx, float(dt)))


def gd_optical_depth(ctx, tau_out=0, grid_out=0):
    return _check("gd_optical_depth", load().gd_optical_depth(ctx, tau_out or None, grid_out or None))


def gd_collide(ctx, tau, reuse_lists=False, max_intervals=1 << 20):
    """Returns the number of intervals the bounded collision step took."""
    n = C.c_int32(0)
    _check("gd_collide", load().gd_collide(ctx, float(tau), 1 if reuse_lists else 0, int(max_intervals),
                                           C.byref(n)))
    return n.value


def gd_step(ctx, dt, reuse_lists=False):
    """Returns the number of collision intervals of the split timestep."""
    n = C.c_int32(0)
    _check("gd_step", load().gd_step(ctx, float(dt), 1 if reuse_lists else 0, C.byref(n)))
    return n.value


def gd_timestep(ctx, rule: DtRule, dti_out=0):
    """Returns the common transport timestep dt (Sect. 2.6)."""
    dt = C.c_double(0.0)
    _check("gd_timestep", load().gd_timestep(ctx, C.byref(rule), C.byref(dt), dti_out or None))
    return dt.value


def gd_stats(ctx, n_instances):
    st = Stats()
    inst = (InstanceStats * n_instances)()
    code = load().gd_stats(ctx, C.byref(st), inst)
    return code, st, inst


def gd_run_intervals(ctx, n, push=False):
    return _check("gd_run_intervals", load().gd_run_intervals(ctx, int(n), 1 if push else 0))


def gd_autotune(ctx):
    """Returns (cell edge factor, x division) chosen by the library."""
    f, xs = C.c_double(0.0), C.c_int32(0)
    _check("gd_autotune", load().gd_autotune(ctx, C.byref(f), C.byref(xs)))
    return f.value, xs.value


def gd_controller_bins(ctx, instance):
    """(A_b, B_b) of one instance's last interval choice, as two lists of n_groups floats."""
    A, B, n = (C.c_double * 96)(), (C.c_double * 96)(), C.c_int32(0)
    _check("gd_controller_bins", load().gd_controller_bins(ctx, int(instance), A, B, C.byref(n)))
    return list(A)[:n.value], list(B)[:n.value]


def gd_group_stats(ctx, instance, group):
    """The state of one spatial group of one instance, as a dict."""
    g = GroupStats()
    _check("gd_group_stats", load().gd_group_stats(ctx, int(instance), int(group), C.byref(g)))
    return {f: getattr(g, f) for f, _ in GroupStats._fields_ if not f.startswith("pad")}


def gd_status_string(code):
    return load().gd_status_string(int(code)).decode()


def gd_neighbors_fixed(x, y, z, n, K, params: InstanceParams, nbr_out, d_out=0, stream=0):
    """Neighbour lists of one instance without device allocation (see include/gd.h)."""
    return _check("gd_neighbors_fixed",
                  load().gd_neighbors_fixed(x, y, z, int(n), int(K), C.byref(params), nbr_out,
                                            d_out or None, stream or None))


# ------------------------------------------------------------------ convenience wrapper
_PARAM_KEYS = [f for f, _ in InstanceParams._fields_ if not f.startswith("pad")]


def instance_params(d: dict) -> InstanceParams:
    p = InstanceParams()
    for k in _PARAM_KEYS:
        if k in d:
            setattr(p, k, d[k])
    return p


class Session:
    """Owns torch device copies of a workload and one library context."""

    def __init__(self, instances, K=None, precision=GD_FP64, flags=0, device="cuda:0",
                 stream=None, max_events=0, cell_factor=0.0, cell_xsplit=0, velocities=False):
        import numpy as np
        import torch

        from . import workloads
        cat = workloads.concat(instances)
        self.n_inst = len(instances)
        self.K = int(K if K is not None else instances[0]["params"]["K"])
        self.N = int(cat["offsets"][-1])
        self.offsets = np.ascontiguousarray(cat["offsets"], dtype=np.int64)
        self.params_host = [dict(p) for p in cat["params"]]
        dev = torch.device(device)
        t = {k: torch.as_tensor(np.ascontiguousarray(cat[k], dtype=np.float64), device=dev)
             for k in ("x", "y", "z", "s", "M")}
        if velocities:
            for k in ("vr", "lth", "lph"):
                t[k] = torch.as_tensor(np.ascontiguousarray(cat[k], dtype=np.float64), device=dev)
        self.t = t
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        self._params = (InstanceParams * self.n_inst)(*[instance_params(p) for p in cat["params"]])
        cfg = Config()
        cfg.n_instances = self.n_inst
        cfg.K = self.K
        cfg.precision = precision
        cfg.flags = flags
        cfg.offsets = self.offsets.ctypes.data
        cfg.params = C.cast(self._params, C.c_void_p)
        for k in ("x", "y", "z", "s", "M"):
            setattr(cfg, k, t[k].data_ptr())
        if velocities:
            for k in ("vr", "lth", "lph"):
                setattr(cfg, k, t[k].data_ptr())
        cfg.stream = self.stream.cuda_stream
        cfg.max_events_per_interval = max_events
        cfg.cell_factor = cell_factor
        cfg.cell_xsplit = cell_xsplit
        torch.cuda.synchronize(dev)
        self.cfg = cfg
        self.ctx = gd_create(cfg)
        self.device = dev

    def close(self):
        if self.ctx is not None:
            gd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build_neighbors(self, want=False):
        import torch
        if want:
            nbr = torch.empty((self.N, self.K), dtype=torch.int32, device=self.device)
            d = torch.empty(self.N, dtype=torch.float64, device=self.device)
            gd_build_neighbors(self.ctx, nbr.data_ptr(), d.data_ptr())
            self.stream.synchronize()
            return nbr, d
        gd_build_neighbors(self.ctx)
        return None

    def collision_rates(self, want=False, chan=False):
        import torch
        lam = torch.empty(self.N, dtype=torch.float64, device=self.device) if want else None
        ch = torch.empty((self.N, self.K, 2), dtype=torch.float64, device=self.device) if chan else None
        gd_collision_rates(self.ctx, lam.data_ptr() if lam is not None else 0,
                           ch.data_ptr() if ch is not None else 0)
        if want or chan:
            self.stream.synchronize()
        return lam, ch

    def sample_collisions(self, want=False):
        import torch
        if want:
            ec = torch.empty(self.N, dtype=torch.int32, device=self.device)
            eh = torch.empty(self.N, dtype=torch.int32, device=self.device)
            nn = torch.empty(self.N, dtype=torch.int32, device=self.device)
            gd_sample_collisions(self.ctx, ec.data_ptr(), eh.data_ptr(), nn.data_ptr())
            self.stream.synchronize()
            return ec, eh, nn
        gd_sample_collisions(self.ctx)
        return None

    def push_staggered(self, dt=-1.0):
        gd_push_staggered(self.ctx, dt)

    def diffuse(self, dt=-1.0):
        gd_diffuse(self.ctx, dt)

    def optical_depth(self, want_grid=False):
        """tau at every particle (float64 [N]) and, with want_grid, the face grids of the
        instances with a grid, concatenated ([column][face] each)."""
        import torch
        tau = torch.empty(self.N, dtype=torch.float64, device=self.device)
        grid = None
        if want_grid:
            n = 0
            for p in self._params:
                if p.tau_nr > 0 and p.kappa0 > 0.0:
                    nm = 1 if p.tau_geom == GD_TAU_2D else p.tau_nmu
                    n += nm * p.tau_nphi * (p.tau_nr + 1)
            grid = torch.empty(max(n, 1), dtype=torch.float64, device=self.device)
        torch.cuda.synchronize(self.device)
        gd_optical_depth(self.ctx, tau.data_ptr(), grid.data_ptr() if grid is not None else 0)
        self.stream.synchronize()
        return (tau, grid[:n]) if want_grid else tau

    def collide(self, tau, reuse_lists=False, max_intervals=1 << 20):
        return gd_collide(self.ctx, tau, reuse_lists, max_intervals)

    def step(self, dt, reuse_lists=False):
        return gd_step(self.ctx, dt, reuse_lists)

    def timestep(self, dt_max, dt_out=math.inf, f_orb=0.0, dx_H=0.0, c_adv=0.0, c_diff=0.0, want=False):
        """The common transport timestep; with want=True also every particle's dt_i."""
        import torch
        rule = DtRule(dt_max, dt_out, f_orb, dx_H, c_adv, c_diff)
        dti = torch.empty(self.N, dtype=torch.float64, device=self.device) if want else None
        dt = gd_timestep(self.ctx, rule, dti.data_ptr() if dti is not None else 0)
        return (dt, dti) if want else dt

    def run_intervals(self, n, push=False):
        gd_run_intervals(self.ctx, n, push)

    def autotune(self):
        return gd_autotune(self.ctx)

    def controller_bins(self, instance=0):
        return gd_controller_bins(self.ctx, instance)

    def group_stats(self, instance=0):
        """Every spatial group of one instance (one entry for a one-group instance)."""
        G = max(1, int(self._params[instance].spatial_groups))
        return [gd_group_stats(self.ctx, instance, g) for g in range(G)]

    def stats(self, check=True):
        code, st, inst = gd_stats(self.ctx, self.n_inst)
        if check and code != GD_OK:
            raise GDError("gd_stats", code)
        out = {f: getattr(st, f) for f, _ in Stats._fields_ if f not in ("kernel_ms", "kernel_calls")}
        out["kernel_ms"] = dict(zip(TIMING_SLOTS, list(st.kernel_ms)))
        out["kernel_calls"] = dict(zip(TIMING_SLOTS, list(st.kernel_calls)))
        out["code"] = code
        out["instances"] = [{f: (list(getattr(x, f)) if f == "spectrum" else getattr(x, f))
                             for f, _ in InstanceStats._fields_} for x in inst]
        return out
