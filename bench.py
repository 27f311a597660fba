#!/usr/bin/env python3
"""Benchmark of the collision step: particle-interval updates per second.

A step is one frozen-neighbour interval of the whole hot path over every particle:
gd_build_neighbors (cell list + K-NN), gd_collision_rates (pair rates, bin moments,
interval choice) and gd_sample_collisions (events, mass/weight updates, audit).

Default workload: the global disk of 2^22 particles with log-normal diameters
(median 10 um, sigma_ln 1), K = 32, measured in the mixed form (value) and in the
plain FP64 form (reported beside it).  Its working set (neighbour lists alone are
512 MB) is larger than the 129 MB L2, so no L2 flush is added between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload disk22|disk20|patches256|disk24|patch4096|disk22_rz|disk22_rphi|disk22_r]

Under torchrun (N > 1) every rank runs an independent replica (seed + rank) on its
own GPU: the path does not shard without a halo exchange, so this is weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-collision updates/s (K-NN+rates+MC) mixed vs FP64 on 1 GB300; % HBM roofline"
UNIT = "particle-interval updates/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def pipe_peaks():
    """FP32 and FP64 FMA-pipe peaks of this GPU (TFLOP/s), measured by the FMA-chain
    microbenchmark in libgdpeaks.so (CUDA events, best of five launches)."""
    import ctypes
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_2609_35967_gb300", "libgdpeaks.so"))
    lib.gdp_fma_tflops.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.gdp_fma_tflops.restype = ctypes.c_int
    out = {}
    for name, fp64 in (("fp32_tflops", 0), ("fp64_tflops", 1)):
        v, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
        rc = lib.gdp_fma_tflops(fp64, ctypes.byref(v), ctypes.byref(ms))
        if rc != 0:
            raise RuntimeError(f"gdp_fma_tflops({fp64}) failed: {rc}")
        out[name] = v.value
    out["how"] = ("FMA chains (8 independent per thread, 256-thread blocks, 8 per SM), "
                  "2 flops per FMA, CUDA events, best of 5 launches")
    return out


def shard(n_items, rank, world):
    """Instances of a batch a rank takes when the batch is split across ranks: rank r takes
    r, r + world, r + 2 world, ... (disjoint, all covered, sizes within one)."""
    return list(range(rank, n_items, world))


def make_workload(name, rank=0, world=1):
    """The workload and its config.  Every workload runs as one replica per rank (its own
    seed: weak scaling), except the 256-patch batch, whose instances are split across the
    ranks (the same batch on any number of ranks: strong scaling, no exchange)."""
    from paper_2609_35967_gb300 import workloads as W
    if name == "disk22":
        return W.config2(seed=1 + rank), dict(workload="global disk 5-100 au, 2^22 particles, "
                                               "log-normal a (median 10 um, sigma_ln 1), K=32")
    if name == "disk20":
        return W.config1(seed=1 + rank), dict(workload="global disk 5-100 au, 2^20 particles, "
                                               "a = 1 um, K=32")
    if name == "patches256":
        insts = W.config3(seed0=1000)
        cfg = dict(workload="256 local patches, N_b log-uniform 2^10-2^16, K=32")
        if world > 1:
            cfg["sharding"] = f"instances r, r + {world}, ... on rank r (the same 256 patches split across ranks)"
            cfg["n_particles_total"] = int(sum(len(i["x"]) for i in insts))
            insts = [insts[b] for b in shard(len(insts), rank, world)]
        return insts, cfg
    if name == "disk24":
        return W.config4(seed=1 + rank), dict(workload="global disk, 2^24 particles, log-normal a "
                                               "(median 1 um, sigma_ln 0.5), K=48, with push")
    if name == "patch4096":
        return W.config0(), dict(workload="local patch at 10 au, 4096 particles, K=32")
    models = {"disk22_rz": (W.MODEL_RZ, "2D radial-polar model (meridional plane)"),
              "disk22_rphi": (W.MODEL_RPHI, "vertically integrated radial-azimuthal model (midplane)"),
              "disk22_r": (W.MODEL_R, "1D radial model")}
    if name in models:
        model, what = models[name]
        insts = W.config2(seed=1 + rank)
        for ins in insts:
            ins["params"] = dict(ins["params"], model=model)
        return insts, dict(workload="global disk 5-100 au, 2^22 particles, log-normal a (median 10 um, "
                                    f"sigma_ln 1), K=32, {what}")
    raise SystemExit(f"unknown workload {name}")


# per-kernel algorithmic HBM bytes per particle (what a launch must read and write)
def algo_bytes(kernel, K, mixed):
    if kernel == "knn":
        # own position (16 B FP32 or 32 B FP64), the list row (4K), d_i and V_i (16 B)
        return (16 if mixed else 32) + 4 * K + 16
    if kernel == "rates":
        # list row (4K), one partner snapshot per particle (16 / 32 B), own position,
        # snapshot, M and V (32 + 32 + 8 + 8), lambda* written (8)
        return 4 * K + (16 if mixed else 32) + 88
    if kernel == "sample":
        return 8 + 8 + 4 + 8          # lambda*, state of the interval, perm, diameter
    if kernel == "cells":
        return 40 + 4 + 4 + 8 + 32 + 32 + (32 if mixed else 0) + 8
    return 0


# DRAM bytes (read + write) of one launch at full size, from a one-pass ncu capture of the
# bench command (dram__bytes_read.sum + dram__bytes_write.sum), per particle.  The records
# hold only while the sources the measured kernels compile from (their files and the shared
# headers) have the content they had at the capture.
TRAFFIC_CSRC_SHA256 = "1cee01f75e8560e8e8e3c027c926c2417346d94da4c0722d7aa176479ea4aa51"
TRAFFIC = {
    "knn": {"workload": "disk22", "bytes_per_particle": 392.34},
    "rates": {"workload": "disk22", "bytes_per_particle": 196.20},
    "sample": {"workload": "disk22", "bytes_per_particle": 161.97},
}


# Instructions of one launch at full size, per particle, from an ncu capture of the bench
# command (smsp__inst_executed.sum: warp instructions issued; sm__inst_executed_pipe_fp64.sum:
# warp instructions on the FP64 pipe), under the same source digest rule as TRAFFIC.
INST_CSRC_SHA256 = TRAFFIC_CSRC_SHA256
INST = {
    "knn": {"workload": "disk22", "inst": 654.53, "fp64_inst": 2.0289},
    "rates": {"workload": "disk22", "inst": 321.52, "fp64_inst": 0.18779},
    "sample": {"workload": "disk22", "inst": 291.51, "fp64_inst": 6.8512},
}

# Issue rate of the SMs: 4 schedulers per SM, one warp instruction each per cycle.
SCHEDULERS_PER_SM = 4


KERNEL_SOURCES = ("gd_common.cuh", "gd_ctx.h", "gd_physics.cuh", "k_cells.cu", "k_knn.cu", "k_mc.cu")


def csrc_digest():
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2609_35967_gb300", "csrc")
    for name in KERNEL_SOURCES:
        h.update(name.encode())
        with open(os.path.join(d, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def kernel_traffic(kernel, workload, n):
    rec = TRAFFIC.get(kernel)
    if not rec or rec["workload"] != workload or csrc_digest() != TRAFFIC_CSRC_SHA256:
        return None
    return rec["bytes_per_particle"] * n


class ClockSampler:
    def __init__(self, index=0):
        self.samples = []
        self.proc = None
        self.index = index

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([t.strip() for t in line.split(",")])

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        rows = [r for r in self.samples if len(r) >= 9]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        for r in rows:
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                "sw_power_cap"), r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def measure_form(gd, insts, dev, precision, steps, warmup, world, push=False, graph=False,
                 cell_factor=0.0, cell_xsplit=0, timing=True):
    """Times `steps` whole intervals of one form after `warmup` (CUDA events on the library's
    stream, barrier and synchronize on both sides).  graph: the intervals are replayed as a
    captured CUDA graph (gd_run_intervals), which per-kernel timing cannot see into."""
    import torch
    sess = gd.Session(insts, precision=precision, device=str(dev), velocities=push,
                      flags=gd.GD_FLAG_TIMING if (timing and not graph) else 0, cell_factor=cell_factor,
                      cell_xsplit=cell_xsplit)
    cf, xs = (cell_factor, max(1, cell_xsplit)) if cell_factor > 0 else sess.autotune()
    st = sess.stream

    def step():
        if graph:
            sess.run_intervals(1, push)
            return
        sess.build_neighbors()
        sess.collision_rates()
        sess.sample_collisions()
        if push:
            sess.push_staggered(-1.0)

    for _ in range(warmup):
        step()
    pre = sess.stats()
    clocks = ClockSampler(dev.index)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        step()
    e1.record(st)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    ck = clocks.stop()
    post = sess.stats()
    res = {"ms": ms, "clocks": ck, "launches": post["launches"] - pre["launches"],
           "kernel_ms": {k: post["kernel_ms"][k] - pre["kernel_ms"][k] for k in post["kernel_ms"]},
           "kernel_calls": {k: post["kernel_calls"][k] - pre["kernel_calls"][k]
                            for k in post["kernel_calls"]},
           "events": post["events"] - pre["events"], "status": post["status"], "cell_factor": cf,
           "cell_xsplit": xs, "knn_redo": post["knn_redo"] - pre["knn_redo"],
           "rate_redo": post["rate_redo"] - pre["rate_redo"],
           "sample_redo": post["sample_redo"] - pre["sample_redo"],
           "sample_deferred": post["sample_deferred"] - pre["sample_deferred"],
           "dt_exe": post["instances"][0]["dt_exe"]}
    sess.close()
    return res


def measure_collide(gd, insts, dev, G, steps, warmup, cell_factor, cell_xsplit):
    """Whole collision steps (gd_collide over dt_coll, one neighbour build each) of the
    workload split into G spatial groups per instance, mixed form: CUDA events on the library
    stream around the timed steps (gd_collide synchronises after every round inside them)."""
    import torch
    xi = [dict(i, params=dict(i["params"], spatial_groups=G)) for i in insts]
    sess = gd.Session(xi, precision=gd.GD_MIXED, device=str(dev), flags=gd.GD_FLAG_TIMING,
                      cell_factor=cell_factor, cell_xsplit=cell_xsplit)
    tau = insts[0]["params"]["dt_coll"]
    for _ in range(warmup):
        sess.collide(tau)
    g0 = sess.group_stats(0)
    pre = sess.stats()
    st = sess.stream
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    rounds = 0
    for _ in range(steps):
        rounds += sess.collide(tau)
    e1.record(st)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    post = sess.stats()
    g1 = sess.group_stats(0)
    sess.close()
    iv = [b["intervals"] - a["intervals"] for a, b in zip(g0, g1)]
    upd = sum(b["members"] * d for b, d in zip(g1, iv))
    return {"ms_per_step": ms / steps, "rounds_per_step": rounds / steps,
            "intervals_per_step": [d / steps for d in iv], "members": [b["members"] for b in g1],
            "updates_per_step": upd / steps, "updates_per_s": upd / (ms * 1e-3),
            "delayed_per_step": (g1[0]["delayed"] - g0[0]["delayed"]) / steps,
            "breaks": g1[0]["breaks"], "events_per_step": (post["events"] - pre["events"]) / steps,
            "kernels_ms_per_step": {k: (post["kernel_ms"][k] - pre["kernel_ms"][k]) / steps
                                    for k in post["kernel_ms"] if post["kernel_ms"][k] > pre["kernel_ms"][k]},
            "status": post["status"]}


def run_gpu(args, rank, world):
    import torch

    from paper_2609_35967_gb300 import binding as gd
    from paper_2609_35967_gb300 import workloads as W

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    insts, cfg = make_workload(args.workload, rank, world)
    K = insts[0]["params"]["K"]
    push = args.workload == "disk24"
    graph = args.workload == "patches256"
    N = int(sum(len(i["x"]) for i in insts))
    hbm, peak_kind = peaks()

    mixed = measure_form(gd, insts, dev, gd.GD_MIXED, args.steps, args.warmup, world, push=push,
                         cell_factor=args.cell_factor, cell_xsplit=args.cell_xsplit)
    fp64 = None
    if not args.skip_fp64:
        fp64 = measure_form(gd, insts, dev, gd.GD_FP64, max(1, args.steps // 3), max(1, args.warmup // 3), world,
                            push=push, cell_factor=args.cell_factor, cell_xsplit=args.cell_xsplit)

    # end to end through the C ABI with host buffers: H2D of the step's inputs from
    # pinned memory and D2H of the diameters inside the timed region, every step
    cat = W.concat(insts)
    sess = gd.Session(insts, precision=gd.GD_MIXED, device=str(dev), velocities=push,
                      cell_factor=mixed["cell_factor"], cell_xsplit=mixed["cell_xsplit"])
    host = {k: torch.as_tensor(cat[k]).pin_memory() for k in ("x", "y", "z", "s", "M")}
    s_back = torch.empty(N, dtype=torch.float64).pin_memory()
    st = sess.stream
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = s_back.numel() * s_back.element_size()

    def e2e_step():
        with torch.cuda.stream(st):
            for k, v in host.items():
                sess.t[k].copy_(v, non_blocking=True)
        sess.build_neighbors()
        sess.collision_rates()
        sess.sample_collisions()
        if push:
            sess.push_staggered(-1.0)
        with torch.cuda.stream(st):
            s_back.copy_(sess.t["s"], non_blocking=True)

    for _ in range(max(1, args.warmup)):
        e2e_step()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        e2e_step()
    e1.record(st)
    torch.cuda.synchronize(dev)
    e2e_ms = max(e0.elapsed_time(e1), (time.perf_counter() - t0) * 1e3)
    sess.close()
    del graph

    # the other single-GPU workloads of the benchmark, each in both forms: the 2^24, K = 48
    # disk with a push after every interval, and the 256-patch batch replayed as a graph
    extras = {}
    if not args.skip_extra and args.workload == "disk22":
        for name, xsteps, xwarm in (("disk24", 3, 3), ("patches256", 10, 3)):
            xinsts, xcfg = make_workload(name, rank)
            xpush, xgraph = name == "disk24", name == "patches256"
            m = measure_form(gd, xinsts, dev, gd.GD_MIXED, xsteps, xwarm, world, push=xpush, graph=xgraph)
            # the graph's per-kernel split, from a short timed run of the same intervals
            split = (measure_form(gd, xinsts, dev, gd.GD_MIXED, 2, 1, world, push=xpush,
                                  cell_factor=m["cell_factor"], cell_xsplit=m["cell_xsplit"])
                     if xgraph else m)
            f = measure_form(gd, xinsts, dev, gd.GD_FP64, 1, 1, world, push=xpush, graph=xgraph,
                             timing=False)
            t = max_over_ranks([m["ms"], f["ms"]], world, dev)
            extras[name] = dict(cfg=xcfg, N=int(sum(len(i["x"]) for i in xinsts)),
                                K=xinsts[0]["params"]["K"], mixed=m, split=split, fp64=f,
                                times=t, steps=xsteps, graph=xgraph, push=xpush)

    # spatial groups (Sect. 2.5.3): whole collision steps of the bench disk in one group and
    # in eight radial groups
    groups = None
    if not args.skip_extra and args.workload == "disk22":
        groups = {f"G{G}": measure_collide(gd, insts, dev, G, 2, 1, mixed["cell_factor"], mixed["cell_xsplit"])
                  for G in (1, 8)}

    times = max_over_ranks([mixed["ms"], fp64["ms"] if fp64 else 0.0, e2e_ms], world, dev)
    pp = None
    try:
        pp = pipe_peaks()
    except Exception as e:          # reported, never fatal: the HBM roofline stands alone
        pp = {"error": str(e)}
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return dict(N=N, K=K, cfg=cfg, mixed=mixed, fp64=fp64, times=times, hbm=hbm, num_sms=num_sms,
                peak_kind=peak_kind, h2d=h2d, d2h=d2h, push=push, extras=extras, pipe_peaks=pp,
                groups=groups)


def max_over_ranks(times, world, dev):
    """Element-wise maximum of the ranks' timings (every rank gets the result)."""
    import torch
    t = torch.tensor(times, dtype=torch.float64)
    if world > 1:
        t = t.to(dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t = t.cpu()
    return t.tolist()


def host_cpu():
    """nproc and the CPU model of this host (from /proc/cpuinfo where it names one)."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read().splitlines()
        for key in ("model name", "Model", "CPU part"):
            for line in info:
                if line.split(":")[0].strip() == key:
                    model = f"{key}: {line.split(':', 1)[1].strip()}"
                    break
            if model:
                break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu": model or platform.processor() or platform.machine(),
            "machine": platform.machine()}


def cpu_oracle_rate(insts, budget_s=12.0, max_q=4096, dt_exe=None, threads=1):
    """The oracle (plain C, FP64, brute-force K-NN) on a bounded sample of query particles of
    the largest instance: each query's K-NN, rates and sampling over one interval of length
    dt_exe (the GPU's, when given).  threads > 1 spreads batches of queries over host threads
    (the particles of an interval are independent and ctypes releases the GIL in the C calls);
    the oracle's code is the same."""
    import concurrent.futures as cf

    import numpy as np

    from oracle import gdo
    ins = max(insts, key=lambda i: len(i["x"]))
    P = gdo.params(ins["params"])
    n = len(ins["x"])
    dt = dt_exe if dt_exe else P.dt_fn_max / 64.0
    gdo.lib()
    t0 = time.perf_counter()

    def work(seed):
        rng = np.random.default_rng(seed)
        done = 0
        while done < max_q // threads and time.perf_counter() - t0 < budget_s:
            q = rng.choice(n, 8, replace=False)
            nbr, d = gdo.knn(P, ins["x"], ins["y"], ins["z"], q)
            gdo.rates_subset(P, ins["x"], ins["y"], ins["z"], ins["s"], ins["M"], q, nbr, d)
            gdo.sample_subset(P, ins["x"], ins["y"], ins["z"], ins["s"], ins["M"], q, nbr, d, dt, 0)
            done += len(q)
        return done

    if threads > 1:
        with cf.ThreadPoolExecutor(max_workers=threads) as ex:
            done = sum(ex.map(work, range(threads)))
    else:
        done = work(0)
    el = time.perf_counter() - t0
    return done / el, done, el, n


def split_step_line(args):
    """Whole numerical timesteps of Sect. 2.6 on the 2^22 disk with velocities, mixed form:
    each step takes dt from gd_timestep and runs C(dt/2) D(dt/2) T(dt) D(dt/2) C(dt/2)
    (gd_step), the first C reusing the previous step's lists.  CUDA events on the library
    stream around the whole loop (gd_collide and gd_timestep synchronise inside it)."""
    import torch
    from paper_2609_35967_gb300 import binding as gd
    from paper_2609_35967_gb300 import workloads as W
    ins = W.disk_instance(1 << 22, seed=1, K=32, sizes=("lognormal", 10.0, 1.0), velocities=True)
    N = len(ins["x"])
    rule = dict(dt_max=ins["params"]["dt_coll"], f_orb=0.05, dx_H=0.1, c_adv=0.5, c_diff=0.5)

    def run(timing):
        sess = gd.Session([ins], precision=gd.GD_MIXED, velocities=True,
                          flags=gd.GD_FLAG_TIMING if timing else 0)
        for k in range(args.warmup):
            sess.step(sess.timestep(**rule), reuse_lists=k > 0)
        pre = sess.stats()
        st = sess.stream
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        n_iv, t_sim = 0, 0.0
        for _ in range(args.steps):
            dt = sess.timestep(**rule)
            n_iv += sess.step(dt, reuse_lists=True)
            t_sim += dt
        e1.record(st)
        torch.cuda.synchronize()
        post = sess.stats()
        sess.close()
        split = {k: (post["kernel_ms"][k] - pre["kernel_ms"][k]) / args.steps for k in post["kernel_ms"]}
        return e0.elapsed_time(e1), n_iv, t_sim, split, post["status"]

    ms, n_iv, t_sim, _, status = run(False)
    _, _, _, split, _ = run(True)
    return {"metric": "particle timesteps/s (Sect. 2.6 split step C D T D C with gd_timestep)",
            "value": N * args.steps / (ms * 1e-3), "unit": "particle-steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "dtype": "f32+f64 (mixed)", "data": "synthetic",
            "config": {"workload": "global disk 5-100 au, 2^22 particles, log-normal a (median 10 um, "
                                   "sigma_ln 1), K=32, with velocities; dt from gd_timestep (f_orb 0.05, "
                                   "dx_H 0.1, c_adv 0.5, c_diff 0.5, dt_max one orbit at 5 au)",
                       "n_particles": N},
            "collision_intervals_per_step": n_iv / args.steps, "dt_mean_s": t_sim / args.steps,
            "kernels_ms_per_step": {k: v for k, v in split.items() if v > 0.0}, "status": status}


def push_line(args):
    """The staggered step (Sect. 2.3.3) on the 2^22 disk with velocities, plain and with the
    radiation forces of Sect. 2.3.2 (beta0 = 0.05 at s0 = 2 um, P-R drag, a 3D optical depth
    grid of 256 x 16 x 256 cells over 5-100 au and |z/r| < 0.2; kappa0 = 3 cm^2/g at 2 um
    gives an outer tau of about 2 at the median column, 40 in the midplane), both forms;
    CUDA events on the library stream.  Algorithmic bytes: the state read (x, y, z, s, v_r,
    l_theta, l_phi; M too with radiation) and written (six FP64), and with radiation the
    grid's accumulators read and cleared and its faces written."""
    import torch
    from paper_2609_35967_gb300 import binding as gd
    from paper_2609_35967_gb300 import workloads as W
    ins = W.disk_instance(1 << 22, seed=1, K=32, sizes=("lognormal", 10.0, 1.0), velocities=True)
    N = len(ins["x"])
    dt = 0.05 * ins["params"]["dt_coll"]
    nr, nm, nph = 256, 16, 256
    rad = dict(ins["params"], beta0=0.05, kappa0=3.0, rad_s0=2e-4, rad_pr=1, tau_geom=0, tau_nr=nr,
               tau_nmu=nm, tau_nphi=nph, tau_rmin=5 * W.AU, tau_rmax=100 * W.AU, tau_mu=0.2)
    hbm, peak_kind = peaks()

    def timed(params, precision):
        sess = gd.Session([dict(ins, params=params)], precision=precision, velocities=True,
                          flags=gd.GD_FLAG_TIMING)
        for _ in range(args.warmup):
            sess.push_staggered(dt)
        pre = sess.stats()["kernel_ms"]["push"]
        st = sess.stream
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            sess.push_staggered(dt)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        kms = (sess.stats()["kernel_ms"]["push"] - pre) / args.steps
        tau_max = 0.0
        if params.get("tau_nr"):
            tau_max = float(sess.optical_depth().max())
        sess.close()
        return ms, kms, tau_max

    out = {"metric": "particle push steps/s (Sect. 2.3.3, with the radiation forces of Sect. 2.3.2)",
           "unit": "particle-steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "higher_is_better": True, "data": "synthetic",
           "config": {"workload": "global disk 5-100 au, 2^22 particles with velocities, dt = dt_coll/20",
                      "n_particles": N, "tau_grid": [nr, nm, nph]}, "forms": {}}
    plain_b = 7 * 8 + 6 * 8
    rad_b = 8 * 8 + 6 * 8
    cells = nr * nm * nph
    grid_b = cells * (16 + 16) + (nr + 1) * nm * nph * 8
    for name, prec in (("mixed", gd.GD_MIXED), ("fp64", gd.GD_FP64)):
        ms0, k0, _ = timed(ins["params"], prec)
        ms1, k1, tmax = timed(rad, prec)
        out["forms"][name] = {
            "plain": {"ms": ms0, "value": N / (ms0 * 1e-3),
                      "roofline": {"bound": "hbm", "achieved": plain_b * N / (k0 * 1e-3) / 1e9, "peak": hbm,
                                   "frac": plain_b * N / (k0 * 1e-3) / 1e9 / hbm, "algo_bytes_per_particle": plain_b}},
            "radiation": {"ms": ms1, "value": N / (ms1 * 1e-3), "tau_max": tmax,
                          "roofline": {"bound": "hbm", "achieved": (rad_b * N + grid_b) / (k1 * 1e-3) / 1e9,
                                       "peak": hbm, "frac": (rad_b * N + grid_b) / (k1 * 1e-3) / 1e9 / hbm,
                                       "algo_bytes": rad_b * N + grid_b}}}
    out["value"] = out["forms"]["mixed"]["radiation"]["value"]
    out["ms_per_step"] = out["forms"]["mixed"]["radiation"]["ms"]
    out["peak_kind"] = peak_kind
    return out


def diffusion_line(args):
    """The dust diffusion step (Sect. 2.4) alone on the 2^22 disk: positions only in the
    mixed form (FP32 draws and coefficients, FP64 positions), and with velocities (the
    velocity basis change in FP64 from direction cosines); CUDA events on the library stream."""
    import torch
    from paper_2609_35967_gb300 import binding as gd
    from paper_2609_35967_gb300 import workloads as W
    ins = W.disk_instance(1 << 22, seed=1, K=32, sizes=("lognormal", 10.0, 1.0), velocities=True)
    N = len(ins["x"])
    dt = 0.05 * ins["params"]["dt_coll"]
    hbm, peak_kind = peaks()

    def timed(velocities):
        sess = gd.Session([ins], precision=gd.GD_MIXED, velocities=velocities, flags=gd.GD_FLAG_TIMING)
        for _ in range(args.warmup):
            sess.diffuse(dt)
        pre = sess.stats()["kernel_ms"]["diffuse"]
        st = sess.stream
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            sess.diffuse(dt)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        kms = (sess.stats()["kernel_ms"]["diffuse"] - pre) / args.steps
        sess.close()
        return ms, kms

    def timed_timestep(precision):
        # Sect. 2.6: the common transport timestep with every limit on (one kernel, a
        # 16-byte copy back and a synchronisation per call)
        sess = gd.Session([ins], precision=precision, velocities=True)
        rule = dict(dt_max=ins["params"]["dt_coll"], f_orb=0.05, dx_H=0.1, c_adv=0.5, c_diff=0.5)
        for _ in range(args.warmup):
            sess.timestep(**rule)
        st = sess.stream
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            dt_g = sess.timestep(**rule)
        e1.record(st)
        torch.cuda.synchronize()
        sess.close()
        return e0.elapsed_time(e1) / args.steps, dt_g

    ms, kms = timed(False)
    ms_t, dt_g = timed_timestep(gd.GD_MIXED)
    ms_t64, dt_g64 = timed_timestep(gd.GD_FP64)
    bytes_t = 7 * 8              # reads x y z s vr lth lph (FP64)
    bytes_pp = 4 * 8 + 3 * 8     # reads x y z s, writes x y z (FP64)
    ach = bytes_pp * N / (kms * 1e-3) / 1e9
    ms_v, kms_v = timed(True)
    bytes_v = 7 * 8 + 6 * 8
    ach_v = bytes_v * N / (kms_v * 1e-3) / 1e9
    return {"metric": "particle diffusion steps/s (Sect. 2.4 Euler-Maruyama)",
            "value": N * args.steps / (ms * 1e-3), "unit": "particle-steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "dtype": "f32 coefficients, f64 positions", "data": "synthetic",
            "config": {"workload": "global disk 5-100 au, 2^22 particles, dt = dt_coll/20, positions only",
                       "n_particles": N},
            "roofline": {"bound": "hbm", "kernel": "diffuse (mixed)", "achieved": ach, "peak": hbm, "unit": "GB/s",
                         "frac": ach / hbm, "peak_kind": peak_kind, "algo_bytes_per_particle": bytes_pp},
            "with_velocities": {"value": N * args.steps / (ms_v * 1e-3), "ms_per_step": ms_v / args.steps,
                                "dtype": "f32 coefficients, f64 positions and velocity basis change",
                                "roofline": {"bound": "hbm", "achieved": ach_v, "peak": hbm,
                                                             "frac": ach_v / hbm,
                                                             "algo_bytes_per_particle": bytes_v}},
            "timestep": {"what": "gd_timestep, every limit on, with velocities (kernel + copy back + sync), "
                                 "mixed form (FP32 limits)",
                         "ms_per_call": ms_t, "dt_over_dt_coll": dt_g / ins["params"]["dt_coll"],
                         "fp64": {"ms_per_call": ms_t64, "dt_rel_diff": dt_g / dt_g64 - 1.0},
                         "roofline": {"bound": "hbm", "achieved": bytes_t * N / (ms_t * 1e-3) / 1e9, "peak": hbm,
                                      "frac": bytes_t * N / (ms_t * 1e-3) / 1e9 / hbm,
                                      "algo_bytes_per_particle": bytes_t}}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--workload", default="disk22")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-extra", action="store_true",
                    help="only the main workload (no disk24 / patches256 keys)")
    ap.add_argument("--cell-factor", type=float, default=0.0,
                    help="cell edge factor; 0 = pick it and the x division with gd_autotune")
    ap.add_argument("--cell-xsplit", type=int, default=0, choices=(0, 1, 2, 4),
                    help="x division of the cell edge when --cell-factor is given (0: 1)")
    ap.add_argument("--diffusion", action="store_true",
                    help="time the dust diffusion step alone (one JSON line, 1 GPU)")
    ap.add_argument("--split-step", action="store_true",
                    help="time whole split timesteps with gd_timestep (one JSON line, 1 GPU)")
    ap.add_argument("--push", action="store_true",
                    help="time the staggered step, plain and with radiation forces (one JSON line, 1 GPU)")
    ap.add_argument("--peaks", action="store_true",
                    help="measure the FP32 / FP64 FMA-pipe peaks alone (one JSON line, 1 GPU)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        insts, cfg = make_workload(args.workload, 0)
        hc = host_cpu()
        nth = max(1, hc["nproc"] or 1)
        for _ in range(args.warmup):
            cpu_oracle_rate(insts, budget_s=1.0, max_q=64 * nth, threads=nth)
        total_q, total_t = 0, 0.0
        for _ in range(args.steps):
            v, q, el, n = cpu_oracle_rate(insts, budget_s=5.0, max_q=1024 * nth, threads=nth)
            total_q += q
            total_t += el
        value = total_q / total_t
        sample = (f"{total_q} query particles of the {n}-particle instance over {args.steps} steps on {nth} "
                  "host threads: brute-force K-NN, FP64 rates and Philox sampling of each (serial C per "
                  "particle, -O2)")
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nth, "kind": "oracle", "sample": sample,
                             "host": hc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return

    if args.peaks:
        if rank == 0:
            import torch
            torch.cuda.init()
            print(json.dumps({"pipe_peaks": pipe_peaks()}))
        return
    if args.diffusion:
        if rank == 0:
            print(json.dumps(diffusion_line(args)))
        return
    if args.split_step:
        if rank == 0:
            print(json.dumps(split_step_line(args)))
        return
    if args.push:
        if rank == 0:
            print(json.dumps(push_line(args)))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group(backend="nccl")
    r = run_gpu(args, rank, world)
    if rank == 0:
        out = result_line(r, args, world)
        if world == 1 and not args.skip_cpu:
            insts, _ = make_workload(args.workload, 0)
            hc = host_cpu()
            nth = max(1, hc["nproc"] or 1)
            dt = r["mixed"]["dt_exe"]
            v1, q1, el1, n = cpu_oracle_rate(insts, budget_s=8.0, max_q=1024, dt_exe=dt)
            v, q, el, n = cpu_oracle_rate(insts, budget_s=12.0, max_q=65536, dt_exe=dt, threads=nth)
            out["cpu_baseline"] = {
                "value": v, "unit": UNIT, "cores": nth, "kind": "oracle", "host": hc,
                "sample": f"{q} query particles of the {n}-particle instance in {el:.1f} s on {nth} host threads: "
                          f"brute-force K-NN, FP64 rates and sampling over the GPU's interval ({dt:.4g} s) "
                          "(serial C, -O2, the same calls spread over threads)",
                "serial": {"value": v1, "cores": 1, "sample": f"{q1} query particles in {el1:.1f} s"}}
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


def kernel_inst(kernel, workload, n):
    rec = INST.get(kernel)
    if not rec or rec["workload"] != workload or csrc_digest() != INST_CSRC_SHA256:
        return None
    return {k: rec[k] * n for k in ("inst", "fp64_inst")}


def roofline_of(km, kc, K, N, hbm, peak_kind, workload, pp=None, sm_mhz=None, num_sms=None):
    """Roofline of the kernel with the largest share of the step, from its mean launch time
    (CUDA events on the library stream).  HBM: algorithmic bytes per launch over that time.
    None of these kernels is HBM-bound; with the launch's instruction counts recorded from
    ncu (INST), the issue fraction (warp instructions over 4 per SM and cycle at the sampled
    SM clock) is the bound reported, and the FP64-pipe fraction (FP64 warp instructions over
    the measured FP64 FMA peak, 32 lanes x 2 flops each) beside it."""
    dom = max(("knn", "rates", "sample", "cells"), key=lambda k: km.get(k, 0.0))
    avg_s = km[dom] / max(1, kc[dom]) * 1e-3
    ach = algo_bytes(dom, K, True) * N / avg_s / 1e9
    hbm_rl = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
              "traffic": kernel_traffic(dom, workload, N), "peak_kind": peak_kind,
              "algo_bytes_per_particle": algo_bytes(dom, K, True), "launch_ms": avg_s * 1e3}
    ins = kernel_inst(dom, workload, N)
    if not ins or not sm_mhz or not num_sms:
        return hbm_rl
    issue_peak = SCHEDULERS_PER_SM * num_sms * sm_mhz * 1e6
    issue = ins["inst"] / avg_s
    out = {"bound": "alu", "kernel": dom, "achieved": issue, "peak": issue_peak, "unit": "warp-instructions/s",
           "frac": issue / issue_peak, "peak_kind": f"{SCHEDULERS_PER_SM} schedulers x {num_sms} SMs x "
                                                    f"{sm_mhz:.0f} MHz (sampled)",
           "traffic": hbm_rl["traffic"], "launch_ms": avg_s * 1e3,
           "inst_per_particle": INST[dom]["inst"], "hbm": {k: hbm_rl[k] for k in
                                                              ("achieved", "peak", "unit", "frac", "peak_kind",
                                                               "algo_bytes_per_particle")}}
    if pp and pp.get("fp64_tflops"):
        fp64_peak = pp["fp64_tflops"] * 1e12 / 64.0       # FP64 FMA warp instructions per second
        out["fp64_pipe"] = {"achieved": ins["fp64_inst"] / avg_s, "peak": fp64_peak,
                            "unit": "FP64 warp-instructions/s", "frac": ins["fp64_inst"] / avg_s / fp64_peak,
                            "peak_kind": "measured FP64 FMA chain (pipe_peaks)"}
    return out


def result_line(r, args, world):
    """The JSON line of the GPU arm from one rank's results with max-over-ranks times."""
    N, K = r["N"], r["K"]
    ms_mixed, ms_fp64, ms_e2e = r["times"]
    # the units all ranks processed: N each (replicas), or the whole batch split across them
    n_job = r["cfg"].get("n_particles_total", world * N)
    value = n_job * args.steps / (ms_mixed * 1e-3)
    km = r["mixed"]["kernel_ms"]
    kc = r["mixed"]["kernel_calls"]
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_mixed / args.steps, "higher_is_better": True,
        "scaling": "strong" if "sharding" in r["cfg"] else "weak", "vs_baseline": None,
        "dtype": "f32+f64 (mixed)", "data": "synthetic",
        "config": dict(r["cfg"], n_particles=N, K=K, precision="mixed",
                       l2="no flush: working set > 129 MB L2 (lists alone 4K B/particle)",
                       parallelism=("1 GPU" if world == 1 else
                                    f"instances split across {world} ranks" if "sharding" in r["cfg"] else
                                    f"{world} independent replicas"),
                       cell_factor=r["mixed"]["cell_factor"],
                       cell_xsplit=r["mixed"].get("cell_xsplit", 1)),
        "events_per_step": r["mixed"]["events"] / args.steps,
        "knn_fp64_redo_per_step": r["mixed"].get("knn_redo", 0) / args.steps,
        "mixed_fp64_settled_per_step": {"rates": r["mixed"]["rate_redo"] / args.steps,
                                        "sampling": r["mixed"]["sample_redo"] / args.steps,
                                        "sampling_deferred": r["mixed"].get("sample_deferred", 0) / args.steps},
        "roofline": roofline_of(km, kc, K, N, r["hbm"], r["peak_kind"], args.workload, r.get("pipe_peaks"),
                                (r["mixed"]["clocks"] or {}).get("sm_mhz"), r.get("num_sms")),
        "kernels_ms_per_step": {k: v / args.steps for k, v in km.items() if v > 0 and k != "stats"},
        "gpu_launches": r["mixed"]["launches"],
        "clocks": r["mixed"]["clocks"],
        "e2e": {"value": n_job * args.steps / (ms_e2e * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"]},
    }
    if r.get("pipe_peaks"):
        out["pipe_peaks"] = r["pipe_peaks"]
    if r["fp64"]:
        st = max(1, args.steps // 3)
        out["fp64"] = {"value": n_job * st / (ms_fp64 * 1e-3), "ms_per_step": ms_fp64 / st,
                       "cell_factor": r["fp64"]["cell_factor"],
                       "kernels_ms_per_step": {k: v / st for k, v in r["fp64"]["kernel_ms"].items()
                                               if v > 0 and k != "stats"}}
        out["mixed_over_fp64"] = out["value"] / out["fp64"]["value"]
    if r.get("groups"):
        g = r["groups"]
        out["spatial_groups"] = {
            "config": "the same disk, whole collision steps of dt_coll (gd_collide, one neighbour build "
                      "each), mixed form, one group against eight equal-width radial groups",
            **g, "step_time_8_over_1": g["G8"]["ms_per_step"] / g["G1"]["ms_per_step"],
            "updates_8_over_1": g["G8"]["updates_per_step"] / g["G1"]["updates_per_step"]}
    for name, x in r.get("extras", {}).items():
        xm, xf = x["times"]
        sp = x["split"]
        sst = 2 if x["graph"] else x["steps"]
        v = world * x["N"] * x["steps"] / (xm * 1e-3)
        vf = world * x["N"] / (xf * 1e-3)
        out[name] = {
            "value": v, "unit": UNIT, "ms_per_step": xm / x["steps"], "steps": x["steps"],
            "config": dict(x["cfg"], n_particles=x["N"], K=x["K"], precision="mixed",
                           timed="one CUDA graph replay per interval (gd_run_intervals)" if x["graph"]
                           else "gd_build_neighbors, gd_collision_rates, gd_sample_collisions"
                           + (", gd_push_staggered" if x["push"] else ""),
                           cell_factor=x["mixed"]["cell_factor"], cell_xsplit=x["mixed"]["cell_xsplit"]),
            "kernels_ms_per_step": {k: w / sst for k, w in sp["kernel_ms"].items() if w > 0 and k != "stats"},
            "roofline": roofline_of(sp["kernel_ms"], sp["kernel_calls"], x["K"], x["N"], r["hbm"],
                                    r["peak_kind"], name, r.get("pipe_peaks"),
                                    (sp.get("clocks") or {}).get("sm_mhz"), r.get("num_sms")),
            "events_per_step": x["mixed"]["events"] / x["steps"],
            "mixed_fp64_settled_per_step": {"rates": x["mixed"]["rate_redo"] / x["steps"],
                                            "sampling": x["mixed"]["sample_redo"] / x["steps"]},
            "fp64": {"value": vf, "ms_per_step": xf},
            "mixed_over_fp64": v / vf,
            "status": x["mixed"]["status"],
        }
    return out


if __name__ == "__main__":
    main()
