"""bench.py's multi-rank logic on the CPU: two gloo ranks, max-over-ranks timing, the
whole-job value assembled by rank 0, and the reference arm printing on rank 0 only."""
import json
import os
import socket
import subprocess
import sys
import types

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench as b
    # rank r is the slow one on a different timer each
    times = b.max_over_ranks([10.0 + rank, 30.0 - rank, 5.0 * (rank + 1)], world, "cpu")
    dist.barrier()
    q.put((rank, times))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0] == got[1] == [11.0, 30.0, 10.0]


def _fake_rank_result(N=1000, K=32, ms=(20.0, 60.0, 25.0)):
    kernel_ms = {"cells": 1.0, "knn": 10.0, "rates": 3.0, "interval": 0.1, "sample": 5.0, "stats": 0.2}
    calls = {k: 10 for k in kernel_ms}
    mixed = {"ms": ms[0], "clocks": None, "launches": 170, "kernel_ms": kernel_ms, "kernel_calls": calls,
             "events": 1234, "status": 0, "cell_factor": 0.8, "rate_redo": 3, "sample_redo": 1,
             "dt_exe": 1.0}
    fp64 = dict(mixed, ms=ms[1])
    return dict(N=N, K=K, cfg={"workload": "test"}, mixed=mixed, fp64=fp64, times=list(ms),
                hbm=6696.8, peak_kind="measured", h2d=40 * N, d2h=8 * N, push=False)


def test_result_line_whole_job_value():
    args = types.SimpleNamespace(steps=10, warmup=3, workload="disk22")
    for world in (1, 2, 4):
        r = _fake_rank_result()
        out = bench.result_line(r, args, world)
        # the units all ranks processed over the slowest rank's time
        assert out["value"] == world * r["N"] * args.steps / (r["times"][0] * 1e-3)
        assert out["n_gpus"] == world and out["scaling"] == "weak"
        assert out["e2e"]["value"] == world * r["N"] * args.steps / (r["times"][2] * 1e-3)
        assert out["roofline"]["kernel"] == "knn"
        assert "stats" not in out["kernels_ms_per_step"]
        assert ("replicas" in out["config"]["parallelism"]) == (world > 1)
        json.dumps(out)


def test_reference_arm_prints_on_rank0_only():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "patch4096", "--steps", "1", "--warmup", "3"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0 and p.stdout.strip() == ""
    env.update(RANK="0", LOCAL_RANK="0")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "patch4096", "--steps", "1", "--warmup", "3"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    line = json.loads(p.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_batch_sharding_splits_instances():
    """The 256-patch batch on N ranks: disjoint shards that cover every instance, sizes within
    one; the whole-job value counts the whole batch once (strong scaling)."""
    for world in (1, 2, 3, 4, 8):
        parts = [bench.shard(256, r, world) for r in range(world)]
        flat = sorted(b for p in parts for b in p)
        assert flat == list(range(256))
        assert max(map(len, parts)) - min(map(len, parts)) <= 1
    args = types.SimpleNamespace(steps=10, warmup=3, workload="patches256")
    r = _fake_rank_result(N=500)
    r["cfg"] = {"workload": "test", "sharding": "r::2", "n_particles_total": 1000}
    out = bench.result_line(r, args, 2)
    assert out["scaling"] == "strong"
    assert out["value"] == 1000 * args.steps / (r["times"][0] * 1e-3)


def test_counter_records_match_the_kernel_sources():
    """The instruction and DRAM records the bench's roofline uses were taken on the kernel
    sources as committed: their digest matches, and the bench-workload roofline of the K-NN
    comes out as the issue bound with its traffic."""
    import bench
    assert bench.csrc_digest() == bench.TRAFFIC_CSRC_SHA256 == bench.INST_CSRC_SHA256
    N = 1 << 22
    km = {"knn": 49.7, "rates": 16.1, "sample": 38.6, "cells": 13.7}
    kc = {k: 10 for k in km}
    rl = bench.roofline_of(km, kc, 32, N, 6790.0, "measured", "disk22", {"fp64_tflops": 1.05}, 2070.0, 152)
    assert rl["bound"] == "alu" and rl["kernel"] == "knn"
    issue = bench.INST["knn"]["inst"] * N / 4.97e-3
    assert abs(rl["frac"] - issue / (4 * 152 * 2070e6)) < 1e-9
    assert abs(rl["traffic"] - bench.TRAFFIC["knn"]["bytes_per_particle"] * N) < 1.0
    assert 0.0 < rl["fp64_pipe"]["frac"] < 1.0 and 0.0 < rl["hbm"]["frac"] < 1.0
