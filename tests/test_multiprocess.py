"""The N > 1 path of bench.py on CPU: two gloo ranks on 127.0.0.1.

The hot path shards as independent replicas (one trajectory per rank, no
data-path collective), so the only cross-rank operations are the barrier
around the timed region and the max over ranks of the measured time; the
whole-job value is the units of all ranks over that max. Also checked: the
reference arm prints one JSON line on rank 0 only (other ranks exit 0 without
work) with the same metric, unit and config as the GPU arm.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    import torch
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    t_max = bench.reduce_max(times[rank], torch.device("cpu"))
    value = bench.job_value(1000, world, t_max)
    dist.barrier()
    out[rank] = (t_max, value)
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo():
    world = 2
    times = [1.25, 2.5]   # seconds: rank 1 is the slowest
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, times, out), nprocs=world, join=True)
    for r in range(world):
        t_max, value = out[r]
        assert t_max == 2.5
        assert value == pytest.approx(1000 * world / 2.5)


def _run_bench(env_extra, args):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, env=env, cwd=ROOT,
                          capture_output=True, text=True, timeout=300)


def test_reference_arm_rank0_prints_one_line():
    import bench
    r = _run_bench({"WORLD_SIZE": "1", "RANK": "0", "LOCAL_RANK": "0"},
                   ["--impl", "reference", "--workload", "si8", "--steps", "1", "--warmup", "0",
                    "--ref-sample-s", "0.5"])
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.metric_name("si8", "mixed") and d["unit"] == bench.UNIT
    assert bench.metric_name("si216", "mixed") == bench.METRIC
    assert d["higher_is_better"] is True and d["value"] > 0
    assert d["config"] == bench.workload_config("si8", "mixed", 1)
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    r = _run_bench({"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"},
                   ["--impl", "reference", "--workload", "si8", "--steps", "1", "--warmup", "0", "--gpus", "2"])
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
