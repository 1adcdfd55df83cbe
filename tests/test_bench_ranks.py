"""Host side of bench.py's multi-rank path (independent replicas, one rank
per GPU): the timed region's duration is the slowest rank's, every rank
learns it, and the whole-job throughput counts every rank's replica.  Run as
two gloo ranks on the CPU."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_CODE = r"""
import json, os, sys
sys.path.insert(0, os.environ["BENCH_ROOT"])
import torch.distributed as dist
import bench
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
ms = 100.0 + 50.0 * rank                      # rank 1 is the slow one
m = bench.max_over_ranks(ms, dist, "cpu")
v = bench.throughput(4608000, 3, world, m)
print(json.dumps({"rank": rank, "ms_max": m, "value": v}))
dist.barrier()
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_take_the_slowest_time():
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   BENCH_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_CODE], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["ms_max"] == 150.0
        # 2 replicas x 4.608 M nodes x 5 fields x 3 steps in 0.150 s
        assert abs(o["value"] - 2 * 5 * 4608000 * 3 / 0.150 / 1e9) < 1e-12


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(123.0, None, "cpu") == 123.0
    assert abs(bench.throughput(1000, 2, 1, 10.0) - 5 * 1000 * 2 / 0.01 / 1e9) < 1e-15


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the FP64 oracle on host cores) needs no
    GPU: one JSON line with the contract's keys, its e2e copying nothing."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], cwd=ROOT, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1
    assert line["config"]["workload"] == "hill3d_60x60x20_r3_fp64_R2"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
