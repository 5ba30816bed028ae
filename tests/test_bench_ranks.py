"""The multi-rank logic of bench.py on CPU: two gloo ranks (127.0.0.1).  With
N GPUs the bench runs N independent replicas of the workload (the solve does
not shard); the ranks only meet at barriers and in the max-over-ranks of the
step time, and only rank 0 prints.  No GPU is used here."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, os.environ["ROOT"])
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
ws, rank, local = bench._dist()
bench._barrier()
m = bench._max_over_ranks(10.0 + 5.0 * rank, "cpu")
bench._barrier()
print(json.dumps({"rank": rank, "ws": ws, "max": m}))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_agree_on_the_slowest_step():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    assert all(o["ws"] == 2 and o["max"] == 15.0 for o in outs)


def test_single_process_helpers_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(3.5, "cpu") == 3.5
    bench._barrier()


def test_reference_arm_other_ranks_exit_without_work():
    # rank 1 of a reference run returns before building or timing anything
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_reference_arm_line_on_the_small_workload():
    # the oracle as the reference arm on the 3,072-unknown workload: one JSON
    # line with the contract's keys, the same config dict as the GPU arm's
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "0",
                        "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300,
                       env=dict(os.environ, RANK="0", LOCAL_RANK="0", WORLD_SIZE="1"))
    assert p.returncode == 0, p.stderr
    d = json.loads(p.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["unit"] == "s" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    from paper_2002_04958_gb300 import inputs
    args = argparse.Namespace(config=0, kind="amg", interp=0, tol=1e-8, nvcyc="1,1,1", inner=0, smoother=0,
                              agg=0, precision=0, batched=1, graph=1)
    assert d["config"] == json.loads(json.dumps(bench._config(args, inputs.preset(0), 1)))
    assert d["metric"] == bench.METRIC


def test_roofline_traffic_entries_match_the_kernel_sources():
    # the stored DRAM traffic of each roofline class applies to the kernel
    # source it was captured on: every class's source region is found, and
    # an entry whose hash differs is reported as null by the bench (not used)
    import json
    import bench
    with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
        table = json.load(f)
    for name in bench.TRAFFIC_SOURCES:
        h = bench.kernel_source_sha256(name)
        assert h is not None, name
        entry = table.get(name)
        if entry and entry.get("kernel_source_sha256") == h:
            assert bench._traffic_from_profiles(name, entry["workload"]) == entry["traffic_bytes_per_launch"]
        else:
            assert bench._traffic_from_profiles(name, (entry or {}).get("workload", "")) is None
