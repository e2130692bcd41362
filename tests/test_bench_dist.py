"""The benchmark's multi-process logic on CPU (gloo, world size 2): the job
time is the maximum over ranks, the work is summed over ranks, and under
torchrun only rank 0 prints the JSON line."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    ws, r, _ = bench.dist_init()
    assert (ws, r) == (world, rank)
    bench.barrier(ws)
    mx = bench.max_over_ranks(10.0 + rank, ws)    # per-rank step times 10 ms and 11 ms
    sm = bench.sum_over_ranks(100.0 * (rank + 1), ws)
    q.put((rank, mx, sm))
    dist.destroy_process_group()


def test_max_and_sum_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 11.0, 300.0), (1, 11.0, 300.0)]


def test_reference_arm_under_torchrun_prints_one_line():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--workload", "c1_tiny", "--steps", "1", "--warmup", "0", "--ref-nodes", "1"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GUPS" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_resized_workload_is_named_and_has_no_stress_traffic():
    """--n / --bins build a smaller copy of a workload (for captures that must fit on the
    device); the JSON line's config says so, and the stress shape's scaled DRAM traffic is
    not attached to it."""
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    from paper_2410_06106_gb300 import synth
    args = argparse.Namespace(n=512, bins=725)
    assert bench.size_override(args) == {"N": 512, "B": 725}
    assert bench.size_override(argparse.Namespace(n=None, bins=None)) == {}
    cfg = bench.workload_config("c5_stress", 4, 512, 725)
    assert cfg["workload"] == "c5_stress resized" and cfg["N"] == 512 and cfg["bins"] == 725
    assert cfg["slices"] == 4 and cfg["nodes"] == synth.CONFIGS["c5_stress"]["M"]
    full = bench.workload_config("c5_stress")
    assert full["workload"] == "c5_stress" and full["N"] == 2048
    prob = synth.make_problem("c5_stress", slices=1, **bench.size_override(args))
    assert prob["geometry"]["N"] == 512 and prob["geometry"]["B"] == 725 and prob["M"] == 64
    assert bench.profile_traffic("backproject_ustep", None) is None


def test_reference_arm_on_a_problem_with_fewer_nodes_than_sampled():
    """the reference arm samples --ref-nodes nodes (8 by default); a problem with fewer
    (c1_tiny has 4) is sampled whole instead of failing"""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "c1_tiny", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([x for x in out.stdout.splitlines() if x.startswith("{")][-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert "nodes 0..3 " in line["cpu_baseline"]["sample"]
