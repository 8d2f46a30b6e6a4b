"""Multi-rank host logic on CPU: replicas across gloo ranks, and the reference arm."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2106_07694_gb300.replicas import replica_glups
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    local_ms = 100.0 * (rank + 1)          # rank 1 is the slow one
    v, t = replica_glups(local_ms, nodes_per_rank=1_000_000, steps=10)
    q.put((rank, v, t))
    dist.destroy_process_group()


def test_replica_throughput_is_max_time_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, v, t in out:
        assert t == 200.0                                   # the slowest rank's time
        assert abs(v - 2 * 1_000_000 * 10 / 0.2 / 1e9) < 1e-12  # nodes of both ranks


def test_single_process_replicas_are_identity():
    sys.path.insert(0, ROOT)
    from paper_2106_07694_gb300.replicas import replica_glups
    v, t = replica_glups(50.0, 2_000_000, 5)
    assert t == 50.0 and abs(v - 0.2) < 1e-12


def test_reference_arm_prints_one_json_line_on_rank0_only():
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GLUPS" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
    env1 = dict(env, RANK="1", WORLD_SIZE="2")
    r1 = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"],
                        cwd=ROOT, env=env1, capture_output=True, text=True, timeout=600)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
