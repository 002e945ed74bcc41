"""The N > 1 path of bench.py on CPU: world-size-2 gloo ranks, each with its
own film (seed offset = rank) and its own time; the whole-job value uses the
slowest rank's time on every rank (no collective on the data path)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 100.0 + 50.0 * rank                     # rank 1 is the slow one
    ms_max, value = bench.replica_throughput(ms_local, 1000, world)
    w = bench.make_workload("grounded", seed_offset=rank, size=(8, 8, 4))
    q.put((rank, ms_max, value, float(w.P0.sum())))
    dist.destroy_process_group()


def test_two_gloo_replicas_share_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, ms0, v0, s0), (_, ms1, v1, s1) = out
    assert ms0 == ms1 == 150.0
    assert v0 == v1 == pytest.approx(2 * 1000 / 0.150)
    assert s0 != s1                                    # every rank advances its own film


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.replica_throughput(200.0, 500, 1) == (200.0, pytest.approx(2500.0))


def test_bench_launches_replicas_itself():
    """`bench.py --gpus 2` with no launcher around it starts two ranks itself
    (torch's launcher, rendezvous on 127.0.0.1); the self-test mode runs the
    same rank arithmetic on gloo without a GPU, and rank 0 alone prints."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2", "--replica-selftest",
                        "--steps", "10"], capture_output=True, text=True, timeout=300, env=env, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1                              # rank 0 only
    line = lines[0]
    assert line["n_gpus"] == 2
    assert line["ms_per_step"] == pytest.approx(20.0 / 10)   # the slower rank: 10 ms x 2
    assert line["value"] == pytest.approx(2 * 1000 * 10 / 0.020)
