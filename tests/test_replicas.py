"""The multi-GPU path is replicas: one process per GPU on its own events, no data-path
collective; the only exchange is the timing (max over ranks) and the unit count (sum).  Tested
here with two gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    from paper_2312_11728_gb300 import pipeline, synth as S
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r works on events drawn with seed r: same shape, different content
        g = S.geometry_barrel()
        ev = S.simulate_event(g, 40, rank, 0, eta_max=1.0, noise_per_layer=5)
        value, wall, total = pipeline.replica_throughput(1.0 + rank, 100 * (rank + 1), dist)
        out.put((rank, value, wall, total, float(ev.hit_xyz.sum()), ev.hit_xyz.shape))
    finally:
        dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    import torch.multiprocessing as tmp
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, wall, total, _, _ in res:
        assert wall == 2.0 and total == 300.0          # slowest rank's time, all ranks' units
        assert value == pytest.approx(150.0)
    assert res[0][4] != res[1][4]                       # different events on the two ranks


def test_replica_throughput_single_process():
    from paper_2312_11728_gb300 import pipeline
    value, wall, total = pipeline.replica_throughput(0.5, 1000)
    assert (value, wall, total) == (2000.0, 0.5, 1000.0)


def test_bench_spawns_its_own_ranks():
    """`bench.py --gpus 2` without a launcher re-runs itself as two ranks (torch.distributed.run on
    127.0.0.1); rank 0 alone prints the one JSON line, which reports both ranks.  The reference arm
    (the FP64 oracle on the host cores) needs no GPU, so the ranks run here."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "0"], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 1 and d["value"] > 0
