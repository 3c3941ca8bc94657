"""Host-side logic of the multi-GPU benchmark path on CPU (gloo, world size 2):
rank rendezvous on 127.0.0.1, max-over-ranks timing, and weak-scaling
shards (each rank an independent seeded population, no data-path
collective)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    from paper_2311_08927_gb300 import inputs as I
    ws, r, local = bench.dist_env()
    dist = bench.init_dist(ws, "gloo")
    t = bench.max_over_ranks(dist, 10.0 + rank)
    pop = I.config_population(3, n=64, seed_offset=bench.shard_seed_offset(r))
    bench.barrier(dist)
    out[rank] = (ws, r, t, float(pop.y.sum()))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_max_time_and_own_shards():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        ps = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in ps:
            p.start()
        for p in ps:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][:3] == (2, 0, 11.0) and res[1][:3] == (2, 1, 11.0)
    assert res[0][3] != res[1][3]  # independent populations per rank


def test_single_process_needs_no_process_group():
    import bench
    assert bench.init_dist(1, "gloo") is None
    assert bench.max_over_ranks(None, 3.5) == 3.5


def test_reference_arm_under_torchrun_two_ranks():
    """bench.py --impl reference launched as a multi-GPU benchmark run is
    (torch.distributed.run, two ranks, 127.0.0.1): rank 0 alone times the
    oracle and prints one JSON line; rank 1 exits 0 without work."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3",
           "--cpu-seconds", "0.5"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
