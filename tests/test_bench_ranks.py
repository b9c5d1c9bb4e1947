"""The benchmark's multi-rank control plane on CPU: two gloo ranks, each timing its own
replica; rank 0 must see the max of the times and the sum of the units (replicas, no
data-path collective)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    r, w, local = bench.dist_env()
    dist = bench.dist_init(w)
    bench.barrier(dist)
    t, u = bench.reduce_max_sum(dist, 1.0 + rank, 100.0 * (rank + 1))
    bench.barrier(dist)
    q.put((r, w, t, u))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for r, w, t, u in out:
        assert w == 2
        assert t == 2.0          # max over ranks of the timed seconds
        assert u == 300.0        # total units of all replicas


def test_single_rank_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_init(1) is None
    assert bench.reduce_max_sum(None, 3.0, 7.0) == (3.0, 7.0)


@pytest.mark.slow
def test_reference_arm_line():
    # the reference arm (the FP64 oracle on the host cores) prints one JSON line
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--cpu-samples", "128"], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
