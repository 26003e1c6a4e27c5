"""The N > 1 path of bench.py on CPU: two gloo ranks on 127.0.0.1.

Each rank simulates its own event (weak scaling, no collective on the data
path); the timing reduces with a barrier and max/sum over ranks, and under
torchrun the reference arm prints one line from rank 0 while the other rank
exits 0 without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench._dist()
    assert (w, r) == (world, rank)
    dist = bench._init_pg(w, "gloo")
    bench._barrier(dist)
    mx = bench._max_over_ranks(dist, 10.0 + rank, "cpu")
    sm = bench._sum_over_ranks(dist, 1.0 + rank, "cpu")
    wl = bench.make_workload("three_planes", rank)
    d = wl.events[0][0]
    out.put((rank, mx, sm, wl.seed, d.n, float(d.q[:100].sum()), float(d.x_mm[:100].sum())))
    bench._barrier(dist)
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_shard():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, mx0, sm0, seed0, n0, qs0, xs0), (r1, mx1, sm1, seed1, n1, qs1, xs1) = res
    # timing reductions: max and sum over the two ranks on both ranks
    assert mx0 == mx1 == 11.0
    assert sm0 == sm1 == 3.0
    # each rank its own event of the same size (weak scaling)
    assert seed0 != seed1 and n0 == n1 == 100_000
    assert qs0 != qs1 and xs0 != xs1


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
