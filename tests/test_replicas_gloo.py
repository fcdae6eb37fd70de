"""Host path of the multi-GPU form, on CPU over gloo with world size 2.

The method shards only across independent decompositions (replicas): every
rank runs its own problem with its own seeds, there is no data-path
collective, and the job's time is the slowest rank's.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    from paper_2103_04081_gb300 import inputs as IN
    dist, r, w, _ = bench.dist_setup()
    assert (r, w) == (rank, world)
    mx = bench.max_over_ranks(dist, 10.0 * (rank + 1), "cpu")
    wl = dict(IN.WORKLOADS["c1_60cube_f64"])
    X, A0 = bench.make_inputs(wl, rank, "cpu")
    digest = [float(X.double().sum()), float(A0[0].double().sum())]
    seen = [None] * world
    dist.all_gather_object(seen, digest)
    q.put((rank, mx, bench.whole_job_rate(w, 100, mx), seen))
    dist.destroy_process_group()


def test_two_replicas_time_and_seeds():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, rate, seen in out:
        assert mx == 20.0                          # the slower rank's time, on every rank
        assert rate == pytest.approx(2 * 100 / 0.020)   # whole-job iterations per second
        assert seen[0] != seen[1]                  # each replica has its own data and init
        assert seen[0][0] == out[0][3][0][0]       # and every rank sees the same digests


def test_reference_arm_under_torchrun_prints_one_line():
    """`bench.py --impl reference` launched like the GPU arm: rank 0 times the
    oracle and prints the line; rank 1 exits 0 without work."""
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--workload", "c1_60cube_f64"]
    res = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
