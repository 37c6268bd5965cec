"""The multi-rank (replica) path of the benchmark on CPU with gloo ranks:
the max-over-ranks timing, the weak-scaling value, and the reference arm
under torchrun with two ranks (rank 0 prints the one JSON line)."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank), PMACE_DIST_BACKEND="gloo")
    sys.path.insert(0, ROOT)
    import bench
    dist, w, r, _ = bench.dist_setup()
    assert w == world and r == rank and dist.get_backend() == "gloo"
    dist.barrier()
    vals = bench.max_over_ranks(dist, [10.0 + rank, 5.0 - rank])
    out[rank] = vals
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_with_gloo():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        assert res[rank] == [11.0, 5.0]


def test_weak_scaling_value():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.weak_scaling_value(1, 324 * 10, 2.0) == 1620.0
    assert bench.weak_scaling_value(4, 324 * 10, 2.0) == 6480.0
    assert bench.max_over_ranks(None, [1, 2]) == [1.0, 2.0]


@pytest.mark.timeout(600)
def test_reference_arm_under_torchrun_two_ranks():
    env = dict(os.environ, PMACE_DIST_BACKEND="gloo", OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}", "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--ref-seconds", "0.3",
           "--workload", "small"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
