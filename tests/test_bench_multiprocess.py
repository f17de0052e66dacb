"""The multi-process (N > 1) host logic of bench.py, on CPU with the gloo backend.

Under torchrun every timing is the maximum over ranks and only rank 0 prints (the
partitioned step's exchange itself is covered by tests/test_partition_gloo.py).  These
tests run world size 2 on 127.0.0.1 without a GPU."""
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


def _worker(rank, world, port, values, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.max_over_ranks(values[rank], dist, "cpu")
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_timings_are_the_maximum_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    port = _free_port()
    values = [3.25, 7.5]
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, values, out), nprocs=2, join=True)
        assert dict(out) == {0: 7.5, 1: 7.5}


def test_replica_value_counts_every_replica():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_value(9.0, 6.0, 1) == pytest.approx(1500.0)
    assert bench.replica_value(9.0, 6.0, 4) == pytest.approx(6000.0)
    assert bench.max_over_ranks(2.5, None, "cpu") == 2.5


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    port = _free_port()
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                        "--master-port", str(port), "bench.py", "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
