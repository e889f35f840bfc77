"""The multi-rank (replica) path of bench.py on CPU: two gloo ranks agree on the slowest
rank's time and on the whole-job throughput; the reference arm runs on rank 0 only."""
import io
import os
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_max, value = bench.replica_throughput(1.0 + rank, 3.0e9, world, dist, "cpu")
    out.put((rank, t_max, value))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import socket
    mp = torch.multiprocessing.get_context("spawn")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    q = mp.Queue()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # slowest rank 2.0 s; both ranks' units (2 x 3e9) over it
    for _, t_max, value in res:
        assert t_max == 2.0
        assert value == pytest.approx(3.0)


def test_replica_throughput_single_rank():
    import bench
    t_max, value = bench.replica_throughput(0.5, 1.0e9, 1, None, "cpu")
    assert t_max == 0.5 and value == pytest.approx(2.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.reference_arm(argparse.Namespace(steps=1, warmup=3, gpus=2))
    assert buf.getvalue() == ""
