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


def test_shard_cases_partitions_and_balances():
    """Every case on exactly one rank, each rank's cases in order, and the loads within one
    case of each other (largest-first to the least loaded rank)."""
    import bench
    from paper_1903_06304_gb300 import inputs as inp
    cs = inp.batch_cases(seed=0, ncases=64)
    dofs = [4 * c.n * c.n * (c.p + 1) ** 2 for c in cs]
    for world in (1, 2, 3, 4, 8):
        parts = bench.shard_cases(dofs, world)
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(len(cs)))
        assert all(p == sorted(p) for p in parts)
        loads = [sum(dofs[k] for k in p) for p in parts]
        assert max(loads) - min(loads) <= max(dofs), (world, loads)
    assert bench.shard_cases(dofs, 1) == [list(range(len(cs)))]
    assert bench.shard_cases([5, 5], 3)[2] == []          # more ranks than cases: one idles


def _shard_rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # a fixed total of 6e9 units shared by the ranks; rank r needed 2 + r seconds
    t_max, value = bench.sharded_throughput(2.0 + rank, 6.0e9, world, dist, "cpu")
    out.put((rank, t_max, value))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_throughput_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import socket
    mp = torch.multiprocessing.get_context("spawn")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    q = mp.Queue()
    procs = [mp.Process(target=_shard_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest rank's 3 s; the whole job did 6e9 units in it
    assert [r[1] for r in res] == [3.0, 3.0]
    assert all(abs(r[2] - 2.0) < 1e-12 for r in res)


def test_batch_arm_refuses_on_every_rank_before_any_collective(monkeypatch):
    """Fewer cases than ranks: each rank reaches the same decision from the deterministic
    partition and exits before a process group exists, so no rank is left waiting in a
    barrier or all-reduce of the others."""
    import argparse
    import bench
    import torch.distributed as dist
    for rank in (0, 1):
        monkeypatch.setenv("WORLD_SIZE", "2")
        monkeypatch.setenv("RANK", str(rank))
        monkeypatch.setenv("LOCAL_RANK", str(rank))
        with pytest.raises(SystemExit):
            bench.batch_arm(argparse.Namespace(batch_cases=1))
        assert not dist.is_initialized()
