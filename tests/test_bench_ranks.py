"""Host logic of bench.py's multi-rank runs, on CPU with the gloo backend.

The job's step time is the slowest rank's and its work the sum over ranks.
Under N > 1 the step is row-sharded: every rank takes a flop-balanced range of
rows (the partition is host logic) and the shards' sizes are all-gathered.
The reference arm runs on rank 0 only.
"""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, f = bench.reduce_over_ranks(10.0 + rank, 100.0 * (rank + 1), world, device="cpu")
    q.put((rank, t, f))
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_and_total_work_over_two_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    for _, t, f in res:
        assert t == 11.0      # max over ranks
        assert f == 300.0     # sum over ranks


def _shard_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads as w
    A = w.stencil3d_27pt(12, seed=1)
    lens = np.diff(A.rowptr)
    rf = np.zeros(A.nrows, np.int64)
    np.add.at(rf, A.row_ids(), lens[A.colidx])
    prefix = np.concatenate([[0], np.cumsum(rf)])
    r0, r1 = bench.shard_bounds(prefix, rank, world)
    # shard sizes: this rank's rows of A*A and a second product's rows
    nnz = [int(prefix[r1] - prefix[r0]), 10 * (rank + 1)]
    first, total = bench.shard_exchange(nnz, world, device="cpu")
    q.put((rank, r0, r1, nnz, first, total, int(prefix[-1]), A.nrows))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_step_partition_and_exchange_over_two_ranks():
    """The row ranges of the ranks tile [0, m) and each holds about half the
    flops; the all-gather places every shard after the lower ranks' shards."""
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, a0, a1, n0, f0, t0, fm, m), (_, b0, b1, n1, f1, t1, _, _) = res
    assert a0 == 0 and a1 == b0 and b1 == m
    assert abs(n0[0] - fm / 2) <= 0.05 * fm
    assert f0 == [0, 0] and f1 == [n0[0], n0[1]]
    assert t0 == t1 == [n0[0] + n1[0], n0[1] + n1[1]]


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(7.5, 42.0, 1, device="cpu") == (7.5, 42.0)


def test_reference_arm_other_ranks_do_nothing(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    bench.run_reference(bench.parse_args(["--impl", "reference", "--gpus", "2"]))
    assert capsys.readouterr().out == ""
