"""Host logic of bench.py's multi-rank runs, on CPU with the gloo backend.

Each rank times its own problem (weak scaling); the job's step time is the
slowest rank's and its work the sum over ranks.  The reference arm runs on
rank 0 only.
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
