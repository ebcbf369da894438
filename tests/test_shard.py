"""Row-range sharding of C = A*B across devices (1-D row partition by flops).

CPU: the host partitioner through the C ABI (no GPU needed) and the nnz
exchange over gloo with two ranks.  GPU: shards computed one after another on
one device concatenate to the full product, checked against the oracle.
"""

import os
import socket
import sys

import numpy as np
import pytest

import oracle
import workloads as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _ops():
    from paper_1801_03065_gb300 import build
    build.build()
    from paper_1801_03065_gb300 import ops
    return ops


def _check_bounds(b, m, parts):
    assert len(b) == parts + 1 and b[0] == 0 and b[-1] == m
    assert all(x <= y for x, y in zip(b, b[1:]))


@pytest.mark.parametrize("parts", [1, 2, 3, 7, 16])
def test_partition_balances_flops(parts):
    ops = _ops()
    A = w.rmat_symmetric(scale=10, seed=3)
    lens = np.diff(A.rowptr)
    rf = np.zeros(A.nrows, np.int64)
    np.add.at(rf, A.row_ids(), lens[A.colidx])
    prefix = np.concatenate([[0], np.cumsum(rf)])
    b = ops.partition_rows(prefix, parts)
    _check_bounds(b, A.nrows, parts)
    share = prefix[-1] / parts
    for p in range(1, parts):
        # each boundary is the row nearest to its target (rows are indivisible)
        t = share * p
        r = b[p]
        cands = [abs(prefix[x] - t) for x in range(max(b[p - 1], r - 1), min(A.nrows, r + 1) + 1)]
        assert abs(prefix[r] - t) <= min(cands) + 1e-9
        assert abs(prefix[r] - t) <= rf.max()


def test_partition_edge_cases():
    ops = _ops()
    # all work in one row: the other shards are empty around it
    pre = np.array([0, 0, 0, 100, 100, 100], np.int64)
    b = ops.partition_rows(pre, 4)
    _check_bounds(b, 5, 4)
    assert sum(1 for p in range(4) if b[p] <= 2 < b[p + 1]) == 1
    # no work: equal row counts
    b = ops.partition_rows(np.zeros(11, np.int64), 5)
    assert b == [0, 2, 4, 6, 8, 10]
    # more shards than rows
    b = ops.partition_rows(np.array([0, 5, 10], np.int64), 4)
    _check_bounds(b, 2, 4)
    # empty matrix
    assert ops.partition_rows(np.zeros(1, np.int64), 3) == [0, 0, 0, 0]
    from paper_1801_03065_gb300._binding import SpGEMMError
    with pytest.raises(SpGEMMError):
        ops.partition_rows(np.array([0, 5, 3], np.int64), 2)    # decreasing prefix
    with pytest.raises(SpGEMMError):
        ops.partition_rows(np.array([0, 5], np.int64), 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1801_03065_gb300 import ops
    # the same prefix on every rank gives the same bounds; nnz of the shards are exchanged
    pre = np.concatenate([[0], np.cumsum(np.arange(1, 101))]).astype(np.int64)
    b = ops.partition_rows(pre, world)
    q.put((rank, b, ops.shard_offsets(10 * (rank + 1))))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_offsets_over_two_gloo_ranks():
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
    (r0, b0, o0), (r1, b1, o1) = res
    assert b0 == b1 and b0[0] == 0 and b0[-1] == 100
    assert o0 == (0, 30) and o1 == (10, 30)


@pytest.mark.gpu
@pytest.mark.parametrize("parts", [2, 3, 5])
def test_shards_concatenate_to_the_full_product(parts):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ops = _ops()
    from _util import dev, tol_of
    A = w.rmat_symmetric(scale=11, seed=5)
    A.values = np.random.default_rng(6).uniform(-1, 1, A.nnz)
    Ad = dev(A)
    h = ops.SpGEMM()
    prefix = h.row_flops(Ad, Ad)
    lens = np.diff(A.rowptr)
    rf = np.zeros(A.nrows, np.int64)
    np.add.at(rf, A.row_ids(), lens[A.colidx])
    assert np.array_equal(prefix.cpu().numpy(), np.concatenate([[0], np.cumsum(rf)]))
    bounds = ops.partition_rows(prefix, parts)
    rps, cjs, vxs = [np.zeros(1, np.int64)], [], []
    for p in range(parts):
        Cb, r0, off, total = ops.shard_multiply(h, Ad, Ad, p, parts)
        assert r0 == bounds[p]
        rp, cj, vx = Cb.to_host()
        rps.append(rp[1:] + rps[-1][-1])
        cjs.append(cj)
        vxs.append(vx)
    rp = np.concatenate(rps)
    cj = np.concatenate(cjs)
    vx = np.concatenate(vxs)
    C, S = oracle.spgemm(A, A)
    assert np.array_equal(rp, C.rowptr) and np.array_equal(cj, C.colidx)
    assert np.all(np.abs(vx - C.values) <= tol_of(np.float64) * S)


def test_row_block_rebases_and_views_on_host_tensors():
    ops = _ops()
    A = w.random_csr(50, 40, 4.0, seed=91)
    Ah = ops.CsrMatrix(torch.from_numpy(A.rowptr.copy()), torch.from_numpy(A.colidx.copy()),
                       torch.from_numpy(A.values.copy()), A.shape)
    for r0, r1 in ((0, 50), (0, 0), (7, 23), (49, 50), (50, 50)):
        blk = ops.row_block(Ah, r0, r1)
        assert blk.shape == (r1 - r0, 40)
        rp = blk.rowptr.numpy()
        assert rp[0] == 0 and np.array_equal(rp, A.rowptr[r0:r1 + 1] - A.rowptr[r0])
        lo, hi = A.rowptr[r0], A.rowptr[r1]
        assert np.array_equal(blk.colidx.numpy(), A.colidx[lo:hi])
        assert np.array_equal(blk.values.numpy(), A.values[lo:hi])
        if hi > lo:   # views of A's arrays, not copies
            assert blk.colidx.data_ptr() == Ah.colidx[lo:].data_ptr()


def test_partition_rows_accepts_tensors():
    ops = _ops()
    pre = torch.tensor([0, 3, 3, 9, 12, 20], dtype=torch.int64)
    assert ops.partition_rows(pre, 2) == ops.partition_rows(pre.numpy(), 2)
    b = ops.partition_rows(pre, 2)
    _check_bounds(b, 5, 2)
    assert b[1] in (3, 4)   # 10 of 20 flops: after row 2 (9) or row 3 (12), whichever is nearer
    assert b[1] == 3
