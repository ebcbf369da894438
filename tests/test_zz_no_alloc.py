"""The allocation-free transpose (spgemm_transpose_noalloc) against spgemm_transpose
and the oracle's counting transpose.

It exists for callers that cannot allocate GPU memory at the moment they need
a transpose (inside an allocator or out-of-memory handler, on paths that must
not synchronise the device, under a fixed memory budget): its scratch is a
fixed buffer inside the library.  The tests call it several times in a row
through the C ABI, on problems of different shapes, so later calls also run on
the buffer contents the earlier ones left behind, and compare every result
with the regular entry point and with the oracle (integer outputs and the
gathered values must be identical).  The shapes reach all three column sorts:
warp teams (columns of at most 256 entries), CTA teams (257 to 16 384) and
columns longer than 16 384 entries, whose sort buffers are carved out of the
fixed buffer.  It lives in a file of its own that pytest collects last.
"""

import ctypes as C

import numpy as np
import pytest

import oracle
import workloads as w
from workloads.csr import csr_from_coo

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _noalloc_transpose(lib, B, Ad):
    dev = Ad.colidx.device
    rp = torch.empty(Ad.ncols + 1, dtype=torch.int64, device=dev)
    cj = torch.empty(Ad.nnz, dtype=torch.int32, device=dev)
    vx = torch.empty(Ad.nnz, dtype=Ad.values.dtype, device=dev)
    perm = torch.empty(Ad.nnz, dtype=torch.int64, device=dev)
    desc = Ad.desc()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.spgemm_transpose_noalloc(C.byref(desc), C.c_void_p(rp.data_ptr()), C.c_void_p(cj.data_ptr()),
                                      C.c_void_p(vx.data_ptr()), C.c_void_p(perm.data_ptr()), stream)
    return rc, rp, cj, vx, perm


def test_transpose_noalloc_matches_transpose():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_03065_gb300 import build
    build.build()
    from paper_1801_03065_gb300 import _binding as B
    from paper_1801_03065_gb300 import ops
    lib = B.load()
    cases = [
        w.shuffle_rows(w.random_csr(3000, 500, 6.0, seed=21, dtype=np.float64), 3),
        w.random_csr(1200, 40000, 4.0, seed=22, dtype=np.float32),
        _long_columns(),
    ]
    results = []
    for A in cases:   # calls in a row on the shared scratch buffer
        Ad = ops.CsrMatrix.from_host(A.rowptr, A.colidx, A.values, A.shape, device="cuda:0")
        rc, rp, cj, vx, perm = _noalloc_transpose(lib, B, Ad)
        assert rc == 0, B.STATUS_NAMES.get(rc, rc)
        results.append((A, Ad, rp, cj, vx, perm))
    torch.cuda.synchronize()
    h = ops.SpGEMM()
    for A, Ad, rp, cj, vx, perm in results:
        ref, perm_ref = oracle.transpose(A)
        assert np.array_equal(rp.cpu().numpy(), ref.rowptr)
        assert np.array_equal(cj.cpu().numpy(), ref.colidx)
        assert np.array_equal(perm.cpu().numpy(), perm_ref)
        assert np.array_equal(vx.cpu().numpy().astype(np.float64), ref.values)
        At, perm_gpu = h.transpose(Ad)
        h.sync()
        assert torch.equal(rp, At.rowptr)
        assert torch.equal(cj, At.colidx)
        assert torch.equal(perm, perm_gpu)
        assert torch.equal(vx, At.values)
    h.close()


def _long_columns():
    """40 000 x 8, FP64, two or three entries per row: column 0 holds every row
    (40 000 entries, sorted in buffers carved out of the fixed scratch), column
    1 every 40th row (1 000 entries, a CTA sort), the rest random short columns;
    rows are shuffled so every column's entries arrive out of order."""
    m = 40000
    rng = np.random.default_rng(23)
    rows = [np.arange(m), np.arange(0, m, 40), np.arange(m)]
    cols = [np.zeros(m, np.int64), np.ones(m // 40, np.int64), rng.integers(2, 8, m)]
    A = csr_from_coo(m, 8, np.concatenate(rows), np.concatenate(cols),
                     rng.uniform(-1.0, 1.0, m + m // 40 + m))
    assert int(np.bincount(A.colidx, minlength=8)[0]) > 16384
    return w.shuffle_rows(A, 5)


def test_transpose_noalloc_malformed_rowptr():
    """Row pointers that do not cover the entries give SPGEMM_ERR_BAD_INDEX (the
    kernels' own range checks; no entry is read through a bad pointer)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_03065_gb300 import _binding as B
    from paper_1801_03065_gb300 import ops
    lib = B.load()
    cj = torch.tensor([0, 1, 2, 0, 1, 2, 0, 1], dtype=torch.int32, device="cuda:0")
    vx = torch.arange(8, dtype=torch.float64, device="cuda:0")
    for rowptr in ([0, 100, 8], [0, 3, 9], [1, 4, 8]):
        rp = torch.tensor(rowptr, dtype=torch.int64, device="cuda:0")
        Ad = ops.CsrMatrix(rp, cj, vx, (2, 3))
        rc = _noalloc_transpose(lib, B, Ad)[0]
        assert rc == 8, (rowptr, B.STATUS_NAMES.get(rc, rc))   # SPGEMM_ERR_BAD_INDEX
    # the next call on the same buffer is still correct
    A = w.random_csr(500, 300, 5.0, seed=24, dtype=np.float64)
    Ad = ops.CsrMatrix.from_host(A.rowptr, A.colidx, A.values, A.shape, device="cuda:0")
    rc, rp, cjt, vxt, perm = _noalloc_transpose(lib, B, Ad)
    assert rc == 0
    ref, perm_ref = oracle.transpose(A)
    assert np.array_equal(rp.cpu().numpy(), ref.rowptr) and np.array_equal(cjt.cpu().numpy(), ref.colidx)
    assert np.array_equal(perm.cpu().numpy(), perm_ref) and np.array_equal(vxt.cpu().numpy(), ref.values)


def test_transpose_noalloc_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_03065_gb300 import _binding as B
    lib = B.load()
    d = B.CsrT()
    d.nrows, d.ncols, d.nnz = 10, 10, 5_000_000   # 60 MB of staging: beyond the fixed buffer
    d.rowptr_is_64, d.dtype = 1, B.SPGEMM_R64
    d.rowptr = 1   # never dereferenced: the size check comes first
    d.colidx = 1
    d.values = None
    rc = lib.spgemm_transpose_noalloc(C.byref(d), C.c_void_p(1), C.c_void_p(1), None, None, None)
    assert rc == 3   # SPGEMM_ERR_OOM
