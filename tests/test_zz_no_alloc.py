"""The allocation-free transpose (spgemm_transpose_noalloc) against spgemm_transpose.

It exists for callers that cannot allocate GPU memory at the moment they need
a transpose (inside an allocator or out-of-memory handler, on paths that must
not synchronise the device, under a fixed memory budget): its scratch is a
fixed buffer inside the library.  This test calls it twice in a row through
the C ABI, on problems of different shapes, so the second call also runs on
the buffer contents the first call left behind, and compares both results
with the regular entry point (integer outputs and the gathered values must be
identical).  It lives in a file of its own that pytest collects last.
"""

import ctypes as C

import numpy as np
import pytest

import workloads as w

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
    ]
    results = []
    for A in cases:   # two calls in a row on the shared scratch buffer
        Ad = ops.CsrMatrix.from_host(A.rowptr, A.colidx, A.values, A.shape, device="cuda:0")
        rc, rp, cj, vx, perm = _noalloc_transpose(lib, B, Ad)
        assert rc == 0, B.STATUS_NAMES.get(rc, rc)
        results.append((Ad, rp, cj, vx, perm))
    torch.cuda.synchronize()
    h = ops.SpGEMM()
    for Ad, rp, cj, vx, perm in results:
        At, perm_ref = h.transpose(Ad)
        h.sync()
        assert torch.equal(rp, At.rowptr)
        assert torch.equal(cj, At.colidx)
        assert torch.equal(perm, perm_ref)
        assert torch.equal(vx, At.values)
    h.close()


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
