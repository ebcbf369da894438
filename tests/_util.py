"""Shared helpers of the GPU parity tests (device transfer, oracle comparison)."""

from __future__ import annotations

import numpy as np

import oracle
from workloads.csr import Csr

TOL = {np.float64: 1e-13, np.float32: 1e-5}


def tol_of(dtype) -> float:
    return TOL[np.dtype(dtype).type]


def dev(M: Csr, dtype=np.float64, rp64=True, device="cuda:0", with_values=True):
    import torch
    from paper_1801_03065_gb300 import ops
    vals = None
    if with_values and M.values is not None:
        vals = M.values.astype(dtype)
    return ops.CsrMatrix.from_host(M.rowptr, M.colidx, vals, M.shape, device=device,
                                   rowptr_dtype=torch.int64 if rp64 else torch.int32)


def host_inputs(M: Csr, dtype):
    """The matrix exactly as the GPU sees it (values rounded to dtype)."""
    return Csr(M.nrows, M.ncols, M.rowptr, M.colidx,
               None if M.values is None else M.values.astype(dtype))


def assert_matches_oracle(A: Csr, B: Csr, Cd, dtype, ref=None):
    """Structure bit-exact, values within tol * sum |a||b| (per entry)."""
    Ah, Bh = host_inputs(A, dtype), host_inputs(B, dtype)
    if ref is None:
        ref = oracle.spgemm(Ah, Bh)
    C, S = ref
    rp, cj, vx = Cd.to_host()
    assert rp.shape == C.rowptr.shape
    assert np.array_equal(rp, C.rowptr), "row pointers differ"
    assert np.array_equal(cj, C.colidx), "column indices differ"
    err = np.abs(vx.astype(np.float64) - C.values)
    bound = tol_of(dtype) * S
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, "values out of tolerance at %s (err %s, bound %s)" % (
        bad[:5], err[bad[:5]], bound[bad[:5]])
    return ref


def row_sample(A: Csr, rows: np.ndarray) -> Csr:
    """The rows `rows` of A as a matrix (for oracle checks of sampled rows of C)."""
    rows = np.asarray(rows, dtype=np.int64)
    lens = A.rowptr[rows + 1] - A.rowptr[rows]
    rp = np.zeros(rows.size + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    idx = np.concatenate([np.arange(A.rowptr[r], A.rowptr[r + 1]) for r in rows]) if rows.size else np.zeros(0, np.int64)
    vals = None if A.values is None else A.values[idx]
    return Csr(rows.size, A.ncols, rp, A.colidx[idx], vals)


def assert_rows_match_oracle(A: Csr, B: Csr, Cd, dtype, rows):
    """Check sampled rows of the GPU C against the oracle on those rows of A."""
    Ah, Bh = host_inputs(A, dtype), host_inputs(B, dtype)
    sub = row_sample(Ah, rows)
    Cref, S = oracle.spgemm(sub, Bh)
    import torch
    rp = Cd.rowptr.to(torch.int64).cpu().numpy()
    rows = np.asarray(rows, dtype=np.int64)
    for t, r in enumerate(rows):
        a, b = int(rp[r]), int(rp[r + 1])
        ra, rb = int(Cref.rowptr[t]), int(Cref.rowptr[t + 1])
        assert b - a == rb - ra, "row %d size %d != %d" % (r, b - a, rb - ra)
        if b == a:
            continue
        cj = Cd.colidx[a:b].cpu().numpy()
        vx = Cd.values[a:b].cpu().numpy().astype(np.float64)
        assert np.array_equal(cj, Cref.colidx[ra:rb]), "row %d columns differ" % r
        err = np.abs(vx - Cref.values[ra:rb])
        assert np.all(err <= tol_of(dtype) * S[ra:rb]), "row %d values out of tolerance" % r
