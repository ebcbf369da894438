"""Minimal host-side CSR container used by generators, oracle wrappers and tests."""

from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np


@dataclass
class Csr:
    """CSR matrix: ``rowptr`` int64[nrows+1], ``colidx`` int32[nnz], ``values`` or None."""

    nrows: int
    ncols: int
    rowptr: np.ndarray
    colidx: np.ndarray
    values: Optional[np.ndarray] = None

    def __post_init__(self):
        self.rowptr = np.ascontiguousarray(self.rowptr, dtype=np.int64)
        self.colidx = np.ascontiguousarray(self.colidx, dtype=np.int32)
        if self.values is not None:
            self.values = np.ascontiguousarray(self.values)
        assert self.rowptr.shape == (self.nrows + 1,)
        assert int(self.rowptr[-1]) == self.colidx.shape[0]

    @property
    def nnz(self) -> int:
        return int(self.colidx.shape[0])

    @property
    def shape(self):
        return (self.nrows, self.ncols)

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.rowptr)

    def with_values(self, values: np.ndarray) -> "Csr":
        return Csr(self.nrows, self.ncols, self.rowptr, self.colidx, values)

    def astype(self, dtype) -> "Csr":
        v = None if self.values is None else self.values.astype(dtype)
        return Csr(self.nrows, self.ncols, self.rowptr, self.colidx, v)

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.nrows, self.ncols), dtype=np.float64)
        rows = np.repeat(np.arange(self.nrows), self.row_lengths())
        vals = np.ones(self.nnz) if self.values is None else self.values.astype(np.float64)
        np.add.at(d, (rows, self.colidx.astype(np.int64)), vals)
        return d

    def row_ids(self) -> np.ndarray:
        return np.repeat(np.arange(self.nrows, dtype=np.int64), self.row_lengths())


def csr_from_coo(nrows, ncols, rows, cols, vals=None, sum_duplicates=False) -> Csr:
    """Build a row-sorted CSR (columns ascending within each row) from COO triples."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    if vals is not None:
        vals = np.asarray(vals)[order]
    if sum_duplicates and rows.size:
        key = rows * max(ncols, 1) + cols
        first = np.ones(key.size, dtype=bool)
        first[1:] = key[1:] != key[:-1]
        idx = np.cumsum(first) - 1
        rows, cols = rows[first], cols[first]
        if vals is not None:
            acc = np.zeros(int(first.sum()), dtype=vals.dtype)
            np.add.at(acc, idx, vals)
            vals = acc
    counts = np.bincount(rows, minlength=nrows) if rows.size else np.zeros(nrows, np.int64)
    rowptr = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return Csr(nrows, ncols, rowptr, cols.astype(np.int32), vals)


def shuffle_rows(a: Csr, seed: int) -> Csr:
    """Same matrix with the column order inside every row randomly permuted."""
    rng = np.random.default_rng(seed)
    rid = a.row_ids()
    key = rid.astype(np.float64) + rng.random(a.nnz) * 0.5
    order = np.argsort(key, kind="stable")
    v = None if a.values is None else a.values[order]
    return Csr(a.nrows, a.ncols, a.rowptr.copy(), a.colidx[order], v)


def identity(n: int, dtype=np.float64) -> Csr:
    return Csr(n, n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32),
               np.ones(n, dtype=dtype))


def permutation_matrix(perm: np.ndarray, dtype=np.float64) -> Csr:
    """Row i has a single 1 in column perm[i]  (so (Pi·X)(i,:) = X(perm[i],:))."""
    n = perm.shape[0]
    return Csr(n, n, np.arange(n + 1, dtype=np.int64), perm.astype(np.int32),
               np.ones(n, dtype=dtype))


def lower_triangle(A: Csr) -> Csr:
    """The strictly lower triangle of A's pattern (values dropped): the input
    of triangle counting on an undirected graph."""
    rid = A.row_ids()
    keep = A.colidx < rid
    rp = np.zeros(A.nrows + 1, dtype=np.int64)
    np.cumsum(np.bincount(rid[keep], minlength=A.nrows), out=rp[1:])
    return Csr(A.nrows, A.ncols, rp, A.colidx[keep].astype(np.int32), None)
