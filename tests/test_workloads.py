"""CPU pins of the seeded input generators: the sizes and value ranges of the
synthetic workloads the tests and the bench run (closed forms where the
structure has one; the recorded sizes of the seeded random workloads, so a
change to a generator cannot silently change the measured problem)."""

import numpy as np
import pytest

import workloads as w


def test_laplace5_64():
    A = w.laplace2d_5pt(64)
    assert A.shape == (4096, 4096)
    assert A.nnz == 5 * 64 * 64 - 4 * 64          # interior 5, edges 4, corners 3
    d = A.to_dense()
    assert np.all(np.diag(d) == 4.0) and set(np.unique(d[d != 0])) == {4.0, -1.0}


def test_stencil27_100_and_aggregation():
    g = 100
    A = w.stencil3d_27pt(g, seed=1)
    assert A.shape == (g ** 3, g ** 3)
    assert A.nnz == (3 * g - 2) ** 3 == 26_463_592   # a 3-point line per axis, (3g - 2)^3 entries
    rows = A.row_ids()
    diag = rows == A.colidx
    assert diag.sum() == g ** 3
    assert np.all(np.abs(A.values[diag] - 26.0) <= 1e-3)
    assert np.all(np.abs(A.values[~diag] + 1.0) <= 1e-3)
    P = w.aggregation(g, 3)
    assert P.shape == (g ** 3, 34 ** 3) and P.nnz == g ** 3
    assert np.all(P.values == 1.0) and np.all(np.diff(P.rowptr) == 1)


def test_rmat18_sizes():
    G = w.rmat_symmetric(scale=18, seed=7)
    deg = np.diff(G.rowptr)
    assert G.shape == (2 ** 18, 2 ** 18)
    assert G.nnz == 7_610_508 and deg.max() == 25_125 and (deg == 0).sum() == 88_099
    assert G.values.dtype == np.float32 and G.values.min() > 0.0 and G.values.max() <= 1.0
    assert np.all(G.row_ids() != G.colidx)            # no self-loops


def test_rmat_is_symmetric_small():
    G = w.rmat_symmetric(scale=10, seed=7)
    d = G.to_dense() != 0
    assert np.array_equal(d, d.T) and not np.any(np.diag(d))


def test_batched_first_products():
    pairs = w.batched_pairs(count=8, seed=11)
    assert [a.nrows for a, _ in pairs] == [1976, 17084, 3696, 4504, 30604, 52482, 3442, 89781]
    fm = sum(int(np.diff(b.rowptr)[a.colidx].sum()) for a, b in pairs)
    assert fm == 190_524_205
    assert sum(a.nnz for a, _ in pairs) == 6_276_229 and sum(b.nnz for _, b in pairs) == 6_138_219
    for a, b in pairs:
        assert a.shape == (a.nrows, a.nrows) and b.shape == a.shape
        assert np.all(np.abs(a.values) <= 1.0) and np.all(np.abs(b.values) <= 1.0)
        for M in (a, b):   # columns increase inside every row (no repeats)
            c = M.colidx.astype(np.int64)
            same_row = M.row_ids()[1:] == M.row_ids()[:-1]
            assert np.all(c[1:][same_row] > c[:-1][same_row])
