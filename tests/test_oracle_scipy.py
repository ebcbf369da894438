"""Pins of the CPU oracle at sizes beyond the dense brute force: scipy.sparse
products (an independent library routine, not the oracle's C code) give the
structural pattern (a product of 0/1 patterns counts the paths i -> j -> l, so
it is free of cancellation), the products' values, the transpose, the
Galerkin triple product, the masked gradients and the masked counts.  All CPU.
"""

import numpy as np
import pytest

import oracle
import workloads as w
from workloads.csr import Csr

sp = pytest.importorskip("scipy.sparse")


def _sp(M: Csr, ones=False):
    vals = np.ones(M.nnz, dtype=np.int64) if ones else np.asarray(M.values, dtype=np.float64)
    return sp.csr_matrix((vals, M.colidx.astype(np.int64), M.rowptr.astype(np.int64)), shape=M.shape)


def _canon(X):
    X = X.tocsr()
    X.sort_indices()
    return X


def _on_pattern(X, M: Csr):
    """X's entries at M's (row, column) positions, in M's storage order."""
    X = X.tocsr()
    return np.asarray(X[M.row_ids(), M.colidx.astype(np.int64)]).ravel()


def _cases():
    A1 = w.random_csr(3000, 2000, 10.0, seed=1)
    B1 = w.random_csr(2000, 4000, 8.0, seed=2)
    A2 = w.shuffle_rows(w.random_csr(2500, 2500, 6.0, seed=3, empty_frac=0.1), 4)
    B2 = w.shuffle_rows(w.random_csr(2500, 1800, 12.0, seed=5), 6)
    return [(A1, B1), (A2, B2), (w.stencil3d_27pt(12, seed=1),) * 2]


@pytest.mark.parametrize("case", range(3))
def test_spgemm_against_scipy(case):
    A, B = _cases()[case]
    C, S = oracle.spgemm(A, B)
    paths = _canon(_sp(A, ones=True) @ _sp(B, ones=True))   # structural pattern, path counts
    assert np.array_equal(C.rowptr, paths.indptr) and np.array_equal(C.colidx, paths.indices)
    # the path counts of a row add up to its multiplications (f_m of Section 2)
    rf, fm, maxrf = oracle.row_flops(A, B)
    assert fm == int(paths.data.sum()) and maxrf == int(np.add.reduceat(paths.data, paths.indptr[:-1]).max())
    ref = _on_pattern(_sp(A) @ _sp(B), C)
    assert np.all(np.abs(C.values - ref) <= 1e-13 * S)
    absref = _on_pattern(abs(_sp(A)) @ abs(_sp(B)), C)
    assert np.allclose(S, absref, rtol=1e-13, atol=0.0)


def test_transpose_against_scipy():
    for seed in range(3):
        A = w.shuffle_rows(w.random_csr(1500, 900, 7.0, seed=seed, empty_frac=0.05), seed + 10)
        At, perm = oracle.transpose(A)
        T = _canon(_sp(A).T)
        assert np.array_equal(At.rowptr, T.indptr) and np.array_equal(At.colidx, T.indices)
        assert np.array_equal(At.values, T.data) and np.array_equal(At.values, A.values[perm])


def test_galerkin_against_scipy():
    rng = np.random.default_rng(7)
    A = w.stencil3d_27pt(15, seed=1)
    P = w.aggregation(15, 3, rng=rng, lo=0.5, hi=1.5)
    C, S = oracle.galerkin(A, P)
    paths = _canon(_sp(P, ones=True).T @ _sp(A, ones=True) @ _sp(P, ones=True))
    assert np.array_equal(C.rowptr, paths.indptr) and np.array_equal(C.colidx, paths.indices)
    ref = _on_pattern(_sp(P).T @ _sp(A) @ _sp(P), C)
    assert np.all(np.abs(C.values - ref) <= 1e-13 * S)


def test_masked_gradients_against_scipy():
    A = w.random_csr(1200, 800, 6.0, seed=11)
    B = w.random_csr(800, 1500, 6.0, seed=12)
    C, _ = oracle.spgemm(A, B)
    G = C.with_values(np.random.default_rng(13).uniform(-1, 1, C.nnz))
    dA, SA = oracle.masked_dA(A, B, G)
    dB, SB = oracle.masked_dB(A, B, G)
    assert np.all(np.abs(dA - _on_pattern(_sp(G) @ _sp(B).T, A)) <= 1e-13 * SA)
    assert np.all(np.abs(dB - _on_pattern(_sp(A).T @ _sp(G), B)) <= 1e-13 * SB)


def test_masked_count_against_scipy():
    G = w.rmat_symmetric(scale=11, seed=7)
    L = w.lower_triangle(G)
    counts = oracle.masked_count(L, L, L)
    paths = _sp(L, ones=True) @ _sp(L, ones=True)
    ref = np.asarray(paths.multiply(_sp(L, ones=True)).sum(axis=1)).ravel()
    assert np.array_equal(counts, ref.astype(np.int64))
