"""CPU oracle for the two-phase SpGEMM C = A·B (FP64, OpenMP over rows).

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
benchmark's CPU-baseline leg are the only callers.  The GPU path neither
imports this package nor shares code with it.

Each function states the definition it writes out (paper section in
brackets):

* ``row_flops``        – rf_i = Σ_{j∈A(i,:)} |B(j,:)|, f_m = Σ rf_i, maxrf
                         [§2, multiplication count of Algorithm 1; §3.1.2]
* ``compress``         – CSI = col >> 5, CS = OR of 1 << (col & 31) per distinct CSI [§3.2]
* ``symbolic_plain``   – |C(i,:)| = #distinct l reachable through A(i,:) [Algorithm 2, symbolic phase]
* ``symbolic_compressed`` – Σ popcount of the OR-union of B_c rows [§3.2, Alg. 3]
* ``spgemm``           – C = A·B by gather / stable sort / in-order sum [Alg. 1]
* ``transpose``        – counting transpose with value permutation
* ``masked_dA/dB``     – dA = (G·Bᵀ) on A's pattern, dB = (Aᵀ·G) on B's pattern
* ``stats``            – f_m, maxrf, nnz(C), maxrs, CF, CMRF [§4 table columns]
* ``galerkin``         – C = Pᵀ·A·P (the R×A×P products of §4 with R = Pᵀ) as
                         Pᵀ·(A·P) and its bound |P|ᵀ|A||P|

All values are computed in FP64 (FP32 inputs are widened first).
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

from workloads.csr import Csr

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        i64, p = C.c_int64, C.c_void_p
        L.oracle_row_flops.argtypes = [i64, p, p, p, p, p, p]
        L.oracle_compress_count.argtypes = [i64, p, p, p]
        L.oracle_compress_fill.argtypes = [i64, p, p, p, p, p]
        L.oracle_symbolic_plain.argtypes = [i64, i64, p, p, p, p, p]
        L.oracle_symbolic_compressed.argtypes = [i64, i64, p, p, p, p, p, p, p]
        L.oracle_numeric.argtypes = [i64, p, p, p, p, p, p, p, p, p, p]
        L.oracle_transpose.argtypes = [i64, i64, p, p, p, p, p, p, p]
        L.oracle_masked_dA.argtypes = [i64, i64, p, p, p, p, p, p, p, p, p, p]
        L.oracle_masked_dB.argtypes = [i64, i64, i64, p, p, p, p, p, p, p, p, p, p]
        L.oracle_masked_count.argtypes = [i64, i64, p, p, p, p, p, p, p]
        for f in ("oracle_row_flops", "oracle_compress_count", "oracle_compress_fill",
                  "oracle_symbolic_plain", "oracle_symbolic_compressed", "oracle_numeric",
                  "oracle_transpose", "oracle_masked_dA", "oracle_masked_dB", "oracle_masked_count",
                  "oracle_num_threads"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(v):
    return None if v is None else np.ascontiguousarray(v, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed with code %d" % (what, rc))


def row_flops(A: Csr, B: Csr):
    """(rf int64[m], f_m, maxrf)."""
    rf = np.zeros(A.nrows, dtype=np.int64)
    fm, mx = C.c_int64(0), C.c_int64(0)
    _check(lib().oracle_row_flops(A.nrows, _ptr(A.rowptr), _ptr(A.colidx), _ptr(B.rowptr),
                                  _ptr(rf), C.byref(fm), C.byref(mx)), "row_flops")
    return rf, int(fm.value), int(mx.value)


def compress(B: Csr):
    """Compressed B: (rowptr int64[n+1], csi int32[], cs uint32[])."""
    cnt = np.zeros(B.nrows, dtype=np.int64)
    _check(lib().oracle_compress_count(B.nrows, _ptr(B.rowptr), _ptr(B.colidx), _ptr(cnt)),
           "compress_count")
    rp = np.zeros(B.nrows + 1, dtype=np.int64)
    np.cumsum(cnt, out=rp[1:])
    csi = np.zeros(int(rp[-1]), dtype=np.int32)
    cs = np.zeros(int(rp[-1]), dtype=np.uint32)
    _check(lib().oracle_compress_fill(B.nrows, _ptr(B.rowptr), _ptr(B.colidx), _ptr(rp),
                                      _ptr(csi), _ptr(cs)), "compress_fill")
    return rp, csi, cs


def symbolic_plain(A: Csr, B: Csr) -> np.ndarray:
    """C row pointers (int64[m+1]) from the definition of the structural product."""
    rs = np.zeros(A.nrows, dtype=np.int64)
    _check(lib().oracle_symbolic_plain(A.nrows, B.ncols, _ptr(A.rowptr), _ptr(A.colidx),
                                       _ptr(B.rowptr), _ptr(B.colidx), _ptr(rs)), "symbolic")
    rp = np.zeros(A.nrows + 1, dtype=np.int64)
    np.cumsum(rs, out=rp[1:])
    return rp


def symbolic_compressed(A: Csr, Bc, k: int):
    """(C row pointers, compressed row flops rfc int64[m]) from the compressed B."""
    bcp, csi, cs = Bc
    rs = np.zeros(A.nrows, dtype=np.int64)
    rfc = np.zeros(A.nrows, dtype=np.int64)
    kc = (k + 31) // 32
    _check(lib().oracle_symbolic_compressed(A.nrows, kc, _ptr(A.rowptr), _ptr(A.colidx),
                                            _ptr(bcp), _ptr(csi), _ptr(cs), _ptr(rs), _ptr(rfc)),
           "symbolic_compressed")
    rp = np.zeros(A.nrows + 1, dtype=np.int64)
    np.cumsum(rs, out=rp[1:])
    return rp, rfc


def spgemm(A: Csr, B: Csr, with_bounds: bool = True):
    """C = A·B in FP64 with sorted rows; returns (C, S) with S = Σ|a||b| per entry."""
    assert A.ncols == B.nrows
    cp = symbolic_plain(A, B)
    nnz = int(cp[-1])
    cj = np.zeros(nnz, dtype=np.int32)
    cx = np.zeros(nnz, dtype=np.float64)
    s = np.zeros(nnz, dtype=np.float64) if with_bounds else None
    ax, bx = _f64(A.values), _f64(B.values)
    _check(lib().oracle_numeric(A.nrows, _ptr(A.rowptr), _ptr(A.colidx), _ptr(ax),
                                _ptr(B.rowptr), _ptr(B.colidx), _ptr(bx),
                                _ptr(cp), _ptr(cj), _ptr(cx), _ptr(s)), "numeric")
    return Csr(A.nrows, B.ncols, cp, cj, cx), s


def transpose(A: Csr):
    """(Aᵀ with rows sorted, perm) where Aᵀ.values = A.values[perm]."""
    tp = np.zeros(A.ncols + 1, dtype=np.int64)
    tj = np.zeros(A.nnz, dtype=np.int32)
    ax = _f64(A.values)
    tx = np.zeros(A.nnz, dtype=np.float64) if ax is not None else None
    perm = np.zeros(A.nnz, dtype=np.int64)
    _check(lib().oracle_transpose(A.nrows, A.ncols, _ptr(A.rowptr), _ptr(A.colidx), _ptr(ax),
                                  _ptr(tp), _ptr(tj), _ptr(tx), _ptr(perm)), "transpose")
    return Csr(A.ncols, A.nrows, tp, tj, tx), perm


def masked_dA(A: Csr, B: Csr, G: Csr):
    """dA(i,j) = Σ_l G(i,l)·B(j,l) on A's pattern; returns (dA values, S)."""
    out = np.zeros(A.nnz, dtype=np.float64)
    s = np.zeros(A.nnz, dtype=np.float64)
    gx, bx = _f64(G.values), _f64(B.values)
    _check(lib().oracle_masked_dA(A.nrows, B.ncols, _ptr(A.rowptr), _ptr(A.colidx),
                                  _ptr(G.rowptr), _ptr(G.colidx), _ptr(gx),
                                  _ptr(B.rowptr), _ptr(B.colidx), _ptr(bx), _ptr(out), _ptr(s)),
           "masked_dA")
    return out, s


def masked_dB(A: Csr, B: Csr, G: Csr):
    """dB(j,l) = Σ_i A(i,j)·G(i,l) on B's pattern; returns (dB values, S)."""
    out = np.zeros(B.nnz, dtype=np.float64)
    s = np.zeros(B.nnz, dtype=np.float64)
    ax, gx = _f64(A.values), _f64(G.values)
    _check(lib().oracle_masked_dB(A.nrows, A.ncols, B.ncols, _ptr(A.rowptr), _ptr(A.colidx),
                                  _ptr(ax), _ptr(G.rowptr), _ptr(G.colidx), _ptr(gx),
                                  _ptr(B.rowptr), _ptr(B.colidx), _ptr(out), _ptr(s)),
           "masked_dB")
    return out, s


def stats(A: Csr, B: Csr):
    """Paper's per-multiplication statistics (§4 results table columns)."""
    rf, fm, maxrf = row_flops(A, B)
    cp = symbolic_plain(A, B)
    rs = np.diff(cp)
    Bc = compress(B)
    cpc, rfc = symbolic_compressed(A, Bc, B.ncols)
    out = {
        "m": A.nrows, "n": A.ncols, "k": B.ncols, "f_m": fm, "maxrf": maxrf,
        "nnzC": int(cp[-1]), "maxrs": int(rs.max()) if rs.size else 0,
        "f_m_compressed": int(rfc.sum()), "maxrf_compressed": int(rfc.max()) if rfc.size else 0,
    }
    out["CF"] = out["f_m_compressed"] / fm if fm else 1.0
    out["CMRF"] = out["maxrf_compressed"] / maxrf if maxrf else 1.0
    out["rowsizes_match"] = bool(np.array_equal(cp, cpc))
    return out


def masked_count(X: Csr, Y: Csr, S: Csr):
    """counts[i] = sum over l in S(i,:) of |{j : (i,j) in X, (j,l) in Y}| (int64[X.nrows])."""
    assert X.ncols == Y.nrows and S.nrows == X.nrows
    out = np.zeros(X.nrows, dtype=np.int64)
    _check(lib().oracle_masked_count(X.nrows, Y.ncols, _ptr(X.rowptr), _ptr(X.colidx), _ptr(Y.rowptr),
                                     _ptr(Y.colidx), _ptr(S.rowptr), _ptr(S.colidx), _ptr(out)),
           "masked_count")
    return out


def _abs(M: Csr) -> Csr:
    return Csr(M.nrows, M.ncols, M.rowptr, M.colidx, np.abs(np.asarray(M.values, dtype=np.float64)))


def galerkin(A: Csr, P: Csr):
    """C = Pᵀ·A·P and the entrywise bound S = Σ_{i,j} |p_iI||a_ij||p_jJ|.

    The R×A×P product of multigrid setup (§4) with R = Pᵀ, written out as its
    definition by two products: C = Pᵀ·(A·P) with the counting transpose and
    the Gustavson product above (Algorithm 1), and S the same products of the
    absolute values.  The pattern is the structural product (every (I, J) with
    some stored P(i,I), A(i,j), P(j,J)), which both factorisations give.
    """
    assert A.nrows == A.ncols == P.nrows
    Pt, _ = transpose(P)
    AP, _ = spgemm(A, P, with_bounds=False)
    C, _ = spgemm(Pt, AP, with_bounds=False)
    Pta, _ = transpose(_abs(P))
    APa, _ = spgemm(_abs(A), _abs(P), with_bounds=False)
    S, _ = spgemm(Pta, APa, with_bounds=False)
    assert np.array_equal(S.rowptr, C.rowptr) and np.array_equal(S.colidx, C.colidx)
    return C, np.asarray(S.values, dtype=np.float64)
