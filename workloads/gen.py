"""Seeded generators for the five synthetic workloads and for small test cases.

All randomness comes from numpy ``default_rng`` (PCG64).  Generated CSR rows
have ascending column indices unless a test shuffles them on purpose.

Workloads (names used across tests and the benchmark):

* ``laplace5_64``   – 2-D 5-point Laplacian on a 64×64 grid, 4 / −1, FP64;  C = A·A.
* ``stencil27_100`` – 27-point stencil on a 100³ grid, 26 / −1 plus a
  uniform(−1e-3, 1e-3) perturbation of every stored entry (seed 1), FP64;
  C = A·A and the multigrid triple product Pᵀ·(A·P) with P the piecewise
  constant aggregation over 3×3×3 blocks (agg(x) = x // 3, 34³ aggregates).
* ``rmat18``        – symmetrised R-MAT, scale 18, edge factor 16,
  (a, b, c, d) = (0.57, 0.19, 0.19, 0.05), seed 7, self-loops and duplicates
  removed, FP32 values uniform(0, 1];  C = A·A.
* ``batched512``    – 512 independent square pairs (A_i, B_i), n_i log-uniform
  in [1e3, 2e5], geometric row lengths with means uniform in [3, 40], uniform
  columns without replacement, values uniform(−1, 1), seed 11.
* ``laplace7_64``   – 7-point Laplacian on a 64³ grid, 6 / −1 plus a
  uniform(−0.1, 0.1) perturbation (seed 3), P the 2×2×2 aggregation with
  values uniform(0.5, 1.5), W uniform(−1, 1) on the pattern of A·P.
"""

from __future__ import annotations

import numpy as np

from .csr import Csr, csr_from_coo


# --------------------------------------------------------------------------
# structured grids
# --------------------------------------------------------------------------

def _grid_stencil(dims, offsets, diag, off):
    """Stencil matrix on a grid with x fastest; offsets is a list of integer tuples."""
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    coords = np.indices(dims[::-1]).reshape(len(dims), -1)[::-1]  # coords[0] = x (fastest)
    strides = np.cumprod((1,) + dims[:-1])
    rows_l, cols_l, vals_l = [], [], []
    base = np.arange(n, dtype=np.int64)
    for off_vec in offsets:
        ok = np.ones(n, dtype=bool)
        shift = 0
        for ax, dlt in enumerate(off_vec):
            c = coords[ax] + dlt
            ok &= (c >= 0) & (c < dims[ax])
            shift += dlt * strides[ax]
        r = base[ok]
        rows_l.append(r)
        cols_l.append(r + shift)
        is_diag = all(v == 0 for v in off_vec)
        vals_l.append(np.full(r.size, diag if is_diag else off, dtype=np.float64))
    rows = np.concatenate(rows_l)
    cols = np.concatenate(cols_l)
    vals = np.concatenate(vals_l)
    return csr_from_coo(n, n, rows, cols, vals)


def laplace2d_5pt(g: int = 64) -> Csr:
    offs = [(0, -1), (-1, 0), (0, 0), (1, 0), (0, 1)]
    return _grid_stencil((g, g), offs, 4.0, -1.0)


def stencil3d_27pt(g: int = 100, seed: int = 1, perturb: float = 1e-3) -> Csr:
    offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    a = _grid_stencil((g, g, g), offs, 26.0, -1.0)
    if perturb:
        rng = np.random.default_rng(seed)
        a.values = a.values + rng.uniform(-perturb, perturb, size=a.nnz)
    return a


def laplace3d_7pt(g: int = 64, rng=None, perturb: float = 0.1) -> Csr:
    offs = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    a = _grid_stencil((g, g, g), offs, 6.0, -1.0)
    if perturb:
        a.values = a.values + rng.uniform(-perturb, perturb, size=a.nnz)
    return a


def aggregation(g: int, block: int, ndim: int = 3, rng=None, lo=None, hi=None) -> Csr:
    """Piecewise-constant aggregation prolongator P (g^ndim × na^ndim), one entry per row.

    agg(x) = x // block per axis (the last aggregate of an axis is partial when
    block does not divide g).  Values are 1.0, or uniform(lo, hi) from ``rng``.
    """
    na = -(-g // block)
    n = g ** ndim
    coords = np.indices((g,) * ndim).reshape(ndim, -1)[::-1]
    agg = np.zeros(n, dtype=np.int64)
    stride = 1
    for ax in range(ndim):
        agg += (coords[ax] // block) * stride
        stride *= na
    if rng is None:
        vals = np.ones(n, dtype=np.float64)
    else:
        vals = rng.uniform(lo, hi, size=n)
    return Csr(n, na ** ndim, np.arange(n + 1, dtype=np.int64), agg.astype(np.int32), vals)


# --------------------------------------------------------------------------
# R-MAT
# --------------------------------------------------------------------------

def rmat_symmetric(scale: int = 18, edge_factor: int = 16, a=0.57, b=0.19, c=0.19,
                   seed: int = 7, dtype=np.float32, with_values: bool = True) -> Csr:
    """Symmetrised R-MAT graph as a CSR matrix.

    Each of edge_factor·2^scale edges picks one quadrant per bit level
    (most significant bit first) with probabilities (a, b, c, 1-a-b-c); there
    is no noise and no vertex permutation.  The edge set is symmetrised,
    self-loops and duplicates are dropped, then one value uniform(0, 1] is
    drawn per stored entry in CSR order.
    """
    rng = np.random.default_rng(seed)
    n = 1 << scale
    ne = edge_factor << scale
    rows = np.zeros(ne, dtype=np.int64)
    cols = np.zeros(ne, dtype=np.int64)
    for lvl in range(scale):
        u = rng.random(ne)
        rbit = u >= (a + b)
        cbit = ((u >= a) & (u < a + b)) | (u >= a + b + c)
        sh = scale - 1 - lvl
        rows |= rbit.astype(np.int64) << sh
        cols |= cbit.astype(np.int64) << sh
    r = np.concatenate([rows, cols])
    cc = np.concatenate([cols, rows])
    keep = r != cc
    key = np.unique(r[keep] * n + cc[keep])
    rr = key // n
    c2 = key - rr * n
    counts = np.bincount(rr, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    vals = None
    if with_values:
        vals = (1.0 - rng.random(key.size)).astype(dtype)
    return Csr(n, n, rowptr, c2.astype(np.int32), vals)


# --------------------------------------------------------------------------
# random rows (batched workload and small tests)
# --------------------------------------------------------------------------

def _distinct_random_rows(rng, nrows, ncols, lengths):
    """Uniform column sets without replacement, sorted within each row.

    Draws with replacement, then redraws duplicated entries until every row is
    distinct; by exchangeability the resulting set is uniform over subsets.
    """
    lengths = np.minimum(lengths.astype(np.int64), ncols)
    rowptr = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(lengths, out=rowptr[1:])
    total = int(rowptr[-1])
    rid = np.repeat(np.arange(nrows, dtype=np.int64), lengths)
    cols = rng.integers(0, ncols, size=total, dtype=np.int64)
    # keys row * ncols + col, sorted; equal keys are equal values, so sorting
    # the keys themselves orders (row, col) exactly as a stable argsort would
    key = rid * ncols + cols
    del rid, cols
    while True:
        key.sort()
        dup = np.zeros(total, dtype=bool)
        if total > 1:
            np.equal(key[1:], key[:-1], out=dup[1:])
        nd = int(np.count_nonzero(dup))
        if nd == 0:
            break
        key[dup] = (key[dup] // ncols) * ncols + rng.integers(0, ncols, size=nd, dtype=np.int64)
    return Csr(nrows, ncols, rowptr, (key % ncols).astype(np.int32), None)


def random_csr(m, n, mean_len=4.0, seed=0, dtype=np.float64, lengths=None,
               empty_frac=0.0, vmin=-1.0, vmax=1.0) -> Csr:
    """Random CSR with geometric row lengths (or given lengths), sorted columns."""
    rng = np.random.default_rng(seed)
    if lengths is None:
        if mean_len <= 0 or n == 0:
            lengths = np.zeros(m, dtype=np.int64)
        else:
            lengths = rng.geometric(min(1.0, 1.0 / mean_len), size=m)
            if empty_frac > 0:
                lengths[rng.random(m) < empty_frac] = 0
    lengths = np.asarray(lengths, dtype=np.int64)
    if n == 0:
        lengths = np.zeros(m, dtype=np.int64)
    a = _distinct_random_rows(rng, m, max(n, 1), lengths) if m else Csr(0, n, np.zeros(1, np.int64), np.zeros(0, np.int32))
    a.ncols = n
    a.values = rng.uniform(vmin, vmax, size=a.nnz).astype(dtype)
    return a


def values_on_pattern(nnz: int, rng, lo=-1.0, hi=1.0, dtype=np.float64) -> np.ndarray:
    return rng.uniform(lo, hi, size=nnz).astype(dtype)


def batched_pairs(count: int = 512, seed: int = 11, nmin: int = 1000, nmax: int = 200000,
                  mu_lo: float = 3.0, mu_hi: float = 40.0, dtype=np.float64):
    """List of ``count`` independent (A_i, B_i) square CSR pairs.

    n_i = floor(exp(uniform(ln nmin, ln nmax))); mean row lengths mu_A, mu_B
    uniform in [mu_lo, mu_hi]; lengths geometric on {1, 2, ...} with mean mu,
    capped at n_i; columns uniform without replacement; values uniform(-1, 1)
    drawn in FP64 (FP32 = round-to-nearest of those draws).  Instances are
    drawn in order from one stream, so a smaller ``count`` gives a prefix.
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(np.floor(np.exp(rng.uniform(np.log(nmin), np.log(nmax)))))
        mu_a, mu_b = rng.uniform(mu_lo, mu_hi, size=2)
        la = np.minimum(rng.geometric(1.0 / mu_a, size=n), n)
        lb = np.minimum(rng.geometric(1.0 / mu_b, size=n), n)
        A = _distinct_random_rows(rng, n, n, la)
        B = _distinct_random_rows(rng, n, n, lb)
        A.values = rng.uniform(-1.0, 1.0, size=A.nnz).astype(dtype)
        B.values = rng.uniform(-1.0, 1.0, size=B.nnz).astype(dtype)
        out.append((A, B))
    return out


def batched_fresh_values(pairs, repeat: int, seed: int = 11, dtype=np.float64):
    """Fresh uniform(-1, 1) values for numeric-reuse repeat ``repeat`` (rng([seed, repeat]))."""
    rng = np.random.default_rng([seed, repeat])
    out = []
    for A, B in pairs:
        va = rng.uniform(-1.0, 1.0, size=A.nnz).astype(dtype)
        vb = rng.uniform(-1.0, 1.0, size=B.nnz).astype(dtype)
        out.append((va, vb))
    return out


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

def config_workload(name: str, **kw):
    """Return a dict describing a named workload (matrices + metadata)."""
    if name == "laplace5_64":
        g = kw.get("g", 64)
        A = laplace2d_5pt(g)
        return {"name": name, "A": A, "B": A, "dtype": "f64"}
    if name == "stencil27_100":
        g = kw.get("g", 100)
        A = stencil3d_27pt(g, seed=1)
        P = aggregation(g, 3)
        return {"name": name, "A": A, "B": A, "P": P, "dtype": "f64"}
    if name == "rmat18":
        scale = kw.get("scale", 18)
        A = rmat_symmetric(scale=scale, seed=7)
        return {"name": name, "A": A, "B": A, "dtype": "f32"}
    if name == "batched512":
        count = kw.get("count", 512)
        dtype = kw.get("dtype", np.float64)
        return {"name": name, "pairs": batched_pairs(count=count, seed=11, dtype=dtype),
                "dtype": "f64" if dtype == np.float64 else "f32"}
    if name == "laplace7_64":
        g = kw.get("g", 64)
        rng = np.random.default_rng(3)
        A = laplace3d_7pt(g, rng=rng, perturb=0.1)
        P = aggregation(g, 2, rng=rng, lo=0.5, hi=1.5)
        return {"name": name, "A": A, "B": P, "rng": rng, "dtype": "f64"}
    raise KeyError(name)
