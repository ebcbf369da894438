"""Pins for the CPU oracle: checks against facts fixed by the paper and by the
mathematics (brute-force dense products, closed forms, invariants), never
against the oracle itself.  All CPU, no GPU.
"""

import itertools

import numpy as np
import pytest

import oracle
import workloads as w
from workloads.csr import Csr, csr_from_coo

pytestmark = pytest.mark.filterwarnings("ignore")


def _dense_pattern(a: Csr) -> np.ndarray:
    d = np.zeros(a.shape, dtype=np.int64)
    d[a.row_ids(), a.colidx] = 1
    return d


def _rand(m, n, density, seed, shuffle=False):
    rng = np.random.default_rng(seed)
    mask = rng.random((m, n)) < density
    r, c = np.nonzero(mask)
    a = csr_from_coo(m, n, r, c, rng.uniform(-1, 1, size=r.size))
    if shuffle:
        a = w.shuffle_rows(a, seed + 1000)
    return a


def _assert_sorted_rows(c: Csr):
    for i in range(c.nrows):
        cols = c.colidx[c.rowptr[i]:c.rowptr[i + 1]]
        assert np.all(np.diff(cols) > 0), "row %d not strictly increasing" % i


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("seed", range(40))
def test_spgemm_matches_dense_product(seed):
    """Algorithm 1 result equals the dense product on tiny matrices (all densities)."""
    rng = np.random.default_rng(seed)
    m, n, k = (int(x) for x in rng.integers(0, 13, size=3))
    da, db = rng.choice([0.0, 0.1, 0.3, 0.7, 1.0], size=2)
    A = _rand(m, n, da, seed, shuffle=bool(seed % 2))
    B = _rand(n, k, db, seed + 77, shuffle=bool(seed % 3 == 0))
    C, S = oracle.spgemm(A, B)
    assert C.shape == (m, k)
    pat = (_dense_pattern(A) @ _dense_pattern(B)) > 0
    assert np.array_equal(_dense_pattern(C) > 0, pat)
    dense = A.to_dense() @ B.to_dense()
    got = C.to_dense()
    sabs = np.abs(A.to_dense()) @ np.abs(B.to_dense())
    assert np.all(np.abs(got - dense) <= 1e-13 * sabs + 1e-300)
    # S is the sum of absolute products on C's pattern
    assert np.allclose(C.to_dense() * 0 + np.where(pat, sabs, 0), _scatter(C, S), rtol=1e-14, atol=0)
    _assert_sorted_rows(C)


def _scatter(c: Csr, vals):
    d = np.zeros(c.shape)
    d[c.row_ids(), c.colidx] = vals
    return d


def test_row_flops_brute_force():
    for seed in range(10):
        A = _rand(9, 11, 0.4, seed)
        B = _rand(11, 7, 0.5, seed + 1)
        rf, fm, mx = oracle.row_flops(A, B)
        expect = [sum(B.rowptr[j + 1] - B.rowptr[j] for j in A.colidx[A.rowptr[i]:A.rowptr[i + 1]])
                  for i in range(A.nrows)]
        assert list(rf) == expect
        assert fm == sum(expect)
        assert mx == (max(expect) if expect else 0)
        C, _ = oracle.spgemm(A, B)
        assert C.nnz <= fm


# ---------------------------------------------------------------- invariants
def test_identity():
    A = w.random_csr(50, 40, 5.0, seed=3)
    C, _ = oracle.spgemm(A, w.identity(40))
    assert np.array_equal(C.rowptr, A.rowptr) and np.array_equal(C.colidx, A.colidx)
    assert np.array_equal(C.values, A.values)
    C, _ = oracle.spgemm(w.identity(50), A)
    assert np.array_equal(C.colidx, A.colidx) and np.array_equal(C.values, A.values)


def test_permutation_equivariance():
    rng = np.random.default_rng(5)
    A = w.random_csr(60, 50, 6.0, seed=8)
    B = w.random_csr(50, 70, 6.0, seed=9)
    C, _ = oracle.spgemm(A, B)
    pr = rng.permutation(60)
    PA, _ = oracle.spgemm(w.permutation_matrix(pr), A)       # rows of A permuted
    PC, _ = oracle.spgemm(PA, B)
    PC2, _ = oracle.spgemm(w.permutation_matrix(pr), C)
    assert np.array_equal(PC.rowptr, PC2.rowptr) and np.array_equal(PC.colidx, PC2.colidx)
    assert np.allclose(PC.values, PC2.values, rtol=1e-14, atol=1e-15)
    pc = rng.permutation(70)                                 # columns of B relabelled
    Bp = Csr(B.nrows, B.ncols, B.rowptr, pc[B.colidx].astype(np.int32), B.values)
    Cp, _ = oracle.spgemm(A, Bp)
    d1 = Cp.to_dense()
    d2 = np.zeros_like(d1)
    d2[:, pc] = C.to_dense()
    assert np.allclose(d1, d2, rtol=1e-14, atol=1e-15)


def test_matvec_consistency():
    A = w.random_csr(300, 200, 8.0, seed=21)
    B = w.random_csr(200, 250, 8.0, seed=22)
    C, S = oracle.spgemm(A, B)
    x = np.random.default_rng(0).uniform(-1, 1, 250)

    def spmv(M, v):
        return np.bincount(M.row_ids(), weights=M.values * v[M.colidx], minlength=M.nrows)

    lhs = spmv(C, x)
    rhs = spmv(A, spmv(B, x))
    bound = spmv(Csr(C.nrows, C.ncols, C.rowptr, C.colidx, S), np.abs(x))
    assert np.all(np.abs(lhs - rhs) <= 1e-12 * bound + 1e-300)


def test_empty_and_degenerate():
    for (m, n, k) in [(0, 0, 0), (0, 5, 3), (4, 0, 3), (4, 5, 0), (1, 1, 1)]:
        A = w.random_csr(m, n, 2.0, seed=1)
        B = w.random_csr(n, k, 2.0, seed=2)
        C, _ = oracle.spgemm(A, B)
        assert C.shape == (m, k)
        assert np.array_equal(C.to_dense(), A.to_dense() @ B.to_dense())


# ---------------------------------------------------------------- closed forms
def _laplace5_closed_form(g):
    """C = A·A for the 5-point 4/-1 Laplacian, entry by entry from the stencil algebra:
    C_ii = 16 + deg(i); neighbours -8; distance-2 on an axis +1; diagonal neighbours +2."""
    idx = lambda x, y: x + g * y
    rows, cols, vals = [], [], []
    for y in range(g):
        for x in range(g):
            deg = sum(0 <= x + dx < g and 0 <= y + dy < g for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)))
            ent = {(0, 0): 16.0 + deg}
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                if 0 <= x + dx < g and 0 <= y + dy < g:
                    ent[(dx, dy)] = -8.0
                if 0 <= x + 2 * dx < g and 0 <= y + 2 * dy < g:
                    ent[(2 * dx, 2 * dy)] = 1.0
            for dx, dy in itertools.product((1, -1), (1, -1)):
                if 0 <= x + dx < g and 0 <= y + dy < g:
                    ent[(dx, dy)] = 2.0
            for (dx, dy), v in ent.items():
                rows.append(idx(x, y)); cols.append(idx(x + dx, y + dy)); vals.append(v)
    return csr_from_coo(g * g, g * g, rows, cols, vals)


def test_laplace5_squared_closed_form():
    """5-point Laplacian squared: 13-point pattern and integer values, exact."""
    A = w.laplace2d_5pt(64)
    C, _ = oracle.spgemm(A, A)
    ref = _laplace5_closed_form(64)
    assert np.array_equal(C.rowptr, ref.rowptr)
    assert np.array_equal(C.colidx, ref.colidx)
    assert np.array_equal(C.values, ref.values)
    assert C.nnz == 51972
    rs = np.diff(C.rowptr)
    assert rs.max() == 13
    # every interior row has the full 13-point stencil
    g = 64
    interior = [x + g * y for y in range(2, g - 2) for x in range(2, g - 2)]
    assert np.all(rs[interior] == 13)
    _, fm, mx = oracle.row_flops(A, A)
    assert fm == 100104 and mx == 25


def test_stencil27_squared_closed_form():
    """A = 27 I - N with N the 27-point all-ones stencil, so A² = 729 I - 54 N + N²,
    N = N1 ⊗ N1 ⊗ N1 (Kronecker), and on a g³ grid nnz(A²) = (5g-6)³, f_m = (9g-10)³."""
    g = 6
    A = w.stencil3d_27pt(g, perturb=0.0)
    n1 = np.zeros((g, g))
    for i in range(g):
        for j in range(max(0, i - 1), min(g, i + 2)):
            n1[i, j] = 1.0
    N = np.kron(np.kron(n1, n1), n1)   # x fastest: index = x + g y + g² z -> kron(z, y, x)
    ref = 729.0 * np.eye(g ** 3) - 54.0 * N + N @ N
    C, _ = oracle.spgemm(A, A)
    assert np.array_equal(C.to_dense(), ref)
    # -54 + (N²)_ij < 0 wherever N_ij = 1, so no entry of the 125-point pattern cancels
    assert np.array_equal(_dense_pattern(C) > 0, ref != 0)
    for g in (7, 12):
        A = w.stencil3d_27pt(g, perturb=0.0)
        st = oracle.stats(A, A)
        assert st["nnzC"] == (5 * g - 6) ** 3
        assert st["f_m"] == (9 * g - 10) ** 3
        assert st["maxrs"] == 125 and st["maxrf"] == 729


def test_galerkin_triple_product_invariants():
    """Pᵀ A P with piecewise-constant aggregation: (PᵀAP)_IJ = Σ_{i∈I, j∈J} a_ij."""
    g = 7
    A = w.stencil3d_27pt(g, seed=1)
    P = w.aggregation(g, 3)
    Pt, _ = oracle.transpose(P)
    AP, _ = oracle.spgemm(A, P)
    RAP, _ = oracle.spgemm(Pt, AP)
    agg = P.colidx.astype(np.int64)
    na = P.ncols
    ref = np.zeros((na, na))
    np.add.at(ref, (agg[A.row_ids()], agg[A.colidx]), A.values)
    assert np.allclose(RAP.to_dense(), ref, rtol=1e-13, atol=1e-12)
    assert abs(RAP.values.sum() - A.values.sum()) <= 1e-9 * np.abs(A.values).sum()
    # row sums of A·P equal row sums of A
    rs_ap = np.bincount(AP.row_ids(), weights=AP.values, minlength=AP.nrows)
    rs_a = np.bincount(A.row_ids(), weights=A.values, minlength=A.nrows)
    assert np.allclose(rs_ap, rs_a, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("seed", range(24))
def test_galerkin_matches_dense_triple_product(seed):
    """oracle.galerkin equals the dense Pᵀ·A·P (values, structural pattern, bound) on tiny inputs."""
    rng = np.random.default_rng(500 + seed)
    n, K = int(rng.integers(0, 12)), int(rng.integers(0, 8))
    da, dp = rng.choice([0.0, 0.15, 0.4, 1.0], size=2)
    A = _rand(n, n, da, 600 + seed, shuffle=bool(seed % 2))
    P = _rand(n, K, dp, 700 + seed, shuffle=bool(seed % 3 == 0))
    C, S = oracle.galerkin(A, P)
    assert C.shape == (K, K)
    pa, pp = _dense_pattern(A), _dense_pattern(P)
    pat = (pp.T @ pa @ pp) > 0
    assert np.array_equal(_dense_pattern(C) > 0, pat)
    Ad, Pd = A.to_dense(), P.to_dense()
    sabs = np.abs(Pd).T @ np.abs(Ad) @ np.abs(Pd)
    assert np.all(np.abs(C.to_dense() - Pd.T @ Ad @ Pd) <= 1e-13 * sabs + 1e-300)
    assert np.allclose(_scatter(C, S), np.where(pat, sabs, 0), rtol=1e-14, atol=0)
    _assert_sorted_rows(C)


def test_galerkin_aggregation_closed_form_and_sum():
    """Aggregation P with unit values: C_IJ = Σ_{i∈I, j∈J} a_ij (every entry); with
    general values Σ_IJ C_IJ = uᵀ A u for u = P·1."""
    g = 6
    A = w.stencil3d_27pt(g, seed=2)
    P = w.aggregation(g, 2)
    C, _ = oracle.galerkin(A, P)
    agg = P.colidx.astype(np.int64)
    ref = np.zeros((P.ncols, P.ncols))
    np.add.at(ref, (agg[A.row_ids()], agg[A.colidx]), A.values)
    assert np.allclose(C.to_dense(), ref, rtol=1e-13, atol=1e-12)
    patref = np.zeros(ref.shape, dtype=bool)
    patref[agg[A.row_ids()], agg[A.colidx]] = True
    assert np.array_equal(_dense_pattern(C) > 0, patref)
    rng = np.random.default_rng(5)
    P2 = Csr(P.nrows, P.ncols, P.rowptr, P.colidx, rng.uniform(0.5, 1.5, size=P.nnz))
    C2, _ = oracle.galerkin(A, P2)
    u = np.bincount(P2.row_ids(), weights=P2.values, minlength=P2.nrows)
    Au = np.bincount(A.row_ids(), weights=A.values * u[A.colidx], minlength=A.nrows)
    assert abs(C2.values.sum() - u @ Au) <= 1e-12 * (np.abs(A.values).sum() * 2.25)


def test_galerkin_planted_mistakes_are_caught():
    """A·P·Pᵀ-style slips (untransposed restriction, dropped factor) fail the dense pin."""
    rng = np.random.default_rng(9)
    A = _rand(9, 9, 0.4, 31)
    P = _rand(9, 9, 0.3, 32)
    Ad, Pd = A.to_dense(), P.to_dense()
    ref = Pd.T @ Ad @ Pd
    wrong_r, _ = oracle.spgemm(P, oracle.spgemm(A, P, with_bounds=False)[0], with_bounds=False)
    assert not np.allclose(wrong_r.to_dense(), ref)
    Pt, _ = oracle.transpose(P)
    dropped, _ = oracle.spgemm(Pt, P, with_bounds=False)
    assert not np.allclose(dropped.to_dense(), ref)
    C, _ = oracle.galerkin(A, P)
    assert np.allclose(C.to_dense(), ref, rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------- compression (§3.2)
def test_compression_bit_semantics():
    """Bit b of CS at CSI s is set iff column 32·s + b is in the row; CSI distinct."""
    for seed, shuffle in ((0, False), (1, True), (2, True)):
        B = w.random_csr(80, 300, 12.0, seed=seed)
        if shuffle:
            B = w.shuffle_rows(B, seed)
        rp, csi, cs = oracle.compress(B)
        for j in range(B.nrows):
            cols = set(B.colidx[B.rowptr[j]:B.rowptr[j + 1]].tolist())
            sets = csi[rp[j]:rp[j + 1]]
            assert len(set(sets.tolist())) == len(sets)
            got = set()
            for s, mask in zip(sets, cs[rp[j]:rp[j + 1]]):
                for b in range(32):
                    if (int(mask) >> b) & 1:
                        got.add(32 * int(s) + b)
            assert got == cols


def test_compressed_symbolic_equals_plain():
    """Compression changes the number of inserts, never nnz(C) (§3.2)."""
    cases = [
        (w.random_csr(120, 90, 7.0, seed=4), w.random_csr(90, 500, 9.0, seed=5)),
        (w.laplace2d_5pt(20), w.laplace2d_5pt(20)),
        (w.stencil3d_27pt(6), w.stencil3d_27pt(6)),
        (w.shuffle_rows(w.random_csr(50, 64, 10.0, seed=6), 1), w.shuffle_rows(w.random_csr(64, 33, 5.0, seed=7), 2)),
    ]
    for A, B in cases:
        cp = oracle.symbolic_plain(A, B)
        cpc, rfc = oracle.symbolic_compressed(A, oracle.compress(B), B.ncols)
        assert np.array_equal(cp, cpc)
        rf, fm, _ = oracle.row_flops(A, B)
        assert np.all(rfc <= rf)


def test_compression_ratio_laplace5():
    """CF for the 5-point 64² Laplacian: compressed f_m / f_m."""
    A = w.laplace2d_5pt(64)
    st = oracle.stats(A, A)
    # each grid line of 64 columns spans exactly 2 column sets; a row of B has
    # one set for its x-line (or two when x is 31/32 or crosses) and one per y neighbour
    assert st["f_m_compressed"] == 60800
    assert abs(st["CF"] - 60800 / 100104) < 1e-15


# ---------------------------------------------------------------- transpose / gradients
def test_transpose():
    for seed in range(5):
        A = _rand(13, 9, 0.3, seed, shuffle=True)
        At, perm = oracle.transpose(A)
        assert np.array_equal(At.to_dense(), A.to_dense().T)
        assert np.array_equal(At.values, A.values[perm])
        _assert_sorted_rows(At)
        Att, _ = oracle.transpose(At)
        As = csr_from_coo(A.nrows, A.ncols, A.row_ids(), A.colidx, A.values)
        assert np.array_equal(Att.colidx, As.colidx) and np.array_equal(Att.values, As.values)


@pytest.mark.parametrize("seed", range(8))
def test_masked_gradients_dense(seed):
    """dA = (G·Bᵀ)∘S_A and dB = (Aᵀ·G)∘S_B for L = Σ W∘(A·B), G = W on C's pattern."""
    rng = np.random.default_rng(seed)
    A = _rand(10, 8, 0.35, seed)
    B = _rand(8, 11, 0.35, seed + 50)
    C, _ = oracle.spgemm(A, B)
    G = C.with_values(rng.uniform(-1, 1, C.nnz))
    dA, _ = oracle.masked_dA(A, B, G)
    dB, _ = oracle.masked_dB(A, B, G)
    ref_a = (G.to_dense() @ B.to_dense().T)[A.row_ids(), A.colidx]
    ref_b = (A.to_dense().T @ G.to_dense())[B.row_ids(), B.colidx]
    assert np.allclose(dA, ref_a, rtol=1e-13, atol=1e-14)
    assert np.allclose(dB, ref_b, rtol=1e-13, atol=1e-14)


def test_masked_gradient_closed_form_aggregation():
    """P with one entry per row: dA_ij = W(i,agg(j))·P(j,agg(j)),
    dB(j,agg(j)) = Σ_i A_ij W(i,agg(j))."""
    rng = np.random.default_rng(3)
    A = w.laplace3d_7pt(6, rng=rng, perturb=0.1)
    P = w.aggregation(6, 2, rng=rng, lo=0.5, hi=1.5)
    C, _ = oracle.spgemm(A, P)
    Wv = rng.uniform(-1, 1, C.nnz)
    G = C.with_values(Wv)
    dA, _ = oracle.masked_dA(A, P, G)
    Wd = G.to_dense()
    agg = P.colidx
    expect = Wd[A.row_ids(), agg[A.colidx]] * P.values[A.colidx]
    assert np.allclose(dA, expect, rtol=1e-14, atol=0)
    dB, _ = oracle.masked_dB(A, P, G)
    expect_b = np.zeros(P.nnz)
    np.add.at(expect_b, A.colidx, A.values * Wd[A.row_ids(), agg[A.colidx]])
    assert np.allclose(dB, expect_b, rtol=1e-13, atol=1e-14)


def test_planted_mistakes_are_caught():
    """Mutants of the numeric result (a dropped product, a transposed operand, a
    sign slip, an off-by-one row of B) must each fail the dense brute-force pin."""
    rng = np.random.default_rng(11)
    A = _rand(8, 8, 0.5, 1)
    B = _rand(8, 8, 0.5, 2)
    dense = A.to_dense() @ B.to_dense()
    sabs = np.abs(A.to_dense()) @ np.abs(B.to_dense())

    def passes(c):
        return np.all(np.abs(c - dense) <= 1e-13 * sabs + 1e-300)

    assert passes(oracle.spgemm(A, B)[0].to_dense())
    # dropped term: one stored A(i,j) removed from the product
    keep = np.ones(A.nnz, bool)
    keep[int(rng.integers(A.nnz))] = False
    Ad = csr_from_coo(8, 8, A.row_ids()[keep], A.colidx[keep], A.values[keep])
    assert not passes(oracle.spgemm(Ad, B)[0].to_dense())
    # transposed operand
    At, _ = oracle.transpose(A)
    assert not passes(oracle.spgemm(At, B)[0].to_dense())
    # sign slip on one value
    An = A.with_values(A.values.copy())
    An.values[0] = -An.values[0]
    assert not passes(oracle.spgemm(An, B)[0].to_dense())
    # wrong index: row j+1 of B used for A(i,j)
    Ash = Csr(8, 8, A.rowptr, ((A.colidx + 1) % 8).astype(np.int32), A.values)
    assert not passes(oracle.spgemm(Ash, B)[0].to_dense())


# ------------------------------------------------------------------ masked counts (triangles)
def _graph(n, edges):
    """Undirected simple graph as a symmetric CSR pattern."""
    e = np.array(sorted({(min(a, b), max(a, b)) for a, b in edges if a != b}), dtype=np.int64).reshape(-1, 2)
    rows = np.concatenate([e[:, 0], e[:, 1]])
    cols = np.concatenate([e[:, 1], e[:, 0]])
    return csr_from_coo(n, n, rows, cols, np.ones(rows.size))


def _triangles(G):
    L = w.lower_triangle(G)
    return int(oracle.masked_count(L, L, L).sum())


@pytest.mark.parametrize("n", [3, 4, 5, 10, 17])
def test_masked_count_complete_graph(n):
    G = _graph(n, itertools.combinations(range(n), 2))
    assert _triangles(G) == n * (n - 1) * (n - 2) // 6


@pytest.mark.parametrize("n", [4, 7, 30])
def test_masked_count_cycle_and_wheel(n):
    cycle = [(i, (i + 1) % n) for i in range(n)]
    assert _triangles(_graph(n, cycle)) == 0
    wheel = cycle + [(n, i) for i in range(n)]   # hub n joined to every cycle vertex
    assert _triangles(_graph(n + 1, wheel)) == n


@pytest.mark.parametrize("seed", range(8))
def test_masked_count_against_dense(seed):
    rng = np.random.default_rng(seed)
    # general patterns: counts are the row sums of (X @ Y) * S over 0/1 matrices
    m, n, k = rng.integers(1, 40, size=3)
    X = w.random_csr(int(m), int(n), float(rng.uniform(0.5, 6)), seed=seed)
    Y = w.random_csr(int(n), int(k), float(rng.uniform(0.5, 6)), seed=seed + 100)
    S = w.random_csr(int(m), int(k), float(rng.uniform(0.5, 8)), seed=seed + 200)
    Xd, Yd, Sd = _dense_pattern(X), _dense_pattern(Y), _dense_pattern(S)
    ref = ((Xd.astype(np.int64) @ Yd.astype(np.int64)) * Sd).sum(axis=1)
    assert np.array_equal(oracle.masked_count(X, Y, S), ref)
    # triangles of a random graph: trace(A^3) / 6
    nv = 30
    edges = [tuple(e) for e in rng.integers(0, nv, size=(120, 2))]
    G = _graph(nv, edges)
    Gd = _dense_pattern(G).astype(np.int64)
    assert _triangles(G) == int(np.trace(Gd @ Gd @ Gd)) // 6


def test_masked_count_planted_mistake_is_caught():
    """Counting every product of the row (dropping the mask) breaks the dense pin."""
    X = w.random_csr(20, 15, 4.0, seed=1)
    Y = w.random_csr(15, 25, 4.0, seed=2)
    S = w.random_csr(20, 25, 3.0, seed=3)
    Xd, Yd, Sd = _dense_pattern(X), _dense_pattern(Y), _dense_pattern(S)
    ref = ((Xd.astype(np.int64) @ Yd.astype(np.int64)) * Sd).sum(axis=1)
    unmasked = (Xd.astype(np.int64) @ Yd.astype(np.int64)).sum(axis=1)
    assert not np.array_equal(unmasked, ref)
    assert np.array_equal(oracle.masked_count(X, Y, S), ref)
