"""GPU parity of the Galerkin triple product C = Pᵀ·A·P (one plan) against the oracle.

Structure bit-exact; values within tol * Σ |p_iI||a_ij||p_jJ| (tol 1e-13 FP64,
1e-5 FP32), through spgemm_rap_symbolic / spgemm_rap_numeric.
"""

import numpy as np
import pytest

import oracle
import workloads as w
from workloads.csr import Csr, csr_from_coo

from _util import dev, host_inputs, tol_of

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ops():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_03065_gb300 import build
    build.build()
    from paper_1801_03065_gb300 import ops as _ops
    return _ops


def check(A, P, Cd, dtype, ref=None):
    if ref is None:
        ref = oracle.galerkin(host_inputs(A, dtype), host_inputs(P, dtype))
    C, S = ref
    rp, cj, vx = Cd.to_host()
    assert np.array_equal(rp, C.rowptr), "row pointers differ"
    assert np.array_equal(cj, C.colidx), "column indices differ"
    err = np.abs(vx.astype(np.float64) - C.values)
    bad = np.nonzero(err > tol_of(dtype) * S)[0]
    assert bad.size == 0, "values out of tolerance at %s" % bad[:5]
    return ref


def run(ops, A, P, dtype=np.float64, rp64=True, h=None):
    h = h or ops.SpGEMM()
    Ad, Pd = dev(A, dtype, rp64), dev(P, dtype, rp64)
    Cd = h.rap(Ad, Pd)
    h.sync()
    return h, Ad, Pd, Cd


def _hub_problem(n, K, hubs, hub_rows, seed):
    """A random square A; P with ~2 random columns per row plus, in the first
    hub_rows rows, one of `hubs` shared columns (rows of C with many products)."""
    rng = np.random.default_rng(seed)
    A = w.random_csr(n, n, 6.0, seed=seed)
    base = w.random_csr(n, K - hubs, 2.0, seed=seed + 1)
    r = base.row_ids()
    c = base.colidx.astype(np.int64) + hubs
    hr = np.arange(hub_rows, dtype=np.int64)
    rows = np.concatenate([r, hr])
    cols = np.concatenate([c, hr % hubs])
    P = csr_from_coo(n, K, rows, cols, rng.uniform(-1, 1, size=rows.size))
    return A, P


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("rp64", [True, False])
def test_rap_random(ops, dtype, rp64):
    A = w.random_csr(700, 700, 8.0, seed=21)
    P = w.random_csr(700, 90, 2.0, seed=22, empty_frac=0.1)
    _, _, _, Cd = run(ops, A, P, dtype, rp64)
    check(A, P, Cd, dtype)


def test_rap_unsorted_inputs(ops):
    A = w.shuffle_rows(w.random_csr(400, 400, 10.0, seed=31), 32)
    P = w.shuffle_rows(w.random_csr(400, 50, 3.0, seed=33), 34)
    _, _, _, Cd = run(ops, A, P)
    check(A, P, Cd, np.float64)


def test_rap_aggregation_stencil(ops):
    """The multigrid case: 27-point stencil with 3x3x3 aggregation (partial last layer)."""
    g = 20
    A = w.stencil3d_27pt(g, seed=4)
    P = w.aggregation(g, 3, rng=np.random.default_rng(5), lo=0.5, hi=1.5)
    h, _, _, Cd = run(ops, A, P)
    check(A, P, Cd, np.float64)
    st = h.stats()
    assert st["f_m"] == int(np.sum((A.rowptr[1:] - A.rowptr[:-1])))   # one P entry per row: |R(I,:)|·|A(i,:)|·1
    assert st["maxrs"] == 27


def test_rap_cta_classes(ops):
    """Rows whose symbolic bitmap (K = 100 000) and numeric table exceed a warp's share."""
    A, P = _hub_problem(4000, 100000, 10, 1500, seed=41)
    h, _, _, Cd = run(ops, A, P)
    check(A, P, Cd, np.float64)
    st = h.stats()
    assert st["bin_rows_numeric"][3] >= 10     # CTA rows of the numeric phase
    assert st["bin_rows_numeric"][2] > 0       # warp rows


def test_rap_row_too_large(ops):
    """A row of C above the CTA numeric table is refused by the symbolic call."""
    from paper_1801_03065_gb300._binding import SpGEMMError
    A, P = _hub_problem(6000, 100000, 1, 3000, seed=43)
    h = ops.SpGEMM()
    with pytest.raises(SpGEMMError) as e:
        h.rap_symbolic(dev(A), dev(P))
    assert e.value.status == 5
    # the handle stays usable
    A2 = w.random_csr(200, 200, 5.0, seed=44)
    P2 = w.random_csr(200, 30, 2.0, seed=45)
    _, _, _, Cd = run(ops, A2, P2, h=h)
    check(A2, P2, Cd, np.float64)


@pytest.mark.parametrize("case", ["k1", "p_empty", "a_empty_rows", "n0", "empty_cols"])
def test_rap_edge_cases(ops, case):
    rng = np.random.default_rng(7)
    if case == "k1":
        A = w.random_csr(300, 300, 5.0, seed=51)
        P = csr_from_coo(300, 1, np.arange(300), np.zeros(300, np.int64), rng.uniform(-1, 1, 300))
    elif case == "p_empty":
        A = w.random_csr(300, 300, 5.0, seed=52)
        P = Csr(300, 40, np.zeros(301, np.int64), np.zeros(0, np.int32), np.zeros(0))
    elif case == "a_empty_rows":
        A = w.random_csr(300, 300, 5.0, seed=53, empty_frac=0.7)
        P = w.random_csr(300, 40, 2.0, seed=54)
    elif case == "n0":
        A = Csr(0, 0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
        P = Csr(0, 12, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    else:
        A = w.random_csr(300, 300, 5.0, seed=55)
        Pb = w.random_csr(300, 40, 2.0, seed=56)
        P = Csr(300, 80, Pb.rowptr, (Pb.colidx * 2).astype(np.int32), Pb.values)   # odd columns empty
    _, _, _, Cd = run(ops, A, P)
    check(A, P, Cd, np.float64)


def test_rap_numeric_reuse_and_graph(ops):
    """New values on the same patterns: numeric only, eagerly and as a CUDA graph replay."""
    A = w.random_csr(900, 900, 7.0, seed=61)
    P = w.random_csr(900, 120, 2.0, seed=62)
    h = ops.SpGEMM()
    Ad, Pd = dev(A), dev(P)
    rp, nnz = h.rap_symbolic(Ad, Pd)
    Cd = h.rap_numeric(Ad, Pd, rp, nnz)
    h.sync()
    check(A, P, Cd, np.float64)
    rng = np.random.default_rng(63)
    A2 = Csr(A.nrows, A.ncols, A.rowptr, A.colidx, rng.uniform(-2, 2, A.nnz))
    P2 = Csr(P.nrows, P.ncols, P.rowptr, P.colidx, rng.uniform(-2, 2, P.nnz))
    Ad2 = Ad.with_values(torch.from_numpy(A2.values).cuda())
    Pd2 = Pd.with_values(torch.from_numpy(P2.values).cuda())
    h.rap_numeric(Ad2, Pd2, rp, nnz, Cd.colidx, Cd.values)
    h.sync()
    check(A2, P2, Cd, np.float64)
    # graph: capture once, then update the values in place and replay
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            h.rap_numeric(Ad2, Pd2, rp, nnz, Cd.colidx, Cd.values, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    A3v = rng.uniform(-1, 1, A.nnz)
    P3v = rng.uniform(-1, 1, P.nnz)
    Ad2.values.copy_(torch.from_numpy(A3v))
    Pd2.values.copy_(torch.from_numpy(P3v))
    g.replay()
    torch.cuda.synchronize()
    h.sync()
    check(Csr(A.nrows, A.ncols, A.rowptr, A.colidx, A3v), Csr(P.nrows, P.ncols, P.rowptr, P.colidx, P3v),
          Cd, np.float64)


def test_rap_errors(ops):
    from paper_1801_03065_gb300._binding import SpGEMMError
    A = w.random_csr(100, 100, 4.0, seed=71)
    P = w.random_csr(100, 20, 2.0, seed=72)
    h = ops.SpGEMM()
    Ad, Pd = dev(A), dev(P)
    # numeric before symbolic
    rp = torch.zeros(21, dtype=torch.int64, device="cuda")
    with pytest.raises(SpGEMMError) as e:
        h.rap_numeric(Ad, Pd, rp, 0)
    assert e.value.status == 2
    # shapes: P with the wrong number of rows
    Pbad = w.random_csr(99, 20, 2.0, seed=73)
    with pytest.raises(SpGEMMError) as e:
        h.rap_symbolic(Ad, dev(Pbad))
    assert e.value.status == 1
    # another P after the plan: not ready
    rp, nnz = h.rap_symbolic(Ad, Pd)
    with pytest.raises(SpGEMMError) as e:
        h.rap_numeric(Ad, dev(P), rp, nnz)
    assert e.value.status == 2
    # out-of-range columns of P and of A
    Pc = Csr(P.nrows, P.ncols, P.rowptr, P.colidx.copy(), P.values)
    Pc.colidx[5] = 20
    with pytest.raises(SpGEMMError) as e:
        h.rap_symbolic(Ad, dev(Pc))
    assert e.value.status == 8
    Ac = Csr(A.nrows, A.ncols, A.rowptr, A.colidx.copy(), A.values)
    Ac.colidx[3] = 100
    with pytest.raises(SpGEMMError) as e:
        h.rap_symbolic(dev(Ac), Pd)
    assert e.value.status == 8
    # still usable afterwards
    _, _, _, Cd = run(ops, A, P, h=h)
    check(A, P, Cd, np.float64)


def test_rap_stencil27_100_full(ops):
    """The bench's triple product at full size (1 M rows, 39 304 aggregates), every entry."""
    A = w.stencil3d_27pt(100, seed=1)
    P = w.aggregation(100, 3)
    _, _, _, Cd = run(ops, A, P)
    check(A, P, Cd, np.float64)
