"""Gradients of L = sum W * (A·P) through the CUDA masked-product backward.

dL/dC = W on C's pattern, so dA = (W·Pᵀ) on A's pattern and dB = (Aᵀ·W) on P's
pattern.  Checked against the oracle's masked gradients (entrywise tolerance
with S = sum of absolute products), against central finite differences in FP64
(the loss is bilinear, so the difference quotient is exact up to rounding),
against the closed form for a one-entry-per-row P, and the backward is timed
against the forward.
"""

import statistics

import numpy as np
import pytest

import oracle
import workloads as w
from workloads.csr import Csr

from _util import dev, host_inputs, tol_of

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ag():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_03065_gb300 import build
    build.build()
    from paper_1801_03065_gb300 import autograd as _ag
    return _ag


def diff_workload(g):
    rng = np.random.default_rng(3)
    A = w.laplace3d_7pt(g, rng=rng, perturb=0.1)
    P = w.aggregation(g, 2, rng=rng, lo=0.5, hi=1.5)
    C, _ = oracle.spgemm(A, P)
    W = rng.uniform(-1, 1, C.nnz)
    return A, P, C, W


def make(ag, A, P, dtype):
    Ad, Pd = dev(A, dtype), dev(P, dtype)
    pat = ag.SpGEMMPattern(Ad, Pd)
    return Ad, Pd, pat


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_gradients_match_oracle_full_size(ag, dtype):
    A, P, C, W = diff_workload(64)
    Ad, Pd, pat = make(ag, A, P, dtype)
    assert np.array_equal(pat.C.colidx.cpu().numpy(), C.colidx)
    a = Ad.values.clone().requires_grad_(True)
    b = Pd.values.clone().requires_grad_(True)
    Wd = torch.as_tensor(W.astype(dtype), device="cuda")
    c = ag.spgemm_values(a, b, pat)
    loss = (Wd * c).sum()
    loss.backward()
    Ah, Ph = host_inputs(A, dtype), host_inputs(P, dtype)
    G = C.with_values(W.astype(dtype).astype(np.float64))
    ref_a, sa = oracle.masked_dA(Ah, Ph, G)
    ref_b, sb = oracle.masked_dB(Ah, Ph, G)
    t = tol_of(dtype)
    ga, gb = a.grad.cpu().numpy(), b.grad.cpu().numpy()
    assert np.all(np.abs(ga - ref_a) <= t * sa)
    assert np.all(np.abs(gb - ref_b) <= t * sb)
    # forward values on C's pattern
    Cref, S = oracle.spgemm(Ah, Ph)
    assert np.all(np.abs(c.detach().cpu().numpy() - Cref.values) <= t * S)
    pat.close()


def test_gradient_closed_form_aggregation(ag):
    """One entry per row of P: dA_ij = W(i, agg j) P(j, agg j); dB(j, agg j) = sum_i A_ij W(i, agg j)."""
    A, P, C, W = diff_workload(16)
    Ad, Pd, pat = make(ag, A, P, np.float64)
    a = Ad.values.clone().requires_grad_(True)
    b = Pd.values.clone().requires_grad_(True)
    (torch.as_tensor(W, device="cuda") * ag.spgemm_values(a, b, pat)).sum().backward()
    Wd = np.zeros(C.shape)
    Wd[C.row_ids(), C.colidx] = W
    agg = P.colidx
    exp_a = Wd[A.row_ids(), agg[A.colidx]] * P.values[A.colidx]
    exp_b = np.zeros(P.nnz)
    np.add.at(exp_b, A.colidx, A.values * Wd[A.row_ids(), agg[A.colidx]])
    assert np.allclose(a.grad.cpu().numpy(), exp_a, rtol=1e-13, atol=1e-14)
    assert np.allclose(b.grad.cpu().numpy(), exp_b, rtol=1e-12, atol=1e-13)
    pat.close()


def test_finite_differences_fp64(ag):
    """Central differences (h = 1e-6) in random directions and 32 single coordinates:
    |FD - <grad, V>| <= 1e-8 * T with T = sum_il |W_il| sum_j |A_ij||B_jl|."""
    A, P, C, W = diff_workload(24)
    Ad, Pd, pat = make(ag, A, P, np.float64)
    Wt = torch.as_tensor(W, device="cuda")
    a0, b0 = Ad.values.clone(), Pd.values.clone()

    def loss(a, b):
        return float((Wt * pat.forward_values(a, b)).sum().item())

    a = a0.clone().requires_grad_(True)
    b = b0.clone().requires_grad_(True)
    (Wt * ag.spgemm_values(a, b, pat)).sum().backward()
    ga, gb = a.grad.clone(), b.grad.clone()
    T = float((Wt.abs() * pat.forward_values(a0.abs(), b0.abs())).sum().item())
    h = 1e-6
    gen = torch.Generator(device="cuda").manual_seed(0)
    for _ in range(4):
        va = torch.rand(a0.shape, generator=gen, device="cuda", dtype=torch.float64) * 2 - 1
        vb = torch.rand(b0.shape, generator=gen, device="cuda", dtype=torch.float64) * 2 - 1
        fd_a = (loss(a0 + h * va, b0) - loss(a0 - h * va, b0)) / (2 * h)
        fd_b = (loss(a0, b0 + h * vb) - loss(a0, b0 - h * vb)) / (2 * h)
        assert abs(fd_a - float((ga * va).sum())) <= 1e-8 * T
        assert abs(fd_b - float((gb * vb).sum())) <= 1e-8 * T
    rng = np.random.default_rng(7)
    for _ in range(32):
        which = rng.integers(2)
        base, grad = (a0, ga) if which == 0 else (b0, gb)
        q = int(rng.integers(base.numel()))
        e = torch.zeros_like(base)
        e[q] = 1.0
        if which == 0:
            fd = (loss(a0 + h * e, b0) - loss(a0 - h * e, b0)) / (2 * h)
        else:
            fd = (loss(a0, b0 + h * e) - loss(a0, b0 - h * e)) / (2 * h)
        assert abs(fd - float(grad[q])) <= 1e-8 * T
    pat.close()


def test_gradcheck_tiny(ag):
    A = w.random_csr(9, 7, 3.0, seed=1)
    B = w.random_csr(7, 8, 3.0, seed=2)
    Ad, Bd = dev(A), dev(B)
    pat = ag.SpGEMMPattern(Ad, Bd)
    a = Ad.values.clone().requires_grad_(True)
    b = Bd.values.clone().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda x, y: ag.spgemm_values(x, y, pat), (a, b), eps=1e-6, atol=1e-9)
    pat.close()


def test_backward_within_three_forwards(ag):
    A, P, C, W = diff_workload(64)
    Ad, Pd, pat = make(ag, A, P, np.float64)
    Wt = torch.as_tensor(W, device="cuda")
    a = Ad.values.clone().requires_grad_(True)
    b = Pd.values.clone().requires_grad_(True)

    def fwd():
        return ag.spgemm_values(a, b, pat)

    def timed(fn, n=20):
        ts = []
        for _ in range(n):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            fn()
            e.record()
            torch.cuda.synchronize()
            ts.append(s.elapsed_time(e))
        return statistics.median(ts)

    for _ in range(3):
        (Wt * fwd()).sum().backward()
    a0, b0, g = a.detach(), b.detach(), Wt.clone()
    out = torch.empty(pat.C.nnz, dtype=torch.float64, device="cuda")
    # both paths captured as CUDA graphs, so the timing excludes Python launch overhead
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        pat.forward_values(a0, b0, out=out)
        pat.grads(g, a0, b0)
    torch.cuda.current_stream().wait_stream(side)
    gf, gb = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.graph(gf):
        pat.forward_values(a0, b0, out=out)
    with torch.cuda.graph(gb):
        da, db = pat.grads(g, a0, b0)
    t_f = timed(gf.replay)
    t_b = timed(gb.replay)
    print("forward %.4f ms, backward %.4f ms" % (t_f, t_b))
    gb.replay()
    torch.cuda.synchronize()
    ref_a = pat.grad_a(g, b0)
    assert torch.allclose(da, ref_a, rtol=1e-12, atol=1e-13)
    assert t_b <= 3.0 * t_f
    pat.close()
