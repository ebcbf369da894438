"""Differentiable C = A·B over the value arrays of A and B on fixed patterns.

With G = dL/dC on C's pattern, the gradients restricted to the operands'
patterns are

    dA(i,j) = sum_l G(i,l) B(j,l)   (i,j) in S_A     i.e. (G·Bᵀ) sampled on S_A
    dB(j,l) = sum_i A(i,j) G(i,l)   (j,l) in S_B     i.e. (Aᵀ·G) sampled on S_B

Both are masked products (libkkspgemm's spgemm_masked: accumulators keyed by
the target pattern).  The symbolic structure of C and the transposes of A and
B (patterns plus value permutations) are built once per pattern and kept; a
forward is a numeric reuse on C's pattern, a backward two gathers and two
masked products.  All arithmetic runs in the CUDA library.
"""

from __future__ import annotations

from typing import Optional

import torch

from .ops import CsrMatrix, SpGEMM


class SpGEMMPattern:
    """Fixed patterns of A (m×n) and B (n×k) with C = A·B's structure kept for reuse."""

    def __init__(self, A: CsrMatrix, B: CsrMatrix, **options):
        assert A.values is not None and B.values is not None, "patterns need initial values"
        self.A, self.B = A, B
        self.h_fwd = SpGEMM(**options)
        self.h_da = SpGEMM(**options)
        self.h_db = SpGEMM(**options)
        rp, nnz = self.h_fwd.symbolic(A, B)
        C = self.h_fwd.numeric(A, B, rp, nnz)
        self.C = C                                   # pattern (rowptr, colidx) of C
        self.At, self.At_perm = self.h_da.transpose(A, with_values=True)
        self.Bt, self.Bt_perm = self.h_da.transpose(B, with_values=True)
        # int64 row pointers of the target patterns (kept: the masked plans are
        # cached by pattern pointers)
        self.A_rp64 = A.rowptr if A.rowptr.dtype == torch.int64 else A.rowptr.to(torch.int64)
        self.B_rp64 = B.rowptr if B.rowptr.dtype == torch.int64 else B.rowptr.to(torch.int64)
        self.h_fwd.sync()
        self.h_da.sync()

    @property
    def shape(self):
        return (self.A.nrows, self.B.ncols)

    def forward_values(self, a_vals: torch.Tensor, b_vals: torch.Tensor,
                       out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Values of C on its pattern (numeric reuse, no sort)."""
        if out is None:
            out = torch.empty(self.C.nnz, dtype=a_vals.dtype, device=a_vals.device)
        Cm = CsrMatrix(self.C.rowptr, self.C.colidx, out, self.C.shape)
        self.h_fwd.numeric_reuse(self.A.with_values(a_vals.contiguous()), self.B.with_values(b_vals.contiguous()), Cm)
        return out

    def grad_a(self, g_vals: torch.Tensor, b_vals: torch.Tensor) -> torch.Tensor:
        """dA on A's pattern: (G·Bᵀ) sampled on S_A (Bᵀ's values read through its permutation)."""
        G = CsrMatrix(self.C.rowptr, self.C.colidx, g_vals.contiguous(), self.C.shape)
        return self.h_da.masked(G, self.Bt.with_values(b_vals.contiguous()), self.A_rp64, self.A.colidx,
                                y_perm=self.Bt_perm)

    def grad_b(self, g_vals: torch.Tensor, a_vals: torch.Tensor) -> torch.Tensor:
        """dB on B's pattern: (Aᵀ·G) sampled on S_B (Aᵀ's values read through its permutation)."""
        G = CsrMatrix(self.C.rowptr, self.C.colidx, g_vals.contiguous(), self.C.shape)
        return self.h_db.masked(self.At.with_values(a_vals.contiguous()), G, self.B_rp64, self.B.colidx,
                                x_perm=self.At_perm)

    def grads(self, g_vals: torch.Tensor, a_vals: torch.Tensor, b_vals: torch.Tensor,
              need_a: bool = True, need_b: bool = True):
        """(dA, dB); the two masked products run concurrently on two streams."""
        main = torch.cuda.current_stream()
        if not (need_a and need_b):
            return (self.grad_a(g_vals, b_vals) if need_a else None,
                    self.grad_b(g_vals, a_vals) if need_b else None)
        if getattr(self, "_side", None) is None:
            self._side = torch.cuda.Stream(device=g_vals.device)
        side = self._side
        side.wait_stream(main)
        with torch.cuda.stream(side):
            db = self.grad_b(g_vals, a_vals)
        da = self.grad_a(g_vals, b_vals)
        main.wait_stream(side)
        db.record_stream(main)
        return da, db

    def close(self):
        for h in (self.h_fwd, self.h_da, self.h_db):
            h.close()


class SpGEMMFunction(torch.autograd.Function):
    """c_vals = values of A·B on C's pattern, differentiable in a_vals and b_vals."""

    @staticmethod
    def forward(ctx, a_vals: torch.Tensor, b_vals: torch.Tensor, pattern: SpGEMMPattern):
        ctx.pattern = pattern
        ctx.save_for_backward(a_vals, b_vals)
        return pattern.forward_values(a_vals, b_vals)

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        a_vals, b_vals = ctx.saved_tensors
        da, db = ctx.pattern.grads(g, a_vals, b_vals, ctx.needs_input_grad[0], ctx.needs_input_grad[1])
        return da, db, None


def spgemm_values(a_vals: torch.Tensor, b_vals: torch.Tensor, pattern: SpGEMMPattern) -> torch.Tensor:
    """Differentiable values of C = A·B on the pattern kept by ``pattern``."""
    return SpGEMMFunction.apply(a_vals, b_vals, pattern)
