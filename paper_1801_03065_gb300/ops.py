"""PyTorch-facing wrappers over the C ABI (device memory and streams only).

Tensors provide the device buffers and torch's current CUDA stream is passed
to every call; all arithmetic runs in libkkspgemm's kernels.
"""

from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import torch

from . import _binding as B


def _dtype_code(t: Optional[torch.dtype]) -> int:
    if t is None or t == torch.float64:
        return B.SPGEMM_R64
    if t == torch.float32:
        return B.SPGEMM_R32
    raise TypeError("values must be float32 or float64, got %s" % t)


def _stream(stream=None) -> C.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    if t is None or t.numel() == 0:
        return None
    return C.c_void_p(t.data_ptr())


@dataclass
class CsrMatrix:
    """CSR matrix held in device tensors.

    rowptr: int32 or int64 [nrows + 1]; colidx: int32 [nnz]; values: float32 /
    float64 [nnz] or None (pattern only).
    """

    rowptr: torch.Tensor
    colidx: torch.Tensor
    values: Optional[torch.Tensor]
    shape: Tuple[int, int]

    def __post_init__(self):
        assert self.rowptr.dtype in (torch.int32, torch.int64)
        assert self.colidx.dtype == torch.int32
        assert self.rowptr.is_contiguous() and self.colidx.is_contiguous()
        if self.values is not None:
            assert self.values.is_contiguous() and self.values.numel() == self.colidx.numel()

    @property
    def nrows(self) -> int:
        return int(self.shape[0])

    @property
    def ncols(self) -> int:
        return int(self.shape[1])

    @property
    def nnz(self) -> int:
        return int(self.colidx.numel())

    @property
    def dtype(self):
        return None if self.values is None else self.values.dtype

    def with_values(self, values: Optional[torch.Tensor]) -> "CsrMatrix":
        return CsrMatrix(self.rowptr, self.colidx, values, self.shape)

    def desc(self, dtype_hint=None) -> B.CsrT:
        d = B.CsrT()
        d.nrows, d.ncols, d.nnz = self.nrows, self.ncols, self.nnz
        d.rowptr_is_64 = 1 if self.rowptr.dtype == torch.int64 else 0
        d.dtype = _dtype_code(self.dtype if self.values is not None else dtype_hint)
        d.rowptr = self.rowptr.data_ptr()
        d.colidx = self.colidx.data_ptr() if self.nnz > 0 else None
        d.values = self.values.data_ptr() if (self.values is not None and self.nnz > 0) else None
        return d

    @staticmethod
    def from_host(rowptr, colidx, values, shape, device="cuda", rowptr_dtype=torch.int64):
        rp = torch.as_tensor(rowptr).to(device=device, dtype=rowptr_dtype).contiguous()
        cj = torch.as_tensor(colidx).to(device=device, dtype=torch.int32).contiguous()
        vx = None if values is None else torch.as_tensor(values).to(device=device).contiguous()
        return CsrMatrix(rp, cj, vx, (int(shape[0]), int(shape[1])))

    def to_host(self):
        """(rowptr int64, colidx int32, values or None) as numpy arrays."""
        rp = self.rowptr.to(torch.int64).cpu().numpy()
        cj = self.colidx.cpu().numpy()
        vx = None if self.values is None else self.values.cpu().numpy()
        return rp, cj, vx


class SpGEMM:
    """A handle of the two-phase SpGEMM library (owns all device scratch)."""

    def __init__(self, compression: int = -1, compress_threshold: float = 0.85,
                 l1_max_occupancy: float = 0.5, l1_max_log2_slots: int = 0, dense: int = -1,
                 method: int = 0, workspace_limit_bytes: int = 0, pool_limit_bytes: int = 0,
                 device: int = 0, hash_function: int = 1, slots_per_key_log2: int = 0,
                 tune: bool = False, verbose: bool = False, numeric_positions: bool = True,
                 cta_partition: int = 0, window_positions: int = 1, stage_b: bool = False,
                 sym_merge: bool = True):
        self._lib = B.load()
        opt = B.OptionsT()
        B.check(self._lib.spgemm_options_default(C.byref(opt)), "spgemm_options_default")
        opt.compression = compression
        opt.compress_threshold = compress_threshold
        opt.l1_max_occupancy = l1_max_occupancy
        opt.l1_max_log2_slots = l1_max_log2_slots
        opt.dense = dense
        opt.method = method
        opt.workspace_limit_bytes = workspace_limit_bytes
        opt.pool_limit_bytes = pool_limit_bytes
        opt.device = device
        opt.hash_function = hash_function
        opt.slots_per_key_log2 = slots_per_key_log2
        opt.tune = 1 if tune else 0
        opt.verbose = 1 if verbose else 0
        opt.numeric_positions = 1 if numeric_positions else 0
        opt.cta_partition = int(cta_partition)
        opt.window_positions = int(window_positions)
        opt.stage_b = 1 if stage_b else 0
        opt.sym_merge = 1 if sym_merge else 0
        self.device = torch.device("cuda", device)
        h = C.c_void_p()
        B.check(self._lib.spgemm_handle_create(C.byref(h), C.byref(opt)), "spgemm_handle_create")
        self._h = h
        self._keep = None

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.spgemm_handle_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- phases
    def symbolic(self, A: CsrMatrix, Bm: CsrMatrix, C_rowptr: Optional[torch.Tensor] = None, stream=None):
        """The symbolic phase of Algorithm 2: returns (C_rowptr int64 tensor, nnz(C))."""
        if C_rowptr is None:
            C_rowptr = torch.empty(A.nrows + 1, dtype=torch.int64, device=A.rowptr.device)
        hint = A.dtype or Bm.dtype
        da, db = A.desc(hint), Bm.desc(hint)
        nnz = C.c_int64(0)
        self._keep = (A, Bm, C_rowptr)
        B.check(self._lib.spgemm_symbolic(self._h, C.byref(da), C.byref(db), C.c_void_p(C_rowptr.data_ptr()),
                                          C.byref(nnz), _stream(stream)), "spgemm_symbolic")
        return C_rowptr, int(nnz.value)

    def numeric(self, A: CsrMatrix, Bm: CsrMatrix, C_rowptr: torch.Tensor, nnz: Optional[int] = None,
                C_colidx: Optional[torch.Tensor] = None, C_values: Optional[torch.Tensor] = None,
                stream=None) -> CsrMatrix:
        """The numeric phase of Algorithm 2: C's columns and values (rows sorted)."""
        if nnz is None:
            nnz = int(C_rowptr[-1].item()) if C_colidx is None else C_colidx.numel()
        dev = C_rowptr.device
        if C_colidx is None:
            C_colidx = torch.empty(nnz, dtype=torch.int32, device=dev)
        if C_values is None:
            C_values = torch.empty(nnz, dtype=A.dtype, device=dev)
        da, db = A.desc(), Bm.desc()
        B.check(self._lib.spgemm_numeric(self._h, C.byref(da), C.byref(db), C.c_void_p(C_rowptr.data_ptr()),
                                         _ptr(C_colidx), _ptr(C_values), _stream(stream)), "spgemm_numeric")
        return CsrMatrix(C_rowptr, C_colidx, C_values, (A.nrows, Bm.ncols))

    def numeric_reuse(self, A: CsrMatrix, Bm: CsrMatrix, Cm: CsrMatrix, stream=None) -> CsrMatrix:
        """Values of C on its known (sorted) pattern for new values of A and B."""
        da, db = A.desc(), Bm.desc()
        B.check(self._lib.spgemm_numeric_reuse(self._h, C.byref(da), C.byref(db),
                                               C.c_void_p(Cm.rowptr.data_ptr()), _ptr(Cm.colidx),
                                               _ptr(Cm.values), _stream(stream)), "spgemm_numeric_reuse")
        return Cm

    def multiply(self, A: CsrMatrix, Bm: CsrMatrix, stream=None) -> CsrMatrix:
        rp, nnz = self.symbolic(A, Bm, stream=stream)
        return self.numeric(A, Bm, rp, nnz, stream=stream)

    # ---------------------------------------------------------------- Galerkin triple product
    def rap_symbolic(self, A: CsrMatrix, P: CsrMatrix, C_rowptr: Optional[torch.Tensor] = None, stream=None):
        """Row pointers and nnz of C = P^T A P, planned in one pass (A*P is never formed)."""
        if C_rowptr is None:
            C_rowptr = torch.empty(P.ncols + 1, dtype=torch.int64, device=A.rowptr.device)
        hint = A.dtype or P.dtype
        da, dp = A.desc(hint), P.desc(hint)
        nnz = C.c_int64(0)
        self._keep = (A, P, C_rowptr)
        B.check(self._lib.spgemm_rap_symbolic(self._h, C.byref(da), C.byref(dp), C.c_void_p(C_rowptr.data_ptr()),
                                              C.byref(nnz), _stream(stream)), "spgemm_rap_symbolic")
        return C_rowptr, int(nnz.value)

    def rap_numeric(self, A: CsrMatrix, P: CsrMatrix, C_rowptr: torch.Tensor, nnz: Optional[int] = None,
                    C_colidx: Optional[torch.Tensor] = None, C_values: Optional[torch.Tensor] = None,
                    stream=None) -> CsrMatrix:
        """Columns (sorted per row) and values of C = P^T A P on the last rap_symbolic plan."""
        if nnz is None:
            nnz = int(C_rowptr[-1].item()) if C_colidx is None else C_colidx.numel()
        dev = C_rowptr.device
        if C_colidx is None:
            C_colidx = torch.empty(nnz, dtype=torch.int32, device=dev)
        if C_values is None:
            C_values = torch.empty(nnz, dtype=A.dtype, device=dev)
        da, dp = A.desc(), P.desc()
        B.check(self._lib.spgemm_rap_numeric(self._h, C.byref(da), C.byref(dp), C.c_void_p(C_rowptr.data_ptr()),
                                             _ptr(C_colidx), _ptr(C_values), _stream(stream)),
                "spgemm_rap_numeric")
        return CsrMatrix(C_rowptr, C_colidx, C_values, (P.ncols, P.ncols))

    def rap(self, A: CsrMatrix, P: CsrMatrix, stream=None) -> CsrMatrix:
        """C = P^T A P (both phases)."""
        rp, nnz = self.rap_symbolic(A, P, stream=stream)
        return self.rap_numeric(A, P, rp, nnz, stream=stream)

    def sync(self, stream=None):
        B.check(self._lib.spgemm_handle_sync(self._h, _stream(stream)), "spgemm_handle_sync")

    def row_flops(self, A: CsrMatrix, Bm: CsrMatrix, prefix: Optional[torch.Tensor] = None,
                  stream=None) -> torch.Tensor:
        """Inclusive prefix of the per-row multiplications of A*B (int64 [m + 1], on A's device)."""
        if prefix is None:
            prefix = torch.empty(A.nrows + 1, dtype=torch.int64, device=A.rowptr.device)
        hint = A.dtype or Bm.dtype
        da, db = A.desc(hint), Bm.desc(hint)
        B.check(self._lib.spgemm_row_flops(self._h, C.byref(da), C.byref(db), C.c_void_p(prefix.data_ptr()),
                                           _stream(stream)), "spgemm_row_flops")
        return prefix

    def stats(self) -> dict:
        st = B.StatsT()
        B.check(self._lib.spgemm_get_stats(self._h, C.byref(st)), "spgemm_get_stats")
        out = {name: getattr(st, name) for name, _ in B.StatsT._fields_ if name != "bin_rows_numeric"}
        out["bin_rows_numeric"] = list(st.bin_rows_numeric)
        return out

    # ---------------------------------------------------------------- masked / transpose
    def masked(self, X: CsrMatrix, Y: CsrMatrix, S_rowptr: torch.Tensor, S_colidx: torch.Tensor,
               out: Optional[torch.Tensor] = None, x_perm: Optional[torch.Tensor] = None,
               y_perm: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """out(i,l) = sum_j X(i,j) Y(j,l) for (i,l) in the pattern S.

        x_perm / y_perm: X's (Y's) entry p takes its value from values[perm[p]].
        """
        n = S_colidx.numel()
        if out is None:
            out = torch.empty(n, dtype=X.dtype, device=S_colidx.device)
        dx, dy = X.desc(), Y.desc()
        B.check(self._lib.spgemm_masked(self._h, C.byref(dx), C.byref(dy), C.c_void_p(S_rowptr.data_ptr()),
                                        _ptr(S_colidx), n, _ptr(out), _ptr(x_perm), _ptr(y_perm),
                                        _stream(stream)), "spgemm_masked")
        return out

    def masked_count(self, X: CsrMatrix, Y: CsrMatrix, S_rowptr: torch.Tensor, S_colidx: torch.Tensor,
                     out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """Per-row structural counts of (X·Y) on the pattern S (int64[X.nrows]):
        out[i] = sum over l in S(i,:) of |{j : (i,j) in X, (j,l) in Y}|; values
        are not read.  S_rowptr must be int64."""
        if out is None:
            out = torch.empty(X.nrows, dtype=torch.int64, device=S_colidx.device)
        assert S_rowptr.dtype == torch.int64
        dx, dy = X.desc(torch.float64), Y.desc(torch.float64)
        B.check(self._lib.spgemm_masked_count(self._h, C.byref(dx), C.byref(dy), C.c_void_p(S_rowptr.data_ptr()),
                                              _ptr(S_colidx), S_colidx.numel(), _ptr(out), _stream(stream)),
                "spgemm_masked_count")
        return out

    def transpose(self, A: CsrMatrix, with_values: bool = True, out=None, stream=None):
        """(A^T as CsrMatrix with int64 row pointers, perm) with At.values = A.values[perm].

        out: optional (At, perm) from an earlier call on the same shape to write into.
        """
        dev = A.colidx.device
        if out is not None:
            At0, perm = out
            Atp, Atj, Atx = At0.rowptr, At0.colidx, At0.values
        else:
            Atp = torch.empty(A.ncols + 1, dtype=torch.int64, device=dev)
            Atj = torch.empty(A.nnz, dtype=torch.int32, device=dev)
            perm = torch.empty(A.nnz, dtype=torch.int64, device=dev)
            Atx = None
            if with_values and A.values is not None:
                Atx = torch.empty(A.nnz, dtype=A.values.dtype, device=dev)
        d = A.desc() if (with_values and A.values is not None) else A.with_values(None).desc(A.dtype)
        B.check(self._lib.spgemm_transpose(self._h, C.byref(d), C.c_void_p(Atp.data_ptr()), _ptr(Atj), _ptr(Atx),
                                           _ptr(perm), _stream(stream)), "spgemm_transpose")
        return CsrMatrix(Atp, Atj, Atx, (A.ncols, A.nrows)), perm

    def gather(self, src: torch.Tensor, perm: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None):
        if out is None:
            out = torch.empty(perm.numel(), dtype=src.dtype, device=src.device)
        B.check(self._lib.spgemm_gather(self._h, _dtype_code(src.dtype), _ptr(src), _ptr(perm), _ptr(out),
                                        perm.numel(), _stream(stream)), "spgemm_gather")
        return out

    # ---------------------------------------------------------------- batched
    def batch_symbolic(self, As: Sequence[CsrMatrix], Bs: Sequence[CsrMatrix], stream=None):
        n = len(As)
        hint = As[0].dtype if n else None
        da = (B.CsrT * max(n, 1))(*[a.desc(hint) for a in As])
        db = (B.CsrT * max(n, 1))(*[b.desc(hint) for b in Bs])
        rps = [torch.empty(a.nrows + 1, dtype=torch.int64, device=a.rowptr.device) for a in As]
        prp = (C.c_void_p * max(n, 1))(*[r.data_ptr() for r in rps])
        nnz = (C.c_int64 * max(n, 1))()
        self._keep = (As, Bs, rps)
        B.check(self._lib.spgemm_batch_symbolic(self._h, n, da, db, prp, nnz, _stream(stream)),
                "spgemm_batch_symbolic")
        return rps, [int(nnz[i]) for i in range(n)]

    def batch_numeric(self, As, Bs, rowptrs, nnzs, colidx=None, values=None, stream=None) -> List[CsrMatrix]:
        n = len(As)
        if colidx is None:
            colidx = [torch.empty(z, dtype=torch.int32, device=r.device) for r, z in zip(rowptrs, nnzs)]
        if values is None:
            values = [torch.empty(z, dtype=a.dtype, device=r.device) for a, r, z in zip(As, rowptrs, nnzs)]
        da = (B.CsrT * max(n, 1))(*[a.desc() for a in As])
        db = (B.CsrT * max(n, 1))(*[b.desc() for b in Bs])
        prp = (C.c_void_p * max(n, 1))(*[r.data_ptr() for r in rowptrs])
        pcj = (C.c_void_p * max(n, 1))(*[(c.data_ptr() if c.numel() else 0) for c in colidx])
        pcx = (C.c_void_p * max(n, 1))(*[(v.data_ptr() if v.numel() else 0) for v in values])
        B.check(self._lib.spgemm_batch_numeric(self._h, n, da, db, prp, pcj, pcx, _stream(stream)),
                "spgemm_batch_numeric")
        return [CsrMatrix(r, c, v, (a.nrows, b.ncols)) for r, c, v, a, b in zip(rowptrs, colidx, values, As, Bs)]


# -------------------------------------------------------------------- row-range sharding
def partition_rows(prefix, parts: int) -> List[int]:
    """Row bounds [0 = b_0 <= ... <= b_parts = m] that split the flops in
    `prefix` (int64 [m + 1], host or device) into `parts` near-equal shares."""
    import numpy as np
    if isinstance(prefix, torch.Tensor):
        prefix = prefix.detach().cpu().numpy()
    pre = np.ascontiguousarray(prefix, dtype=np.int64)
    bounds = np.zeros(int(parts) + 1, dtype=np.int64)
    B.check(B.load().spgemm_partition_rows(C.c_void_p(pre.ctypes.data), int(pre.size - 1), int(parts),
                                           C.c_void_p(bounds.ctypes.data)), "spgemm_partition_rows")
    return [int(x) for x in bounds]


def row_block(A: CsrMatrix, r0: int, r1: int) -> CsrMatrix:
    """Rows [r0, r1) of A: row pointers rebased to 0, columns and values as views."""
    ends = A.rowptr[[r0, r1]].to("cpu").tolist()
    rp = (A.rowptr[r0:r1 + 1].to(torch.int64) - int(ends[0])).contiguous()
    cj = A.colidx[int(ends[0]):int(ends[1])]
    vx = None if A.values is None else A.values[int(ends[0]):int(ends[1])]
    return CsrMatrix(rp, cj, vx, (r1 - r0, A.ncols))


def shard_offsets(local_nnz: int, group=None) -> Tuple[int, int]:
    """(this shard's first entry in the global C, nnz of the global C): the one
    exchange of row-range sharding, an all-gather of the shards' nnz."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return 0, int(local_nnz)
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    mine = torch.tensor([int(local_nnz)], dtype=torch.int64, device=dev)
    allv = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(allv, mine, group=group)
    counts = [int(t.item()) for t in allv]
    return sum(counts[:rank]), sum(counts)


def shard_multiply(h: "SpGEMM", A: CsrMatrix, Bm: CsrMatrix, rank: int, parts: int, stream=None):
    """Row shard `rank` of `parts` of C = A*B on this device (B replicated):
    returns (C block, its first row, its first entry in the global C, global nnz)."""
    bounds = partition_rows(h.row_flops(A, Bm, stream=stream), parts)
    r0, r1 = bounds[rank], bounds[rank + 1]
    Cb = h.multiply(row_block(A, r0, r1), Bm, stream=stream)
    off, total = shard_offsets(Cb.nnz)
    return Cb, r0, off, total


def launch_count() -> int:
    """Kernels launched by libkkspgemm so far in this process."""
    return int(B.load().spgemm_launch_count())


def spgemm(A: CsrMatrix, Bm: CsrMatrix, **options) -> CsrMatrix:
    """One-shot C = A·B (symbolic + numeric) on a fresh handle."""
    h = SpGEMM(**options)
    try:
        Cm = h.multiply(A, Bm)
        h.sync()
        return Cm
    finally:
        h.close()
