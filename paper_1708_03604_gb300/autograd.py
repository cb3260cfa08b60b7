"""Differentiable block-sparse tensors over libbsm.

``BlockSparseTensor`` pairs a libbsm handle (the block pattern) with its
values as a CUDA tensor that the handle borrows.  ``matmul`` and ``add`` are
``torch.autograd.Function``s whose backward passes call the library's
hand-written adjoints:

* C = alpha*A.B (on-the-fly filtered): dA = alpha*dC.B^T on A's pattern and
  dB = alpha*A^T.dC on B's pattern, over the products the forward kept
  (``bsm_multiply_backward``);
* Z = a*X + b*Y (norm filtered): dX = a*dZ, dY = b*dZ on the blocks that
  reached Z (``bsm_add_backward``).

The gradient is that of the implemented function at fixed keep-decisions.
``mcweeny`` runs the purification chain X <- 3X^2 - 2X^3 with optional
checkpointing of every ``checkpoint_every`` steps (the intermediate products
of a segment are recomputed in backward).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.utils.checkpoint as _ckpt

from . import bsm


class BlockSparseTensor:
    """A libbsm block pattern plus its values (CUDA tensor borrowed by the handle)."""

    def __init__(self, handle: bsm.Matrix, data: torch.Tensor):
        self.handle = handle
        self.data = data

    @classmethod
    def from_bcsr(cls, X, requires_grad: bool = False, dtype=torch.float64) -> "BlockSparseTensor":
        data = torch.tensor(np.asarray(X.data), dtype=dtype, device="cuda")
        h = bsm.Matrix.from_device(X, data, borrow=True)
        data.requires_grad_(requires_grad)
        return cls(h, data)

    @property
    def row_bs(self):
        return self.handle.row_bs

    @property
    def col_bs(self):
        return self.handle.col_bs

    def pattern(self):
        return self.handle.pattern()

    def to_host(self):
        rp, ci, bo = self.pattern()
        from types import SimpleNamespace
        return SimpleNamespace(row_bs=self.row_bs, col_bs=self.col_bs, row_ptr=rp, col_idx=ci, blk_off=bo,
                               data=self.data.detach().cpu().numpy())


class _MatMul(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a, b, A, B, alpha, eps, prec, sink):
        Cm = bsm.multiply(alpha, A, B, eps=eps, prec=prec)
        c = Cm.data_tensor()
        Cm.borrow(c)
        sink.append(Cm)
        ctx.save_for_backward(a, b)
        ctx.handles = (A, B, Cm)
        ctx.alpha, ctx.prec = alpha, prec
        return c

    @staticmethod
    def backward(ctx, gc):
        a, b = ctx.saved_tensors
        A, B, Cm = ctx.handles
        dA = torch.empty_like(a) if ctx.needs_input_grad[0] else None
        dB = torch.empty_like(b) if ctx.needs_input_grad[1] else None
        bsm.multiply_backward(ctx.alpha, Cm, gc.contiguous(), A, B, dA, dB, prec=ctx.prec)
        return dA, dB, None, None, None, None, None, None


class _Add(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, y, X, Y, a, b, eps, sink):
        Z = bsm.add(a, X, b, Y, eps=eps)
        z = Z.data_tensor()
        Z.borrow(z)
        sink.append(Z)
        ctx.save_for_backward(x, y)
        ctx.handles = (X, Y, Z)
        return z

    @staticmethod
    def backward(ctx, gz):
        x, y = ctx.saved_tensors
        X, Y, Z = ctx.handles
        dX = torch.empty_like(x) if ctx.needs_input_grad[0] else None
        dY = torch.empty_like(y) if ctx.needs_input_grad[1] else None
        bsm.add_backward(Z, gz.contiguous(), X, Y, dX, dY)
        return dX, dY, None, None, None, None, None, None


def matmul(X: BlockSparseTensor, Y: BlockSparseTensor, alpha: float = 1.0, eps: float = 0.0,
           prec: str = "fp64") -> BlockSparseTensor:
    """alpha * X.Y with on-the-fly filtering at eps (differentiable)."""
    sink: list = []
    c = _MatMul.apply(X.data, Y.data, X.handle, Y.handle, float(alpha), float(eps), prec, sink)
    return BlockSparseTensor(sink[0], c)


def add(X: BlockSparseTensor, Y: BlockSparseTensor, a: float = 1.0, b: float = 1.0,
        eps: float = 0.0) -> BlockSparseTensor:
    """a*X + b*Y over the union pattern, blocks with norm <= eps dropped (differentiable)."""
    sink: list = []
    z = _Add.apply(X.data, Y.data, X.handle, Y.handle, float(a), float(b), float(eps), sink)
    return BlockSparseTensor(sink[0], z)


def mcweeny_step(X: BlockSparseTensor, eps: float, prec: str = "fp64") -> BlockSparseTensor:
    """One purification step 3X^2 - 2X^3, every multiply and the add filtered at eps."""
    X2 = matmul(X, X, eps=eps, prec=prec)
    X3 = matmul(X2, X, eps=eps, prec=prec)
    return add(X2, X3, 3.0, -2.0, eps=eps)


def mcweeny(X0: BlockSparseTensor, steps: int, eps: float, prec: str = "fp64",
            checkpoint_every: int = 0) -> BlockSparseTensor:
    """Purification chain; with checkpoint_every = c > 0 only every c-th
    iterate is kept for backward and each segment of c steps is recomputed."""
    X = X0
    k = 0
    while k < steps:
        seg = min(checkpoint_every, steps - k) if checkpoint_every > 0 else 1
        if checkpoint_every > 0 and torch.is_grad_enabled() and X.data.requires_grad:
            sink: list = []
            handle = X.handle

            def run(x_data, _h=handle, _n=seg, _sink=sink):
                Y = BlockSparseTensor(_h, x_data)
                for _ in range(_n):
                    Y = mcweeny_step(Y, eps, prec)
                _sink.append(Y.handle)
                return Y.data

            z = _ckpt.checkpoint(run, X.data, use_reentrant=True)
            X = BlockSparseTensor(sink[0], z)
        else:
            for _ in range(seg):
                X = mcweeny_step(X, eps, prec)
        k += seg
    return X


def block_pair_index(X, W, transpose_w: bool = False):
    """Element index pairs (into X.data, into W.data) of the blocks both
    patterns hold: X block (i, j) against W block (i, j), or W block (j, i)
    transposed when transpose_w.  Host-side bookkeeping for losses."""
    xr, xc, xo = (np.asarray(v) for v in X.pattern())
    wr, wc, wo = (np.asarray(v) for v in W.pattern())
    rbs, cbs = np.asarray(X.row_bs, np.int64), np.asarray(X.col_bs, np.int64)
    nbc = max(len(cbs), len(rbs))
    xrow = np.repeat(np.arange(len(xr) - 1, dtype=np.int64), np.diff(xr))
    wrow = np.repeat(np.arange(len(wr) - 1, dtype=np.int64), np.diff(wr))
    wkey = wrow * nbc + wc.astype(np.int64)          # ascending (CSR order)
    xcol = xc.astype(np.int64)
    xkey = xcol * nbc + xrow if transpose_w else xrow * nbc + xcol
    pos = np.searchsorted(wkey, xkey)
    hit = pos < len(wkey)
    hit[hit] = wkey[pos[hit]] == xkey[hit]
    if not hit.any():
        return (torch.zeros(0, dtype=torch.int64, device="cuda"),) * 2
    qx = np.nonzero(hit)[0]
    m, n = rbs[xrow[qx]], cbs[xcol[qx]]
    size = m * n
    start = np.concatenate([[0], np.cumsum(size)[:-1]])
    blk = np.repeat(np.arange(len(qx)), size)
    e = np.arange(int(size.sum()), dtype=np.int64) - start[blk]     # element inside the block
    ix = xo[qx][blk] + e
    if transpose_w:
        nn = n[blk]
        r, c = e // nn, e % nn
        iw = wo[pos[qx]][blk] + c * m[blk] + r
    else:
        iw = wo[pos[qx]][blk] + e
    return torch.tensor(ix, device="cuda"), torch.tensor(iw, device="cuda")


def trace_product(X: BlockSparseTensor, W: BlockSparseTensor) -> torch.Tensor:
    """trace(X.W) = sum over blocks of X_ij . W_ji^T (elementwise)."""
    ix, iw = block_pair_index(X, W, transpose_w=True)
    return (X.data[ix] * W.data[iw]).sum()
