"""Seeded synthetic block-sparse inputs.

This module only *builds inputs*: block-size vectors, block patterns and
block values.  It holds none of the multiply's arithmetic (no norms, no
filtering, no products) and imports nothing from the CUDA binding or from the
oracle, so both sides of every parity test are fed from here.

The paper's own matrices come from CP2K runs (Table 1 of the paper: S-E,
H2O-DFT-LS, AMORPH) that are not available; these generators stand in for
them with the same geometry:

* ``uniform`` patterns: exactly ``round(occ * nbr * nbc)`` distinct blocks
  drawn without replacement (uniformly at random);
* ``banded`` patterns: block (i, j) present iff ``|i - j| <= W`` and a
  uniform draw is < 0.5 (the diagonal always present), ``W = round(occ * nb)``,
  followed by one symmetric random permutation of the block indices (DBCSR
  permutes rows and columns randomly for load balance, §1.1 of the paper);
  values are scaled by ``exp(-d / 50)`` with ``d`` the pre-permutation
  block distance, mimicking the decay of a localised-basis operator.

Seeds: A=1, B=2, T=3, X0=5, W=6, block sizes=7, permutation=8.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

SEED_A, SEED_B, SEED_T, SEED_X0, SEED_W, SEED_SIZES, SEED_PERM = 1, 2, 3, 5, 6, 7, 8


@dataclass
class BCSR:
    """Host-side block-CSR matrix (row-major elements inside each block)."""

    row_bs: np.ndarray   # int32 [nbr]
    col_bs: np.ndarray   # int32 [nbc]
    row_ptr: np.ndarray  # int64 [nbr + 1]
    col_idx: np.ndarray  # int32 [nnzb], ascending within each row
    blk_off: np.ndarray  # int64 [nnzb], element offset of each block
    data: np.ndarray     # float64 or float32 [data_len]

    @property
    def nbr(self) -> int:
        return int(self.row_bs.shape[0])

    @property
    def nbc(self) -> int:
        return int(self.col_bs.shape[0])

    @property
    def nnzb(self) -> int:
        return int(self.row_ptr[-1])

    def block_rows(self) -> np.ndarray:
        """Block-row index of every stored block."""
        return np.repeat(np.arange(self.nbr, dtype=np.int32), np.diff(self.row_ptr))

    def astype(self, dtype) -> "BCSR":
        return replace(self, data=self.data.astype(dtype))


# --------------------------------------------------------------------------
# block sizes
# --------------------------------------------------------------------------
def uniform_sizes(nb: int, s: int) -> np.ndarray:
    return np.full(nb, s, dtype=np.int32)


def mixed_sizes(nb: int, sizes, probs, seed: int = SEED_SIZES) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.asarray(rng.choice(np.asarray(sizes, dtype=np.int32), size=nb, p=probs), dtype=np.int32)


# --------------------------------------------------------------------------
# patterns: (rows, cols, dist) with dist the pre-permutation |i - j|
# --------------------------------------------------------------------------
def uniform_pattern(nbr: int, nbc: int, occ: float, seed: int):
    rng = np.random.default_rng(seed)
    count = int(round(occ * nbr * nbc))
    lin = np.sort(rng.choice(nbr * nbc, size=count, replace=False))
    rows = (lin // nbc).astype(np.int64)
    cols = (lin % nbc).astype(np.int64)
    return rows, cols, None


def permutation(nb: int, seed: int = SEED_PERM) -> np.ndarray:
    return np.random.default_rng(seed).permutation(nb).astype(np.int64)


def banded_pattern(nb: int, occ: float, seed: int, perm: np.ndarray | None,
                   half: float = 0.5, symmetric: bool = False):
    """Band of half-width W = round(occ * nb), each off-diagonal block kept
    with probability ``half``; then rows and columns go through ``perm``.

    ``symmetric=True`` draws the upper triangle and mirrors it."""
    W = int(round(occ * nb))
    rng = np.random.default_rng(seed)
    i0 = np.repeat(np.arange(nb, dtype=np.int64), 2 * W + 1)
    d0 = np.tile(np.arange(-W, W + 1, dtype=np.int64), nb)
    j0 = i0 + d0
    ok = (j0 >= 0) & (j0 < nb)
    i0, j0, d0 = i0[ok], j0[ok], d0[ok]
    u = rng.random(i0.shape[0])
    if symmetric:
        # decide on the upper triangle only, then mirror it
        keep = (d0 >= 0) & ((u < half) | (d0 == 0))
        i0, j0 = i0[keep], j0[keep]
        off = i0 != j0
        i0, j0 = np.concatenate([i0, j0[off]]), np.concatenate([j0, i0[off]])
        d0 = j0 - i0
        keep = np.ones(i0.shape[0], dtype=bool)
    else:
        keep = (u < half) | (d0 == 0)
    i0, j0, d0 = i0[keep], j0[keep], d0[keep]
    if perm is not None:
        rows, cols = perm[i0], perm[j0]
    else:
        rows, cols = i0, j0
    return rows, cols, np.abs(d0)


# --------------------------------------------------------------------------
# assembling a BCSR matrix
# --------------------------------------------------------------------------
def assemble(row_bs, col_bs, rows, cols, dist, seed: int, decay: float | None = None,
             dtype=np.float64, values: str = "normal") -> BCSR:
    """Sort the (row, col) pattern into CSR order, lay the blocks out
    contiguously and fill them with N(0, 1) values (times exp(-dist/decay)
    when ``decay`` is given)."""
    row_bs = np.asarray(row_bs, dtype=np.int32)
    col_bs = np.asarray(col_bs, dtype=np.int32)
    nbr, nbc = row_bs.shape[0], col_bs.shape[0]
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    if dist is not None:
        dist = np.asarray(dist)[order]
    counts = np.bincount(rows, minlength=nbr)
    row_ptr = np.zeros(nbr + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    sizes = row_bs[rows].astype(np.int64) * col_bs[cols].astype(np.int64)
    blk_off = np.zeros(rows.shape[0], dtype=np.int64)
    if rows.shape[0] > 1:
        np.cumsum(sizes[:-1], out=blk_off[1:])
    total = int(sizes.sum())
    rng = np.random.default_rng(seed)
    if values == "normal":
        data = rng.standard_normal(total)
    elif values == "zeros":
        data = np.zeros(total)
    else:
        raise ValueError(values)
    if decay is not None and dist is not None and total:
        scale = np.exp(-dist.astype(np.float64) / decay)
        # block by block (in chunks of blocks, so no element-sized temporary)
        step = 1 << 20
        for b0 in range(0, rows.shape[0], step):
            b1 = min(b0 + step, rows.shape[0])
            e0 = int(blk_off[b0])
            e1 = int(blk_off[b1 - 1] + sizes[b1 - 1])
            data[e0:e1] *= np.repeat(scale[b0:b1], sizes[b0:b1])
    return BCSR(row_bs, col_bs, row_ptr, cols.astype(np.int32), blk_off, data.astype(dtype, copy=False))


def empty(row_bs, col_bs, dtype=np.float64) -> BCSR:
    row_bs = np.asarray(row_bs, dtype=np.int32)
    col_bs = np.asarray(col_bs, dtype=np.int32)
    return BCSR(row_bs, col_bs, np.zeros(row_bs.shape[0] + 1, dtype=np.int64),
                np.zeros(0, dtype=np.int32), np.zeros(0, dtype=np.int64), np.zeros(0, dtype=dtype))


def identity(bs) -> BCSR:
    """Block-diagonal identity with blocking ``bs``."""
    bs = np.asarray(bs, dtype=np.int32)
    nb = bs.shape[0]
    m = assemble(bs, bs, np.arange(nb), np.arange(nb), None, seed=0, values="zeros")
    for b in range(nb):
        s = int(bs[b])
        m.data[m.blk_off[b]:m.blk_off[b] + s * s] = np.eye(s).ravel()
    return m


def permutation_matrix(bs, perm) -> BCSR:
    """Block permutation P with P[i, perm[i]] = I, so (P.A) row i = A row perm[i].
    Requires bs[i] == bs[perm[i]]."""
    bs = np.asarray(bs, dtype=np.int32)
    perm = np.asarray(perm, dtype=np.int64)
    nb = bs.shape[0]
    m = assemble(bs, bs, np.arange(nb), perm, None, seed=0, values="zeros")
    for i in range(nb):
        s = int(bs[i])
        b = m.row_ptr[i]
        m.data[m.blk_off[b]:m.blk_off[b] + s * s] = np.eye(s).ravel()
    return m


def _shape_groups(X: BCSR):
    """Yield (block indices, m, n) for every distinct block shape of X."""
    brow = X.block_rows()
    m = X.row_bs[brow].astype(np.int64)
    n = X.col_bs[X.col_idx].astype(np.int64)
    key = m * 65536 + n
    for kv in np.unique(key):
        idx = np.nonzero(key == kv)[0]
        yield idx, int(kv // 65536), int(kv % 65536)


def _gather_blocks(X: BCSR, idx, m, n):
    e = X.blk_off[idx][:, None] + np.arange(m * n, dtype=np.int64)[None, :]
    return X.data[e].reshape(-1, m, n), e


def transpose(X: BCSR) -> BCSR:
    """Block transpose (pattern and every block transposed)."""
    rows = X.block_rows().astype(np.int64)
    cols = X.col_idx.astype(np.int64)
    T = assemble(X.col_bs, X.row_bs, cols, rows, None, seed=0, values="zeros", dtype=X.data.dtype)
    src = np.lexsort((rows, cols))          # transposed CSR order -> source block
    dst = np.empty_like(src)
    dst[src] = np.arange(src.shape[0])     # source block -> transposed position
    for idx, m, n in _shape_groups(X):
        blk, _ = _gather_blocks(X, idx, m, n)
        e = T.blk_off[dst[idx]][:, None] + np.arange(m * n, dtype=np.int64)[None, :]
        T.data[e] = blk.transpose(0, 2, 1).reshape(-1, m * n)
    return T


# --------------------------------------------------------------------------
# the five workloads (sizes can be scaled down for oracle-speed tests)
# --------------------------------------------------------------------------
def uniform_23(nb: int = 200, occ: float = 0.20, s: int = 23):
    """Plain FP64 C = A.B, uniform s x s blocks, occupancy ``occ`` chosen
    uniformly at random, N(0,1) values, beta = 0, no filtering."""
    bs = uniform_sizes(nb, s)
    A = assemble(bs, bs, *uniform_pattern(nb, nb, occ, SEED_A), seed=SEED_A + 100)
    B = assemble(bs, bs, *uniform_pattern(nb, nb, occ, SEED_B), seed=SEED_B + 100)
    return dict(A=A, B=B, eps=0.0, alpha=1.0, beta=0.0)


def mixed_banded(nb: int = 3000, occ: float = 0.10, sizes=(5, 13, 23), probs=(0.6, 0.2, 0.2),
                 eps: float = 1e-6, decay: float = 50.0):
    """Mixed block sizes drawn per block row/column, banded-local pattern then
    randomly permuted (about ``occ`` occupancy), values N(0,1)*exp(-d/decay),
    filter threshold ``eps`` on block-norm products."""
    bs = mixed_sizes(nb, sizes, probs)
    perm = permutation(nb)
    A = assemble(bs, bs, *banded_pattern(nb, occ, SEED_A, perm), seed=SEED_A + 100, decay=decay)
    B = assemble(bs, bs, *banded_pattern(nb, occ, SEED_B, perm), seed=SEED_B + 100, decay=decay)
    return dict(A=A, B=B, eps=eps, alpha=1.0, beta=0.0)


def large_banded_23(nb: int = 6912, occ: float = 0.05, eps: float = 1e-8, decay: float = 50.0):
    """Uniform 23 x 23 blocks with the banded-then-permuted pattern
    (H2O-DFT-LS geometry: 6912 * 23 = 158,976 rows)."""
    bs = uniform_sizes(nb, 23)
    perm = permutation(nb)
    A = assemble(bs, bs, *banded_pattern(nb, occ, SEED_A, perm), seed=SEED_A + 100, decay=decay)
    B = assemble(bs, bs, *banded_pattern(nb, occ, SEED_B, perm), seed=SEED_B + 100, decay=decay)
    return dict(A=A, B=B, eps=eps, alpha=1.0, beta=0.0)


def differentiation_13(nb: int = 800, occ: float = 0.15, dtype=np.float64):
    """Loss ||A.B - T||_F^2 workload: 13 x 13 blocks, uniform random
    patterns for A, B and T, N(0,1) values."""
    bs = uniform_sizes(nb, 13)
    A = assemble(bs, bs, *uniform_pattern(nb, nb, occ, SEED_A), seed=SEED_A + 100, dtype=dtype)
    B = assemble(bs, bs, *uniform_pattern(nb, nb, occ, SEED_B), seed=SEED_B + 100, dtype=dtype)
    T = assemble(bs, bs, *uniform_pattern(nb, nb, occ, SEED_T), seed=SEED_T + 100, dtype=dtype)
    return dict(A=A, B=B, T=T, eps=0.0, alpha=1.0, beta=0.0)


def purification_start(nb: int = 20000, occ: float = 0.02, sizes=(4, 1), probs=(0.5, 0.5),
                       decay: float = 50.0):
    """Symmetric block-sparse X0 for the McWeeny chain: banded pattern with
    decaying N(0,1) values, symmetrised, then shifted and scaled by its
    Gershgorin interval so that every eigenvalue lies in [0, 1]; W has X0's
    pattern with N(0,1) values (the weight of the trace objective)."""
    bs = mixed_sizes(nb, sizes, probs)
    perm = permutation(nb)
    rows, cols, dist = banded_pattern(nb, occ, SEED_X0, perm, symmetric=True)
    H = assemble(bs, bs, rows, cols, dist, seed=SEED_X0 + 100, decay=decay)
    # symmetrise: H <- (H + H^T) / 2 block by block (pattern is symmetric)
    Ht = transpose(H)
    H.data = 0.5 * (H.data + Ht.data)
    # Gershgorin interval over scalar rows
    ro = np.concatenate([[0], np.cumsum(bs.astype(np.int64))])
    n = int(ro[-1])
    diag = np.zeros(n)
    absum = np.zeros(n)
    brow = H.block_rows()
    for idx, m, k in _shape_groups(H):
        blk, _ = _gather_blocks(H, idx, m, k)
        r = ro[brow[idx]][:, None] + np.arange(m)[None, :]
        np.add.at(absum, r.ravel(), np.abs(blk).sum(axis=2).ravel())
        isd = brow[idx] == H.col_idx[idx]
        if isd.any():
            d = np.diagonal(blk[isd], axis1=1, axis2=2)
            np.add.at(diag, r[isd].ravel(), d.ravel())
    radius = absum - np.abs(diag)
    lo = float(np.min(diag - radius))
    hi = float(np.max(diag + radius))
    X0 = H
    X0.data = X0.data / (hi - lo)
    for idx, m, k in _shape_groups(X0):
        isd = idx[brow[idx] == X0.col_idx[idx]]
        if isd.size:
            e = X0.blk_off[isd][:, None] + (np.arange(m) * (m + 1))[None, :]
            X0.data[e] -= lo / (hi - lo)
    Wm = assemble(bs, bs, rows, cols, None, seed=SEED_W + 100)
    return dict(X0=X0, W=Wm, eps=1e-7, steps=10)
