"""Test-side helpers: densify block-sparse matrices and compare results.

Nothing here implements the multiply; dense products use numpy/BLAS."""
from __future__ import annotations

import numpy as np

from paper_1708_03604_gb300 import inputs as I


def offsets(bs):
    return np.concatenate([[0], np.cumsum(np.asarray(bs, dtype=np.int64))])


def to_dense(X) -> np.ndarray:
    ro, co = offsets(X.row_bs), offsets(X.col_bs)
    D = np.zeros((int(ro[-1]), int(co[-1])))
    row_ptr = np.asarray(X.row_ptr)
    for i in range(len(X.row_bs)):
        for b in range(int(row_ptr[i]), int(row_ptr[i + 1])):
            j = int(X.col_idx[b])
            m, n = int(X.row_bs[i]), int(X.col_bs[j])
            D[ro[i]:ro[i] + m, co[j]:co[j] + n] = np.asarray(X.data[X.blk_off[b]:X.blk_off[b] + m * n],
                                                            dtype=np.float64).reshape(m, n)
    return D


def block_mask(X) -> np.ndarray:
    ro, co = offsets(X.row_bs), offsets(X.col_bs)
    M = np.zeros((int(ro[-1]), int(co[-1])), dtype=bool)
    row_ptr = np.asarray(X.row_ptr)
    for i in range(len(X.row_bs)):
        for b in range(int(row_ptr[i]), int(row_ptr[i + 1])):
            j = int(X.col_idx[b])
            M[ro[i]:ro[i] + X.row_bs[i], co[j]:co[j] + X.col_bs[j]] = True
    return M


def pattern_set(X):
    row_ptr = np.asarray(X.row_ptr)
    return {(i, int(X.col_idx[b])) for i in range(len(X.row_bs))
            for b in range(int(row_ptr[i]), int(row_ptr[i + 1]))}


def random_bcsr(row_bs, col_bs, occ, seed, dtype=np.float64):
    rows, cols, _ = I.uniform_pattern(len(row_bs), len(col_bs), occ, seed)
    return I.assemble(row_bs, col_bs, rows, cols, None, seed=seed + 1000, dtype=dtype)


def rel_fro(x, ref) -> float:
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / (den if den > 0 else 1.0))
