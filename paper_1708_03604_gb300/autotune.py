"""Autotuner of the numeric kernels' per-shape variants.

For every output block shape (m, n) that a multiply produces there are two
ways to compute its block products:

* variant 0: one warp per output block (FP64: lanes over its elements;
  split paths: tensor-core MMAs on packed fragments);
* variant 1, for blocks of at most 16 elements (FP64 also 5 x 5 and 6 x 6):
  one lane per output block on CUDA cores (split paths: the same narrow
  pieces multiplied with FP32 FMA).

Which is faster depends on the shape and the product mix, so it is measured:
starting from variant 0 everywhere, each shape in turn is switched to
variant 1 and kept there if the numeric kernel (timed with CUDA events by
the library) gets faster.  The table is process-wide in libbsm and can be
saved to / loaded from JSON.
"""
from __future__ import annotations

import json
import statistics

import numpy as np

from . import bsm


def _shapes(A: bsm.Matrix, B: bsm.Matrix):
    ms = sorted(set(int(x) for x in np.asarray(A.row_bs)))
    ns = sorted(set(int(x) for x in np.asarray(B.col_bs)))
    return sorted(((m, n) for m in ms for n in ns), key=lambda t: (t[0] * t[1], t))


def _numeric_ms(A, B, eps, prec, reps, Cm):
    t = []
    for _ in range(reps):
        bsm.multiply(1.0, A, B, 0.0, Cm, eps, prec=prec, build_stacks=False)
        t.append(Cm.timings()["numeric"])
    return statistics.median(t)


def tune(A: bsm.Matrix, B: bsm.Matrix, eps: float = 0.0, prec: str = "tf32x3", reps: int = 3,
         gain: float = 0.01) -> dict:
    """Choose the variant of every output shape of A.B for `prec`; returns
    {"prec": ..., "variants": {"m x n": 0|1}, "numeric_ms": {...}}.  The
    tcgen05 row-panel engine has no per-shape variants: tune "tf32x3" for the
    kernel it falls back to."""
    if prec == "tf32x3_panel":
        raise ValueError("the tf32x3_panel engine has no per-shape variants")
    # larger shapes have one variant
    fp64 = prec in ("fp64", "fp64_dmma", "ozaki")  # lane variant = plain FP64 FMA
    shapes = [(m, n) for m, n in _shapes(A, B) if m * n <= 16 or (fp64 and (m, n) in ((5, 5), (6, 6)))]
    for m, n in shapes:
        bsm.bsm_set_variant(prec, m, n, 0)
    Cm = bsm.Matrix.empty(A.row_bs, B.col_bs)
    bsm.bsm_set_profiling(True)
    try:
        _numeric_ms(A, B, eps, prec, 1, Cm)  # warm-up
        best = _numeric_ms(A, B, eps, prec, reps, Cm)
        start = best
        chosen = {}
        for m, n in shapes:
            bsm.bsm_set_variant(prec, m, n, 1)
            t = _numeric_ms(A, B, eps, prec, reps, Cm)
            if t < best * (1.0 - gain):
                best = t
                chosen[f"{m}x{n}"] = 1
            else:
                bsm.bsm_set_variant(prec, m, n, 0)
                chosen[f"{m}x{n}"] = 0
    finally:
        bsm.bsm_set_profiling(False)
    return {"prec": prec, "variants": chosen, "numeric_ms": {"all_mma": start, "tuned": best}}


def apply(table: dict):
    for key, v in table["variants"].items():
        m, n = (int(x) for x in key.split("x"))
        bsm.bsm_set_variant(table["prec"], m, n, int(v))


def reset(prec: str, sizes):
    """Back to the library's default variants for these block sizes."""
    for m in sizes:
        for n in sizes:
            bsm.bsm_set_variant(prec, int(m), int(n), -1)


def save(tables, path: str):
    with open(path, "w") as f:
        json.dump(tables, f, indent=1, sort_keys=True)


def load(path: str):
    with open(path) as f:
        tables = json.load(f)
    for t in (tables if isinstance(tables, list) else [tables]):
        apply(t)
    return tables
