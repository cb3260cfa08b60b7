"""Autotuner of the numeric kernels (the paper's GPU library finds its kernel
parameters per block shape by auto-tuning, §2; this is the same idea over
the knobs of this library's kernels).

What it searches, per precision, by timing the numeric kernel (CUDA events
recorded by the library around the launch) on the caller's operands:

* per output block shape (m, n): the variant -- one warp per block (FP64:
  lanes over its elements; split and Ozaki paths: tensor-core MMAs on packed
  fragments) or, for blocks of at most 16 elements and 5 x 5 ones (FP64 and
  Ozaki also 6 x 6), one lane per block on the CUDA cores;
* the FP64 FMA kernel build (how many output elements a lane holds per pass:
  up to 9 or up to 24) -- BSM_P_FP64;
* warps per CTA (4 or 2) of the persistent mma.sync kernels;
* persistent CTAs per SM;
* the fragment-tile pass shape (tiles along rows and columns that one pass
  over a block's products covers) of the split, Ozaki and FP64-MMA kernels
  (on the split paths also the default split: blocks of one tile row in a
  kernel instance of their own, compiled for 1-row passes);
* the order of the output blocks: by block row, or by 2-D tiles of ranked
  rows x ranked columns so that the blocks in flight share A's and B's
  blocks in L2;
* for TF32x3, the engine: the per-C-block mma.sync kernel or the tcgen05
  row-panel engine (where it applies), and for the latter the k-steps summed
  in one tensor-memory accumulator before each drain -- the fastest within
  ``err_target`` of the FP64 path;
* for the split paths, the interval F of the cross-product sum (FP32
  accumulation in the tensor core over at most F block products, then an FP64
  running sum or a compensated FP32 pair), the fastest form and F whose result
  is within ``err_target`` (relative Frobenius) of the FP64 path on the same
  operands.

Each knob is searched in turn (coordinate descent from the library
defaults), a value kept only when it is faster by more than ``gain``.  The
chosen table is process-wide in libbsm, saved to / loaded from JSON.

Run as a module to tune the bench workloads and write a table:
``python -m paper_1708_03604_gb300.autotune --workload mixed3000 --out t.json``.
"""
from __future__ import annotations

import argparse
import json
import statistics

import numpy as np

from . import bsm

SPLIT = ("tf32x3", "bf16x3", "bf16x6")
TILES = ("sched_tile", [0, 16, 32, 64, 128])
SEARCH = {
    "fp64": [("fp64_build", [0, 1, 2]), ("ctas_per_sm", [0, 1, 2, 3, 4]), TILES],
    "fp64_dmma": [("pass_mt", [3, 2, 1]), ("pass_nt", [3, 2, 1]), ("ctas_per_sm", [0, 1, 2, 4]), TILES],
    "ozaki": [("cta_warps", [4, 2]), ("pass_nt", [3, 2, 1]), ("ctas_per_sm", [0, 1, 2, 3]), TILES],
}
for _p in SPLIT:
    # pass_mt -1: blocks of one tile row in a 1-row kernel instance, the rest in a 2-row one
    SEARCH[_p] = [("cta_warps", [4, 2]), ("pass_mt", [-1, 2, 1]), ("pass_nt", [3, 2, 1]),
                  ("ctas_per_sm", [0, 1, 2, 3, 4]), TILES]
# TF32x3 may also run on the tcgen05 row-panel engine where it applies
SEARCH["tf32x3"] = SEARCH["tf32x3"] + [("engine", [0, 1])]
# flush_every: F > 0 an FP64 running sum every F block products, -F a
# compensated FP32 pair refreshed every F products
FLUSH_CANDIDATES = [-1, -2, -4, -8, 1, 2, 4, 8, 16]
PANEL_STEPS = [3, 4, 6, 8]


def _shapes(A: bsm.Matrix, B: bsm.Matrix):
    ms = sorted(set(int(x) for x in np.asarray(A.row_bs)))
    ns = sorted(set(int(x) for x in np.asarray(B.col_bs)))
    return sorted(((m, n) for m in ms for n in ns), key=lambda t: (t[0] * t[1], t))


def _numeric_ms(A, B, eps, prec, reps, Cm, flush_every=0, phase="numeric"):
    t = []
    for _ in range(reps):
        bsm.multiply(1.0, A, B, 0.0, Cm, eps, prec=prec, build_stacks=False, flush_every=flush_every)
        t.append(Cm.timings()[phase])
    return statistics.median(t)


def reset(prec: str, sizes=()):
    """Back to the library's defaults for `prec` (launch knobs, and the
    variants of these block sizes)."""
    for name, _ in SEARCH.get(prec, []):
        bsm.bsm_set_tuning(prec, name, -1)
    if prec == "tf32x3":
        bsm.bsm_set_tuning(prec, "panel_steps", -1)
    for m in sizes:
        for n in sizes:
            bsm.bsm_set_variant(prec, int(m), int(n), -1)


def _rel_err(torch, x, ref):
    return float(torch.linalg.vector_norm(x - ref) / torch.linalg.vector_norm(ref))


def tune(A: bsm.Matrix, B: bsm.Matrix, eps: float = 0.0, prec: str = "tf32x3", reps: int = 3,
         gain: float = 0.01, tune_flush: bool = True, err_target: float = 1e-6) -> dict:
    """Choose the variants and launch knobs of `prec` for A.B; returns the
    table (also left in effect in the library)."""
    if prec == "tf32x3_panel":
        raise ValueError("the tf32x3_panel engine is tuned through 'tf32x3' (its engine and panel_steps knobs)")
    fp64_like = prec in ("fp64", "fp64_dmma", "ozaki")  # lane variant = plain FP64 FMA
    shapes = [(m, n) for m, n in _shapes(A, B)
              if m * n <= 16 or (m, n) == (5, 5) or (fp64_like and (m, n) == (6, 6))]
    reset(prec)
    for m, n in shapes:
        bsm.bsm_set_variant(prec, m, n, 0)
    Cm = bsm.Matrix.empty(A.row_bs, B.col_bs)
    bsm.bsm_set_profiling(True)
    try:
        _numeric_ms(A, B, eps, prec, 1, Cm)  # warm-up
        start = best = _numeric_ms(A, B, eps, prec, reps, Cm)
        variants = {}
        for m, n in shapes:
            bsm.bsm_set_variant(prec, m, n, 1)
            t = _numeric_ms(A, B, eps, prec, reps, Cm)
            if t < best * (1.0 - gain):
                best = t
                variants[f"{m}x{n}"] = 1
            else:
                bsm.bsm_set_variant(prec, m, n, 0)
                variants[f"{m}x{n}"] = 0
        params = {}
        for name, values in SEARCH.get(prec, []):
            if name == "engine":
                continue       # decided last, on the whole multiply's time
            chosen = values[0]
            bsm.bsm_set_tuning(prec, name, chosen)
            for v in values[1:]:
                bsm.bsm_set_tuning(prec, name, v)
                t = _numeric_ms(A, B, eps, prec, reps, Cm)
                if t < best * (1.0 - gain):
                    best, chosen = t, v
            bsm.bsm_set_tuning(prec, name, chosen)
            params[name] = chosen
        flush = None
        flush_trials = {}
        if tune_flush and prec in SPLIT:
            import torch
            ref = bsm.multiply(1.0, A, B, 0.0, None, eps, build_stacks=False).data_tensor()
            fbest = None
            for f in FLUSH_CANDIDATES:
                t = _numeric_ms(A, B, eps, prec, reps, Cm, flush_every=f)
                err = _rel_err(torch, Cm.data_tensor_view(), ref)
                flush_trials[str(f)] = {"numeric_ms": t, "rel_fro_err_vs_fp64_path": err}
                if err <= err_target and (fbest is None or t < fbest[1]):
                    fbest = (f, t)
            if fbest is not None:
                flush = fbest[0]
                best = min(best, fbest[1])
        engine_trials = {}
        if any(name == "engine" for name, _ in SEARCH.get(prec, [])):
            # the engines differ in their preparation too: compare whole multiplies
            bsm.bsm_set_tuning(prec, "engine", 0)
            t0 = _numeric_ms(A, B, eps, prec, reps, Cm, flush_every=flush or 0, phase="total")
            bsm.bsm_set_tuning(prec, "engine", 1)
            t1 = _numeric_ms(A, B, eps, prec, reps, Cm, flush_every=0, phase="total")
            panel_ran = Cm.engine() == "panel_tcgen05"
            engine_trials = {"mma_sync_total_ms": t0, "panel_total_ms": t1 if panel_ran else None}
            if panel_ran and t1 < t0 * (1.0 - gain):
                params["engine"] = 1
                flush = None       # the panel engine keeps its own compensated sum
                # k-steps per accumulator buffer: the fastest within the error target
                import torch
                ref = bsm.multiply(1.0, A, B, 0.0, None, eps, build_stacks=False).data_tensor()
                steps_best, steps_trials = (PANEL_STEPS[0], t1), {}
                for v in PANEL_STEPS:
                    bsm.bsm_set_tuning(prec, "panel_steps", v)
                    t = _numeric_ms(A, B, eps, prec, reps, Cm, phase="total")
                    err = _rel_err(torch, Cm.data_tensor_view(), ref)
                    steps_trials[str(v)] = {"total_ms": t, "rel_fro_err_vs_fp64_path": err}
                    if err <= err_target and t < steps_best[1] * (1.0 - gain):
                        steps_best = (v, t)
                bsm.bsm_set_tuning(prec, "panel_steps", steps_best[0])
                params["panel_steps"] = steps_best[0]
                engine_trials["panel_steps_trials"] = steps_trials
            else:
                bsm.bsm_set_tuning(prec, "engine", 0)
                params["engine"] = 0
        tuned_ms = _numeric_ms(A, B, eps, prec, reps, Cm, flush_every=flush or 0)
    finally:
        bsm.bsm_set_profiling(False)
    return {"prec": prec, "variants": variants, "params": params, "flush_every": flush,
            "flush_trials": flush_trials, "engine_trials": engine_trials,
            "numeric_ms": {"default": start, "tuned": tuned_ms},
            "workload": {"nbr": int(len(A.row_bs)), "block_sizes": sorted(set(int(x) for x in np.asarray(A.row_bs))),
                         "eps": eps}}


def apply(table: dict):
    """Put a table (from tune or load) into effect in the library."""
    prec = table["prec"]
    for key, v in table.get("variants", {}).items():
        m, n = (int(x) for x in key.split("x"))
        bsm.bsm_set_variant(prec, m, n, int(v))
    for name, v in table.get("params", {}).items():
        bsm.bsm_set_tuning(prec, name, int(v))


def save(tables, path: str):
    with open(path, "w") as f:
        json.dump(tables, f, indent=1, sort_keys=True)


def load(path: str):
    """Load a table or a list of tables and put them into effect."""
    with open(path) as f:
        tables = json.load(f)
    for t in (tables if isinstance(tables, list) else [tables]):
        apply(t)
    return tables


def main():
    import torch
    from . import inputs as I
    p = argparse.ArgumentParser(description="tune the numeric kernels on a bench workload and write the table")
    p.add_argument("--workload", default="mixed3000", choices=["mixed3000", "banded23_6912"])
    p.add_argument("--nb", type=int, default=0, help="block rows/cols (default: the workload's)")
    p.add_argument("--precs", default="fp64,ozaki,tf32x3,bf16x6,bf16x3,fp64_dmma")
    p.add_argument("--reps", type=int, default=3)
    p.add_argument("--out", required=True)
    a = p.parse_args()
    torch.cuda.set_device(0)
    w = (I.mixed_banded(nb=a.nb or 3000) if a.workload == "mixed3000" else I.large_banded_23(nb=a.nb or 6912))
    A, B = bsm.Matrix.from_host(w["A"]), bsm.Matrix.from_host(w["B"])
    tables = []
    for prec in a.precs.split(","):
        t = tune(A, B, w["eps"], prec=prec, reps=a.reps)
        t["workload"]["name"] = a.workload
        tables.append(t)
        print(json.dumps({k: t[k] for k in ("prec", "params", "flush_every", "numeric_ms")}), flush=True)
    save(tables, a.out)


if __name__ == "__main__":
    main()
