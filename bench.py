#!/usr/bin/env python
"""Benchmark of the local block-sparse multiply on one GB300 (or N replicas).

A step is one full ``bsm_multiply`` -- block norms, symbolic count, C pattern
and product list, stacks by shape, numeric products -- of C = A.B with
inputs already resident in HBM.  The default workload is the H2O-DFT-LS
geometry: 6912 x 6912 block rows/columns of uniform 23 x 23 blocks (158,976
rows), banded-local pattern of half-width 346, half filled, then randomly
permuted (about 5% occupancy), values N(0,1)*exp(-|i-j|/50), filter
threshold 1e-8 on block-norm products.

The metric is useful TFLOP/s (sum of 2*m*n*k over the kept block products,
whatever the precision path) of the FP64 path.  The same line carries:

* ``roofline``: the FP64 numeric kernel's rate against the FP64 FMA peak
  (derived from unit counts and clocks, and the rate the library's own probe
  measures in this run);
* ``split_precision``: the FP64 tensor-core (DMMA) path, the Ozaki slices,
  TF32x3 / BF16x6 / BF16x3 with a compensated FP32 sum (TF32x3 on the engine
  the tuned table picks, and on the per-C-block mma.sync kernel), TF32x3 with
  an FP64 running sum every F block products (F = 1, 2, 4, 8), the tcgen05
  row-panel engine -- each with its step time, speedup over the FP64 path, error
  against the oracle on sampled C block rows and against the FP64 path over
  all of C, and its own roofline;
* ``e2e``: the same multiply through the C ABI from pinned host buffers;
* ``cpu_baseline``: the CPU oracle on sampled rows, single-threaded and on
  every host core;
* ``secondary``: the mixed 5/13/23-block workload (3000 x 3000 block rows)
  with both filter readings.

``--impl reference`` times the CPU oracle instead (sampled rows per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1708_03604_gb300 import inputs as I  # noqa: E402

METRIC = "block-SpGEMM useful TFLOP/s"
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
# FP64 FMA: the nominal 1.25 TFLOP/s of GB300 at 2070 MHz on 152 SMs is 2 FMA
# per clock per SM
FP64_FMA_PER_CLK_PER_SM = 2
FP64_PEAK_TFLOPS = SM_COUNT * FP64_FMA_PER_CLK_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12   # 1.2586
TF32_PER_BF16 = 1.1 / 2.25       # nominal dense TF32 / BF16 tensor rates of GB300

WORKLOADS = {
    "banded23_6912": dict(
        desc=("uniform 23x23 blocks, 6912x6912 block rows/cols (158,976 rows; H2O-DFT-LS geometry), banded "
              "half-width 346 half-filled then permuted (~5% occupancy), N(0,1)*exp(-d/50), filter_eps=1e-8"),
        block_sizes=[23], occupancy=0.05, eps=1e-8),
    "mixed3000": dict(
        desc=("mixed 5/13/23 blocks (p=0.6/0.2/0.2), 3000x3000 block rows/cols, banded half-width 300 "
              "half-filled then permuted (~10% occupancy), N(0,1)*exp(-d/50), filter_eps=1e-6"),
        block_sizes=[5, 13, 23], occupancy=0.10, eps=1e-6),
}
OTHER = ["uniform23_200", "diff13_800", "purify_2000", "smm_sweep"]


def make_inputs(name, args):
    if name == "banded23_6912":
        return I.large_banded_23(nb=args.nb_banded)
    return I.mixed_banded(nb=args.nb_mixed)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def hbm_peak_gbs():
    """Measured copy bandwidth of this GPU model (MEASURED_PEAKS.json), else the fallback 6800."""
    v = measured_peaks().get("hbm_gbs")
    return (float(v), "measured") if v else (6800.0, "fallback")


def tensor_peaks():
    """Dense BF16 and TF32 tensor-core peaks (TFLOP/s): the measured cuBLAS
    BF16 burst rate of MEASURED_PEAKS.json (fallback 1900) and TF32 at the
    nominal TF32/BF16 ratio."""
    mp = measured_peaks()
    bf16 = float(mp.get("bf16_tflops") or 1900.0)
    basis = "measured" if mp.get("bf16_tflops") else "fallback"
    return {"bf16": bf16, "tf32": bf16 * TF32_PER_BF16, "basis": basis}


TUNING_DIR = os.path.join(ROOT, "paper_1708_03604_gb300", "tuning")


def load_tuning(spec, name):
    """Put the autotuner's tables for this workload into effect; returns a
    summary for the JSON line (None when no table is loaded)."""
    if spec == "none":
        return None
    path = os.path.join(TUNING_DIR, f"{name}.json") if spec == "auto" else spec
    if not os.path.exists(path):
        return None
    from paper_1708_03604_gb300 import autotune
    tables = autotune.load(path)
    return {"table": os.path.relpath(path, ROOT),
            "tables": [{k: t.get(k) for k in ("prec", "params", "variants", "flush_every", "numeric_ms")}
                       for t in (tables if isinstance(tables, list) else [tables])]}


PROFILE_TRAFFIC = {"banded23_6912": os.path.join(ROOT, "profiles", "numeric_fp64_banded6912.md")}


def traffic_from_profile(name):
    """DRAM bytes per launch of the FP64 numeric kernel from the committed ncu
    summary of this workload (None when absent or marked stale)."""
    path = PROFILE_TRAFFIC.get(name)
    if not path:
        return None
    try:
        for line in open(path):
            if line.startswith("traffic_bytes_per_launch:"):
                v = line.split(":", 1)[1].strip()
                return None if v in ("", "null", "stale") else float(v)
    except OSError:
        pass
    return None


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--workload", default="banded23_6912", choices=list(WORKLOADS) + OTHER,
                   help="banded23_6912 is the headline line; the others measure the remaining configurations")
    p.add_argument("--no-split", action="store_true", help="skip the other-precision legs")
    p.add_argument("--legs", default="", help="comma list of legs to run (default: all)")
    p.add_argument("--leg-steps", type=int, default=3, help="timed steps per leg")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-secondary", action="store_true", help="skip the mixed-workload secondary leg")
    p.add_argument("--cpu-seconds", type=float, default=10.0, help="target length of each oracle sample")
    p.add_argument("--oracle-rows", type=int, default=64, help="sampled C block rows for the parity checks")
    p.add_argument("--nb-banded", type=int, default=6912,
                   help="block rows/cols of banded23_6912 (smaller cases for profiling; quoted at 6912)")
    p.add_argument("--nb", "--nb-mixed", dest="nb_mixed", type=int, default=3000,
                   help="block rows/cols of mixed3000 (smaller cases for profiling; quoted at 3000)")
    p.add_argument("--tune", default="auto",
                   help="autotuner tables (JSON) to load before timing: 'auto' = the committed tables of the "
                        "workload under paper_1708_03604_gb300/tuning/ when present, 'none', or a path")
    return p.parse_args()


def config(name, args, extra=None):
    wl = WORKLOADS[name]
    nb = args.nb_banded if name == "banded23_6912" else args.nb_mixed
    c = {"workload": f"{name}: {wl['desc']}", "nb": nb, "block_sizes": wl["block_sizes"],
         "occupancy": wl["occupancy"], "filter_eps": wl["eps"], "alpha": 1.0, "beta": 0.0,
         "l2": "inputs larger than L2 (A+B FP64 data >> 129 MB L2); no flush between steps"}
    if extra:
        c.update(extra)
    return c


# --------------------------------------------------------------------------
# the CPU oracle on sampled C block rows (single thread, or one thread per
# host core; ctypes releases the GIL during the C oracle's calls)
# --------------------------------------------------------------------------
def oracle_rows(w, rows, threads=1):
    """Oracle results for the given C block rows; returns (list of results,
    seconds, useful FLOP)."""
    from oracle import oracle as O
    O.build()
    rows = np.sort(np.asarray(rows))
    chunks = [c for c in np.array_split(rows, max(1, threads)) if len(c)]
    t0 = time.perf_counter()
    if len(chunks) == 1:
        res = [O.multiply(1.0, w["A"], w["B"], eps=w["eps"], rows=chunks[0])]
    else:
        with ThreadPoolExecutor(len(chunks)) as ex:
            res = list(ex.map(lambda rr: O.multiply(1.0, w["A"], w["B"], eps=w["eps"], rows=rr), chunks))
    dt = time.perf_counter() - t0
    return res, dt, sum(r.useful_flop for r in res)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def calibrate_rows(w, target_s, threads, seed=11):
    """Rows per thread so that one oracle call takes about target_s (each call
    also pays a fixed cost: the block norms of all of A and B)."""
    rng = np.random.default_rng(seed)
    order = rng.permutation(w["A"].nbr)
    dts = []
    for m in (1, 3):
        _, dt, _ = oracle_rows(w, order[:m], 1)
        dts.append(dt)
    per_row = max((dts[1] - dts[0]) / 2, 1e-4)
    fixed = max(dts[0] - per_row, 0.0)
    return int(max(1, min(w["A"].nbr // max(threads, 1), (target_s - fixed) / per_row))), per_row, fixed


def cpu_baseline(w, target_s):
    """The oracle as it stands, timed on this host: single-threaded and with
    one thread per core, each on a seeded sample of C block rows."""
    cores = host_cores()
    per, per_row, fixed = calibrate_rows(w, target_s, 1)
    rng = np.random.default_rng(12)
    rows1 = rng.permutation(w["A"].nbr)[:per]
    _, dt1, fl1 = oracle_rows(w, rows1, 1)
    nrows = min(w["A"].nbr, per * cores)
    rowsn = np.random.default_rng(13).permutation(w["A"].nbr)[:nrows]
    _, dtn, fln = oracle_rows(w, rowsn, cores)
    single = {"value": fl1 / dt1 / 1e12, "unit": "TFLOP/s", "cores": 1,
              "sample": f"{len(rows1)} of {w['A'].nbr} C block rows (seeded), {fl1:.3e} useful FLOP in {dt1:.1f} s"}
    return {"value": fln / dtn / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "sample": (f"{nrows} of {w['A'].nbr} C block rows (seeded), one thread per host core "
                       f"({cores}), each thread one oracle call on its share of the rows (every call also "
                       f"computes all block norms of A and B); {fln:.3e} useful FLOP in {dtn:.1f} s; "
                       "plain C oracle (-O2), single-threaded code"),
            "single_thread": single}


# --------------------------------------------------------------------------
# parity of GPU results on sampled rows against the oracle's rows
# --------------------------------------------------------------------------
class RowSample:
    """Oracle rows (pattern and values) and where they sit in the GPU's C."""

    def __init__(self, w, rows, res):
        self.rows = np.sort(np.asarray(rows))
        self.ref = {}
        self.bs_r, self.bs_c = np.asarray(w["A"].row_bs), np.asarray(w["B"].col_bs)
        for r in res:
            C = r.C
            for i in range(len(C.row_ptr) - 1):
                o0, o1 = int(C.row_ptr[i]), int(C.row_ptr[i + 1])
                if o1 > o0:
                    e0 = int(C.blk_off[o0])
                    e1 = int(C.blk_off[o1 - 1]) + int(self.bs_r[i]) * int(self.bs_c[C.col_idx[o1 - 1]])
                    self.ref[i] = (C.col_idx[o0:o1].copy(), C.data[e0:e1].copy())
        for i in self.rows:
            self.ref.setdefault(int(i), (np.zeros(0, np.int32), np.zeros(0)))

    def compare(self, Cm, pattern=None):
        """(pattern equal on the sampled rows, rel. Frobenius error over all of
        C in those rows)."""
        rp, ci, bo = pattern if pattern is not None else Cm.pattern()
        dev = Cm.data_tensor_view()
        same, num, den = True, 0.0, 0.0
        for i in self.rows:
            cols, vals = self.ref[int(i)]
            g0, g1 = int(rp[i]), int(rp[i + 1])
            if not np.array_equal(ci[g0:g1], cols):
                same = False
                continue
            if g1 > g0:
                e0 = int(bo[g0])
                e1 = int(bo[g1 - 1]) + int(self.bs_r[i]) * int(self.bs_c[ci[g1 - 1]])
                got = dev[e0:e1].cpu().numpy()
                num += float(np.sum((got - vals) ** 2))
                den += float(np.sum(vals ** 2))
        return same, ((num / den) ** 0.5 if den else 0.0)


def rel_err_full(torch, x, ref, chunk=1 << 28):
    """||x - ref|| / ||ref|| over two device vectors, in chunks."""
    num = den = 0.0
    for s in range(0, ref.numel(), chunk):
        a, b = x[s:s + chunk], ref[s:s + chunk]
        num += float(torch.sum((a - b) ** 2))
        den += float(torch.sum(b * b))
    return (num / den) ** 0.5 if den else 0.0


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"bsm_bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
            if vis.strip().isdigit():
                cmd += ["-i", vis.strip()]
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        first_idx = None
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            if first_idx is None:
                first_idx = parts[0]
            if parts[0] != first_idx:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power)}


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """Maximum of a per-rank scalar (the step time) over all ranks; the
    whole-job rate divides the units every rank processed by it."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, max_ms: float) -> float:
    """Whole-job throughput of `world` replicas (weak scaling), in units/ms."""
    return world * units_per_rank / max_ms


# --------------------------------------------------------------------------
# issued tensor work per block product, per engine (for the legs' rooflines)
# --------------------------------------------------------------------------
def _cdiv(a, b):
    return -(-a // b)


def issued_flop(prec, shapes, counts):
    """FLOP the tensor cores (or the FP64 units) issue for the kept products
    of each shape (m, n, k): tile padding and piece products included."""
    tot = 0.0
    for (m, n, k), c in zip(shapes, counts):
        m, n, k = int(m), int(n), int(k)
        if prec == "fp64":
            f = 2.0 * m * n * k
        elif prec == "fp64_dmma":
            f = (_cdiv(m, 8) * _cdiv(n, 8) * _cdiv(k, 4) * 512.0) if (m >= 8 and n >= 8) else 2.0 * m * n * k
        elif prec == "tf32x3":
            f = 3 * _cdiv(m, 16) * _cdiv(n, 8) * _cdiv(k, 8) * 2048.0
        elif prec == "bf16x3":
            f = 3 * _cdiv(m, 16) * _cdiv(n, 8) * _cdiv(k, 16) * 4096.0
        elif prec == "bf16x6":
            f = 6 * _cdiv(m, 16) * _cdiv(n, 8) * _cdiv(k, 16) * 4096.0
        elif prec == "ozaki":
            f = 21 * _cdiv(m, 16) * _cdiv(n, 8) * _cdiv(k, 16) * 4096.0
        else:
            return None
        tot += f * int(c)
    return tot


PIECES = {"tf32x3": 3, "bf16x3": 3, "bf16x6": 6, "ozaki": 21, "tf32x3_panel": 3}


def leg_roofline(prec, useful, issued, num_ms, peaks, tpk):
    """Roofline of one leg's numeric kernel: useful and issued rates against
    the peak of the unit the kernel issues on (measured by the probe in this
    run) and, for tensor-core legs, against the dense tcgen05-class peak."""
    s = num_ms * 1e-3
    ach = useful / s / 1e12
    out = {"achieved_useful": ach, "unit": "TFLOP/s", "launch_ms": num_ms}
    if prec in ("fp64",):
        out.update(bound="alu", peak=FP64_PEAK_TFLOPS, frac=ach / FP64_PEAK_TFLOPS,
                   peak_basis="derived FP64 FMA peak", peak_measured_dfma=peaks["fp64_fma"],
                   frac_of_measured=ach / peaks["fp64_fma"])
        return out
    if prec == "fp64_dmma":
        iss = issued / s / 1e12
        out.update(bound="alu", achieved_issued=iss, peak=peaks["fp64_mma"], peak_basis="measured DMMA probe",
                   frac=ach / peaks["fp64_mma"], frac_issued=iss / peaks["fp64_mma"])
        return out
    dt = "tf32" if prec.startswith("tf32") else "bf16"
    npieces = PIECES[prec]
    mma = peaks[f"{dt}_mma"]
    out.update(bound="tensor", pieces=npieces, peak_mma_sync=mma, peak_tcgen05=tpk[dt],
               peak_basis=f"measured mma.sync {dt} probe; tcgen05 peak from MEASURED_PEAKS bf16 "
                          f"({tpk['basis']})" + (" x nominal TF32/BF16" if dt == "tf32" else ""),
               frac=ach / (mma / npieces), frac_useful_vs_tcgen05=ach / (tpk[dt] / npieces))
    if issued is not None:
        iss = issued / s / 1e12
        out.update(achieved_issued=iss, frac_issued=iss / mma, frac_issued_vs_tcgen05=iss / tpk[dt])
    return out


# --------------------------------------------------------------------------
# reference arm: the CPU oracle on every host core
# --------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return
    name = args.workload if args.workload in WORKLOADS else "banded23_6912"
    w = make_inputs(name, args)
    cores = host_cores()
    per, _, _ = calibrate_rows(w, 5.0, cores)
    rng = np.random.default_rng(5)
    times, flops = [], []
    for s in range(args.warmup + args.steps):
        rows = rng.permutation(w["A"].nbr)[:min(w["A"].nbr, per * cores)]
        _, dt, fl = oracle_rows(w, rows, cores)
        if s >= args.warmup:
            times.append(dt)
            flops.append(fl)
    value = sum(flops) / sum(times) / 1e12
    sample = (f"{min(w['A'].nbr, per * cores)} of {w['A'].nbr} C block rows per step (seeded), one thread per "
              f"host core ({cores}), plain C oracle (-O2)")
    line = {"metric": METRIC, "impl": "reference", "value": value, "unit": "TFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config(name, args, {"sample_rows_per_step": min(w['A'].nbr, per * cores)}),
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# the headline workloads
# --------------------------------------------------------------------------
def timed_steps(torch, stream, fn, steps, times_out=None):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        fn()
        if times_out is not None:
            times_out.append(fn.last())
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def e2e_run(torch, bsm, w, eps, flop, world, steps, barrier, max_ms):
    """The multiply through the C ABI from pinned host buffers: per step,
    handles from host patterns (validated on the host) and H2D of A's and
    B's data, the multiply, D2H of C's data and pattern into pinned memory,
    handles destroyed.  Per-stage times are taken in the timed passes (the
    stage ends are points where the ABI synchronises anyway)."""
    pin, pat = {}, {}
    for nm in ("A", "B"):
        pin[nm] = torch.from_numpy(w[nm].data).pin_memory()
        pat[nm] = [torch.from_numpy(np.ascontiguousarray(getattr(w[nm], f))).pin_memory().numpy()
                   for f in ("row_bs", "col_bs", "row_ptr", "col_idx", "blk_off")]
    h2d = sum(w[nm].data.nbytes + w[nm].row_ptr.nbytes + w[nm].col_idx.nbytes + w[nm].blk_off.nbytes +
              w[nm].row_bs.nbytes + w[nm].col_bs.nbytes for nm in ("A", "B"))
    out = {}
    times, stages = [], []
    d2h = 0
    for it in range(steps + 1):
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hA = bsm.bsm_create(*pat["A"], bsm.BSM_FP64, pin["A"].data_ptr(), pin["A"].numel(), bsm.BSM_DATA_COPY)
        hB = bsm.bsm_create(*pat["B"], bsm.BSM_FP64, pin["B"].data_ptr(), pin["B"].numel(), bsm.BSM_DATA_COPY)
        hC = bsm.bsm_create_empty(w["A"].row_bs, w["B"].col_bs, bsm.BSM_FP64)
        t1 = time.perf_counter()
        bsm.bsm_multiply(1.0, hA, hB, 0.0, hC, eps, bsm.make_opts("fp64"))
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        inf = bsm.bsm_get_info(hC)
        if "c" not in out or out["c"].numel() < inf.data_len:
            out["c"] = torch.empty(inf.data_len, dtype=torch.float64).pin_memory()
            out["rp"] = torch.empty(inf.nbr + 1, dtype=torch.int64).pin_memory()
            out["ci"] = torch.empty(max(inf.nnzb, 1), dtype=torch.int32).pin_memory()
            out["bo"] = torch.empty(max(inf.nnzb, 1), dtype=torch.int64).pin_memory()
        bsm.lib().bsm_copy_data(hC, out["c"].data_ptr())
        bsm.lib().bsm_copy_pattern(hC, out["rp"].data_ptr(), out["ci"].data_ptr(), out["bo"].data_ptr())
        t3 = time.perf_counter()
        for h in (hA, hB, hC):
            bsm.bsm_destroy(h)
        torch.cuda.synchronize()
        t4 = time.perf_counter()
        d2h = inf.data_len * 8 + (inf.nbr + 1) * 8 + inf.nnzb * 12
        if it > 0:
            times.append(t4 - t0)
            stages.append((t1 - t0, t2 - t1, t3 - t2, t4 - t3))
    et = max_ms(statistics.mean(times))
    st = np.mean(np.array(stages), axis=0) * 1e3
    del out, pin
    return {"value": world * flop / et / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": et * 1e3, "steps": steps,
            "includes": "host pattern validation, H2D of A and B from pinned memory, multiply, "
                        "D2H of C's data and pattern into pinned memory, handles destroyed",
            "stage_ms_timed_mean": {"create_and_h2d": round(st[0], 2), "multiply": round(st[1], 2),
                                    "d2h": round(st[2], 2), "destroy": round(st[3], 2)}}


def phase_rates(phases, w, cnt, c_blocks):
    """Algorithmic bytes and GB/s of the index phases (block norms, symbolic
    count, fill, stacks) of one FP64 step, against the measured HBM bandwidth."""
    A, B = w["A"], w["B"]
    peak, basis = hbm_peak_gbs()
    cand = cnt.products + cnt.filtered
    per = {
        "norms": (8.0 * (len(A.data) + len(B.data)) + 8.0 * (A.nnzb + B.nnzb),
                  "8 B per element read + 8 B per block written"),
        "symbolic": (12.0 * cand, "12 B per candidate product (B index + norm)"),
        "fill": (12.0 * cnt.products + 24.0 * c_blocks, "12 B per product + 24 B per C block written"),
        "stacks": (36.0 * cnt.products, "12 B per product read + 24 B per triple written"),
    }
    out = {}
    for k, (b, how) in per.items():
        ms = phases.get(k)
        if ms:
            gbs = b / (ms * 1e-3) / 1e9
            out[k] = {"ms": ms, "algorithmic_gb": b / 1e9, "gb_per_s": gbs, "frac_of_hbm": gbs / peak,
                      "bytes": how}
    out["hbm_peak_gbs"] = peak
    out["hbm_peak_basis"] = basis
    return out


LEGS = [  # (key, precision, flush_every, timed steps scale)
    ("fp64_dmma", "fp64_dmma", 0, "one"),
    ("ozaki", "ozaki", 0, "full"),
    ("tf32x3", "tf32x3", 0, "full"),
    ("tf32x3_mma_sync", "tf32x3", 0, "full"),
    ("tf32x3_fp64sum_f1", "tf32x3", 1, "full"),
    ("tf32x3_fp64sum_f2", "tf32x3", 2, "full"),
    ("tf32x3_fp64sum_f4", "tf32x3", 4, "full"),
    ("tf32x3_fp64sum_f8", "tf32x3", 8, "full"),
    ("bf16x6", "bf16x6", 0, "full"),
    ("bf16x6_fp64sum_f4", "bf16x6", 4, "full"),
    ("bf16x3", "bf16x3", 0, "full"),
    ("tf32x3_panel", "tf32x3_panel", 0, "full"),
]


def run_headline(args, name, world, rank, local_rank):
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    def max_ms(x: float) -> float:
        return max_over_ranks(x, world, "cuda")

    from paper_1708_03604_gb300 import bsm

    w = make_inputs(name, args)
    eps = w["eps"]
    A = bsm.Matrix.from_host(w["A"])
    B = bsm.Matrix.from_host(w["B"])
    stream = torch.cuda.current_stream()
    Cm = [bsm.Matrix.empty(w["A"].row_bs, w["B"].col_bs)]

    peaks = {u: bsm.measure_peak(u, 5) / 1e12 for u in ("fp64_fma", "fp64_mma", "tf32_mma", "bf16_mma")}
    tpk = tensor_peaks()
    tuned = load_tuning(args.tune, name)

    class Step:
        def __init__(self, prec="fp64", flush_every=0):
            self.prec, self.fl = prec, flush_every

        def __call__(self):
            bsm.multiply(1.0, A, B, 0.0, Cm[0], eps, prec=self.prec, flush_every=self.fl, build_stacks=True)

        def last(self):
            return Cm[0].timings()

    step = Step()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---------------- timed region: the FP64 path
    bsm.bsm_set_profiling(True)
    clocks = ClockSampler()
    clocks.start()
    time.sleep(0.3)
    launches0 = bsm.bsm_get_launch_count()
    per_step = []
    barrier()
    ms = max_ms(timed_steps(torch, stream, step, args.steps, per_step))
    barrier()
    launches = bsm.bsm_get_launch_count() - launches0
    clk = clocks.stop()
    bsm.bsm_set_profiling(False)
    cnt = Cm[0].counts()
    flop = cnt.useful_flop
    value = job_rate(flop, world, ms) * 1e-9
    num_ms = statistics.mean(t["numeric"] for t in per_step)
    phases = {k: statistics.mean(t[k] for t in per_step) for k in per_step[0]}
    shapes, scounts = Cm[0].stack_shapes()
    roofline = leg_roofline("fp64", flop, None, num_ms, peaks, tpk)
    traffic = traffic_from_profile(name) if world == 1 else None
    roofline.update(kernel=("k_numeric_cc<double> (FP64 FMA, one warp per C block; stream of the multiply, "
                            "CUDA events of the library around the launch)"),
                    traffic=traffic,
                    traffic_note=("dram__bytes_read.sum + dram__bytes_write.sum of one launch at 2000 block rows, "
                                  "scaled by products to the full launch (profiles/numeric_fp64_banded6912.md)")
                    if traffic else "no committed capture for this workload")
    c_blocks = Cm[0].nnzb
    pattern = Cm[0].pattern()
    ref_c = Cm[0].data_tensor()    # the FP64 result, kept for the legs' full-C errors

    # ---------------- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        torch.cuda.empty_cache()
        e2e = e2e_run(torch, bsm, w, eps, flop, world, max(2, min(args.steps, 3)), barrier, max_ms)

    # ---------------- oracle rows (parity of every leg on the same rows)
    sample = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rows = np.random.default_rng(11).permutation(w["A"].nbr)[:min(args.oracle_rows, w["A"].nbr)]
        res, _, _ = oracle_rows(w, rows, host_cores())
        sample = RowSample(w, rows, res)
        same, err = sample.compare(Cm[0], pattern)
        parity = {"rows": len(rows), "pattern_equal": same, "rel_fro_fp64_vs_oracle": err}
    else:
        parity = None

    # ---------------- the other precisions
    split = {}
    if not args.no_split:
        legs = LEGS if not args.legs else [lg for lg in LEGS if lg[0] in args.legs.split(",")]
        for key, prec, fl, scale in legs:
            Cm[0] = bsm.Matrix.empty(w["A"].row_bs, w["B"].col_bs)   # free the previous leg's C first
            torch.cuda.empty_cache()
            ls = Step(prec, fl)
            engine_saved = None
            if key.endswith("_mma_sync"):   # the per-C-block mma.sync kernel whatever the tuned engine
                engine_saved = bsm.bsm_get_tuning(prec, "engine")
                bsm.bsm_set_tuning(prec, "engine", 0)
            ls()
            torch.cuda.synchronize()
            bsm.bsm_set_profiling(True)
            ks = 1 if (scale == "one" and args.leg_steps > 1) else args.leg_steps
            per = []
            sms = max_ms(timed_steps(torch, stream, ls, ks, per))
            bsm.bsm_set_profiling(False)
            lnum = statistics.mean(t["numeric"] for t in per)
            got = Cm[0].data_tensor_view()
            leg = {"precision": prec, "flush_every": fl, "engine": Cm[0].engine(),
                   "value": world * flop / (sms * 1e-3) / 1e12, "ms_per_step": sms, "steps": ks,
                   "numeric_ms": lnum, "speedup_vs_fp64": ms / sms,
                   "rel_fro_err_vs_fp64_path_all_of_C": rel_err_full(torch, got, ref_c),
                   "c_elements_compared": int(ref_c.numel())}
            if sample is not None:
                same, err = sample.compare(Cm[0], pattern)
                leg.update(pattern_equal_on_oracle_rows=same, rel_fro_err_vs_oracle_rows=err)
            rp_prec = "tf32x3" if prec == "tf32x3_panel" else prec
            leg["roofline"] = leg_roofline(prec, flop, issued_flop(rp_prec, shapes, scounts)
                                           if prec != "tf32x3_panel" else None, lnum, peaks, tpk)
            split[key] = leg
            del got
            if engine_saved is not None:
                bsm.bsm_set_tuning(prec, "engine", engine_saved)
        Cm[0] = bsm.Matrix.empty(w["A"].row_bs, w["B"].col_bs)
        torch.cuda.empty_cache()
    compliant = {k: v for k, v in split.items()
                 if "fp64sum" in k and v.get("rel_fro_err_vs_oracle_rows", v["rel_fro_err_vs_fp64_path_all_of_C"]) <= 1e-6}
    best = max(compliant.items(), key=lambda kv: kv[1]["speedup_vs_fp64"]) if compliant else None

    # ---------------- CPU oracle timed on this host
    cpu = cpu_baseline(w, args.cpu_seconds) if (rank == 0 and world == 1 and not args.no_cpu) else None

    # ---------------- secondary: the mixed-size workload, both filter readings
    secondary = None
    if name == "banded23_6912" and not args.no_secondary and world == 1:
        del ref_c
        A = B = None
        Cm[0] = None
        torch.cuda.empty_cache()
        secondary = run_secondary(args, torch, bsm, stream, rank)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": config(name, args, {"products": cnt.products, "filtered": cnt.filtered,
                                              "useful_flop": flop, "c_blocks": c_blocks,
                                              "stacks_built": True, "shapes": shapes.tolist(),
                                              "parallelism": "replicas" if world > 1 else "single GPU"}),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clk, "measured_unit_peaks_tflops": peaks, "tensor_peaks_tflops": tpk,
                "split_precision": split,
                "split_fp64_sum_best": ({"leg": best[0], "speedup_vs_fp64": best[1]["speedup_vs_fp64"],
                                      "rel_fro_err_vs_oracle_rows": best[1].get("rel_fro_err_vs_oracle_rows"),
                                      "form": "split pieces on tensor cores, FP32 accumulation over at most "
                                              "F block products, FP64 running sum"} if best else None),
                "parity_sample": parity, "phase_ms_mean_fp64_step": phases,
                "index_phases": phase_rates(phases, w, cnt, c_blocks), "autotune": tuned,
                "secondary": secondary}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_secondary(args, torch, bsm, stream, rank):
    """The mixed 5/13/23 workload: FP64 step time, the post-filter reading
    (C blocks with norm <= eps dropped after the multiply) beside the
    per-product reading, both patterns against the oracle's."""
    from oracle import oracle as O
    w = make_inputs("mixed3000", args)
    eps = w["eps"]
    tuned = load_tuning(args.tune, "mixed3000")
    A, B = bsm.Matrix.from_host(w["A"]), bsm.Matrix.from_host(w["B"])
    Cm = bsm.Matrix.empty(w["A"].row_bs, w["B"].col_bs)

    def step():
        bsm.multiply(1.0, A, B, 0.0, Cm, eps, build_stacks=True)

    step()
    ms = timed_steps(torch, stream, step, 3)
    cnt = Cm.counts()
    per_product_blocks = Cm.nnzb
    pat1 = Cm.pattern()
    Cp = bsm.multiply(1.0, A, B, 0.0, None, eps, post_filter=True)
    post_blocks = Cp.nnzb
    out = {"workload": WORKLOADS["mixed3000"]["desc"], "nb": args.nb_mixed, "ms_per_step": ms,
           "value": cnt.useful_flop / ms * 1e-9, "unit": "TFLOP/s", "products": cnt.products,
           "filtered_products": cnt.filtered, "c_blocks_per_product_filter": per_product_blocks,
           "c_blocks_post_filter": post_blocks, "autotune": tuned}
    if rank == 0 and not args.no_cpu:
        O.build()
        res, dt, _ = oracle_rows(w, np.arange(w["A"].nbr), host_cores())
        # whole C of the oracle, rows concatenated (each result holds its rows only)
        rp = np.zeros(len(w["A"].row_bs) + 1, np.int64)
        for r in res:
            rp[1:] += np.diff(r.C.row_ptr)
        rp = np.cumsum(np.concatenate([[0], rp[1:]]))
        # the results hold consecutive row ranges in ascending order
        ci = np.concatenate([r.C.col_idx for r in res])
        data = np.concatenate([r.C.data for r in res])
        bs_r, bs_c = np.asarray(w["A"].row_bs), np.asarray(w["B"].col_bs)
        brow = np.repeat(np.arange(len(bs_r)), np.diff(rp))
        sizes = bs_r[brow].astype(np.int64) * bs_c[ci].astype(np.int64)
        bo = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
        Cref = I.BCSR(w["A"].row_bs, w["B"].col_bs, rp, ci.astype(np.int32), bo, data)
        nrm = O.block_norms(Cref)
        post = O.post_filter(Cref, eps)
        g_rp, g_ci, _ = pat1
        p_rp, p_ci, _ = Cp.pattern()
        out.update(oracle_seconds_all_rows=dt,
                   pattern_equal_per_product_filter=bool(np.array_equal(g_rp, rp) and np.array_equal(g_ci, ci)),
                   pattern_equal_post_filter=bool(np.array_equal(p_rp, post.row_ptr) and
                                                  np.array_equal(p_ci, post.col_idx)),
                   oracle_c_blocks_post_filter=int(post.nnzb),
                   post_filter_margin_min_rel=float(np.min(np.abs(nrm - eps)) / eps) if len(nrm) else None)
    return out


# --------------------------------------------------------------------------
# the other configurations (one GPU)
# --------------------------------------------------------------------------
def _timed(torch, fn, steps, warmup):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_other(args):
    import torch
    from paper_1708_03604_gb300 import bsm, chain
    torch.cuda.set_device(0)
    name = args.workload
    out = {"metric": METRIC, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "higher_is_better": True, "dtype": "f64", "data": "synthetic", "vs_baseline": None}
    if name == "uniform23_200":
        w = I.uniform_23()
        A, B = bsm.Matrix.from_host(w["A"]), bsm.Matrix.from_host(w["B"])
        Cm = bsm.Matrix.empty(w["A"].row_bs, w["B"].col_bs)
        legs, ref = {}, None
        for key in ("fp64", "fp64_dmma", "ozaki", "tf32x3", "tf32x3_panel", "bf16x6", "bf16x3"):
            ms = _timed(torch, lambda: bsm.multiply(1.0, A, B, 0.0, Cm, w["eps"], prec=key), args.steps, args.warmup)
            flop = Cm.counts().useful_flop
            c = Cm.data_tensor()
            if ref is None:
                ref = c
            legs[key] = {"value": flop / ms * 1e-9, "ms_per_step": ms, "engine": Cm.engine(),
                         "rel_fro_err_vs_fp64_path": rel_err_full(torch, c, ref)}
        out.update(value=legs["fp64"]["value"], ms_per_step=legs["fp64"]["ms_per_step"],
                   config={"workload": name, "nb": 200, "products": Cm.counts().products, "useful_flop": flop},
                   split_precision=legs)
    elif name == "diff13_800":
        w = I.differentiation_13()
        A, B = bsm.Matrix.from_host(w["A"]), bsm.Matrix.from_host(w["B"])
        Cm = bsm.multiply(1.0, A, B)
        dC = torch.randn(Cm.info().data_len, dtype=torch.float64, device="cuda")
        dA = torch.empty(len(w["A"].data), dtype=torch.float64, device="cuda")
        dB = torch.empty(len(w["B"].data), dtype=torch.float64, device="cuda")
        legs = {}
        for prec in ("fp64", "fp64_dmma", "ozaki", "tf32x3"):
            def step():
                bsm.multiply(1.0, A, B, 0.0, Cm, 0.0, prec=prec)
                bsm.multiply_backward(1.0, Cm, dC, A, B, dA, dB, prec=prec)
            ms = _timed(torch, step, args.steps, args.warmup)
            flop = 3 * Cm.counts().useful_flop      # forward + two adjoint products
            legs[prec] = {"value": flop / ms * 1e-9, "ms_per_step": ms}
        out.update(value=legs["fp64"]["value"], ms_per_step=legs["fp64"]["ms_per_step"],
                   config={"workload": name, "step": "multiply + both adjoints", "products": Cm.counts().products,
                           "useful_flop_per_step": flop},
                   split_precision={k: v for k, v in legs.items() if k != "fp64"})
    elif name == "smm_sweep":
        # square blocks m = n = k = s over the range of the paper's Fig. 1 (4..78):
        # uniform random patterns sized so that A + B hold about 1 GB of FP64 data
        rows = []
        for s_ in (4, 5, 6, 8, 9, 12, 13, 16, 22, 23, 26, 32, 45, 64, 78):
            nb = int(round((2.0e6 / (s_ * s_)) ** 0.5 / 0.1)) if s_ < 16 else int(round((1.0e9 / 8 / (s_ * s_) / 0.1) ** 0.5))
            nb = max(40, min(nb, 6000))
            bs = I.uniform_sizes(nb, s_)
            occ = 0.1
            Ah = I.assemble(bs, bs, *I.uniform_pattern(nb, nb, occ, I.SEED_A), seed=I.SEED_A + 100)
            Bh = I.assemble(bs, bs, *I.uniform_pattern(nb, nb, occ, I.SEED_B), seed=I.SEED_B + 100)
            A, B = bsm.Matrix.from_host(Ah), bsm.Matrix.from_host(Bh)
            Cm = bsm.Matrix.empty(bs, bs)
            row = {"s": s_, "nb": nb, "occupancy": occ}
            bsm.bsm_set_profiling(True)
            for prec in ("fp64", "fp64_dmma", "ozaki", "tf32x3") + (("tf32x3_panel",) if s_ <= 24 else ()):
                num = []
                ms = _timed(torch, lambda: (bsm.multiply(1.0, A, B, 0.0, Cm, 0.0, prec=prec, build_stacks=False),
                                            num.append(Cm.timings()["numeric"])), args.steps, args.warmup)
                flop = Cm.counts().useful_flop
                nm = statistics.median(num[args.warmup:] or num)
                row[prec] = {"step_tflops": flop / ms * 1e-9, "numeric_tflops": flop / nm * 1e-9, "numeric_ms": nm,
                             "engine": Cm.engine()}
            bsm.bsm_set_profiling(False)
            row["products"] = Cm.counts().products
            rows.append(row)
            del A, B, Cm
            torch.cuda.empty_cache()
        out.update(value=None, config={"workload": name, "occupancy": 0.1,
                                       "note": "per block size: one multiply of uniform s x s blocks"}, sweep=rows)
    else:  # purify_2000: the 10-step McWeeny chain as one CUDA graph
        w = I.purification_start(nb=2000)
        X0 = bsm.Matrix.from_host(w["X0"])
        legs = {}
        for prec in ("fp64", "ozaki", "tf32x3"):
            g = chain.McWeenyGraph(X0, w["steps"], w["eps"], prec=prec)
            flop = sum(h.counts().useful_flop for h in g.X2 + g.X3)
            ms = _timed(torch, g.replay, args.steps, args.warmup)
            assert g.status() == 0
            occ = [h.nnzb / 2000 ** 2 for h in g.X]
            legs[prec] = {"value": flop / ms * 1e-9, "ms_per_step": ms, "useful_flop": flop,
                          "block_occupancy_per_iterate": [round(o, 4) for o in occ]}
            del g
        # the first multiply of the chain at its full size (20000 block rows)
        del X0
        torch.cuda.empty_cache()
        wf = I.purification_start(nb=20000)
        Xf = bsm.Matrix.from_host(wf["X0"])
        full = {"nb": 20000, "x0_blocks": int(wf["X0"].nnzb)}
        try:
            Cf = bsm.Matrix.empty(wf["X0"].row_bs, wf["X0"].col_bs)
            t0 = time.perf_counter()
            bsm.multiply(1.0, Xf, Xf, 0.0, Cf, wf["eps"], build_stacks=False)
            torch.cuda.synchronize()
            cnt = Cf.counts()
            full.update(status="ok", seconds=time.perf_counter() - t0, products=cnt.products,
                        useful_flop=cnt.useful_flop, c_blocks=Cf.nnzb)
        except bsm.BsmError as e:
            full.update(status="refused", error=str(e))
        out.update(value=legs["fp64"]["value"], ms_per_step=legs["fp64"]["ms_per_step"],
                   config={"workload": name, "step": "replay of the graph-captured 10-step chain (20 multiplies, "
                                                    "10 filtered adds)", "eps": w["eps"]},
                   split_precision={"ozaki": legs["ozaki"], "tf32x3": legs["tf32x3"]}, chain=legs,
                   full_size_first_multiply=full)
    print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload in WORKLOADS:
        return run_headline(args, args.workload, world, rank, local_rank)
    return run_other(args)


if __name__ == "__main__":
    main()
