#!/usr/bin/env python
"""Benchmark of the local block-sparse multiply on one GB300 (or N replicas).

A step is one full ``bsm_multiply`` -- block norms, symbolic count, C pattern
and product list, stacks by shape, numeric products -- on the mixed-block
workload: 3000 x 3000 block rows/columns, block sizes drawn per row/column
from {5 (p=0.6), 13 (0.2), 23 (0.2)}, banded-local pattern (half-width 300,
half filled) then randomly permuted (about 10% occupancy), values
N(0,1)*exp(-|i-j|/50), filter threshold 1e-6 on block-norm products.

The metric is useful TFLOP/s (sum of 2*m*n*k over the kept block products,
whatever the precision path) of the FP64 path; the same line reports the
split-precision paths (TF32x3, BF16x6, BF16x3) with their speedup and
relative Frobenius error, the roofline of the numeric kernel, the
end-to-end rate through the C ABI with host buffers, and the CPU oracle.

``--impl reference`` times the CPU oracle instead (on a bounded sample of
C block rows per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1708_03604_gb300 import inputs as I  # noqa: E402

WORKLOAD = dict(nb=3000, occ=0.10, sizes=(5, 13, 23), probs=(0.6, 0.2, 0.2), eps=1e-6, decay=50.0)
WORKLOAD_NAME = ("mixed 5/13/23 blocks (p=0.6/0.2/0.2), 3000x3000 block rows/cols, banded half-width 300 "
                 "half-filled then permuted (~10% occupancy), N(0,1)*exp(-d/50), filter_eps=1e-6")
SM_COUNT = 152
FP64_FMA_PER_CLK_PER_SM = 2          # from the nominal 1.25 TFLOP/s FP64 at 2070 MHz on 152 SMs
SM_MAX_MHZ = 2070.0
FP64_PEAK_TFLOPS = SM_COUNT * FP64_FMA_PER_CLK_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12   # 1.2586
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "numeric_fp64_mixed3000.md")


def hbm_peak_gbs():
    """Measured copy bandwidth of this GPU model (MEASURED_PEAKS.json), else 6678."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = json.load(f).get("hbm_gbs")
        return float(v) if v else 6678.0
    except (OSError, ValueError, TypeError):
        return 6678.0


def phase_rates(phases, w, cnt, c_blocks, c_len):
    """Algorithmic bytes and GB/s of the index phases (block norms, symbolic
    fill, stacks) of one FP64 step, against the measured HBM bandwidth."""
    A, B = w["A"], w["B"]
    peak = hbm_peak_gbs()
    cand = cnt.products + cnt.filtered
    per = {
        # every element of A and B read once, one FP64 norm written per block
        "norms": (8.0 * (len(A.data) + len(B.data)) + 8.0 * (A.nnzb + B.nnzb),
                  "8 B per element read + 8 B per block written"),
        # per candidate product one B column index and one B norm (L2-resident re-reads)
        "symbolic": (12.0 * cand, "12 B per candidate product (B index + norm)"),
        # product list (3 x int32) and C pattern (col int32, blk_off int64, rc int32, segment int64)
        "fill": (12.0 * cnt.products + 24.0 * c_blocks, "12 B per product + 24 B per C block written"),
        # product ids read, (a_off, b_off, c_off) int64 triples written
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
    return out


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--no-split", action="store_true", help="skip the split-precision legs")
    p.add_argument("--legs", default="", help="comma list of split-precision legs to run (default: all)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="target length of the oracle sample")
    p.add_argument("--nb", type=int, default=WORKLOAD["nb"],
                   help="block rows/cols (smaller cases for profiling; the metric is quoted at 3000)")
    p.add_argument("--nb-banded", type=int, default=6912,
                   help="block rows/cols of banded23_6912 (smaller cases for profiling; quoted at 6912)")
    p.add_argument("--workload", default="mixed3000",
                   choices=["mixed3000", "uniform23_200", "banded23_6912", "diff13_800", "purify_2000", "smm_sweep"],
                   help="mixed3000 is the headline line; the others measure the remaining configurations")
    a = p.parse_args()
    if a.nb != WORKLOAD["nb"]:
        WORKLOAD["nb"] = a.nb
    return a


def make_inputs():
    return I.mixed_banded(**WORKLOAD)


def config(extra=None):
    c = {"workload": WORKLOAD_NAME, "nb": WORKLOAD["nb"], "block_sizes": list(WORKLOAD["sizes"]),
         "occupancy": WORKLOAD["occ"], "filter_eps": WORKLOAD["eps"], "alpha": 1.0, "beta": 0.0,
         "l2": "inputs larger than L2 (A+B = 1.5 GB of FP64 data vs 129 MB L2); no flush between steps"}
    if extra:
        c.update(extra)
    return c


# --------------------------------------------------------------------------
# CPU oracle on a sample of C block rows
# --------------------------------------------------------------------------
def oracle_sample(w, target_s, seed=11, rows_hint=None):
    """Run the oracle on seeded random C block rows until about target_s
    seconds; returns (rows, result, seconds)."""
    from oracle import oracle as O
    O.build()
    rng = np.random.default_rng(seed)
    order = rng.permutation(w["A"].nbr)
    n = rows_hint or 4
    if rows_hint is None:
        # calibrate on 4 and 16 rows (each call also pays a fixed cost: the block
        # norms of all of A and B), then run the sized sample once
        dts = []
        for m in (4, 16):
            t0 = time.perf_counter()
            O.multiply(1.0, w["A"], w["B"], eps=w["eps"], rows=np.sort(order[:m]))
            dts.append(time.perf_counter() - t0)
        per_row = max((dts[1] - dts[0]) / 12, 1e-6)
        fixed = max(dts[0] - 4 * per_row, 0.0)
        n = int(max(4, min(len(order), (target_s - fixed) / per_row)))
    rows = np.sort(order[:n])
    t0 = time.perf_counter()
    r = O.multiply(1.0, w["A"], w["B"], eps=w["eps"], rows=rows)
    return rows, r, time.perf_counter() - t0


def cpu_baseline(w, target_s):
    rows, r, secs = oracle_sample(w, target_s)
    return dict(value=r.useful_flop / secs / 1e12, unit="TFLOP/s", cores=1, kind="oracle",
                sample=f"{len(rows)} of {w['A'].nbr} C block rows (seeded), full block norms; "
                       f"{r.useful_flop:.3e} useful FLOP in {secs:.1f} s, single-threaded C (-O2)"), rows, r


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
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
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


def traffic_from_profile():
    """DRAM bytes per launch of the numeric kernel from the committed ncu
    summary (None when absent or marked stale)."""
    try:
        for line in open(PROFILE_TRAFFIC):
            if line.startswith("traffic_bytes_per_launch:"):
                v = line.split(":", 1)[1].strip()
                return None if v in ("", "null", "stale") else float(v)
    except OSError:
        pass
    return None


# --------------------------------------------------------------------------
# reference arm: the CPU oracle
# --------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return
    w = make_inputs()
    from oracle import oracle as O
    O.build()
    rng = np.random.default_rng(5)
    per_step_rows = None
    times, flops = [], []
    # calibrate the per-step sample to ~6 s
    rows, r, secs = oracle_sample(w, 6.0)
    per_step_rows = len(rows)
    for s in range(args.warmup + args.steps):
        rows = np.sort(rng.permutation(w["A"].nbr)[:per_step_rows])
        t0 = time.perf_counter()
        r = O.multiply(1.0, w["A"], w["B"], eps=w["eps"], rows=rows)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            flops.append(r.useful_flop)
    value = sum(flops) / sum(times) / 1e12
    line = {"metric": "block-SpGEMM useful TFLOP/s", "impl": "reference", "value": value, "unit": "TFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config({"sample_rows_per_step": per_step_rows}),
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
                             "sample": f"{per_step_rows} of {w['A'].nbr} C block rows per step (seeded), "
                                       "single-threaded C oracle"},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
    out = {"metric": "block-SpGEMM useful TFLOP/s", "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "higher_is_better": True, "dtype": "f64", "data": "synthetic", "vs_baseline": None}
    if name in ("uniform23_200", "banded23_6912"):
        w = I.uniform_23() if name == "uniform23_200" else I.large_banded_23(nb=args.nb_banded)
        A, B = bsm.Matrix.from_host(w["A"]), bsm.Matrix.from_host(w["B"])
        Cm = bsm.Matrix.empty(w["A"].row_bs, w["B"].col_bs)
        legs = {}
        ref = None
        # error over the first 2^28 elements of C (the whole C of the 6912-block case is 38 GB)
        nref = 1 << 28
        run = [("fp64", "fp64"), ("ozaki", "ozaki"), ("tf32x3", "tf32x3"), ("tf32x3_panel", "tf32x3_panel"),
               ("bf16x6", "bf16x6"), ("bf16x3", "bf16x3")]
        if args.legs:
            run = [lg for lg in run if lg[0] in args.legs.split(",")]
        for key, prec in run:
            ms = _timed(torch, lambda: bsm.multiply(1.0, A, B, 0.0, Cm, w["eps"], prec=prec, build_stacks=False),
                        args.steps, args.warmup)
            flop = Cm.counts().useful_flop
            c = Cm.data_tensor()[:nref].clone()
            torch.cuda.empty_cache()
            if ref is None and key == "fp64":
                ref = c
            err = (torch.linalg.vector_norm(c - ref) / torch.linalg.vector_norm(ref)).item() if ref is not None else None
            legs[key] = {"value": flop / ms * 1e-9, "ms_per_step": ms, "rel_fro_err_vs_fp64_path": err,
                         "err_sample_elements": int(c.numel()), "engine": Cm.engine()}
            del c
            torch.cuda.empty_cache()
        head = legs.get("fp64") or next(iter(legs.values()))
        out.update(value=head["value"], ms_per_step=head["ms_per_step"],
                   config={"workload": name, "nb": len(w["A"].row_bs), "products": Cm.counts().products,
                           "useful_flop": flop,
                           "filtered": Cm.counts().filtered, "c_blocks": Cm.nnzb}, split_precision=legs)
    elif name == "diff13_800":
        w = I.differentiation_13()
        A, B = bsm.Matrix.from_host(w["A"]), bsm.Matrix.from_host(w["B"])
        Cm = bsm.multiply(1.0, A, B)
        dC = torch.randn(Cm.info().data_len, dtype=torch.float64, device="cuda")
        dA = torch.empty(len(w["A"].data), dtype=torch.float64, device="cuda")
        dB = torch.empty(len(w["B"].data), dtype=torch.float64, device="cuda")
        legs = {}
        for prec in ("fp64", "ozaki", "tf32x3"):
            def step():
                bsm.multiply(1.0, A, B, 0.0, Cm, 0.0, prec=prec)
                bsm.multiply_backward(1.0, Cm, dC, A, B, dA, dB, prec=prec)
            ms = _timed(torch, step, args.steps, args.warmup)
            flop = 3 * Cm.counts().useful_flop      # forward + two adjoint products
            legs[prec] = {"value": flop / ms * 1e-9, "ms_per_step": ms}
        out.update(value=legs["fp64"]["value"], ms_per_step=legs["fp64"]["ms_per_step"],
                   config={"workload": name, "step": "multiply + both adjoints", "products": Cm.counts().products,
                           "useful_flop_per_step": flop},
                   split_precision={"ozaki": legs["ozaki"], "tf32x3": legs["tf32x3"]})
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
            for prec in ("fp64", "ozaki", "tf32x3") + (("tf32x3_panel",) if s_ <= 24 else ()):
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
        out.update(value=legs["fp64"]["value"], ms_per_step=legs["fp64"]["ms_per_step"],
                   config={"workload": name, "step": "replay of the graph-captured 10-step chain (20 multiplies, "
                                                    "10 filtered adds)", "eps": w["eps"]},
                   split_precision={"ozaki": legs["ozaki"], "tf32x3": legs["tf32x3"]}, chain=legs)
    print(json.dumps(out), flush=True)


# --------------------------------------------------------------------------
# GB300 arm
# --------------------------------------------------------------------------
def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload != "mixed3000":
        return run_other(args)

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

    w = make_inputs()
    A = bsm.Matrix.from_host(w["A"])
    B = bsm.Matrix.from_host(w["B"])
    eps = w["eps"]
    Cm = bsm.Matrix.empty(w["A"].row_bs, w["B"].col_bs)
    stream = torch.cuda.current_stream()

    def step(prec="fp64", flush_every=0):
        bsm.multiply(1.0, A, B, 0.0, Cm, eps, prec=prec, flush_every=flush_every)

    # per-shape kernel variants chosen by measurement (not timed)
    from paper_1708_03604_gb300 import autotune
    tuned_fp64 = autotune.tune(A, B, eps, prec="fp64", reps=2)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---------------- timed region: FP64 path
    bsm.bsm_set_profiling(True)
    clocks = ClockSampler()
    clocks.start()
    time.sleep(0.3)
    launches0 = bsm.bsm_get_launch_count()
    numeric_ms = []
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    phases = None
    for _ in range(args.steps):
        step()
        phases = Cm.timings()
        numeric_ms.append(phases["numeric"])
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = bsm.bsm_get_launch_count() - launches0
    clk = clocks.stop()
    bsm.bsm_set_profiling(False)
    ms = max_ms(e0.elapsed_time(e1)) / args.steps
    cnt = Cm.counts()
    flop = cnt.useful_flop
    value = job_rate(flop, world, ms) * 1e-9
    num_ms = statistics.mean(numeric_ms)
    achieved = flop / (num_ms * 1e-3) / 1e12
    traffic = traffic_from_profile()
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                "kernel": "k_numeric_cc<double, wide build> (FP64 FMA)", "launch_ms": num_ms,
                "peak_basis": "derived: 152 SMs x 2 FP64 FMA/clk x 2 FLOP x 2070 MHz"}
    C64 = Cm.data_tensor()

    # ---------------- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        pin, pat = {}, {}
        for nm in ("A", "B"):  # every input array in pinned host memory
            pin[nm] = torch.from_numpy(w[nm].data).pin_memory()
            pat[nm] = [torch.from_numpy(np.ascontiguousarray(getattr(w[nm], f))).pin_memory().numpy()
                       for f in ("row_bs", "col_bs", "row_ptr", "col_idx", "blk_off")]
        ke = max(3, min(args.steps, 5))
        h2d = sum(w[nm].data.nbytes + w[nm].row_ptr.nbytes + w[nm].col_idx.nbytes + w[nm].blk_off.nbytes +
                  w[nm].row_bs.nbytes + w[nm].col_bs.nbytes for nm in ("A", "B"))
        out_host = None
        d2h = 0
        times = []
        for it in range(ke + 1):
            barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hA = bsm.bsm_create(*pat["A"], bsm.BSM_FP64, pin["A"].data_ptr(), pin["A"].numel(), bsm.BSM_DATA_COPY)
            hB = bsm.bsm_create(*pat["B"], bsm.BSM_FP64, pin["B"].data_ptr(), pin["B"].numel(), bsm.BSM_DATA_COPY)
            hC = bsm.bsm_create_empty(w["A"].row_bs, w["B"].col_bs, bsm.BSM_FP64)
            bsm.bsm_multiply(1.0, hA, hB, 0.0, hC, eps, bsm.make_opts("fp64"))
            inf = bsm.bsm_get_info(hC)
            if out_host is None or out_host.numel() < inf.data_len:
                # pinned host buffers for C's values and pattern
                out_host = torch.empty(inf.data_len, dtype=torch.float64).pin_memory()
                rp_t = torch.empty(inf.nbr + 1, dtype=torch.int64).pin_memory()
                ci_t = torch.empty(max(inf.nnzb, 1), dtype=torch.int32).pin_memory()
                bo_t = torch.empty(max(inf.nnzb, 1), dtype=torch.int64).pin_memory()
                rp, ci, bo = rp_t.numpy(), ci_t.numpy()[:inf.nnzb], bo_t.numpy()[:inf.nnzb]
            bsm.lib().bsm_copy_data(hC, out_host.data_ptr())
            bsm.lib().bsm_copy_pattern(hC, rp.ctypes.data, ci.ctypes.data, bo.ctypes.data)
            for h in (hA, hB, hC):
                bsm.bsm_destroy(h)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            d2h = inf.data_len * 8 + rp.nbytes + ci.nbytes + bo.nbytes
            if it > 0:
                times.append(dt)
        et = max_ms(statistics.mean(times))
        # one more (untimed) pass with a synchronisation after every stage: where the time goes
        parts = {}

        def mark(name, t_prev):
            torch.cuda.synchronize()
            t = time.perf_counter()
            parts[name] = round((t - t_prev) * 1e3, 2)
            return t

        torch.cuda.synchronize()
        t = time.perf_counter()
        hA = bsm.bsm_create(*pat["A"], bsm.BSM_FP64, pin["A"].data_ptr(), pin["A"].numel(), bsm.BSM_DATA_COPY)
        hB = bsm.bsm_create(*pat["B"], bsm.BSM_FP64, pin["B"].data_ptr(), pin["B"].numel(), bsm.BSM_DATA_COPY)
        hC = bsm.bsm_create_empty(w["A"].row_bs, w["B"].col_bs, bsm.BSM_FP64)
        t = mark("create_and_h2d", t)
        bsm.bsm_multiply(1.0, hA, hB, 0.0, hC, eps, bsm.make_opts("fp64"))
        t = mark("multiply", t)
        bsm.lib().bsm_copy_data(hC, out_host.data_ptr())
        bsm.lib().bsm_copy_pattern(hC, rp.ctypes.data, ci.ctypes.data, bo.ctypes.data)
        t = mark("d2h", t)
        for h in (hA, hB, hC):
            bsm.bsm_destroy(h)
        mark("destroy", t)
        e2e = {"value": world * flop / et / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": et * 1e3,
               "includes": "host pattern validation, H2D of A and B from pinned memory, multiply, "
                           "D2H of C's data (pinned) and pattern",
               "stage_ms_untimed_pass": parts}

    # ---------------- split-precision legs (variants per block shape autotuned first)
    split = {}
    tuned = {"fp64": tuned_fp64}
    if not args.no_split:
        from paper_1708_03604_gb300 import autotune
        legs = [("ozaki", "ozaki", 0), ("tf32x3", "tf32x3", 0), ("bf16x6", "bf16x6", 0), ("bf16x3", "bf16x3", 0),
                ("tf32x3_fp64sum", "tf32x3", 1), ("tf32x3_pair2", "tf32x3", -2), ("tf32x3_pair4", "tf32x3", -4),
                ("bf16x6_pair4", "bf16x6", -4)]
        if args.legs:
            legs = [lg for lg in legs if lg[0] in args.legs.split(",")]
        for prec in dict.fromkeys(lg[1] for lg in legs):
            tuned[prec] = autotune.tune(A, B, eps, prec=prec, reps=2)
        ref_norm = torch.linalg.vector_norm(C64).item()
        for key, prec, fl in legs:
            step(prec, fl)
            torch.cuda.synchronize()
            bsm.bsm_set_profiling(True)
            ks = max(3, min(args.steps, 5))
            num = []
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            for _ in range(ks):
                step(prec, fl)
                num.append(Cm.timings()["numeric"])
            f1.record(stream)
            torch.cuda.synchronize()
            bsm.bsm_set_profiling(False)
            sms = max_ms(f0.elapsed_time(f1)) / ks
            err = (torch.linalg.vector_norm(Cm.data_tensor() - C64).item() / ref_norm)
            split[key] = {"value": world * flop / (sms * 1e-3) / 1e12, "ms_per_step": sms,
                           "numeric_ms": statistics.mean(num), "speedup_vs_fp64": ms / sms,
                           "rel_fro_err_vs_fp64_path": err}
        step()  # leave the FP64 result in Cm
        torch.cuda.synchronize()

    # ---------------- CPU oracle on sampled rows (+ parity of those rows)
    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, rows, r = cpu_baseline(w, args.cpu_seconds)
        rp, ci, bo = Cm.pattern()
        got = Cm.data_host()
        same_pattern = True
        num, den = 0.0, 0.0
        for i in rows:
            g0, g1 = rp[i], rp[i + 1]
            o0, o1 = r.C.row_ptr[i], r.C.row_ptr[i + 1]
            if not np.array_equal(ci[g0:g1], r.C.col_idx[o0:o1]):
                same_pattern = False
                continue
            if g1 > g0:
                ge = slice(bo[g0], bo[g1 - 1] + int(w["A"].row_bs[i]) * int(w["B"].col_bs[ci[g1 - 1]]))
                oe = slice(r.C.blk_off[o0], r.C.blk_off[o1 - 1] + int(w["A"].row_bs[i]) *
                           int(w["B"].col_bs[r.C.col_idx[o1 - 1]]))
                num += float(np.sum((got[ge] - r.C.data[oe]) ** 2))
                den += float(np.sum(r.C.data[oe] ** 2))
        parity = {"rows": len(rows), "pattern_equal": same_pattern,
                  "rel_fro_fp64_vs_oracle": (num / den) ** 0.5 if den else None}

    if rank == 0:
        line = {"metric": "block-SpGEMM useful TFLOP/s", "value": value, "unit": "TFLOP/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": config({"products": cnt.products, "filtered": cnt.filtered, "useful_flop": flop,
                                  "c_blocks": Cm.nnzb, "parallelism": "replicas" if world > 1 else "single GPU"}),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clk, "split_precision": split, "split_autotune": tuned, "parity_sample": parity,
                "phase_ms_last_fp64_step": phases,
                "index_phases": phase_rates(phases, w, cnt, Cm.nnzb, Cm.info().data_len)}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
