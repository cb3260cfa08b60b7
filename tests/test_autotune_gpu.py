"""The autotuner's knobs (GPU): every launch and pass shape the tuner may
choose changes what the numeric launch runs (bsm_get_launch_config) and
leaves the results within the precision's tolerance against the oracle; a
tuned table saved to JSON and loaded again puts the same knobs back."""
import numpy as np
import pytest

from paper_1708_03604_gb300 import inputs as I
from tests.helpers import random_bcsr, rel_fro

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp64_dmma": 1e-12, "tf32x3": 1e-6, "bf16x6": 1e-6, "bf16x3": 1e-4, "ozaki": 1e-13}


@pytest.fixture(scope="module")
def bsm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_03604_gb300 import bsm as B
    B.lib()
    return B


@pytest.fixture(scope="module")
def operands(bsm, oracle):
    # blocks up to 40 x 40: several fragment tiles per side, so pass shapes matter
    bs = I.mixed_sizes(60, (5, 13, 23, 40), (0.4, 0.2, 0.2, 0.2), seed=44)
    Ah, Bh = random_bcsr(bs, bs, 0.15, seed=171), random_bcsr(bs, bs, 0.15, seed=172)
    ref = oracle.multiply(1.0, Ah, Bh, eps=0.3)
    return bsm.Matrix.from_host(Ah), bsm.Matrix.from_host(Bh), ref


@pytest.mark.parametrize("prec,knobs", [
    ("tf32x3", {"cta_warps": 2, "pass_mt": 1, "pass_nt": 1, "ctas_per_sm": 1}),
    ("bf16x6", {"cta_warps": 2, "pass_nt": 2}),
    ("bf16x3", {"pass_mt": 1, "pass_nt": 2, "ctas_per_sm": 2}),
    ("ozaki", {"cta_warps": 2, "pass_nt": 1, "ctas_per_sm": 2}),
    ("ozaki", {"pass_nt": 3}),
    ("fp64", {"fp64_build": 1}),
    ("fp64", {"fp64_build": 2, "ctas_per_sm": 1}),
    ("fp64_dmma", {"pass_mt": 1, "pass_nt": 2, "ctas_per_sm": 3}),
])
def test_knobs_change_the_launch_and_keep_results(bsm, operands, prec, knobs):
    from paper_1708_03604_gb300 import autotune
    A, B, ref = operands
    try:
        for k, v in knobs.items():
            bsm.bsm_set_tuning(prec, k, v)
            assert bsm.bsm_get_tuning(prec, k) == v
        Cg = bsm.multiply(1.0, A, B, eps=0.3, prec=prec)
        cfg = Cg.launch_config()
        np.testing.assert_array_equal(Cg.pattern()[1], ref.C.col_idx)
        assert rel_fro(Cg.data_host(), ref.C.data) <= TOL[prec]
        if "cta_warps" in knobs:
            assert cfg["cta_threads"] == 32 * knobs["cta_warps"]
        if "ctas_per_sm" in knobs:
            assert 0 < cfg["grid"] <= 152 * knobs["ctas_per_sm"]
        if "pass_mt" in knobs:
            assert cfg["pass_mt"] == knobs["pass_mt"]
        if "pass_nt" in knobs:
            assert cfg["pass_nt"] == knobs["pass_nt"]
        if "fp64_build" in knobs:
            assert cfg["fp64_build"] == knobs["fp64_build"]
        assert cfg["kernel"] == {"fp64": "fp64_cores", "fp64_dmma": "fp64_mma", "ozaki": "ozaki_mma"}.get(
            prec, "split_mma")
    finally:
        autotune.reset(prec)
    # back to the defaults
    Cd = bsm.multiply(1.0, A, B, eps=0.3, prec=prec)
    d = Cd.launch_config()
    assert d["cta_threads"] == 128
    assert rel_fro(Cd.data_host(), ref.C.data) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "ozaki"])
def test_schedule_tiles_permute_work_only(bsm, prec):
    """The 2-D tiled order of the output blocks is a permutation of work
    that each warp does alone in a fixed order: the result is bit for bit the
    one of the default (row) order, for banded-then-permuted operands whose
    ranked rows and columns make the tiles compact."""
    from paper_1708_03604_gb300 import autotune
    w = I.mixed_banded(nb=400, occ=0.1, eps=1e-6)
    A, B = bsm.Matrix.from_host(w["A"]), bsm.Matrix.from_host(w["B"])
    base = bsm.multiply(1.0, A, B, eps=w["eps"], prec=prec).data_host()
    try:
        for t in (8, 32, 256):
            bsm.bsm_set_tuning(prec, "sched_tile", t)
            got = bsm.multiply(1.0, A, B, eps=w["eps"], prec=prec).data_host()
            np.testing.assert_array_equal(got, base)
    finally:
        autotune.reset(prec)


def test_engine_knob_runs_the_panel_where_it_applies(bsm, oracle):
    """BSM_TUNE_ENGINE = 1: BSM_P_TF32x3 runs on the tcgen05 row-panel engine
    for uniform blocks with nothing filtered, on the mma.sync kernel where the
    engine does not apply (mixed sizes) or when an FP64 running sum is asked
    for; results within 1e-6 of the oracle either way."""
    from paper_1708_03604_gb300 import autotune
    u = I.large_banded_23(nb=60, occ=0.1, eps=1e-8)
    A, B = bsm.Matrix.from_host(u["A"]), bsm.Matrix.from_host(u["B"])
    ref = oracle.multiply(1.0, u["A"], u["B"], eps=u["eps"])
    try:
        bsm.bsm_set_tuning("tf32x3", "engine", 1)
        Cp = bsm.multiply(1.0, A, B, eps=u["eps"], prec="tf32x3")
        assert Cp.engine() == "panel_tcgen05" and Cp.launch_config()["kernel"] == "panel_tcgen05"
        assert rel_fro(Cp.data_host(), ref.C.data) <= 1e-6
        Cf = bsm.multiply(1.0, A, B, eps=u["eps"], prec="tf32x3", flush_every=4)
        assert Cf.engine() == "split_mma"
        assert rel_fro(Cf.data_host(), ref.C.data) <= 1e-6
        w = I.mixed_banded(nb=120, occ=0.1, eps=1e-6)
        Cm = bsm.multiply(1.0, bsm.Matrix.from_host(w["A"]), bsm.Matrix.from_host(w["B"]), eps=w["eps"],
                          prec="tf32x3")
        assert Cm.engine() == "split_mma"
    finally:
        autotune.reset("tf32x3")


def test_knob_ranges_are_checked(bsm):
    with pytest.raises(bsm.BsmError):
        bsm.bsm_set_tuning("fp64", "cta_warps", 2)        # the FP64 kernels run 4 warps per CTA
    with pytest.raises(bsm.BsmError):
        bsm.bsm_set_tuning("tf32x3", "cta_warps", 8)
    with pytest.raises(bsm.BsmError):
        bsm.bsm_set_tuning("tf32x3", "pass_mt", 3)
    with pytest.raises(bsm.BsmError):
        bsm.bsm_set_tuning("ozaki", "fp64_build", 1)
    with pytest.raises(bsm.BsmError):
        bsm.bsm_set_tuning("tf32x3_panel", "ctas_per_sm", 1)
    with pytest.raises(bsm.BsmError):
        bsm.bsm_set_tuning("fp64", "sched_tile", 4)
    with pytest.raises(bsm.BsmError):
        bsm.bsm_set_tuning("bf16x6", "engine", 1)
    with pytest.raises(bsm.BsmError):
        bsm.bsm_set_tuning("tf32x3_panel", "panel_steps", 9)
    with pytest.raises(bsm.BsmError):
        bsm.bsm_set_tuning("ozaki", "panel_steps", 3)


def test_tuned_table_roundtrip(bsm, operands, tmp_path):
    from paper_1708_03604_gb300 import autotune
    A, B, ref = operands
    try:
        table = autotune.tune(A, B, 0.3, prec="tf32x3", reps=1)
        assert table["numeric_ms"]["tuned"] > 0
        keys = {"cta_warps", "pass_mt", "pass_nt", "ctas_per_sm", "sched_tile", "engine"}
        if table["params"]["engine"] == 1:
            keys.add("panel_steps")
        assert set(table["params"]) == keys
        # the flush interval the tuner chose keeps the error within its target
        if table["flush_every"] is not None:
            assert table["flush_trials"][str(table["flush_every"])]["rel_fro_err_vs_fp64_path"] <= 1e-6
        path = str(tmp_path / "t.json")
        autotune.save([table], path)
        autotune.reset("tf32x3")
        autotune.load(path)
        for k, v in table["params"].items():
            assert bsm.bsm_get_tuning("tf32x3", k) == v
        Cg = bsm.multiply(1.0, A, B, eps=0.3, prec="tf32x3", flush_every=table["flush_every"] or 0)
        assert rel_fro(Cg.data_host(), ref.C.data) <= 1e-6
    finally:
        autotune.reset("tf32x3")
