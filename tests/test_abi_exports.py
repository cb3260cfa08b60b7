"""The C-ABI library loads and exports every entry point include/bsm.h
declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "bsm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bsm_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libbsm():
    from paper_1708_03604_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("bsm_create", "bsm_multiply", "bsm_multiply_backward", "bsm_add", "bsm_get_stacks"):
        assert must in names


def test_library_exports_every_declared_symbol(libbsm):
    missing = [n for n in _declared() if not hasattr(libbsm, n)]
    assert not missing, missing


def test_binding_covers_every_export(libbsm):
    from paper_1708_03604_gb300 import bsm
    assert sorted(bsm.EXPORTS) == _declared()
    L = bsm.lib()
    for n in _declared():
        assert getattr(L, n).argtypes is not None or n == "bsm_last_error"


def test_host_side_argument_errors_need_no_gpu(libbsm):
    """Argument checks run on the host before any CUDA call."""
    from paper_1708_03604_gb300 import bsm
    import numpy as np
    L = bsm.lib()
    h = ctypes.c_void_p()
    bs = np.array([2, 3], np.int32)
    rp = np.array([0, 1, 2], np.int64)
    ci = np.array([1, 0], np.int32)
    bo = np.array([0, 6], np.int64)
    # block outside data_len
    st = L.bsm_create(ctypes.byref(h), 2, 2, bs.ctypes.data, bs.ctypes.data, rp.ctypes.data, ci.ctypes.data,
                      bo.ctypes.data, 0, 1, 10, 0)
    assert st == bsm.BSM_ERR_ARG and b"data_len" in L.bsm_last_error()
    # unsorted columns
    rp2 = np.array([0, 2, 2], np.int64)
    ci2 = np.array([1, 0], np.int32)
    st = L.bsm_create(ctypes.byref(h), 2, 2, bs.ctypes.data, bs.ctypes.data, rp2.ctypes.data, ci2.ctypes.data,
                      bo.ctypes.data, 0, 1, 100, 0)
    assert st == bsm.BSM_ERR_ARG and b"ascending" in L.bsm_last_error()
    # bad block size
    bad = np.array([0, 3], np.int32)
    st = L.bsm_create(ctypes.byref(h), 2, 2, bad.ctypes.data, bs.ctypes.data, rp.ctypes.data, ci.ctypes.data,
                      bo.ctypes.data, 0, 1, 100, 0)
    assert st == bsm.BSM_ERR_ARG
    # bad opts are rejected before anything is read from the matrices
    o = bsm.Opts()
    o.prec = 99
    assert L.bsm_multiply(1.0, None, None, 0.0, None, 0.0, ctypes.byref(o)) == bsm.BSM_ERR_ARG


def test_engine_query_and_variant_range_on_host(libbsm):
    """The engine query and the variant table check their arguments on the
    host; the panel precision has no variant table."""
    from paper_1708_03604_gb300 import bsm
    L = bsm.lib()
    v = ctypes.c_int32()
    assert L.bsm_get_engine(None, ctypes.byref(v)) == bsm.BSM_ERR_ARG
    assert L.bsm_set_variant(bsm.BSM_P_TF32x3_PANEL, 4, 4, 1) == bsm.BSM_ERR_ARG
    assert L.bsm_set_variant(bsm.BSM_P_TF32x3, 4, 4, 1) == bsm.BSM_OK
    assert L.bsm_get_variant(bsm.BSM_P_TF32x3, 4, 4, ctypes.byref(v)) == bsm.BSM_OK and v.value == 1
    assert L.bsm_set_variant(bsm.BSM_P_TF32x3, 4, 4, -1) == bsm.BSM_OK
    assert L.bsm_get_variant(bsm.BSM_P_TF32x3, 4, 4, ctypes.byref(v)) == bsm.BSM_OK and v.value == 1


def test_allocator_wait_limit_and_probe_arguments_on_host(libbsm):
    """The allocator hooks, the wait limit and the peak probe check their
    arguments on the host (no CUDA call is reached)."""
    from paper_1708_03604_gb300 import bsm
    L = bsm.lib()
    hook_a = bsm.ALLOC_FN(lambda n, s, c: None)
    # exactly one hook given
    assert L.bsm_set_allocator(hook_a, bsm.FREE_FN(), None) == bsm.BSM_ERR_ARG
    assert b"both" in L.bsm_last_error()
    n = ctypes.c_int64(-1)
    assert L.bsm_get_allocator_stats(ctypes.byref(n)) == bsm.BSM_OK and n.value == 0
    assert L.bsm_get_allocator_stats(None) == bsm.BSM_ERR_ARG
    # wait limits outside [0, 2] s
    for bad in (-1.0, 2.5, float("nan")):
        assert L.bsm_set_wait_limit(bad) == bsm.BSM_ERR_ARG
    assert L.bsm_set_wait_limit(2.0) == bsm.BSM_OK
    v = ctypes.c_double()
    assert L.bsm_measure_peak(9, 1, ctypes.byref(v)) == bsm.BSM_ERR_ARG
    assert L.bsm_measure_peak(0, 0, ctypes.byref(v)) == bsm.BSM_ERR_ARG
    assert L.bsm_measure_peak(0, 1, None) == bsm.BSM_ERR_ARG
    # the binding's hooks are back in place
    bsm.use_torch_allocator()


def test_product_limit_range():
    """The product limit is host state: its range check runs without a GPU."""
    from paper_1708_03604_gb300 import bsm
    L = bsm.lib()
    assert L.bsm_set_product_limit(0) == bsm.BSM_ERR_ARG
    assert L.bsm_set_product_limit(2**31) == bsm.BSM_ERR_ARG
    assert L.bsm_set_product_limit(1000) == bsm.BSM_OK
    assert L.bsm_set_product_limit(2**31 - 1) == bsm.BSM_OK


def test_tuning_knob_ranges_on_host():
    """The tuning table is host state: every knob's range check runs without a
    GPU, and a value set is read back (then the default restored)."""
    from paper_1708_03604_gb300 import bsm
    P, K = bsm.PREC, bsm.TUNE_PARAMS
    L = bsm.lib()
    ok, bad = bsm.BSM_OK, bsm.BSM_ERR_ARG
    cases = [  # (prec, knob, value, expected status)
        ("tf32x3", "panel_steps", 8, ok), ("tf32x3_panel", "panel_steps", 1, ok),
        ("tf32x3_panel", "panel_steps", 9, bad), ("tf32x3", "panel_steps", 0, bad),
        ("ozaki", "panel_steps", 3, bad), ("fp64", "panel_steps", 3, bad),
        ("tf32x3", "pass_mt", 1, ok), ("bf16x6", "pass_mt", 3, bad), ("ozaki", "pass_mt", 1, bad),
        ("ozaki", "pass_nt", 3, ok), ("ozaki", "pass_nt", 4, bad),
        ("tf32x3", "engine", 1, ok), ("bf16x3", "engine", 1, bad),
        ("fp64", "fp64_build", 2, ok), ("fp64", "fp64_build", 3, bad),
        ("fp64", "sched_tile", 16, ok), ("fp64", "sched_tile", 7, bad),
        ("tf32x3", "cta_warps", 3, bad), ("tf32x3", "ctas_per_sm", 17, bad),
    ]
    for prec, knob, value, want in cases:
        got = L.bsm_set_tuning(P[prec], K[knob], value)
        assert got == want, (prec, knob, value, got)
        if got == ok:
            assert bsm.bsm_get_tuning(prec, knob) == value
            assert L.bsm_set_tuning(P[prec], K[knob], -1) == ok
            assert bsm.bsm_get_tuning(prec, knob) == -1
    assert L.bsm_set_tuning(P["tf32x3"], len(K), 1) == bad       # no such knob
