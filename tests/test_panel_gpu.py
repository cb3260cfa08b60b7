"""Row-panel TF32x3 engine on tcgen05 tensor cores (BSM_P_TF32x3_PANEL)
against the CPU oracle.

The engine computes dense tiles of 5 x 5 output blocks; it must give C's
pattern bit for bit (the pattern comes from the FP64 symbolic phase, as on
every path), values within the split-precision bar of 1e-6 relative
Frobenius error, and every element within the TF32x3 method's analytic
worst-case bound.  Where it does not apply (mixed block sizes, blocks above
24, FP32 data, products removed by the filter) the multiply runs the
mma.sync TF32x3 kernel, which the engine query reports.
"""
import numpy as np
import pytest

from paper_1708_03604_gb300 import inputs as I
from tests.helpers import random_bcsr, rel_fro, to_dense

pytestmark = pytest.mark.gpu

TOL = 1e-6


@pytest.fixture(scope="module")
def bsm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_03604_gb300 import bsm as B
    B.lib()
    return B


def _check_pattern(C_gpu, C_ref):
    rp, ci, bo = C_gpu.pattern()
    np.testing.assert_array_equal(rp, C_ref.row_ptr)
    np.testing.assert_array_equal(ci, C_ref.col_idx)
    np.testing.assert_array_equal(bo, C_ref.blk_off)


def _run(bsm, oracle, A, B, eps=0.0, beta=0.0, C0=None, alpha=1.0, prec="tf32x3_panel"):
    gA, gB = bsm.Matrix.from_host(A), bsm.Matrix.from_host(B)
    Cg = bsm.Matrix.from_host(C0) if C0 is not None else None
    Cg = bsm.multiply(alpha, gA, gB, beta=beta, Cm=Cg, eps=eps, prec=prec)
    ref = oracle.multiply(alpha, A, B, beta=beta, Cold=C0, eps=eps)
    return Cg, ref, gA, gB


def _bound_coeff(s, nsteps, group=3):
    """TF32x3 worst case per element as a multiple of sum_k |a_ik||b_kj|: the
    cut into two 11-bit pieces and the left-out lo*lo product (3 * 2^-22), the
    FP32 sum inside the tensor core of `group` k-steps (3 piece products of
    `group` s terms, each addition off by at most 2^-23 of the running
    magnitude: rounding toward zero), the compensated sum across those sums
    (2^-22) with its compensation term rounded to BF16 after every add (2^-33
    each, at most one add per k-step)."""
    return 1.1 * (3 * 2.0 ** -22 + 3 * group * s * 2.0 ** -23 + 2.0 ** -22 + nsteps * 2.0 ** -33)


@pytest.mark.parametrize("case", ["uniform23", "banded23", "s13", "s24", "s4"])
def test_panel_parity(bsm, oracle, case):
    eps = 0.0
    if case == "uniform23":
        w = I.uniform_23(nb=40, occ=0.2)
        A, B = w["A"], w["B"]
    elif case == "banded23":
        # 37 block rows: the last row and column groups are partial; permuted
        # band as on the large 23 x 23 workload, filter that removes nothing
        w = I.large_banded_23(nb=37, occ=0.15, eps=1e-8)
        A, B, eps = w["A"], w["B"], w["eps"]
    elif case == "s13":
        w = I.differentiation_13(nb=60, occ=0.15)
        A, B = w["A"], w["B"]
    else:
        s = 24 if case == "s24" else 4
        bs = np.full(33, s, np.int32)
        A, B = random_bcsr(bs, bs, 0.25, seed=201), random_bcsr(bs, bs, 0.25, seed=202)
    Cg, ref, _, _ = _run(bsm, oracle, A, B, eps)
    assert Cg.engine() == "panel_tcgen05"
    _check_pattern(Cg, ref.C)
    assert Cg.counts().products == len(ref.prods.a)
    assert Cg.counts().filtered == 0
    assert rel_fro(Cg.data_host(), ref.C.data) <= TOL


@pytest.mark.parametrize("group", [3, 1, 6, 8])
def test_panel_elementwise_bound(bsm, oracle, group):
    """Every element within the analytic TF32x3 bound, on 23 x 23 blocks with
    values spread over six decades (the pieces and the FP32 sums see
    magnitudes far apart), for `group` k-steps per accumulator buffer
    (BSM_TUNE_PANEL_STEPS; 3 is the default)."""
    bs = np.full(30, 23, np.int32)
    A, B = random_bcsr(bs, bs, 0.3, seed=211), random_bcsr(bs, bs, 0.3, seed=212)
    rng = np.random.default_rng(5)
    A.data *= 10.0 ** rng.uniform(-3, 3, size=len(A.data))
    B.data *= 10.0 ** rng.uniform(-3, 3, size=len(B.data))
    bsm.bsm_set_tuning("tf32x3_panel", "panel_steps", -1 if group == 3 else group)
    try:
        Cg, ref, _, _ = _run(bsm, oracle, A, B)
    finally:
        bsm.bsm_set_tuning("tf32x3_panel", "panel_steps", -1)
    assert Cg.engine() == "panel_tcgen05"
    _check_pattern(Cg, ref.C)
    Ch = I.BCSR(ref.C.row_bs, ref.C.col_bs, ref.C.row_ptr, ref.C.col_idx, ref.C.blk_off, Cg.data_host())
    err = np.abs(to_dense(Ch) - to_dense(ref.C))
    bound = _bound_coeff(23, len(bs), group) * (np.abs(to_dense(A)) @ np.abs(to_dense(B)))
    assert np.all(err <= bound), float(np.max(err / np.where(bound > 0, bound, 1.0)))
    if group > 3:   # the tighter default's bound is what a longer group may exceed, not must
        assert rel_fro(Cg.data_host(), ref.C.data) <= 1e-6


def test_panel_matches_mma_sync_path(bsm, oracle):
    """Same split, same piece order, same compensated sum: the two engines
    agree far below the error of either against FP64."""
    w = I.uniform_23(nb=60, occ=0.15)
    gA, gB = bsm.Matrix.from_host(w["A"]), bsm.Matrix.from_host(w["B"])
    p = bsm.multiply(1.0, gA, gB, prec="tf32x3_panel")
    q = bsm.multiply(1.0, gA, gB, prec="tf32x3")
    assert p.engine() == "panel_tcgen05" and q.engine() == "split_mma"
    ref = oracle.multiply(1.0, w["A"], w["B"])
    ep, eq = rel_fro(p.data_host(), ref.C.data), rel_fro(q.data_host(), ref.C.data)
    assert ep <= TOL and eq <= TOL
    assert rel_fro(p.data_host(), q.data_host()) <= 2 * max(ep, eq)


def test_panel_alpha_beta_merge(bsm, oracle):
    """beta != 0: old blocks outside the product pattern (tiles with no
    product at all among them) come out as beta * old."""
    bs = np.full(45, 23, np.int32)
    w = I.large_banded_23(nb=45, occ=0.05, eps=1e-8)
    A, B = w["A"], w["B"]
    C0 = random_bcsr(bs, bs, 0.1, seed=221)
    Cg, ref, _, _ = _run(bsm, oracle, A, B, 0.0, beta=-0.5, C0=C0, alpha=2.0)
    assert Cg.engine() == "panel_tcgen05"
    _check_pattern(Cg, ref.C)
    assert rel_fro(Cg.data_host(), ref.C.data) <= TOL


def test_panel_empty_product(bsm, oracle):
    bs = np.full(10, 23, np.int32)
    A = random_bcsr(bs, bs, 0.0, seed=231)
    B = random_bcsr(bs, bs, 0.3, seed=232)
    Cg, ref, _, _ = _run(bsm, oracle, A, B)
    assert Cg.info().nnzb == 0 and len(ref.C.col_idx) == 0


@pytest.mark.parametrize("why", ["mixed_sizes", "block_above_24", "filtered", "fp32"])
def test_panel_falls_back_to_mma_sync(bsm, oracle, why):
    eps = 0.0
    if why == "mixed_sizes":
        w = I.mixed_banded(nb=60, occ=0.1, eps=0.0)
        A, B = w["A"], w["B"]
    elif why == "block_above_24":
        bs = np.full(12, 25, np.int32)
        A, B = random_bcsr(bs, bs, 0.3, seed=241), random_bcsr(bs, bs, 0.3, seed=242)
    elif why == "filtered":
        w = I.large_banded_23(nb=60, occ=0.1, eps=1e-8)
        A, B = w["A"], w["B"]
        nA = np.sort(oracle.block_norms(A))
        eps = float(nA[len(nA) // 2] ** 2)   # removes a good share of the products
    else:
        w = I.differentiation_13(nb=40, occ=0.15, dtype=np.float32)
        A, B = w["A"], w["B"]
    Cg, ref, gA, gB = _run(bsm, oracle, A, B, eps)
    assert Cg.engine() == "split_mma"
    _check_pattern(Cg, ref.C)
    if why == "filtered":
        assert Cg.counts().filtered > 0
    tol = 1e-5 if why == "fp32" else TOL
    assert rel_fro(Cg.data_host(), ref.C.data) <= tol
    # the fallback is the mma.sync TF32x3 kernel itself
    q = bsm.multiply(1.0, gA, gB, eps=eps, prec="tf32x3")
    np.testing.assert_array_equal(Cg.data_host(), q.data_host())


def test_panel_rejects_no_sync(bsm):
    w = I.uniform_23(nb=20, occ=0.2)
    gA, gB = bsm.Matrix.from_host(w["A"]), bsm.Matrix.from_host(w["B"])
    Cm = bsm.multiply(1.0, gA, gB, prec="tf32x3_panel")
    with pytest.raises(bsm.BsmError) as e:
        bsm.multiply(1.0, gA, gB, Cm=Cm, prec="tf32x3_panel", no_sync=True)
    assert e.value.status == bsm.BSM_ERR_UNSUPPORTED


def test_panel_backward_runs_tf32x3(bsm, oracle):
    import torch
    w = I.uniform_23(nb=30, occ=0.2)
    A, B = w["A"], w["B"]
    Cg, ref, gA, gB = _run(bsm, oracle, A, B)
    G = np.random.default_rng(4).standard_normal(ref.C.data_len)
    dA_ref, dB_ref = oracle.multiply_backward(1.0, A, B, ref.C, G, ref.prods)
    dA = torch.empty(len(A.data), dtype=torch.float64, device="cuda")
    dB = torch.empty(len(B.data), dtype=torch.float64, device="cuda")
    bsm.multiply_backward(1.0, Cg, torch.tensor(G, device="cuda"), gA, gB, dA, dB, prec="tf32x3_panel")
    assert rel_fro(dA.cpu().numpy(), dA_ref) <= TOL
    assert rel_fro(dB.cpu().numpy(), dB_ref) <= TOL


def test_panel_repeat_is_deterministic(bsm):
    """Tiles are taken from an atomic ticket in any order, but each output
    element is summed by one thread in a fixed k order: results repeat bit
    for bit."""
    w = I.large_banded_23(nb=120, occ=0.05, eps=1e-8)
    gA, gB = bsm.Matrix.from_host(w["A"]), bsm.Matrix.from_host(w["B"])
    a = bsm.multiply(1.0, gA, gB, eps=w["eps"], prec="tf32x3_panel").data_host()
    b = bsm.multiply(1.0, gA, gB, eps=w["eps"], prec="tf32x3_panel").data_host()
    np.testing.assert_array_equal(a, b)
