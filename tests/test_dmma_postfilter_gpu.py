"""GPU parity of the FP64 tensor-core path (BSM_P_FP64_DMMA), of the FP64
running-sum form of the split paths, of the multiply's post filter, and a
sanity check of the library's peak probes.

* DMMA: same patterns and product lists as the oracle (bit for bit), values
  within a relative Frobenius error of 1e-12 -- uniform 23 x 23 blocks
  (three 8 x 8 tiles per side, the last one padded), ragged sizes 1..40
  (blocks below 8 rows or columns take the FMA code in the same launch),
  blocks of 64 and 78 (more than one pass of 3 x 3 tiles), both adjoints.
* FP64 running sum every F block products (the split form with FP32
  accumulation over at most F products): every element inside the analytic
  bound of the method for that F.
* Post filter (C blocks with norm <= eps dropped after the multiply): C's
  pattern equal to the oracle's post-filtered pattern bit for bit, values
  within 1e-12, with the margin guard that no kept or dropped block's norm
  lies within 1e-9 relative of eps (where FP64 rounding could flip it).
"""
import numpy as np
import pytest

from paper_1708_03604_gb300 import inputs as I
from tests.helpers import random_bcsr, rel_fro, to_dense

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bsm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_03604_gb300 import bsm as B
    B.lib()
    return B


def _pattern_eq(Cg, Cref):
    rp, ci, bo = Cg.pattern()
    np.testing.assert_array_equal(rp, Cref.row_ptr)
    np.testing.assert_array_equal(ci, Cref.col_idx)
    np.testing.assert_array_equal(bo, Cref.blk_off)


@pytest.mark.parametrize("case", ["uniform23", "ragged", "large"])
def test_dmma_forward_vs_oracle(bsm, oracle, case):
    if case == "uniform23":
        w = I.uniform_23(nb=48, occ=0.2)
        A, B, eps = w["A"], w["B"], 0.0
    elif case == "ragged":
        bs = np.random.default_rng(8).integers(1, 41, size=50).astype(np.int32)
        A, B, eps = random_bcsr(bs, bs, 0.2, seed=61), random_bcsr(bs, bs, 0.2, seed=62), 0.5
    else:
        bs = I.mixed_sizes(16, (64, 78, 9), (0.4, 0.4, 0.2), seed=5)
        A, B, eps = random_bcsr(bs, bs, 0.3, seed=63), random_bcsr(bs, bs, 0.3, seed=64), 0.0
    gA, gB = bsm.Matrix.from_host(A), bsm.Matrix.from_host(B)
    Cg = bsm.multiply(1.0, gA, gB, eps=eps, prec="fp64_dmma")
    ref = oracle.multiply(1.0, A, B, eps=eps)
    _pattern_eq(Cg, ref.C)
    p = Cg.products()
    np.testing.assert_array_equal(p.a, ref.prods.a)
    np.testing.assert_array_equal(p.c, ref.prods.c)
    assert rel_fro(Cg.data_host(), ref.C.data) <= 1e-12
    # against the FMA path of the library too (same products, other unit)
    Cf = bsm.multiply(1.0, gA, gB, eps=eps, prec="fp64")
    assert rel_fro(Cg.data_host(), Cf.data_host()) <= 1e-13


def test_dmma_beta_and_adjoint(bsm, oracle):
    import torch
    bs = I.mixed_sizes(40, (8, 13, 23, 5), (0.3, 0.3, 0.3, 0.1), seed=31)
    A, B = random_bcsr(bs, bs, 0.15, seed=71), random_bcsr(bs, bs, 0.15, seed=72)
    C0 = random_bcsr(bs, bs, 0.1, seed=73)
    gA, gB = bsm.Matrix.from_host(A), bsm.Matrix.from_host(B)
    Cg = bsm.multiply(2.0, gA, gB, beta=-0.5, Cm=bsm.Matrix.from_host(C0), prec="fp64_dmma")
    ref = oracle.multiply(2.0, A, B, beta=-0.5, Cold=C0)
    _pattern_eq(Cg, ref.C)
    assert rel_fro(Cg.data_host(), ref.C.data) <= 1e-12
    Cg = bsm.multiply(0.75, gA, gB, prec="fp64_dmma")
    ref = oracle.multiply(0.75, A, B)
    G = np.random.default_rng(3).standard_normal(ref.C.data_len)
    dA_ref, dB_ref = oracle.multiply_backward(0.75, A, B, ref.C, G, ref.prods)
    dA = torch.full((len(A.data),), np.nan, dtype=torch.float64, device="cuda")
    dB = torch.full((len(B.data),), np.nan, dtype=torch.float64, device="cuda")
    bsm.multiply_backward(0.75, Cg, torch.tensor(G, device="cuda"), gA, gB, dA, dB, prec="fp64_dmma")
    assert rel_fro(dA.cpu().numpy(), dA_ref) <= 1e-12
    assert rel_fro(dB.cpu().numpy(), dB_ref) <= 1e-12


def _fp64sum_bound_coeff(prec, kmax, F):
    """Worst-case error of one output element of the split form whose FP32
    accumulator spans at most F block products before it is added into an
    FP64 running sum, as a multiple of sum_k |a_ik||b_kj|: the cut of the
    operands into pieces and the piece products left out (as for the
    compensated form), plus npp * F * kmax FP32 additions inside the tensor
    core, each off by at most 2^-23 of the running magnitude (they round
    toward zero), plus the FP64 additions (2^-52 each, at most one per
    block product)."""
    if prec == "tf32x3":
        trunc, npp = 3 * 2.0 ** -22, 3
    else:                   # bf16x6
        trunc, npp = 5 * 2.0 ** -24, 6
    return 1.1 * (trunc + npp * F * kmax * 2.0 ** -23 + 64 * 2.0 ** -52)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x6"])
@pytest.mark.parametrize("F", [1, 4, 8])
def test_fp64_running_sum_elementwise_bound(bsm, oracle, prec, F):
    bs = I.mixed_sizes(30, (5, 13, 23, 40), (0.3, 0.3, 0.2, 0.2), seed=27)
    A, B = random_bcsr(bs, bs, 0.3, seed=101), random_bcsr(bs, bs, 0.3, seed=102)
    gA, gB = bsm.Matrix.from_host(A), bsm.Matrix.from_host(B)
    Cg = bsm.multiply(1.0, gA, gB, prec=prec, flush_every=F)
    ref = oracle.multiply(1.0, A, B)
    _pattern_eq(Cg, ref.C)
    Ch = I.BCSR(ref.C.row_bs, ref.C.col_bs, ref.C.row_ptr, ref.C.col_idx, ref.C.blk_off, Cg.data_host())
    err = np.abs(to_dense(Ch) - to_dense(ref.C))
    bound = _fp64sum_bound_coeff(prec, int(bs.max()), F) * (np.abs(to_dense(A)) @ np.abs(to_dense(B)))
    assert np.all(err <= bound), float(np.max(err / np.where(bound > 0, bound, 1.0)))
    assert rel_fro(Ch.data, ref.C.data) <= 1e-6


@pytest.mark.parametrize("prec", ["fp64", "fp64_dmma", "tf32x3"])
def test_post_filter_vs_oracle(bsm, oracle, prec):
    # strong decay and a threshold between the C block norms: the post
    # filter drops a good share of C's blocks
    w = I.mixed_banded(nb=300, occ=0.1, eps=1e-3, decay=4.0)
    A, B, eps = w["A"], w["B"], w["eps"]
    ref = oracle.multiply(1.0, A, B, eps=eps)
    post = oracle.post_filter(ref.C, eps)
    nrm = oracle.block_norms(ref.C)
    assert 0 < post.nnzb < ref.C.nnzb
    margin = float(np.min(np.abs(nrm - eps)) / eps)
    assert margin > 1e-9, margin
    gA, gB = bsm.Matrix.from_host(A), bsm.Matrix.from_host(B)
    Cg = bsm.multiply(1.0, gA, gB, eps=eps, prec=prec, post_filter=True)
    rp, ci, bo = Cg.pattern()
    np.testing.assert_array_equal(rp, post.row_ptr)
    np.testing.assert_array_equal(ci, post.col_idx)
    np.testing.assert_array_equal(bo, post.blk_off)
    tol = 1e-12 if prec.startswith("fp64") else 1e-6
    assert rel_fro(Cg.data_host(), post.data) <= tol
    # the product list no longer indexes C: the adjoint refuses, not misreads
    import torch
    with pytest.raises(bsm.BsmError):
        bsm.multiply_backward(1.0, Cg, torch.zeros(Cg.info().data_len, dtype=torch.float64, device="cuda"), gA, gB,
                              torch.zeros(len(A.data), dtype=torch.float64, device="cuda"), None)
    # and the counts still describe the multiply that made it
    assert Cg.counts().products == len(ref.prods.a)


def test_measured_peaks_plausible(bsm):
    p = {u: bsm.measure_peak(u, 2) / 1e12 for u in bsm.PEAK_UNITS}
    # ranges that any working GB300 meets (nominal FP64 1.25, TF32 / BF16
    # mma.sync a few hundred TFLOP/s); the probes must not report nonsense
    assert 0.2 < p["fp64_fma"] < 5.0, p
    assert 0.2 < p["fp64_mma"] < 5.0, p
    assert 20.0 < p["tf32_mma"] < 2500.0, p
    assert 20.0 < p["bf16_mma"] < 5000.0, p
    assert 5.0 < p["fp32_fma"] < 500.0, p
    with pytest.raises(bsm.BsmError):
        bsm.measure_peak("fp64_fma", 0)
