"""Ozaki-style error-free BF16 slicing (BSM_P_OZAKI) against the CPU oracle.

The slices are exact and the exact-sum levels are exact, so the result is
FP64-class: C's pattern bit for bit (the filter is FP64 as on every path),
values within a relative Frobenius error of 1e-13 of the FP64 oracle on
N(0,1)-type data (ten times tighter than the FP64 path's own bar), and every
element within the worst-case bound of the method: per term of k at most
2^-44 of 2^(ex + ey), with 2^ex the power of two below the largest |a| of
the element's row of A and 2^ey that of its column of B (the rounded sum of
slice levels 4..5 dominates it; see the Ozaki section of k_numeric.cu).
"""
import numpy as np
import pytest

from paper_1708_03604_gb300 import inputs as I
from tests.helpers import block_mask, offsets, random_bcsr, rel_fro, to_dense

pytestmark = pytest.mark.gpu

TOL = 1e-13


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


def _ragged():
    # block sizes 1..130: several fragment tiles per block, inner dimensions
    # above the 80-term exact window (flushes inside one block product)
    rng = np.random.default_rng(15)
    rbs = rng.integers(1, 41, size=11).astype(np.int32)
    kbs = np.concatenate([rng.integers(1, 41, size=7), [97, 130]]).astype(np.int32)
    cbs = rng.integers(1, 41, size=12).astype(np.int32)
    return random_bcsr(rbs, kbs, 0.5, seed=121), random_bcsr(kbs, cbs, 0.5, seed=122), 0.0


@pytest.mark.parametrize("case", ["uniform23", "mixed_filtered", "ragged"])
def test_ozaki_parity(bsm, oracle, case):
    if case == "uniform23":
        w = I.uniform_23(nb=40, occ=0.2)
        A, B, eps = w["A"], w["B"], 0.0
    elif case == "mixed_filtered":
        w = I.mixed_banded(nb=300, occ=0.1, eps=1.0, decay=8.0)
        A, B, eps = w["A"], w["B"], w["eps"]
    else:
        A, B, eps = _ragged()
    Cg = bsm.multiply(1.0, bsm.Matrix.from_host(A), bsm.Matrix.from_host(B), eps=eps, prec="ozaki")
    ref = oracle.multiply(1.0, A, B, eps=eps)
    _check_pattern(Cg, ref.C)
    assert Cg.counts().products == len(ref.prods.a)
    err = rel_fro(Cg.data_host(), ref.C.data)
    assert err <= TOL, err


def _scaled_case():
    """All-positive values (no cancellation: the FP32 sums are as large as
    they get), row scales of A and column scales of B spread over 2^-300 ..
    2^300, one zero row of A and one zero column of B."""
    rng = np.random.default_rng(77)
    bs = I.mixed_sizes(30, (1, 5, 13, 23, 40), (0.2, 0.3, 0.2, 0.2, 0.1), seed=13)
    A = random_bcsr(bs, bs, 0.3, seed=131)
    B = random_bcsr(bs, bs, 0.3, seed=132)
    A.data[:] = rng.random(len(A.data))
    B.data[:] = rng.random(len(B.data))
    n = int(np.sum(bs))
    srow = np.ldexp(1.0, rng.integers(-300, 301, size=n))
    scol = np.ldexp(1.0, rng.integers(-300, 301, size=n))
    srow[n // 2] = 0.0
    scol[n // 3] = 0.0
    off = offsets(bs)
    rp = np.asarray(A.row_ptr)
    for i in range(len(bs)):
        for b in range(rp[i], rp[i + 1]):
            j = A.col_idx[b]
            m, k = bs[i], bs[j]
            blk = A.data[A.blk_off[b]:A.blk_off[b] + m * k].reshape(m, k)
            blk *= srow[off[i]:off[i] + m, None]
    rp = np.asarray(B.row_ptr)
    for i in range(len(bs)):
        for b in range(rp[i], rp[i + 1]):
            j = B.col_idx[b]
            k, nn = bs[i], bs[j]
            blk = B.data[B.blk_off[b]:B.blk_off[b] + k * nn].reshape(k, nn)
            blk *= scol[None, off[j]:off[j] + nn]
    return bs, A, B


def test_ozaki_elementwise_bound(bsm, oracle):
    bs, A, B = _scaled_case()
    Cg = bsm.multiply(1.0, bsm.Matrix.from_host(A), bsm.Matrix.from_host(B), prec="ozaki")
    ref = oracle.multiply(1.0, A, B)
    _check_pattern(Cg, ref.C)
    got = Cg.data_host()
    Cg_h = I.BCSR(ref.C.row_bs, ref.C.col_bs, ref.C.row_ptr, ref.C.col_idx, ref.C.blk_off, got)
    Dg, Dr = to_dense(Cg_h), to_dense(ref.C)
    Ad, Bd = to_dense(A), to_dense(B)
    # K_rc: terms of k of every kept product of the element's block
    K = block_mask(A).astype(np.float64) @ block_mask(B).astype(np.float64)
    rowmax = np.max(np.abs(Ad), axis=1)
    colmax = np.max(np.abs(Bd), axis=0)
    ex = np.where(rowmax > 0, np.floor(np.log2(np.where(rowmax > 0, rowmax, 1.0))), -1100)
    ey = np.where(colmax > 0, np.floor(np.log2(np.where(colmax > 0, colmax, 1.0))), -1100)
    scale = np.ldexp(1.0, (ex[:, None] + ey[None, :] - 44).clip(-1074, 1023).astype(np.int64))
    bound = K * scale
    err = np.abs(Dg - Dr)
    assert np.all(err <= bound), float(np.max(err / np.where(bound > 0, bound, 1.0)))
    # the zero row and column give exact zeros
    nz = (rowmax[:, None] > 0) & (colmax[None, :] > 0) & (K > 0)
    assert np.all(Dg[~nz] == 0.0)


def test_ozaki_long_inner_dimension(bsm, oracle):
    """One output block summing 537,600 terms of k (2,100 blocks of 256): more
    than 8192 exact 64-term windows, so the fixed-point sum is moved into the
    output element once before the end."""
    kbs = np.full(2100, 256, dtype=np.int32)
    A = random_bcsr(np.array([16], np.int32), kbs, 1.0, seed=151)
    B = random_bcsr(kbs, np.array([8], np.int32), 1.0, seed=152)
    Cg = bsm.multiply(1.0, bsm.Matrix.from_host(A), bsm.Matrix.from_host(B), prec="ozaki")
    ref = oracle.multiply(1.0, A, B)
    _check_pattern(Cg, ref.C)
    err = rel_fro(Cg.data_host(), ref.C.data)
    assert err <= TOL, err


def test_ozaki_backward(bsm, oracle):
    import torch
    bs = I.mixed_sizes(40, (3, 7, 13, 23), (0.3, 0.3, 0.2, 0.2), seed=23)
    A, B = random_bcsr(bs, bs, 0.15, seed=71), random_bcsr(bs, bs, 0.15, seed=72)
    gA, gB = bsm.Matrix.from_host(A), bsm.Matrix.from_host(B)
    Cg = bsm.multiply(0.75, gA, gB, prec="ozaki")
    ref = oracle.multiply(0.75, A, B)
    assert rel_fro(Cg.data_host(), ref.C.data) <= TOL
    G = np.random.default_rng(3).standard_normal(ref.C.data_len)
    dA_ref, dB_ref = oracle.multiply_backward(0.75, A, B, ref.C, G, ref.prods)
    dA = torch.full((len(A.data),), np.nan, dtype=torch.float64, device="cuda")
    dB = torch.full((len(B.data),), np.nan, dtype=torch.float64, device="cuda")
    bsm.multiply_backward(0.75, Cg, torch.tensor(G, device="cuda"), gA, gB, dA, dB, prec="ozaki")
    assert rel_fro(dA.cpu().numpy(), dA_ref) <= TOL
    assert rel_fro(dB.cpu().numpy(), dB_ref) <= TOL


def test_ozaki_lane_variants(bsm, oracle):
    """Tiny output blocks run one per lane in FP64 (default for <= 16
    elements; 5 x 5 on request) beside tensor-core items in one launch."""
    bs = I.mixed_sizes(60, (1, 2, 4, 5, 9), (0.2, 0.2, 0.2, 0.2, 0.2), seed=41)
    A, B = random_bcsr(bs, bs, 0.2, seed=141), random_bcsr(bs, bs, 0.2, seed=142)
    ref = oracle.multiply(1.0, A, B)
    gA, gB = bsm.Matrix.from_host(A), bsm.Matrix.from_host(B)
    try:
        for v in (0, 1):
            bsm.bsm_set_variant("ozaki", 5, 5, v)
            Cg = bsm.multiply(1.0, gA, gB, prec="ozaki")
            _check_pattern(Cg, ref.C)
            assert rel_fro(Cg.data_host(), ref.C.data) <= TOL
    finally:
        bsm.bsm_set_variant("ozaki", 5, 5, -1)


def test_ozaki_all_lane_shapes_run_fp64(bsm, oracle):
    """Blocks of 1 and 4 rows/columns only: every output block runs one per
    lane in FP64, so the Ozaki request gives the FP64 path's result bit for bit."""
    w = I.purification_start(nb=200)
    X = bsm.Matrix.from_host(w["X0"])
    a = bsm.multiply(1.0, X, X, eps=w["eps"], prec="ozaki").data_host()
    b = bsm.multiply(1.0, X, X, eps=w["eps"], prec="fp64").data_host()
    np.testing.assert_array_equal(a, b)
    ref = oracle.multiply(1.0, w["X0"], w["X0"], eps=w["eps"])
    assert rel_fro(a, ref.C.data) <= TOL


def test_ozaki_no_sync_matches_eager(bsm):
    w = I.mixed_banded(nb=150, occ=0.1, eps=1e-6)
    A, B = bsm.Matrix.from_host(w["A"]), bsm.Matrix.from_host(w["B"])
    Cm = bsm.multiply(1.0, A, B, eps=w["eps"], prec="ozaki")
    x = Cm.data_host()
    bsm.multiply(1.0, A, B, Cm=Cm, eps=w["eps"], prec="ozaki", no_sync=True)
    assert bsm.bsm_get_status(Cm.h) == 0
    np.testing.assert_array_equal(Cm.data_host(), x)


def test_ozaki_rejects_fp32(bsm):
    w = I.differentiation_13(nb=20, occ=0.15, dtype=np.float32)
    with pytest.raises(bsm.BsmError) as e:
        bsm.multiply(1.0, bsm.Matrix.from_host(w["A"]), bsm.Matrix.from_host(w["B"]), prec="ozaki")
    assert e.value.status == bsm.BSM_ERR_UNSUPPORTED


def test_ozaki_integer_data_is_exact(bsm, oracle):
    """Small integers: every slice product and level sum is exact and so is the
    FP64 oracle's sum, so the two agree bit for bit (negative entries, exact
    zeros and values that end a line's digits early included)."""
    rng = np.random.default_rng(23)
    bs = rng.integers(1, 41, size=30).astype(np.int32)
    A, B = random_bcsr(bs, bs, 0.3, seed=131), random_bcsr(bs, bs, 0.3, seed=132)
    A.data[:] = rng.integers(-100, 101, size=A.data.size)
    B.data[:] = rng.integers(-100, 101, size=B.data.size) * 0.25
    Cg = bsm.multiply(1.0, bsm.Matrix.from_host(A), bsm.Matrix.from_host(B), prec="ozaki")
    ref = oracle.multiply(1.0, A, B)
    _check_pattern(Cg, ref.C)
    np.testing.assert_array_equal(Cg.data_host(), ref.C.data)


def test_ozaki_subnormal_lines(bsm, oracle):
    """Rows of A whose entries are all subnormal (the line exponent field is 0,
    so the line is scaled as if its largest entry were 2^-1023) and rows
    mixing subnormal and normal entries: every element within 2^-44 of
    2^(ex + ey) per term of k, ex the line exponent the slicing uses."""
    rng = np.random.default_rng(29)
    bs = rng.integers(1, 24, size=20).astype(np.int32)
    A, B = random_bcsr(bs, bs, 0.4, seed=141), random_bcsr(bs, bs, 0.4, seed=142)
    ro = offsets(bs)
    Ad = to_dense(A)
    rows = np.arange(int(ro[-1]))
    sub = rows % 3 == 0                  # all-subnormal rows
    mix = rows % 3 == 1                  # subnormal and normal entries
    for b in range(len(A.col_idx)):
        i = int(np.searchsorted(np.asarray(A.row_ptr), b, side="right") - 1)
        m, n = int(A.row_bs[i]), int(A.col_bs[A.col_idx[b]])
        blk = A.data[A.blk_off[b]:A.blk_off[b] + m * n].reshape(m, n)
        r = np.arange(ro[i], ro[i] + m)
        tiny = rng.integers(-2**40, 2**40, size=(m, n)) * 2.0 ** -1074
        blk[sub[r]] = tiny[sub[r]]
        pick = rng.random((m, n)) < 0.5
        blk[mix[r]] = np.where(pick[mix[r]], tiny[mix[r]], blk[mix[r]])
    Cg = bsm.multiply(1.0, bsm.Matrix.from_host(A), bsm.Matrix.from_host(B), prec="ozaki")
    ref = oracle.multiply(1.0, A, B)
    _check_pattern(Cg, ref.C)
    got = I.BCSR(ref.C.row_bs, ref.C.col_bs, ref.C.row_ptr, ref.C.col_idx, ref.C.blk_off, Cg.data_host())
    Dg, Dr = to_dense(got), to_dense(ref.C)
    Ad, Bd = to_dense(A), to_dense(B)
    K = block_mask(A).astype(np.float64) @ block_mask(B).astype(np.float64)
    rowmax = np.max(np.abs(Ad), axis=1)
    colmax = np.max(np.abs(Bd), axis=0)
    ex = np.maximum(np.floor(np.log2(np.where(rowmax > 0, rowmax, 1.0))), -1023)
    ey = np.maximum(np.floor(np.log2(np.where(colmax > 0, colmax, 1.0))), -1023)
    bound = K * np.ldexp(1.0, (ex[:, None] + ey[None, :] - 44).clip(-1074, 1023).astype(np.int64))
    # the oracle's own rounding at the bottom of the FP64 range
    bound = bound + K * 2.0 ** -1074
    assert np.all(np.abs(Dg - Dr) <= bound)
    assert np.any(Dg[sub] != 0.0)
