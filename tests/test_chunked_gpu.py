"""Row-panel chunking of the multiply (GPU).

With the product limit set below a multiply's kept products, the library
fills and multiplies C in panels of whole C block rows, each holding at most
the limit.  Every C block is still computed by the same kernel from the same
products in the same order, so the result must be bit for bit that of one
pass, for every precision, with on-the-fly filtering and with beta * C
merged in.  A chunked C keeps no product list (no stacks, no adjoint, no
no_sync replay), and one C block row above the limit is refused with
BSM_ERR_CAPACITY.
"""
import numpy as np
import pytest

from paper_1708_03604_gb300 import inputs as I
from tests.helpers import random_bcsr, rel_fro

pytestmark = pytest.mark.gpu

PRECS = (("fp64", 0), ("fp64_dmma", 0), ("tf32x3", 0), ("tf32x3", 4), ("bf16x6", 0), ("bf16x3", 0), ("ozaki", 0))


@pytest.fixture(scope="module")
def bsm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_03604_gb300 import bsm as B
    B.lib()
    yield B
    B.set_product_limit()


def _with_empty_rows(bs, occ, seed, empty):
    """A random block-sparse matrix whose block rows in `empty` hold no blocks."""
    rows, cols, _ = I.uniform_pattern(len(bs), len(bs), occ, seed)
    keep = ~np.isin(rows, np.asarray(sorted(empty)))
    return I.assemble(bs, bs, rows[keep], cols[keep], None, seed=seed + 1000)


def _row_products(Cm):
    """Kept products per C block row of an unchunked multiply."""
    row_ptr = np.asarray(Cm.pattern()[0])
    c_rows = np.repeat(np.arange(len(row_ptr) - 1), np.diff(row_ptr))
    return np.bincount(c_rows[Cm.products().c], minlength=len(row_ptr) - 1)


@pytest.fixture(scope="module")
def operands():
    bs = np.concatenate([I.mixed_sizes(36, (1, 2, 4, 5, 6), (0.2, 0.2, 0.2, 0.2, 0.2), seed=12),
                         I.mixed_sizes(28, (13, 23, 32), (0.4, 0.4, 0.2), seed=13)]).astype(np.int32)
    Ah = _with_empty_rows(bs, 0.2, 91, {3, 4, 30, 63})
    Bh = random_bcsr(bs, bs, 0.2, seed=92)
    C0 = random_bcsr(bs, bs, 0.1, seed=93)
    return bs, Ah, Bh, C0


@pytest.mark.parametrize("prec,flush", PRECS)
@pytest.mark.parametrize("eps", [0.0, 0.5])
def test_panels_bit_identical(bsm, oracle, operands, prec, flush, eps):
    _, Ah, Bh, _ = operands
    A, B = bsm.Matrix.from_host(Ah), bsm.Matrix.from_host(Bh)
    C1 = bsm.multiply(1.5, A, B, eps=eps, prec=prec, flush_every=flush)
    per_row = _row_products(C1)
    n1 = C1.counts()
    top = int(per_row.max())
    for limit in (top, 3 * top, max(top, int(per_row.sum()) // 3)):
        bsm.set_product_limit(limit)
        try:
            Cp = bsm.multiply(1.5, A, B, eps=eps, prec=prec, flush_every=flush)
        finally:
            bsm.set_product_limit()
        for a, b in zip(Cp.pattern(), C1.pattern()):
            np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(Cp.data_host(), C1.data_host(), err_msg=f"limit {limit}")
        assert Cp.counts() == n1
        assert Cp.products().a.size == 0
        assert len(Cp.stack_shapes()[0]) == 0
    ref = oracle.multiply(1.5, Ah, Bh, eps=eps)
    tol = {"fp64": 1e-12, "fp64_dmma": 1e-12, "ozaki": 1e-12, "bf16x3": 1e-4}.get(prec, 1e-6)
    assert rel_fro(C1.data_host(), ref.C.data) <= tol


@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "ozaki"])
def test_panels_with_beta(bsm, operands, prec):
    _, Ah, Bh, C0 = operands
    A, B = bsm.Matrix.from_host(Ah), bsm.Matrix.from_host(Bh)
    C1 = bsm.multiply(2.0, A, B, -0.5, bsm.Matrix.from_host(C0), eps=0.5, prec=prec)
    limit = int(_row_products(bsm.multiply(2.0, A, B, eps=0.5)).max())
    bsm.set_product_limit(limit)
    try:
        Cp = bsm.multiply(2.0, A, B, -0.5, bsm.Matrix.from_host(C0), eps=0.5, prec=prec)
    finally:
        bsm.set_product_limit()
    np.testing.assert_array_equal(Cp.pattern()[1], C1.pattern()[1])
    np.testing.assert_array_equal(Cp.data_host(), C1.data_host())


def test_chunked_product_holds_no_list(bsm, operands):
    _, Ah, Bh, _ = operands
    import torch
    A, B = bsm.Matrix.from_host(Ah), bsm.Matrix.from_host(Bh)
    limit = int(_row_products(bsm.multiply(1.0, A, B)).max())
    bsm.set_product_limit(limit)
    try:
        Cp = bsm.multiply(1.0, A, B)
        with pytest.raises(bsm.BsmError):
            bsm.multiply(1.0, A, B, 0.0, Cp, no_sync=True)
    finally:
        bsm.set_product_limit()
    G = torch.ones(Cp.info().data_len, dtype=torch.float64, device="cuda")
    dA = torch.zeros(len(Ah.data), dtype=torch.float64, device="cuda")
    with pytest.raises(bsm.BsmError) as e:
        bsm.multiply_backward(1.0, Cp, G, A, B, dA, None)
    assert e.value.status == bsm.BSM_ERR_ARG
    # the same handle takes an unchunked multiply again, with its list
    C1 = bsm.multiply(1.0, A, B, 0.0, Cp)
    assert C1.products().a.size == C1.counts().products
    bsm.multiply_backward(1.0, C1, G, A, B, dA, None)


def test_row_above_limit_refused(bsm, operands):
    _, Ah, Bh, _ = operands
    A, B = bsm.Matrix.from_host(Ah), bsm.Matrix.from_host(Bh)
    top = int(_row_products(bsm.multiply(1.0, A, B)).max())
    Cm = bsm.multiply(1.0, A, B)
    before = Cm.data_host()
    bsm.set_product_limit(top - 1)
    try:
        with pytest.raises(bsm.BsmError) as e:
            bsm.multiply(1.0, A, B, 0.0, Cm)
        assert e.value.status == bsm.BSM_ERR_CAPACITY
    finally:
        bsm.set_product_limit()
    np.testing.assert_array_equal(Cm.data_host(), before)   # C untouched
    with pytest.raises(bsm.BsmError):
        bsm.set_product_limit(0)


def test_panel_engine_falls_back(bsm):
    """The tcgen05 row-panel engine does not take a chunked multiply: the
    mma.sync TF32x3 kernel runs instead, with its result."""
    u = I.large_banded_23(nb=60, occ=0.1, eps=1e-8)
    A, B = bsm.Matrix.from_host(u["A"]), bsm.Matrix.from_host(u["B"])
    Cw = bsm.multiply(1.0, A, B, eps=u["eps"], prec="tf32x3_panel")
    assert Cw.engine() == "panel_tcgen05"
    Cs = bsm.multiply(1.0, A, B, eps=u["eps"], prec="tf32x3")
    bsm.set_product_limit(max(int(_row_products(Cs).max()), Cs.counts().products // 4))
    try:
        Ct = bsm.multiply(1.0, A, B, eps=u["eps"], prec="tf32x3_panel")
    finally:
        bsm.set_product_limit()
    assert Ct.engine() == "split_mma"
    np.testing.assert_array_equal(Ct.data_host(), Cs.data_host())
    assert rel_fro(Ct.data_host(), Cw.data_host()) <= 1e-6
