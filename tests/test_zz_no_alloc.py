"""The allocation-free sizing entry point, bsm_count_products_static.

It exists for callers that must not allocate device memory while they size
a product (code inside another framework's pool or arena, host threads that
may not call cudaMalloc/cudaFree).  Its scratch is a fixed array inside the
library; this test checks, through the C ABI, that two calls in a row agree
exactly with what bsm_multiply (which allocates) reports for the same
operands, and that sizes above the fixed capacity are refused.  The file is
named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_1708_03604_gb300 import inputs as I
from tests.helpers import random_bcsr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bsm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_03604_gb300 import bsm as B
    B.lib()
    return B


def _static_counts(bsm, A, B, eps):
    import torch
    nbr = A.info().nbr
    prod = torch.full((nbr,), -1, dtype=torch.int64, device="cuda")
    cblk = torch.full((nbr,), -1, dtype=torch.int64, device="cuda")
    tot = torch.full((3,), -1, dtype=torch.int64, device="cuda")
    bsm._sync_stream()
    st = bsm.lib().bsm_count_products_static(A.h, B.h, float(eps), ctypes.c_void_p(prod.data_ptr()),
                                              ctypes.c_void_p(cblk.data_ptr()), ctypes.c_void_p(tot.data_ptr()))
    assert st == bsm.BSM_OK, bsm.lib().bsm_last_error()
    torch.cuda.synchronize()
    return prod.cpu().numpy(), cblk.cpu().numpy(), tot.cpu().numpy()


def _reference_counts(bsm, A, B, eps):
    Cm = bsm.multiply(1.0, A, B, eps=eps)
    rp, _, _ = Cm.pattern()
    p = Cm.products()
    crow = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    prod = np.bincount(crow[p.c], minlength=len(rp) - 1) if len(p.c) else np.zeros(len(rp) - 1, np.int64)
    cnt = Cm.counts()
    return prod, np.diff(rp), (cnt.products, cnt.filtered, cnt.useful_flop / 2)


def test_static_count_matches_multiply_twice(bsm):
    w = I.mixed_banded(nb=240, occ=0.1, eps=1.0, decay=8.0)
    A, B = bsm.Matrix.from_host(w["A"]), bsm.Matrix.from_host(w["B"])
    for eps in (1.0, 0.3):      # two calls in a row; the scratch keeps the last call's norms
        prod, cblk, tot = _static_counts(bsm, A, B, eps)
        rprod, rcblk, rtot = _reference_counts(bsm, A, B, eps)
        np.testing.assert_array_equal(prod, rprod)
        np.testing.assert_array_equal(cblk, rcblk)
        assert tuple(int(x) for x in tot) == tuple(int(x) for x in rtot)
        assert tot[1] > 0


def test_static_count_unfiltered_and_square(bsm):
    bs = I.mixed_sizes(50, (2, 5), (0.5, 0.5), seed=4)
    X = bsm.Matrix.from_host(random_bcsr(bs, bs, 0.2, seed=90))
    for _ in range(2):
        prod, cblk, tot = _static_counts(bsm, X, X, 0.0)
        rprod, rcblk, rtot = _reference_counts(bsm, X, X, 0.0)
        np.testing.assert_array_equal(prod, rprod)
        np.testing.assert_array_equal(cblk, rcblk)
        assert tuple(int(x) for x in tot) == tuple(int(x) for x in rtot)


def test_static_count_rejects_sizes_above_capacity(bsm):
    bs = I.uniform_sizes(1100, 1)             # 1.21M blocks per matrix, 2.42M together
    rows, cols = np.divmod(np.arange(1100 * 1100), 1100)
    Xh = I.assemble(bs, bs, rows, cols, None, seed=3)
    X = bsm.Matrix.from_host(Xh)
    Y = bsm.Matrix.from_host(Xh)
    import torch
    buf = torch.zeros(2 * 1100 + 3, dtype=torch.int64, device="cuda")
    st = bsm.lib().bsm_count_products_static(X.h, Y.h, 1e-3, ctypes.c_void_p(buf.data_ptr()),
                                              ctypes.c_void_p(buf.data_ptr() + 8 * 1100),
                                              ctypes.c_void_p(buf.data_ptr() + 16 * 1100))
    assert st == bsm.BSM_ERR_CAPACITY
    assert b"2097152" in bsm.lib().bsm_last_error()
    assert int(buf.abs().sum().item()) == 0      # refused before any device work


def test_static_count_allocates_nothing(bsm):
    """The property the entry point exists for: after one warm-up call (which
    loads the kernel and looks the array up), further filtered calls take no
    memory from the installed allocator hooks and leave the device's free
    memory unchanged."""
    import torch
    w = I.mixed_banded(nb=240, occ=0.1, eps=1.0, decay=8.0)
    A, B = bsm.Matrix.from_host(w["A"]), bsm.Matrix.from_host(w["B"])
    nbr = A.info().nbr
    out = torch.zeros(2 * nbr + 3, dtype=torch.int64, device="cuda")
    calls = []

    def alloc(n, s):
        calls.append(n)
        return torch.cuda.caching_allocator_alloc(int(n), torch.cuda.current_device(), int(s or 0))

    def free(p, n, s):
        torch.cuda.caching_allocator_delete(p)

    args = (A.h, B.h, 1.0, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(out.data_ptr() + 8 * nbr),
            ctypes.c_void_p(out.data_ptr() + 16 * nbr))
    bsm._sync_stream()
    assert bsm.lib().bsm_count_products_static(*args) == bsm.BSM_OK
    torch.cuda.synchronize()
    bsm.set_allocator(alloc, free)
    try:
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(3):
            assert bsm.lib().bsm_count_products_static(*args) == bsm.BSM_OK
        torch.cuda.synchronize()
        assert calls == []
        assert torch.cuda.mem_get_info()[0] == free0
    finally:
        bsm.use_torch_allocator()
