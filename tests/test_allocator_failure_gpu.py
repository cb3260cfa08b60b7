"""Device-memory provider hooks and the failure paths of the library (GPU).

* The binding installs PyTorch's caching allocator: the library's memory
  shows up in ``torch.cuda.memory_allocated()`` and goes back when the
  handles are destroyed.
* Failure injection on the host: a hook that returns NULL at the n-th
  allocation, for every n a create and a multiply make.  Each call returns
  BSM_ERR_ALLOC, everything it had taken goes back to the hooks, and the
  next call, with a working hook, matches the oracle.
* A bounded device wait that runs out: the tcgen05 row-panel kernel with
  its main-loop wait limit set to 0 gives up at its first wait, every CTA
  drains its copies and tensor-core products and frees its tensor memory,
  the multiply returns BSM_ERR_TIMEOUT, and the next multiplies on the same
  stream (the panel engine again, and the FP64 path) match the oracle.
"""
import gc

import numpy as np
import pytest

from paper_1708_03604_gb300 import inputs as I
from tests.helpers import random_bcsr, rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bsm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_03604_gb300 import bsm as B
    B.lib()
    B.use_torch_allocator()
    yield B
    B.use_torch_allocator()


class FailingHooks:
    """Torch-backed hooks that return NULL at allocation number `fail_at`
    (1-based; 0 = never) and count what is outstanding."""

    def __init__(self, fail_at=0):
        import torch
        self.torch = torch
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}

    def alloc(self, nbytes, stream):
        self.calls += 1
        if self.fail_at and self.calls == self.fail_at:
            return None
        p = self.torch.cuda.caching_allocator_alloc(int(nbytes), self.torch.cuda.current_device(), int(stream or 0))
        self.live[p] = nbytes
        return p

    def free(self, ptr, nbytes, stream):
        assert self.live.pop(ptr) == nbytes
        self.torch.cuda.caching_allocator_delete(ptr)


def test_torch_allocator_holds_library_memory(bsm, oracle):
    import torch
    torch.cuda.synchronize()
    gc.collect()
    base_out = bsm.allocator_outstanding()
    base = torch.cuda.memory_allocated()
    w = I.uniform_23(nb=60, occ=0.2)
    A, B = bsm.Matrix.from_host(w["A"]), bsm.Matrix.from_host(w["B"])
    data_ab = 8 * (len(w["A"].data) + len(w["B"].data))
    assert torch.cuda.memory_allocated() - base >= data_ab
    Cm = bsm.multiply(1.0, A, B)
    torch.cuda.synchronize()
    ref = oracle.multiply(1.0, w["A"], w["B"])
    assert torch.cuda.memory_allocated() - base >= data_ab + 8 * ref.C.data_len
    assert rel_fro(Cm.data_host(), ref.C.data) <= 1e-12
    assert bsm.allocator_outstanding() > base_out
    del A, B, Cm
    gc.collect()
    torch.cuda.synchronize()
    assert bsm.allocator_outstanding() == base_out
    assert torch.cuda.memory_allocated() == base


def test_allocation_failure_at_every_point(bsm, oracle):
    import torch
    bs = I.mixed_sizes(40, (5, 13, 23), (0.5, 0.3, 0.2), seed=9)
    Ah, Bh = random_bcsr(bs, bs, 0.15, seed=81), random_bcsr(bs, bs, 0.15, seed=82)
    ref = oracle.multiply(1.0, Ah, Bh, eps=0.5)
    gc.collect()
    base_out = bsm.allocator_outstanding()
    # how many allocations one create + multiply makes, with a working hook
    h = FailingHooks()
    bsm.set_allocator(h.alloc, h.free)
    try:
        A, B = bsm.Matrix.from_host(Ah), bsm.Matrix.from_host(Bh)
        n_create = h.calls
        Cm = bsm.multiply(1.0, A, B, eps=0.5, prec="tf32x3")
        n_total = h.calls
        del A, B, Cm
        gc.collect()
        torch.cuda.synchronize()
        assert not h.live
        assert n_create >= 8 and n_total > n_create
        # a NULL from the hook at each point in turn
        for k in range(1, n_total + 1):
            h = FailingHooks(fail_at=k)
            bsm.set_allocator(h.alloc, h.free)
            made = []
            with pytest.raises(bsm.BsmError) as e:
                made.append(bsm.Matrix.from_host(Ah))
                made.append(bsm.Matrix.from_host(Bh))
                made.append(bsm.multiply(1.0, made[0], made[1], eps=0.5, prec="tf32x3"))
            status, msg = e.value.status, str(e.value)
            del made, e               # the traceback holds the failed call's frames
            gc.collect()
            assert status == bsm.BSM_ERR_ALLOC, (k, msg)
            torch.cuda.synchronize()
            assert not h.live, (k, len(h.live))       # nothing taken is kept
    finally:
        bsm.use_torch_allocator()
    assert bsm.allocator_outstanding() == base_out
    # the next call works and is right
    A, B = bsm.Matrix.from_host(Ah), bsm.Matrix.from_host(Bh)
    Cm = bsm.multiply(1.0, A, B, eps=0.5, prec="tf32x3")
    np.testing.assert_array_equal(Cm.pattern()[1], ref.C.col_idx)
    assert rel_fro(Cm.data_host(), ref.C.data) <= 1e-6


def test_builtin_pool_still_works(bsm, oracle):
    w = I.uniform_23(nb=30, occ=0.2)
    bsm.set_allocator()          # back to the library's own stream-ordered pool
    try:
        A, B = bsm.Matrix.from_host(w["A"]), bsm.Matrix.from_host(w["B"])
        out0 = bsm.allocator_outstanding()
        Cm = bsm.multiply(1.0, A, B)
        assert bsm.allocator_outstanding() == out0
        ref = oracle.multiply(1.0, w["A"], w["B"])
        assert rel_fro(Cm.data_host(), ref.C.data) <= 1e-12
        del A, B, Cm
        gc.collect()
    finally:
        bsm.use_torch_allocator()


def test_panel_wait_runs_out_then_recovers(bsm, oracle):
    import torch
    u = I.large_banded_23(nb=60, occ=0.1, eps=1e-8)
    A, B = bsm.Matrix.from_host(u["A"]), bsm.Matrix.from_host(u["B"])
    ref = oracle.multiply(1.0, u["A"], u["B"], eps=u["eps"])
    Cm = bsm.Matrix.empty(u["A"].row_bs, u["B"].col_bs)
    bsm._check(bsm.lib().bsm_set_wait_limit(0.0))
    try:
        with pytest.raises(bsm.BsmError) as e:
            bsm.multiply(1.0, A, B, 0.0, Cm, u["eps"], prec="tf32x3_panel")
        assert e.value.status == bsm.BSM_ERR_TIMEOUT
    finally:
        bsm._check(bsm.lib().bsm_set_wait_limit(2.0))
    torch.cuda.synchronize()          # the context is still usable
    # the tensor memory was freed: the engine runs again on every SM
    Cp = bsm.multiply(1.0, A, B, 0.0, Cm, u["eps"], prec="tf32x3_panel")
    assert Cp.engine() == "panel_tcgen05"
    np.testing.assert_array_equal(Cp.pattern()[1], ref.C.col_idx)
    assert rel_fro(Cp.data_host(), ref.C.data) <= 1e-6
    Cf = bsm.multiply(1.0, A, B, eps=u["eps"])
    assert rel_fro(Cf.data_host(), ref.C.data) <= 1e-12
    with pytest.raises(bsm.BsmError):
        bsm._check(bsm.lib().bsm_set_wait_limit(3.0))
