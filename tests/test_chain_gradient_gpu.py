"""The purification workload's gradient (GPU): trace(X_10 . W) with respect
to X_0 through the 10-step McWeeny chain X <- 3X^2 - 2X^3, every multiply
and add filtered at eps = 1e-7.

* 2000 x 2000 blocks of 4 x 4 and 1 x 1 (the chain's reduced size): the
  gradient with checkpoints every 2 steps (each 2-step segment recomputed in
  backward) equals the gradient that keeps every intermediate, bit for bit,
  and so does the loss; the first forward iterates match the oracle's
  (patterns bit for bit, values within 1e-12).
* 200 x 200 blocks: the checkpointed 10-step gradient of the unfiltered
  chain (eps = 0, so no keep-decision can flip under a perturbation) matches
  central finite differences along seeded directions.  With eps = 1e-7 the
  10-step chain holds so many block norms near eps that every tested
  perturbation flips some decision; the filtered gradient is checked against
  finite differences over 4 steps in test_autograd_gpu.py.
"""
import numpy as np
import pytest

from paper_1708_03604_gb300 import inputs as I
from tests.helpers import rel_fro

pytestmark = pytest.mark.gpu

STEPS = 10


@pytest.fixture(scope="module")
def ag():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_03604_gb300 import autograd as A
    return A


def _loss(ag, x0h, Wt, eps, ckpt):
    X0 = ag.BlockSparseTensor.from_bcsr(x0h, requires_grad=True)
    Xk = ag.mcweeny(X0, STEPS, eps, checkpoint_every=ckpt)
    return ag.trace_product(Xk, Wt), X0, Xk


def _signature(ag, x0h, eps):
    """Keep decisions of every step of the chain (no autograd)."""
    sig = []
    X = ag.BlockSparseTensor.from_bcsr(x0h)
    for _ in range(STEPS):
        X2 = ag.matmul(X, X, eps=eps)
        X3 = ag.matmul(X2, X, eps=eps)
        X = ag.add(X2, X3, 3.0, -2.0, eps=eps)
        sig.append((X2.handle.counts().products, X2.handle.counts().filtered, X3.handle.counts().products,
                    X3.handle.counts().filtered, X.handle.nnzb))
    return X, sig


def test_gradient_10_steps_nb2000_checkpointed_equals_plain(ag, oracle):
    import torch
    w = I.purification_start(nb=2000)
    eps = w["eps"]
    Wt = ag.BlockSparseTensor.from_bcsr(w["W"])
    l2, X2, Xk2 = _loss(ag, w["X0"], Wt, eps, 2)
    l2.backward()
    g2 = X2.data.grad.clone()
    nnz_last = Xk2.handle.nnzb
    del X2, Xk2
    torch.cuda.empty_cache()
    l1, X1, Xk1 = _loss(ag, w["X0"], Wt, eps, 0)
    l1.backward()
    assert l1.item() == l2.item()
    assert Xk1.handle.nnzb == nnz_last
    torch.testing.assert_close(X1.data.grad, g2, rtol=0, atol=0)
    assert torch.isfinite(g2).all() and float(g2.abs().max()) > 0
    # the chain grows the pattern (fill-in) over the 10 steps
    assert nnz_last > 5 * w["X0"].nnzb
    del X1, Xk1
    torch.cuda.empty_cache()
    # the first forward iterates against the oracle
    xs = oracle.mcweeny(w["X0"], 2, eps)
    X = ag.BlockSparseTensor.from_bcsr(w["X0"])
    with torch.no_grad():
        for k in (1, 2):
            X = ag.mcweeny_step(X, eps)
            g = X.to_host()
            np.testing.assert_array_equal(g.row_ptr, xs[k].row_ptr)
            np.testing.assert_array_equal(g.col_idx, xs[k].col_idx)
            assert rel_fro(g.data, xs[k].data) <= 1e-12, k


def test_gradient_10_steps_nb200_vs_finite_differences(ag):
    import torch
    w = I.purification_start(nb=200)
    eps = 0.0
    Wt = ag.BlockSparseTensor.from_bcsr(w["W"])
    loss, X0, _ = _loss(ag, w["X0"], Wt, eps, 2)
    loss.backward()
    grad = X0.data.grad.cpu().numpy()
    with torch.no_grad():
        _, base = _signature(ag, w["X0"], eps)
    rng = np.random.default_rng(7)
    h = 1e-6
    an, fd, skipped = [], [], 0
    for _ in range(16):
        v = rng.standard_normal(len(w["X0"].data))
        vals, same = [], True
        for sgn in (1.0, -1.0):
            xh = I.BCSR(w["X0"].row_bs, w["X0"].col_bs, w["X0"].row_ptr, w["X0"].col_idx, w["X0"].blk_off,
                        w["X0"].data + sgn * h * v)
            with torch.no_grad():
                Xk, sig = _signature(ag, xh, eps)
                vals.append(ag.trace_product(Xk, Wt).item())
            same = same and sig == base
        if not same:
            skipped += 1
            continue
        fd.append((vals[0] - vals[1]) / (2 * h))
        an.append(float((grad * v).sum()))
    assert len(fd) >= 4, skipped
    an, fd = np.array(an), np.array(fd)
    assert np.linalg.norm(an - fd) / np.linalg.norm(fd) <= 1e-6
