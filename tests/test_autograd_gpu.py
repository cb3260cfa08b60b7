"""Differentiation through the block-sparse multiply and the purification
chain, on the GPU: hand-written adjoints against dense torch autograd,
central finite differences and the CPU oracle's adjoint."""
import numpy as np
import pytest

from paper_1708_03604_gb300 import inputs as I
from tests.helpers import block_mask, rel_fro, to_dense

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ag():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_03604_gb300 import autograd as A
    return A


def _sq_loss(ag, A, B, T):
    """||A.B - T||_F^2 summed over the union of C's and T's patterns."""
    import torch
    Cm = ag.matmul(A, B)
    ic, it = ag.block_pair_index(Cm, T)
    cross = (Cm.data[ic] * T.data[it]).sum()
    return (Cm.data ** 2).sum() - 2 * cross + (T.data ** 2).sum(), Cm


def test_matmul_grad_vs_dense_autograd(ag):
    import torch
    w = I.differentiation_13(nb=40, occ=0.15)
    A = ag.BlockSparseTensor.from_bcsr(w["A"], requires_grad=True)
    B = ag.BlockSparseTensor.from_bcsr(w["B"], requires_grad=True)
    T = ag.BlockSparseTensor.from_bcsr(w["T"])
    loss, _ = _sq_loss(ag, A, B, T)
    loss.backward()
    Ad = torch.tensor(to_dense(w["A"]), requires_grad=True)
    Bd = torch.tensor(to_dense(w["B"]), requires_grad=True)
    ld = ((Ad @ Bd - torch.tensor(to_dense(w["T"]))) ** 2).sum()
    ld.backward()
    assert abs(loss.item() - ld.item()) <= 1e-12 * abs(ld.item())
    gA = to_dense(type(w["A"])(w["A"].row_bs, w["A"].col_bs, w["A"].row_ptr, w["A"].col_idx, w["A"].blk_off,
                               A.data.grad.cpu().numpy()))
    gB = to_dense(type(w["B"])(w["B"].row_bs, w["B"].col_bs, w["B"].row_ptr, w["B"].col_idx, w["B"].blk_off,
                               B.data.grad.cpu().numpy()))
    assert rel_fro(gA, Ad.grad.numpy() * block_mask(w["A"])) <= 1e-12
    assert rel_fro(gB, Bd.grad.numpy() * block_mask(w["B"])) <= 1e-12


def test_matmul_grad_central_fd(ag):
    """32 directional derivatives along random directions on A's and B's
    patterns, central differences with h = 1e-6 (FP64)."""
    import torch
    w = I.differentiation_13(nb=40, occ=0.15)
    A = ag.BlockSparseTensor.from_bcsr(w["A"], requires_grad=True)
    B = ag.BlockSparseTensor.from_bcsr(w["B"], requires_grad=True)
    T = ag.BlockSparseTensor.from_bcsr(w["T"])
    loss, _ = _sq_loss(ag, A, B, T)
    loss.backward()
    ga, gb = A.data.grad.clone(), B.data.grad.clone()
    rng = np.random.default_rng(9)
    h = 1e-6
    an, fd = [], []
    with torch.no_grad():
        a0, b0 = A.data.detach().clone(), B.data.detach().clone()
        for _ in range(32):
            va = torch.tensor(rng.standard_normal(a0.numel()), device="cuda")
            vb = torch.tensor(rng.standard_normal(b0.numel()), device="cuda")
            vals = []
            for s in (1.0, -1.0):
                A.data.copy_(a0 + s * h * va)
                B.data.copy_(b0 + s * h * vb)
                vals.append(_sq_loss(ag, A, B, T)[0].item())
            fd.append((vals[0] - vals[1]) / (2 * h))
            an.append(float((ga * va).sum() + (gb * vb).sum()))
        A.data.copy_(a0)
        B.data.copy_(b0)
    an, fd = np.array(an), np.array(fd)
    bound = np.finfo(np.float64).eps * abs(loss.item()) / h       # rounding bound of the FD quotient
    err = np.linalg.norm(an - fd) / np.linalg.norm(fd)
    assert err <= 1e-6, (err, bound)


def test_ozaki_grad_vs_dense_autograd(ag):
    """The differentiable multiply on the Ozaki path: loss and gradients against
    dense torch autograd in FP64 (FP64-class agreement)."""
    import torch
    w = I.differentiation_13(nb=40, occ=0.15)
    A = ag.BlockSparseTensor.from_bcsr(w["A"], requires_grad=True)
    B = ag.BlockSparseTensor.from_bcsr(w["B"], requires_grad=True)
    Cm = ag.matmul(A, B, prec="ozaki")
    T = ag.BlockSparseTensor.from_bcsr(w["T"])
    ic, it = ag.block_pair_index(Cm, T)
    loss = (Cm.data ** 2).sum() - 2 * (Cm.data[ic] * T.data[it]).sum() + (T.data ** 2).sum()
    loss.backward()
    Ad = torch.tensor(to_dense(w["A"]), requires_grad=True)
    Bd = torch.tensor(to_dense(w["B"]), requires_grad=True)
    ld = ((Ad @ Bd - torch.tensor(to_dense(w["T"]))) ** 2).sum()
    ld.backward()
    assert abs(loss.item() - ld.item()) <= 1e-12 * abs(ld.item())
    gA = to_dense(type(w["A"])(w["A"].row_bs, w["A"].col_bs, w["A"].row_ptr, w["A"].col_idx, w["A"].blk_off,
                               A.data.grad.cpu().numpy()))
    assert rel_fro(gA, Ad.grad.numpy() * block_mask(w["A"])) <= 1e-12


def test_fp32_grad_vs_dense(ag):
    import torch
    w = I.differentiation_13(nb=30, occ=0.15)
    A = ag.BlockSparseTensor.from_bcsr(w["A"], requires_grad=True, dtype=torch.float32)
    B = ag.BlockSparseTensor.from_bcsr(w["B"], requires_grad=True, dtype=torch.float32)
    T = ag.BlockSparseTensor.from_bcsr(w["T"], dtype=torch.float32)
    loss, _ = _sq_loss(ag, A, B, T)
    loss.backward()
    Ad = torch.tensor(to_dense(w["A"]), requires_grad=True)
    Bd = torch.tensor(to_dense(w["B"]), requires_grad=True)
    ((Ad @ Bd - torch.tensor(to_dense(w["T"]))) ** 2).sum().backward()
    gA = to_dense(type(w["A"])(w["A"].row_bs, w["A"].col_bs, w["A"].row_ptr, w["A"].col_idx, w["A"].blk_off,
                               A.data.grad.double().cpu().numpy()))
    assert rel_fro(gA, Ad.grad.numpy() * block_mask(w["A"])) <= 1e-5


@pytest.mark.parametrize("prec", ["fp64", "ozaki", "tf32x3", "bf16x6"])
def test_backward_vs_oracle_13(ag, oracle, prec):
    import torch
    from paper_1708_03604_gb300 import bsm
    w = I.differentiation_13(nb=300, occ=0.15)
    A, B = bsm.Matrix.from_host(w["A"]), bsm.Matrix.from_host(w["B"])
    Cm = bsm.multiply(1.0, A, B)
    ref = oracle.multiply(1.0, w["A"], w["B"])
    G = np.random.default_rng(4).standard_normal(ref.C.data_len)
    dA_ref, dB_ref = oracle.multiply_backward(1.0, w["A"], w["B"], ref.C, G, ref.prods)
    dA = torch.empty(len(w["A"].data), dtype=torch.float64, device="cuda")
    dB = torch.empty(len(w["B"].data), dtype=torch.float64, device="cuda")
    bsm.multiply_backward(1.0, Cm, torch.tensor(G, device="cuda"), A, B, dA, dB, prec=prec)
    tol = {"fp64": 1e-12, "ozaki": 1e-13}.get(prec, 1e-6)
    assert rel_fro(dA.cpu().numpy(), dA_ref) <= tol
    assert rel_fro(dB.cpu().numpy(), dB_ref) <= tol


def test_add_grad_vs_dense(ag):
    import torch
    bs = I.mixed_sizes(20, (1, 4), (0.5, 0.5), seed=3)
    from tests.helpers import random_bcsr
    Xh, Yh = random_bcsr(bs, bs, 0.3, seed=5), random_bcsr(bs, bs, 0.3, seed=6)
    X = ag.BlockSparseTensor.from_bcsr(Xh, requires_grad=True)
    Y = ag.BlockSparseTensor.from_bcsr(Yh, requires_grad=True)
    Z = ag.add(X, Y, 3.0, -2.0)
    (Z.data ** 3).sum().backward()
    Xd = torch.tensor(to_dense(Xh), requires_grad=True)
    Yd = torch.tensor(to_dense(Yh), requires_grad=True)
    ((3 * Xd - 2 * Yd) ** 3).sum().backward()
    gX = to_dense(type(Xh)(Xh.row_bs, Xh.col_bs, Xh.row_ptr, Xh.col_idx, Xh.blk_off, X.data.grad.cpu().numpy()))
    assert rel_fro(gX, Xd.grad.numpy() * block_mask(Xh)) <= 1e-14


def _chain_oracle_close(oracle, X0h, steps, eps, got):
    xs = oracle.mcweeny(X0h, steps, eps)
    ref = xs[-1]
    g = got.to_host()
    return ref, g


def test_mcweeny_chain_vs_oracle(ag, oracle):
    w = I.purification_start(nb=200)
    X0 = ag.BlockSparseTensor.from_bcsr(w["X0"])
    X = X0
    xs_ref = oracle.mcweeny(w["X0"], 10, w["eps"])
    for k in range(1, 11):
        X = ag.mcweeny_step(X, w["eps"])
        g = X.to_host()
        r = xs_ref[k]
        np.testing.assert_array_equal(g.row_ptr, r.row_ptr)
        np.testing.assert_array_equal(g.col_idx, r.col_idx)
        assert rel_fro(g.data, r.data) <= 1e-12, k
    # fill-in grows and the iterate moves towards an idempotent matrix
    assert xs_ref[-1].nnzb > w["X0"].nnzb


def _chain_signature(ag, X0, steps, eps):
    """Forward chain without autograd; returns the loss inputs and the keep
    decisions of every step (kept products of both multiplies, blocks of X)."""
    sig = []
    X = X0
    for _ in range(steps):
        X2 = ag.matmul(X, X, eps=eps)
        X3 = ag.matmul(X2, X, eps=eps)
        X = ag.add(X2, X3, 3.0, -2.0, eps=eps)
        sig.append((X2.handle.counts().products, X2.handle.counts().filtered, X3.handle.counts().products,
                    X3.handle.counts().filtered, X.handle.nnzb))
    return X, sig


@pytest.mark.parametrize("eps_kind", ["unfiltered", "filtered"])
def test_mcweeny_gradient_checkpointed(ag, eps_kind):
    """grad of trace(X_k.W) w.r.t. X0: checkpointing every 2 steps gives the
    same gradient as keeping every intermediate, and it matches central
    finite differences along directions whose +-h steps keep every filter
    decision of the chain (the gradient is taken at fixed keep-decisions)."""
    import torch
    w = I.purification_start(nb=120)
    steps = 4
    eps = 0.0 if eps_kind == "unfiltered" else w["eps"]
    Wt = ag.BlockSparseTensor.from_bcsr(w["W"])

    def loss_of(x0h, ckpt):
        X0 = ag.BlockSparseTensor.from_bcsr(x0h, requires_grad=True)
        Xk = ag.mcweeny(X0, steps, eps, checkpoint_every=ckpt)
        return ag.trace_product(Xk, Wt), X0

    l1, X1 = loss_of(w["X0"], 0)
    l1.backward()
    l2, X2 = loss_of(w["X0"], 2)
    l2.backward()
    assert l1.item() == l2.item()
    torch.testing.assert_close(X1.data.grad, X2.data.grad, rtol=0, atol=0)
    grad = X1.data.grad.cpu().numpy()
    with torch.no_grad():
        _, base_sig = _chain_signature(ag, ag.BlockSparseTensor.from_bcsr(w["X0"]), steps, eps)
    rng = np.random.default_rng(1)
    # a smaller step where the chain filters: fewer near-threshold decisions flip
    h = 1e-6 if eps == 0.0 else 1e-8
    an, fd, skipped = [], [], 0
    for _ in range(12):
        v = rng.standard_normal(len(w["X0"].data))
        vals, same = [], True
        for sgn in (1.0, -1.0):
            xh = I.BCSR(w["X0"].row_bs, w["X0"].col_bs, w["X0"].row_ptr, w["X0"].col_idx, w["X0"].blk_off,
                        w["X0"].data + sgn * h * v)
            with torch.no_grad():
                Xk, sig = _chain_signature(ag, ag.BlockSparseTensor.from_bcsr(xh), steps, eps)
                vals.append(ag.trace_product(Xk, Wt).item())
            same = same and sig == base_sig
        if not same:
            skipped += 1
            continue
        fd.append((vals[0] - vals[1]) / (2 * h))
        an.append(float((grad * v).sum()))
    assert len(fd) >= 4, skipped
    an, fd = np.array(an), np.array(fd)
    assert np.linalg.norm(an - fd) / np.linalg.norm(fd) <= 1e-6
