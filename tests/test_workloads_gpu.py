"""Parity on the five benchmark workloads at their full sizes (GPU).

Where the oracle can run the whole problem in seconds it does (patterns,
product lists and stacks bit-exact, values within tolerance); otherwise it
checks seeded samples of C block rows (the oracle computes them one by one)
and whole-matrix invariants.  These use the same launch configuration as
bench.py (one persistent numeric launch over every block shape).
"""
import numpy as np
import pytest

from paper_1708_03604_gb300 import inputs as I
from tests.helpers import rel_fro

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_03604_gb300 import bsm
    return bsm, torch


def _device_products(bsm, torch, Cm):
    n = Cm.counts().products
    t = torch.empty((3, n), dtype=torch.int32, device="cuda")
    import ctypes
    nn = ctypes.c_int64()
    bsm._sync_stream()
    st = bsm.lib().bsm_get_products(Cm.h, ctypes.byref(nn), t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr())
    assert st == 0
    return t


def _rows_check(bsm, torch, Cm, ref, rows, row_bs, col_bs, tol, prods=None):
    """Pattern, products and values of C block rows `rows` against the
    oracle's row-restricted result."""
    rp, ci, bo = Cm.pattern()
    data = Cm.data_tensor()
    num = den = 0.0
    if prods is None:
        prods = _device_products(bsm, torch, Cm)
    pcs = prods[2]
    for i in rows:
        g0, g1 = int(rp[i]), int(rp[i + 1])
        o0, o1 = int(ref.C.row_ptr[i]), int(ref.C.row_ptr[i + 1])
        np.testing.assert_array_equal(ci[g0:g1], ref.C.col_idx[o0:o1])
        # products of this row: contiguous in canonical order
        lo = int(torch.searchsorted(pcs, torch.tensor([g0], dtype=torch.int32, device="cuda")).item())
        hi = int(torch.searchsorted(pcs, torch.tensor([g1], dtype=torch.int32, device="cuda")).item())
        ro = np.nonzero(np.isin(ref.prods.c, np.arange(o0, o1)))[0]
        np.testing.assert_array_equal(prods[0, lo:hi].cpu().numpy(), ref.prods.a[ro])
        np.testing.assert_array_equal(prods[1, lo:hi].cpu().numpy(), ref.prods.b[ro])
        if g1 > g0:
            end = int(bo[g1 - 1]) + int(row_bs[i]) * int(col_bs[ci[g1 - 1]])
            oend = int(ref.C.blk_off[o1 - 1]) + int(row_bs[i]) * int(col_bs[ref.C.col_idx[o1 - 1]])
            got = data[int(bo[g0]):end].cpu().numpy()
            exp = ref.C.data[int(ref.C.blk_off[o0]):oend]
            num += float(np.sum((got - exp) ** 2))
            den += float(np.sum(exp ** 2))
    assert (num / den) ** 0.5 <= tol


def test_uniform_23_full(env, oracle):
    """200 x 200 blocks of 23 x 23, 20% uniform, no filter: everything."""
    bsm, torch = env
    w = I.uniform_23()
    A, B = bsm.Matrix.from_host(w["A"]), bsm.Matrix.from_host(w["B"])
    ref = oracle.multiply(1.0, w["A"], w["B"])
    for prec, tol in (("ozaki", 1e-13), ("tf32x3", 1e-6), ("tf32x3_panel", 1e-6), ("bf16x6", 1e-6),
                      ("fp64", 1e-12)):
        Cm = bsm.multiply(1.0, A, B, prec=prec)
        if prec == "tf32x3_panel":
            assert Cm.engine() == "panel_tcgen05"
        rp, ci, bo = Cm.pattern()
        np.testing.assert_array_equal(rp, ref.C.row_ptr)
        np.testing.assert_array_equal(ci, ref.C.col_idx)
        np.testing.assert_array_equal(bo, ref.C.blk_off)
        assert rel_fro(Cm.data_host(), ref.C.data) <= tol
    p = Cm.products()
    np.testing.assert_array_equal(p.a, ref.prods.a)
    np.testing.assert_array_equal(p.b, ref.prods.b)
    np.testing.assert_array_equal(p.c, ref.prods.c)
    shapes, ptr, trip = Cm.stacks()
    s_ref, p_ref, t_ref = oracle.stacks(w["A"], w["B"], ref.C, ref.prods)
    np.testing.assert_array_equal(shapes, s_ref)
    np.testing.assert_array_equal(ptr, p_ref)
    np.testing.assert_array_equal(trip, t_ref)


def test_mixed_3000_full_pattern_and_sampled_values(env, oracle):
    """The bench workload: full C pattern, product list and stacks against
    the oracle's symbolic pass; values on 24 seeded C block rows."""
    bsm, torch = env
    w = I.mixed_banded()
    A, B = bsm.Matrix.from_host(w["A"]), bsm.Matrix.from_host(w["B"])
    Cm = bsm.multiply(1.0, A, B, eps=w["eps"])
    sym = oracle.multiply(1.0, w["A"], w["B"], eps=w["eps"], values=False)
    rp, ci, bo = Cm.pattern()
    np.testing.assert_array_equal(rp, sym.C.row_ptr)
    np.testing.assert_array_equal(ci, sym.C.col_idx)
    np.testing.assert_array_equal(bo, sym.C.blk_off)
    cnt = Cm.counts()
    assert (cnt.products, cnt.filtered, cnt.useful_flop) == (len(sym.prods.a), sym.nfiltered, sym.useful_flop)
    prods = _device_products(bsm, torch, Cm)
    for q, ref in enumerate((sym.prods.a, sym.prods.b, sym.prods.c)):
        assert torch.equal(prods[q], torch.tensor(ref, device="cuda"))
    shapes, ptr, trip = Cm.stacks()
    s_ref, p_ref, t_ref = oracle.stacks(w["A"], w["B"], sym.C, sym.prods)
    np.testing.assert_array_equal(shapes, s_ref)
    np.testing.assert_array_equal(ptr, p_ref)
    assert np.array_equal(trip, t_ref)
    del trip, t_ref, sym
    rows = np.sort(np.random.default_rng(11).choice(w["A"].nbr, 24, replace=False))
    ref = oracle.multiply(1.0, w["A"], w["B"], eps=w["eps"], rows=rows)
    _rows_check(bsm, torch, Cm, ref, rows, w["A"].row_bs, w["B"].col_bs, 1e-12, prods)
    for prec, tol in (("ozaki", 1e-13), ("tf32x3", 1e-6), ("bf16x6", 1e-6)):
        Ct = bsm.multiply(1.0, A, B, eps=w["eps"], prec=prec, build_stacks=False)
        _rows_check(bsm, torch, Ct, ref, rows, w["A"].row_bs, w["B"].col_bs, tol)


def test_large_23_sampled_rows(env, oracle):
    """6912 x 6912 blocks of 23 x 23 (H2O-DFT-LS geometry), 5% banded,
    eps = 1e-8: FP64 and split paths on 8 seeded C block rows; whole-matrix
    counts against the closed-form FLOP identity."""
    bsm, torch = env
    w = I.large_banded_23()
    A, B = bsm.Matrix.from_host(w["A"]), bsm.Matrix.from_host(w["B"])
    rows = np.sort(np.random.default_rng(3).choice(w["A"].nbr, 8, replace=False))
    ref = oracle.multiply(1.0, w["A"], w["B"], eps=w["eps"], rows=rows)
    Cm = bsm.multiply(1.0, A, B, eps=w["eps"], build_stacks=False)
    cnt = Cm.counts()
    assert cnt.useful_flop == 2 * 23 ** 3 * cnt.products
    _rows_check(bsm, torch, Cm, ref, rows, w["A"].row_bs, w["B"].col_bs, 1e-12)
    del Cm
    for prec, tol in (("ozaki", 1e-13), ("tf32x3", 1e-6), ("tf32x3_panel", 1e-6), ("bf16x6", 1e-6)):
        Ct = bsm.multiply(1.0, A, B, eps=w["eps"], prec=prec, build_stacks=False)
        assert Ct.counts().products == cnt.products
        if prec == "tf32x3_panel":
            assert Ct.engine() == "panel_tcgen05"
        _rows_check(bsm, torch, Ct, ref, rows, w["A"].row_bs, w["B"].col_bs, tol)
        del Ct


@pytest.mark.parametrize("dtype", ["fp64", "fp32"])
def test_differentiation_13_full(env, oracle, dtype):
    """800 x 800 blocks of 13 x 13, 15% uniform: forward on 16 rows, and
    both adjoints on 64 seeded A blocks / B blocks (the oracle's adjoint over
    exactly the products that touch them)."""
    bsm, torch = env
    npdt = np.float64 if dtype == "fp64" else np.float32
    tdt = torch.float64 if dtype == "fp64" else torch.float32
    w = I.differentiation_13(dtype=npdt)
    A, B = bsm.Matrix.from_host(w["A"]), bsm.Matrix.from_host(w["B"])
    rows = np.sort(np.random.default_rng(5).choice(800, 16, replace=False))
    ref = oracle.multiply(1.0, w["A"], w["B"], rows=rows)
    tol = 1e-12 if dtype == "fp64" else 1e-5
    if dtype == "fp64":  # the Ozaki path: forward rows, then both adjoints below
        Co = bsm.multiply(1.0, A, B, prec="ozaki", build_stacks=False)
        _rows_check(bsm, torch, Co, ref, rows, w["A"].row_bs, w["B"].col_bs, 1e-13)
        del Co
    Cm = bsm.multiply(1.0, A, B, build_stacks=False)
    _rows_check(bsm, torch, Cm, ref, rows, w["A"].row_bs, w["B"].col_bs, tol)
    rp, ci, bo = Cm.pattern()
    C_h = I.BCSR(w["A"].row_bs, w["B"].col_bs, rp, ci, bo, np.zeros(Cm.info().data_len))
    G = np.random.default_rng(8).standard_normal(C_h.data.shape[0])
    dA = torch.empty(len(w["A"].data), dtype=tdt, device="cuda")
    dB = torch.empty(len(w["B"].data), dtype=tdt, device="cuda")
    bsm.multiply_backward(1.0, Cm, torch.tensor(G, dtype=tdt, device="cuda"), A, B, dA, dB)
    outs = [(dA, dB, tol)]
    if dtype == "fp64":
        oA, oB = torch.empty_like(dA), torch.empty_like(dB)
        bsm.multiply_backward(1.0, Cm, torch.tensor(G, dtype=tdt, device="cuda"), A, B, oA, oB, prec="ozaki")
        outs.append((oA, oB, 1e-13))
    p = Cm.products()
    for gA_, gB_, tol_ in outs:
        _adjoint_blocks_check(oracle, w, p, C_h, G, npdt, gA_, gB_, tol_)


def _adjoint_blocks_check(oracle, w, p, C_h, G, npdt, dA, dB, tol):
    rng = np.random.default_rng(6)
    for side, (idx, gout, X) in enumerate(((p.a, dA, w["A"]), (p.b, dB, w["B"]))):
        pick = rng.choice(X.nnzb, 64, replace=False)
        sel = np.nonzero(np.isin(idx, pick))[0]
        sub = type(p)(a=p.a[sel], b=p.b[sel], c=p.c[sel])
        Gd = G.astype(npdt).astype(np.float64)
        rA, rB = oracle.multiply_backward(1.0, w["A"], w["B"], C_h, Gd, sub, want_dA=side == 0,
                                          want_dB=side == 1)
        r = rA if side == 0 else rB
        got = gout.double().cpu().numpy()
        m = np.zeros(len(X.data), dtype=bool)
        rs = X.block_rows()
        for b in pick:
            n = int(X.row_bs[rs[b]]) * int(X.col_bs[X.col_idx[b]])
            m[X.blk_off[b]:X.blk_off[b] + n] = True
        assert rel_fro(got[m], r[m]) <= tol


def test_purification_2000(env, oracle):
    """X0 of 2000 block rows ({4, 1} blocks, 2% banded, Gershgorin-scaled),
    eps = 1e-7: the first 2 steps against the oracle; the graph-captured
    10-step chain replays to its eager result."""
    bsm, torch = env
    from paper_1708_03604_gb300 import chain
    w = I.purification_start(nb=2000)
    X0 = bsm.Matrix.from_host(w["X0"])
    g = chain.McWeenyGraph(X0, 10, w["eps"])
    xs = oracle.mcweeny(w["X0"], 2, w["eps"])
    for k in (1, 2):
        rp, ci, _ = g.X[k].pattern()
        np.testing.assert_array_equal(rp, xs[k].row_ptr)
        np.testing.assert_array_equal(ci, xs[k].col_idx)
        assert rel_fro(g.X[k].data_host(), xs[k].data) <= 1e-12
    eager = g.result.data_host().copy()
    g.replay()
    torch.cuda.synchronize()
    assert g.status() == 0
    np.testing.assert_array_equal(g.result.data_host(), eager)


@pytest.mark.parametrize("s", [4, 32, 45, 78])
def test_square_block_sizes_sweep(env, oracle, s):
    """Uniform s x s blocks over the range of the paper's kernel sweep
    (4..78): several MMA tiles and super-tile passes per block for s > 32."""
    bsm, torch = env
    nb = 24 if s > 40 else 40
    bs = I.uniform_sizes(nb, s)
    Ah = I.assemble(bs, bs, *I.uniform_pattern(nb, nb, 0.25, I.SEED_A), seed=I.SEED_A + 100)
    Bh = I.assemble(bs, bs, *I.uniform_pattern(nb, nb, 0.25, I.SEED_B), seed=I.SEED_B + 100)
    A, B = bsm.Matrix.from_host(Ah), bsm.Matrix.from_host(Bh)
    ref = oracle.multiply(1.0, Ah, Bh)
    for prec, tol in (("fp64", 1e-12), ("ozaki", 1e-13), ("tf32x3", 1e-6), ("bf16x6", 1e-6)):
        Cm = bsm.multiply(1.0, A, B, prec=prec, build_stacks=False)
        rp, ci, bo = Cm.pattern()
        np.testing.assert_array_equal(ci, ref.C.col_idx)
        assert rel_fro(Cm.data_host(), ref.C.data) <= tol, prec
