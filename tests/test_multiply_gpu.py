"""GPU parity of the block-sparse multiply against the CPU oracle.

Integer results (C's pattern, the product list, the stacks, the filter
decisions) must match bit for bit; FP64 values within a relative Frobenius
error of 1e-12 (the accumulation order inside a block product differs from
the oracle's naive loop), split-precision values within 1e-6 (TF32x3,
BF16x6), FP32 data within 1e-5 of the FP64 oracle.
"""
import numpy as np
import pytest

from paper_1708_03604_gb300 import inputs as I
from tests.helpers import random_bcsr, rel_fro

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "tf32x3": 1e-6, "bf16x6": 1e-6, "bf16x3": 1e-4}


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


def _run(bsm, oracle, A, B, eps, prec="fp64", beta=0.0, C0=None, alpha=1.0, **kw):
    dA, dB = bsm.Matrix.from_host(A), (bsm.Matrix.from_host(B) if B is not A else None)
    dB = dB or dA
    Cg = bsm.Matrix.from_host(C0) if C0 is not None else None
    Cg = bsm.multiply(alpha, dA, dB, beta=beta, Cm=Cg, eps=eps, prec=prec, **kw)
    ref = oracle.multiply(alpha, A, B, beta=beta, Cold=C0, eps=eps)
    return Cg, ref, dA, dB


def test_norms_bitexact(bsm, oracle):
    bs = I.mixed_sizes(70, (1, 5, 13, 23, 40), (0.2, 0.3, 0.2, 0.2, 0.1), seed=3)
    X = random_bcsr(bs, bs, 0.2, seed=11)
    g = bsm.Matrix.from_host(X).block_norms()
    np.testing.assert_array_equal(g, oracle.block_norms(X))
    X32 = X.astype(np.float32)
    g32 = bsm.Matrix.from_host(X32).block_norms()
    np.testing.assert_array_equal(g32, oracle.block_norms(X32))


@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "bf16x6", "bf16x3"])
def test_uniform_23_small(bsm, oracle, prec):
    w = I.uniform_23(nb=40, occ=0.2)
    Cg, ref, _, _ = _run(bsm, oracle, w["A"], w["B"], 0.0, prec=prec)
    _check_pattern(Cg, ref.C)
    err = rel_fro(Cg.data_host(), ref.C.data)
    assert err <= TOL[prec], err
    p = Cg.products()
    np.testing.assert_array_equal(p.a, ref.prods.a)
    np.testing.assert_array_equal(p.b, ref.prods.b)
    np.testing.assert_array_equal(p.c, ref.prods.c)
    cnt = Cg.counts()
    assert cnt.products == len(ref.prods.a)
    assert cnt.useful_flop == ref.useful_flop


@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "bf16x6"])
def test_mixed_banded_filtered(bsm, oracle, prec):
    # banded-then-permuted, sizes {5, 13, 23}, a threshold that filters a
    # good share of the candidate products
    w = I.mixed_banded(nb=240, occ=0.1, eps=1.0, decay=8.0)
    Cg, ref, _, _ = _run(bsm, oracle, w["A"], w["B"], w["eps"], prec=prec)
    assert ref.nfiltered > 0
    _check_pattern(Cg, ref.C)
    cnt = Cg.counts()
    assert (cnt.products, cnt.filtered) == (len(ref.prods.a), ref.nfiltered)
    err = rel_fro(Cg.data_host(), ref.C.data)
    assert err <= TOL[prec], err
    shapes, ptr, trip = Cg.stacks()
    s_ref, p_ref, t_ref = oracle.stacks(w["A"], w["B"], ref.C, ref.prods)
    np.testing.assert_array_equal(shapes, s_ref)
    np.testing.assert_array_equal(ptr, p_ref)
    np.testing.assert_array_equal(trip, t_ref)


@pytest.mark.parametrize("prec,flush", [("tf32x3", 1), ("tf32x3", 4), ("bf16x6", 2)])
def test_split_with_fp64_sum(bsm, oracle, prec, flush):
    # cross-product sum in FP64, refreshed every `flush` block products
    w = I.mixed_banded(nb=200, occ=0.1, eps=1e-6)
    Cg, ref, _, _ = _run(bsm, oracle, w["A"], w["B"], w["eps"], prec=prec, flush_every=flush)
    _check_pattern(Cg, ref.C)
    assert rel_fro(Cg.data_host(), ref.C.data) <= TOL[prec]


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x6", "bf16x3"])
def test_cuda_core_split_variant(bsm, oracle, prec):
    """Tiny output shapes on the CUDA-core (lane per block) variant of the
    split arithmetic, larger ones on the tensor cores, in one launch."""
    rng = np.random.default_rng(2)
    bs = rng.integers(1, 9, size=60).astype(np.int32)
    A, B = random_bcsr(bs, bs, 0.2, seed=141), random_bcsr(bs, bs, 0.2, seed=142)
    sizes = sorted(set(int(x) for x in bs))
    try:
        for m in sizes:
            for n in sizes:
                bsm.bsm_set_variant(prec, m, n, 1)
        for fl in (0, 1):
            Cg, ref, gA, gB = _run(bsm, oracle, A, B, 0.0, prec=prec, flush_every=fl)
            _check_pattern(Cg, ref.C)
            assert rel_fro(Cg.data_host(), ref.C.data) <= TOL[prec]
        # adjoints through the same variant
        import torch
        G = np.random.default_rng(3).standard_normal(ref.C.data_len)
        dA_ref, dB_ref = oracle.multiply_backward(1.0, A, B, ref.C, G, ref.prods)
        dA = torch.empty(len(A.data), dtype=torch.float64, device="cuda")
        dB = torch.empty(len(B.data), dtype=torch.float64, device="cuda")
        bsm.multiply_backward(1.0, Cg, torch.tensor(G, device="cuda"), gA, gB, dA, dB, prec=prec)
        assert rel_fro(dA.cpu().numpy(), dA_ref) <= TOL[prec]
        assert rel_fro(dB.cpu().numpy(), dB_ref) <= TOL[prec]
    finally:
        for m in sizes:
            for n in sizes:
                bsm.bsm_set_variant(prec, m, n, -1)


@pytest.mark.parametrize("variant", [0, 1])
def test_fp64_tiny_blocks_both_variants(bsm, oracle, variant):
    """Blocks of 1, 2, 4, 5 and 6 rows/columns: one warp per output block (0)
    or one lane per output block (1, where eligible), forward and adjoints,
    against the oracle."""
    import torch
    bs = I.mixed_sizes(120, (1, 2, 4, 5, 6), (0.3, 0.2, 0.2, 0.15, 0.15), seed=5)
    A, B = random_bcsr(bs, bs, 0.1, seed=151), random_bcsr(bs, bs, 0.1, seed=152)
    sz = (1, 2, 4, 5, 6)
    try:
        for m in sz:
            for n in sz:
                bsm.bsm_set_variant("fp64", m, n, variant)
                eligible = m * n <= 16 or (m, n) in ((5, 5), (6, 6))
                assert bsm.bsm_get_variant("fp64", m, n) == (variant if eligible else 0)
        Cg, ref, gA, gB = _run(bsm, oracle, A, B, 1e-3, beta=0.5, C0=random_bcsr(bs, bs, 0.05, seed=153))
        _check_pattern(Cg, ref.C)
        assert rel_fro(Cg.data_host(), ref.C.data) <= 1e-12
        Cg, ref, gA, gB = _run(bsm, oracle, A, B, 0.0)
        G = np.random.default_rng(4).standard_normal(ref.C.data_len)
        dA_ref, dB_ref = oracle.multiply_backward(1.0, A, B, ref.C, G, ref.prods)
        dA = torch.empty(len(A.data), dtype=torch.float64, device="cuda")
        dB = torch.empty(len(B.data), dtype=torch.float64, device="cuda")
        bsm.multiply_backward(1.0, Cg, torch.tensor(G, device="cuda"), gA, gB, dA, dB)
        assert rel_fro(dA.cpu().numpy(), dA_ref) <= 1e-12
        assert rel_fro(dB.cpu().numpy(), dB_ref) <= 1e-12
        # FP32 data through the same variant
        A32, B32 = A.astype(np.float32), B.astype(np.float32)
        Cg, ref, _, _ = _run(bsm, oracle, A32, B32, 0.0)
        assert rel_fro(Cg.data_host(), ref.C.data) <= 1e-5
    finally:
        for m in sz:
            for n in sz:
                bsm.bsm_set_variant("fp64", m, n, -1)


def test_autotune_table_roundtrip(bsm, oracle, tmp_path):
    from paper_1708_03604_gb300 import autotune
    bs = I.mixed_sizes(200, (1, 2, 4, 7), (0.3, 0.3, 0.3, 0.1), seed=8)
    Ah, Bh = random_bcsr(bs, bs, 0.05, seed=161), random_bcsr(bs, bs, 0.05, seed=162)
    A, B = bsm.Matrix.from_host(Ah), bsm.Matrix.from_host(Bh)
    sizes = (1, 2, 4, 7)
    try:
        for prec in ("tf32x3", "fp64"):
            table = autotune.tune(A, B, 0.0, prec=prec, reps=1)
            assert set(table["variants"]) == {f"{m}x{n}" for m in sizes for n in sizes if m * n <= 16}
            assert "7x7" not in table["variants"]
            path = str(tmp_path / f"tune_{prec}.json")
            autotune.save([table], path)
            autotune.reset(prec, sizes)
            autotune.load(path)
            for key, v in table["variants"].items():
                m, n = (int(x) for x in key.split("x"))
                assert bsm.bsm_get_variant(prec, m, n) == v
            Cg = bsm.multiply(1.0, A, B, prec=prec)
            ref = oracle.multiply(1.0, Ah, Bh)
            assert rel_fro(Cg.data_host(), ref.C.data) <= TOL[prec]
    finally:
        autotune.reset("tf32x3", sizes)
        autotune.reset("fp64", sizes)


@pytest.mark.parametrize("nb", [29, 40])
def test_single_shape_stacks(bsm, oracle, nb):
    """One block shape: the stack is the product list in order (the direct
    path), for an odd and an even product count."""
    w = I.uniform_23(nb=nb, occ=0.2)
    Cg, ref, _, _ = _run(bsm, oracle, w["A"], w["B"], 0.0)
    shapes, ptr, trip = Cg.stacks()
    s_ref, p_ref, t_ref = oracle.stacks(w["A"], w["B"], ref.C, ref.prods)
    np.testing.assert_array_equal(shapes, s_ref)
    np.testing.assert_array_equal(ptr, p_ref)
    np.testing.assert_array_equal(trip, t_ref)


def test_ragged_sizes_and_large_blocks(bsm, oracle):
    # block sizes 1..40 (several fragment tiles and element passes per block)
    rng = np.random.default_rng(5)
    rbs = rng.integers(1, 41, size=17).astype(np.int32)
    kbs = rng.integers(1, 41, size=13).astype(np.int32)
    cbs = rng.integers(1, 41, size=19).astype(np.int32)
    A = random_bcsr(rbs, kbs, 0.4, seed=21)
    B = random_bcsr(kbs, cbs, 0.4, seed=22)
    for prec in ("fp64", "tf32x3", "bf16x6"):
        Cg, ref, _, _ = _run(bsm, oracle, A, B, 0.0, prec=prec)
        _check_pattern(Cg, ref.C)
        assert rel_fro(Cg.data_host(), ref.C.data) <= TOL[prec]
    # about 40 distinct sizes: far more shapes than the two-pass stack builder
    # takes, so the stacks come from the radix-sort path
    shapes, ptr, trip = Cg.stacks()
    s_ref, p_ref, t_ref = oracle.stacks(A, B, ref.C, ref.prods)
    assert len(s_ref) > 256
    np.testing.assert_array_equal(shapes, s_ref)
    np.testing.assert_array_equal(ptr, p_ref)
    np.testing.assert_array_equal(trip, t_ref)


@pytest.mark.parametrize("nsizes", [6, 7])
def test_stacks_at_the_bin_limit(bsm, oracle, nsizes):
    """6 distinct sizes give 216 shape bins (two-pass builder), 7 give 343
    (radix-sort path): both bit-exact against the oracle's stable bucketing."""
    sizes = (1, 2, 3, 5, 7, 9, 11)[:nsizes]
    bs = I.mixed_sizes(60, sizes, (1.0 / nsizes,) * nsizes, seed=33)
    A, B = random_bcsr(bs, bs, 0.2, seed=111), random_bcsr(bs, bs, 0.2, seed=112)
    Cg, ref, _, _ = _run(bsm, oracle, A, B, 0.0)
    _check_pattern(Cg, ref.C)
    shapes, ptr, trip = Cg.stacks()
    s_ref, p_ref, t_ref = oracle.stacks(A, B, ref.C, ref.prods)
    np.testing.assert_array_equal(shapes, s_ref)
    np.testing.assert_array_equal(ptr, p_ref)
    np.testing.assert_array_equal(trip, t_ref)


def test_alpha_beta_merge(bsm, oracle):
    bs = I.mixed_sizes(50, (2, 7, 11), (0.4, 0.3, 0.3), seed=9)
    A, B, C0 = (random_bcsr(bs, bs, 0.15, seed=s) for s in (31, 32, 33))
    for prec in ("fp64", "tf32x3"):
        Cg, ref, _, _ = _run(bsm, oracle, A, B, 0.0, prec=prec, beta=-0.5, C0=C0, alpha=2.0)
        _check_pattern(Cg, ref.C)
        assert rel_fro(Cg.data_host(), ref.C.data) <= TOL[prec]


def test_beta_zero_ignores_old_nan(bsm, oracle):
    bs = I.uniform_sizes(20, 4)
    A, B, C0 = (random_bcsr(bs, bs, 0.2, seed=s) for s in (41, 42, 43))
    C0.data[:] = np.nan
    Cg, ref, _, _ = _run(bsm, oracle, A, B, 0.0, beta=0.0, C0=C0)
    _check_pattern(Cg, ref.C)
    assert np.all(np.isfinite(Cg.data_host()))


def test_edge_cases(bsm, oracle):
    bs = I.mixed_sizes(12, (1, 3), (0.5, 0.5), seed=1)
    A = random_bcsr(bs, bs, 0.3, seed=51)
    E = I.empty(bs, bs)
    # empty operand -> empty C
    for X, Y in ((A, E), (E, A), (E, E)):
        Cg, ref, _, _ = _run(bsm, oracle, X, Y, 0.0)
        assert Cg.nnzb == 0 and ref.C.nnzb == 0
    # huge threshold -> everything filtered
    Cg, ref, _, _ = _run(bsm, oracle, A, A, 1e300)
    assert Cg.nnzb == 0 and Cg.counts().filtered == ref.nfiltered > 0
    # A.A with the same handle (X^2)
    dA = bsm.Matrix.from_host(A)
    Cg = bsm.multiply(1.0, dA, dA)
    ref = oracle.multiply(1.0, A, A)
    _check_pattern(Cg, ref.C)
    assert rel_fro(Cg.data_host(), ref.C.data) <= 1e-12
    # 1x1 blocks only
    b1 = I.uniform_sizes(30, 1)
    A1, B1 = random_bcsr(b1, b1, 0.3, seed=61), random_bcsr(b1, b1, 0.3, seed=62)
    Cg, ref, _, _ = _run(bsm, oracle, A1, B1, 0.0)
    _check_pattern(Cg, ref.C)
    assert rel_fro(Cg.data_host(), ref.C.data) <= 1e-12


def test_blocking_mismatch_is_reported(bsm):
    a = random_bcsr(I.uniform_sizes(5, 3), I.uniform_sizes(5, 3), 0.5, seed=1)
    b = random_bcsr(I.uniform_sizes(5, 4), I.uniform_sizes(5, 4), 0.5, seed=2)
    with pytest.raises(bsm.BsmError) as e:
        bsm.multiply(1.0, bsm.Matrix.from_host(a), bsm.Matrix.from_host(b))
    assert e.value.status == bsm.BSM_ERR_BLOCKING


def test_deterministic(bsm):
    w = I.mixed_banded(nb=200, occ=0.1, eps=1e-6)
    A, B = bsm.Matrix.from_host(w["A"]), bsm.Matrix.from_host(w["B"])
    for prec in ("fp64", "tf32x3"):
        x = bsm.multiply(1.0, A, B, eps=w["eps"], prec=prec).data_host()
        y = bsm.multiply(1.0, A, B, eps=w["eps"], prec=prec).data_host()
        np.testing.assert_array_equal(x, y)


def _split_bound_coeff(prec, kmax):
    """Worst-case error of one output element of a split path, as a multiple
    of sum_k |a_ik||b_kj|: the cut of every operand into np pieces of p
    significant bits (round to nearest, so x - sum(pieces) <= 2^-(np p) |x|)
    plus the piece products left out; the FP32 sums inside the tensor core
    (at most npp * kmax terms per block product, each addition off by at most
    2^-23 of the running magnitude: round toward zero); the compensated sum
    across block products (about 2u, u = 2^-24)."""
    if prec == "tf32x3":   # 2 pieces of 11 bits, 3 products (lo*lo left out)
        trunc, npp = 3 * 2.0 ** -22, 3
    elif prec == "bf16x3":  # 2 pieces of 8 bits, 3 products
        trunc, npp = 3 * 2.0 ** -16, 3
    else:                   # bf16x6: 3 pieces of 8 bits, 6 products
        trunc, npp = 5 * 2.0 ** -24, 6
    return 1.1 * (trunc + npp * kmax * 2.0 ** -23 + 2.0 ** -22)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x6", "bf16x3"])
def test_split_elementwise_analytic_bound(bsm, oracle, prec):
    """Every element of a split-precision product within the analytic bound
    of its method, on blocks of 5..40 (several fragment tiles and k-steps)."""
    from tests.helpers import to_dense
    bs = I.mixed_sizes(30, (5, 13, 23, 40), (0.3, 0.3, 0.2, 0.2), seed=27)
    A, B = random_bcsr(bs, bs, 0.3, seed=101), random_bcsr(bs, bs, 0.3, seed=102)
    Cg, ref, _, _ = _run(bsm, oracle, A, B, 0.0, prec=prec)
    _check_pattern(Cg, ref.C)
    Ch = I.BCSR(ref.C.row_bs, ref.C.col_bs, ref.C.row_ptr, ref.C.col_idx, ref.C.blk_off, Cg.data_host())
    err = np.abs(to_dense(Ch) - to_dense(ref.C))
    absprod = np.abs(to_dense(A)) @ np.abs(to_dense(B))
    bound = _split_bound_coeff(prec, int(bs.max())) * absprod
    assert np.all(err <= bound), float(np.max(err / np.where(bound > 0, bound, 1.0)))


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_all_tiny_blocks(bsm, oracle, dt):
    """Blocks of 1, 2 and 4 rows/columns only (every output block at most 16
    elements: the small-register build of the CUDA-core kernel), FP64 and FP32
    data, with a transposed adjoint."""
    import torch
    bs = I.mixed_sizes(80, (1, 2, 4), (0.4, 0.2, 0.4), seed=17)
    A, B = random_bcsr(bs, bs, 0.2, seed=91, dtype=dt), random_bcsr(bs, bs, 0.2, seed=92, dtype=dt)
    Cg, ref, gA, gB = _run(bsm, oracle, A, B, 0.0)
    _check_pattern(Cg, ref.C)
    tol = 1e-12 if dt == np.float64 else 1e-5
    assert rel_fro(Cg.data_host(), ref.C.data) <= tol
    tdt = torch.float64 if dt == np.float64 else torch.float32
    G = np.random.default_rng(2).standard_normal(ref.C.data_len)
    dA_ref, dB_ref = oracle.multiply_backward(1.0, A.astype(np.float64), B.astype(np.float64), ref.C,
                                              G.astype(dt).astype(np.float64), ref.prods)
    dA = torch.empty(len(A.data), dtype=tdt, device="cuda")
    dB = torch.empty(len(B.data), dtype=tdt, device="cuda")
    bsm.multiply_backward(1.0, Cg, torch.tensor(G, dtype=tdt, device="cuda"), gA, gB, dA, dB)
    assert rel_fro(dA.double().cpu().numpy(), dA_ref) <= tol
    assert rel_fro(dB.double().cpu().numpy(), dB_ref) <= tol


def test_fp32_data(bsm, oracle):
    w = I.differentiation_13(nb=60, occ=0.15, dtype=np.float32)
    Cg, ref, _, _ = _run(bsm, oracle, w["A"], w["B"], 0.0)
    _check_pattern(Cg, ref.C)
    assert rel_fro(Cg.data_host(), ref.C.data) <= 1e-5
    Cg, ref, _, _ = _run(bsm, oracle, w["A"], w["B"], 0.0, prec="tf32x3")
    assert rel_fro(Cg.data_host(), ref.C.data) <= 1e-5


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_backward_matches_oracle(bsm, oracle, prec):
    bs = I.mixed_sizes(40, (3, 7, 13), (0.4, 0.3, 0.3), seed=23)
    A, B = random_bcsr(bs, bs, 0.15, seed=71), random_bcsr(bs, bs, 0.15, seed=72)
    import torch
    gA, gB = bsm.Matrix.from_host(A), bsm.Matrix.from_host(B)
    Cg = bsm.multiply(0.75, gA, gB, eps=0.0)
    ref = oracle.multiply(0.75, A, B)
    G = np.random.default_rng(3).standard_normal(ref.C.data_len)
    dA_ref, dB_ref = oracle.multiply_backward(0.75, A, B, ref.C, G, ref.prods)
    dC = torch.tensor(G, device="cuda")
    dA = torch.full((len(A.data),), np.nan, dtype=torch.float64, device="cuda")
    dB = torch.full((len(B.data),), np.nan, dtype=torch.float64, device="cuda")
    bsm.multiply_backward(0.75, Cg, dC, gA, gB, dA, dB, prec=prec)
    assert rel_fro(dA.cpu().numpy(), dA_ref) <= TOL[prec]
    assert rel_fro(dB.cpu().numpy(), dB_ref) <= TOL[prec]


def test_add_bitexact(bsm, oracle):
    bs = I.mixed_sizes(60, (1, 4), (0.5, 0.5), seed=29)
    X, Y = random_bcsr(bs, bs, 0.1, seed=81), random_bcsr(bs, bs, 0.1, seed=82)
    gX, gY = bsm.Matrix.from_host(X), bsm.Matrix.from_host(Y)
    for eps in (0.0, 1.0):
        Z = bsm.add(3.0, gX, -2.0, gY, eps=eps)
        ref = oracle.add(3.0, X, -2.0, Y, eps=eps)
        _check_pattern(Z, ref)
        np.testing.assert_array_equal(Z.data_host(), ref.data)
