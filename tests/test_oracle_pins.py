"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each pin is chosen so that a plausible slip in the oracle (a dropped
product, a transposed block, a wrong index, a '>=' for '>', a lost beta
term) fails at least one of them.  None of them re-types the oracle's loops.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from paper_1708_03604_gb300 import inputs as I
from tests.helpers import block_mask, pattern_set, random_bcsr, rel_fro, to_dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_mat(d, bs):
    bs = np.asarray(bs, dtype=np.int32)
    return I.BCSR(bs, bs, np.asarray(d["row_ptr"], np.int64), np.asarray(d["col_idx"], np.int32),
                  np.asarray(d["blk_off"], np.int64), np.asarray(d["data"], np.float64))


# ---------------------------------------------------------------------------
# hand-worked example (tests/golden/hand_worked_3x3.json)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("case,eps", [("eps0", 0.0), ("eps3", 3.0)])
def test_hand_worked_example(oracle, case, eps):
    g = json.load(open(os.path.join(GOLDEN, "hand_worked_3x3.json")))
    A, B = _golden_mat(g["A"], g["bs"]), _golden_mat(g["B"], g["bs"])
    r = oracle.multiply(1.0, A, B, eps=eps)
    exp = g[case]
    assert r.C.row_ptr.tolist() == exp["row_ptr"]
    assert r.C.col_idx.tolist() == exp["col_idx"]
    assert r.C.blk_off.tolist() == exp["blk_off"]
    assert r.C.data.tolist() == [float(v) for v in exp["data"]]
    assert r.prods.a.tolist() == exp["prods_a"]
    assert r.prods.b.tolist() == exp["prods_b"]
    assert r.prods.c.tolist() == exp["prods_c"]
    assert r.useful_flop == exp["useful_flop"]
    assert r.nfiltered == exp.get("nfiltered", 0)
    np.testing.assert_array_equal(oracle.block_norms(A), g["norms_A"])
    np.testing.assert_array_equal(oracle.block_norms(B), g["norms_B"])


# ---------------------------------------------------------------------------
# norms
# ---------------------------------------------------------------------------
def test_norms_closed_forms(oracle):
    # 3-4-5 triangle, an all-ones 4x4 block (norm 4), a 1x1 block of -7
    bs = np.array([1, 2, 4], np.int32)
    rows, cols = np.array([0, 1, 2]), np.array([0, 1, 2])
    X = I.assemble(bs, bs, rows, cols, None, seed=0, values="zeros")
    X.data[X.blk_off[0]] = -7.0
    X.data[X.blk_off[1]:X.blk_off[1] + 4] = [3.0, 0.0, 0.0, 4.0]
    X.data[X.blk_off[2]:X.blk_off[2] + 16] = 1.0
    np.testing.assert_array_equal(oracle.block_norms(X), [7.0, 5.0, 4.0])


def test_norms_correctly_rounded_sum(oracle):
    bs = I.mixed_sizes(30, (1, 3, 7, 23), (0.25, 0.25, 0.25, 0.25), seed=11)
    X = random_bcsr(bs, bs, 0.3, seed=5)
    n = oracle.block_norms(X)
    for b in range(X.nnzb):
        i = int(X.block_rows()[b])
        m, k = int(bs[i]), int(bs[X.col_idx[b]])
        x = X.data[X.blk_off[b]:X.blk_off[b] + m * k]
        exact = math.sqrt(math.fsum(float(v) * float(v) for v in x))
        assert abs(n[b] - exact) <= 4 * np.spacing(exact), (b, n[b], exact)


# ---------------------------------------------------------------------------
# multiply vs dense, identity, permutation, transpose, associativity
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_eps0_equals_dense_product(oracle, seed):
    rng = np.random.default_rng(seed)
    nbr, nbk, nbc = rng.integers(3, 12, size=3)
    rbs = rng.integers(1, 8, size=nbr).astype(np.int32)
    kbs = rng.integers(1, 8, size=nbk).astype(np.int32)
    cbs = rng.integers(1, 8, size=nbc).astype(np.int32)
    A = random_bcsr(rbs, kbs, 0.4, seed=10 + seed)
    B = random_bcsr(kbs, cbs, 0.4, seed=20 + seed)
    r = oracle.multiply(1.0, A, B)
    dense = to_dense(A) @ to_dense(B)
    # pattern = boolean product of the block patterns
    pa = to_dense(type(A)(A.row_bs, A.col_bs, A.row_ptr, A.col_idx, A.blk_off, np.ones_like(A.data))) != 0
    bool_prod = set()
    for (i, k) in pattern_set(A):
        for (k2, j) in pattern_set(B):
            if k2 == k:
                bool_prod.add((i, j))
    assert pattern_set(r.C) == bool_prod
    got = to_dense(r.C)
    mask = block_mask(r.C)
    assert np.all(got[~mask] == 0)
    assert np.all(dense[~mask] == 0)
    assert rel_fro(got, dense) <= 1e-14
    del pa


def test_identity_bitexact(oracle):
    bs = I.mixed_sizes(14, (1, 2, 5, 7), (0.25, 0.25, 0.25, 0.25), seed=3)
    A = random_bcsr(bs, bs, 0.35, seed=7)
    Id = I.identity(bs)
    for r in (oracle.multiply(1.0, A, Id), oracle.multiply(1.0, Id, A)):
        np.testing.assert_array_equal(r.C.row_ptr, A.row_ptr)
        np.testing.assert_array_equal(r.C.col_idx, A.col_idx)
        np.testing.assert_array_equal(r.C.data, A.data)


def test_block_permutation_bitexact(oracle):
    bs = np.array([2, 3, 2, 3, 5, 2, 5, 3], np.int32)
    # a permutation that maps each block size class onto itself
    perm = np.arange(len(bs))
    rng = np.random.default_rng(4)
    for s in np.unique(bs):
        idx = np.nonzero(bs == s)[0]
        perm[idx] = rng.permutation(idx)
    A = random_bcsr(bs, bs, 0.5, seed=8)
    P = I.permutation_matrix(bs, perm)
    r = oracle.multiply(1.0, P, A)
    D = to_dense(A)
    ro = np.concatenate([[0], np.cumsum(bs)])
    exp = np.concatenate([D[ro[perm[i]]:ro[perm[i]] + bs[i]] for i in range(len(bs))])
    np.testing.assert_array_equal(to_dense(r.C), exp)


def test_transpose_identity_bitexact(oracle):
    rbs = np.array([3, 1, 4, 1, 5], np.int32)
    kbs = np.array([2, 6, 5, 3], np.int32)
    cbs = np.array([5, 8, 9, 7, 9, 3], np.int32)
    A = random_bcsr(rbs, kbs, 0.5, seed=31)
    B = random_bcsr(kbs, cbs, 0.5, seed=32)
    AB = oracle.multiply(1.0, A, B).C
    BtAt = oracle.multiply(1.0, I.transpose(B), I.transpose(A)).C
    # same products, same order over k: (AB)^T equals B^T A^T exactly
    np.testing.assert_array_equal(to_dense(AB).T, to_dense(BtAt))


def test_associativity(oracle):
    bs = I.mixed_sizes(10, (2, 3, 6), (0.4, 0.3, 0.3), seed=9)
    A, B, Cm = (random_bcsr(bs, bs, 0.4, seed=s) for s in (41, 42, 43))
    left = oracle.multiply(1.0, oracle.multiply(1.0, A, B).C, Cm).C
    right = oracle.multiply(1.0, A, oracle.multiply(1.0, B, Cm).C).C
    assert rel_fro(to_dense(left), to_dense(right)) <= 1e-13


def test_alpha_beta_merge(oracle):
    bs = I.mixed_sizes(9, (1, 4, 6), (0.3, 0.4, 0.3), seed=12)
    A, B, C0 = (random_bcsr(bs, bs, 0.3, seed=s) for s in (51, 52, 53))
    alpha, beta = -0.75, 2.5
    r = oracle.multiply(alpha, A, B, beta=beta, Cold=C0)
    exp = alpha * (to_dense(A) @ to_dense(B)) + beta * to_dense(C0)
    prod_pat = pattern_set(oracle.multiply(1.0, A, B).C)
    assert pattern_set(r.C) == prod_pat | pattern_set(C0)
    assert rel_fro(to_dense(r.C), exp) <= 1e-14
    # beta = 0: old C is neither read nor kept
    C0.data[:] = np.nan
    r0 = oracle.multiply(alpha, A, B, beta=0.0, Cold=C0)
    assert pattern_set(r0.C) == prod_pat
    assert np.all(np.isfinite(r0.C.data))


# ---------------------------------------------------------------------------
# filtering: brute-force enumeration of (i, k, j) on tiny inputs
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 1])
def test_pattern_bruteforce_with_filter(oracle, seed):
    rng = np.random.default_rng(100 + seed)
    nb = 9
    bs = rng.integers(1, 5, size=nb).astype(np.int32)
    A = random_bcsr(bs, bs, 0.45, seed=60 + seed)
    B = random_bcsr(bs, bs, 0.45, seed=70 + seed)
    # norms computed independently (sum of squares via fsum)
    def norms(X):
        out = []
        br = X.block_rows()
        for b in range(X.nnzb):
            m, k = int(X.row_bs[br[b]]), int(X.col_bs[X.col_idx[b]])
            out.append(math.sqrt(math.fsum(v * v for v in X.data[X.blk_off[b]:X.blk_off[b] + m * k])))
        return out
    nA, nB = norms(A), norms(B)
    cand = []
    for i in range(nb):
        for a in range(A.row_ptr[i], A.row_ptr[i + 1]):
            k = A.col_idx[a]
            for b in range(B.row_ptr[k], B.row_ptr[k + 1]):
                cand.append((i, int(B.col_idx[b]), int(k), int(a), int(b), nA[a] * nB[b]))
    vals = sorted({c[5] for c in cand})
    # thresholds half-way between distinct norm products: no tie within rounding
    eps_list = [0.0] + [0.5 * (vals[q] + vals[q + 1]) for q in (len(vals) // 4, len(vals) // 2, 3 * len(vals) // 4)]
    for eps in eps_list:
        kept = sorted([c for c in cand if eps <= 0 or c[5] > eps], key=lambda c: (c[0], c[1], c[2]))
        r = oracle.multiply(1.0, A, B, eps=eps)
        assert pattern_set(r.C) == {(c[0], c[1]) for c in kept}
        assert r.prods.a.tolist() == [c[3] for c in kept]
        assert r.prods.b.tolist() == [c[4] for c in kept]
        assert r.nfiltered == len(cand) - len(kept)
        # c index points at block (i, j)
        crow = r.C.block_rows() if hasattr(r.C, "block_rows") else np.repeat(np.arange(nb), np.diff(r.C.row_ptr))
        assert [(int(crow[c]), int(r.C.col_idx[c])) for c in r.prods.c] == [(c[0], c[1]) for c in kept]


def test_eps_huge_gives_empty(oracle):
    bs = I.uniform_sizes(12, 3)
    A, B = random_bcsr(bs, bs, 0.3, seed=1), random_bcsr(bs, bs, 0.3, seed=2)
    r = oracle.multiply(1.0, A, B, eps=1e300)
    assert r.C.nnzb == 0 and len(r.prods.a) == 0 and r.useful_flop == 0
    assert r.nfiltered == len(oracle.multiply(1.0, A, B).prods.a)


def test_flop_closed_form(oracle):
    bs = I.mixed_sizes(16, (1, 5, 13, 23), (0.3, 0.3, 0.2, 0.2), seed=21)
    A, B = random_bcsr(bs, bs, 0.3, seed=81), random_bcsr(bs, bs, 0.3, seed=82)
    r = oracle.multiply(1.0, A, B)
    Ar, Br = A.block_rows(), B.block_rows()
    total = 0
    for k in range(len(bs)):
        si = sum(int(bs[Ar[a]]) for a in range(A.nnzb) if A.col_idx[a] == k)
        sj = sum(int(bs[B.col_idx[b]]) for b in range(B.row_ptr[k], B.row_ptr[k + 1]))
        total += 2 * si * sj * int(bs[k])
    assert r.useful_flop == total
    assert Br is not None


def test_row_subset_matches_full(oracle):
    w = I.mixed_banded(nb=60, occ=0.1, eps=1e-3)
    full = oracle.multiply(1.0, w["A"], w["B"], eps=w["eps"])
    rows = [3, 17, 41, 59]
    sub = oracle.multiply(1.0, w["A"], w["B"], eps=w["eps"], rows=rows)
    for i in rows:
        cf = slice(full.C.row_ptr[i], full.C.row_ptr[i + 1])
        cs = slice(sub.C.row_ptr[i], sub.C.row_ptr[i + 1])
        np.testing.assert_array_equal(full.C.col_idx[cf], sub.C.col_idx[cs])
        for bf, bsub in zip(range(cf.start, cf.stop), range(cs.start, cs.stop)):
            m = int(full.C.row_bs[i]) * int(full.C.col_bs[full.C.col_idx[bf]])
            np.testing.assert_array_equal(full.C.data[full.C.blk_off[bf]:full.C.blk_off[bf] + m],
                                          sub.C.data[sub.C.blk_off[bsub]:sub.C.blk_off[bsub] + m])
    empty = oracle.multiply(1.0, w["A"], w["B"], eps=w["eps"], rows=[])
    assert empty.C.nnzb == 0


# ---------------------------------------------------------------------------
# stacks: brute-force canonical order
# ---------------------------------------------------------------------------
def test_stacks_bruteforce(oracle):
    bs = I.mixed_sizes(10, (2, 3, 5), (0.4, 0.3, 0.3), seed=13)
    A, B = random_bcsr(bs, bs, 0.4, seed=91), random_bcsr(bs, bs, 0.4, seed=92)
    r = oracle.multiply(1.0, A, B)
    shapes, ptr, trip = oracle.stacks(A, B, r.C, r.prods)
    Cpos = {}
    crow = np.repeat(np.arange(len(bs)), np.diff(r.C.row_ptr))
    for c in range(r.C.nnzb):
        Cpos[(int(crow[c]), int(r.C.col_idx[c]))] = int(r.C.blk_off[c])
    expected = {}
    for i, j, k in itertools.product(range(len(bs)), repeat=3):
        a = [x for x in range(A.row_ptr[i], A.row_ptr[i + 1]) if A.col_idx[x] == k]
        b = [x for x in range(B.row_ptr[k], B.row_ptr[k + 1]) if B.col_idx[x] == j]
        if a and b:
            expected.setdefault((int(bs[i]), int(bs[j]), int(bs[k])), []).append(
                (int(A.blk_off[a[0]]), int(B.blk_off[b[0]]), Cpos[(i, j)]))
    keys = sorted(expected)
    assert [tuple(s) for s in shapes.tolist()] == keys
    for q, key in enumerate(keys):
        assert [tuple(t) for t in trip[ptr[q]:ptr[q + 1]].tolist()] == expected[key]


# ---------------------------------------------------------------------------
# adjoint
# ---------------------------------------------------------------------------
def test_backward_vs_dense_autograd(oracle):
    torch = pytest.importorskip("torch")
    bs = I.mixed_sizes(12, (1, 3, 4), (0.3, 0.4, 0.3), seed=17)
    A, B = random_bcsr(bs, bs, 0.35, seed=101), random_bcsr(bs, bs, 0.35, seed=102)
    alpha = 1.5
    r = oracle.multiply(alpha, A, B)
    G = np.random.default_rng(7).standard_normal(r.C.data_len)
    dA, dB = oracle.multiply_backward(alpha, A, B, r.C, G, r.prods)
    Gd = to_dense(type(A)(r.C.row_bs, r.C.col_bs, r.C.row_ptr, r.C.col_idx, r.C.blk_off, G))
    At = torch.tensor(to_dense(A), requires_grad=True)
    Bt = torch.tensor(to_dense(B), requires_grad=True)
    loss = (torch.tensor(Gd) * (alpha * (At @ Bt))).sum()
    loss.backward()
    mA, mB = block_mask(A), block_mask(B)
    gA = At.grad.numpy() * mA
    gB = Bt.grad.numpy() * mB
    dAd = to_dense(type(A)(A.row_bs, A.col_bs, A.row_ptr, A.col_idx, A.blk_off, dA))
    dBd = to_dense(type(B)(B.row_bs, B.col_bs, B.row_ptr, B.col_idx, B.blk_off, dB))
    assert rel_fro(dAd, gA) <= 1e-13
    assert rel_fro(dBd, gB) <= 1e-13


def test_backward_central_fd(oracle):
    # L = ||C - T||^2 with C = A.B on C's pattern; dC = 2 (C - T)
    bs = I.uniform_sizes(8, 3)
    A, B = random_bcsr(bs, bs, 0.4, seed=111), random_bcsr(bs, bs, 0.4, seed=112)
    r = oracle.multiply(1.0, A, B)
    T = np.random.default_rng(3).standard_normal(r.C.data_len)

    def loss(Ad, Bd):
        Ax = type(A)(A.row_bs, A.col_bs, A.row_ptr, A.col_idx, A.blk_off, Ad)
        Bx = type(B)(B.row_bs, B.col_bs, B.row_ptr, B.col_idx, B.blk_off, Bd)
        c = oracle.multiply(1.0, Ax, Bx).C.data
        return float(np.sum((c - T) ** 2))

    dA, dB = oracle.multiply_backward(1.0, A, B, r.C, 2.0 * (r.C.data - T), r.prods)
    rng = np.random.default_rng(5)
    h = 1e-6
    for _ in range(4):
        va, vb = rng.standard_normal(A.data.shape), rng.standard_normal(B.data.shape)
        fd = (loss(A.data + h * va, B.data + h * vb) - loss(A.data - h * va, B.data - h * vb)) / (2 * h)
        an = float(np.dot(dA, va) + np.dot(dB, vb))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


# ---------------------------------------------------------------------------
# add, post-filter, McWeeny
# ---------------------------------------------------------------------------
def test_add_vs_dense_and_filter(oracle):
    bs = I.mixed_sizes(11, (1, 2, 5), (0.3, 0.4, 0.3), seed=19)
    X, Y = random_bcsr(bs, bs, 0.3, seed=121), random_bcsr(bs, bs, 0.3, seed=122)
    Z = oracle.add(3.0, X, -2.0, Y)
    assert pattern_set(Z) == pattern_set(X) | pattern_set(Y)
    assert rel_fro(to_dense(Z), 3.0 * to_dense(X) - 2.0 * to_dense(Y)) <= 1e-15
    nz = np.sort(oracle.block_norms(Z))
    eps = 0.5 * (nz[len(nz) // 2] + nz[len(nz) // 2 + 1])
    Zf = oracle.add(3.0, X, -2.0, Y, eps=eps)
    assert Zf.nnzb == int(np.sum(nz > eps))
    # every dropped block had norm <= eps, every kept block > eps
    assert np.all(oracle.block_norms(Zf) > eps)


def test_post_filter(oracle):
    bs = I.uniform_sizes(10, 2)
    X = random_bcsr(bs, bs, 0.5, seed=131)
    n = np.sort(oracle.block_norms(X))
    eps = 0.5 * (n[10] + n[11])
    Y = oracle.post_filter(X, eps)
    assert Y.nnzb == int(np.sum(n > eps))
    keepset = {p for p, nn in zip(sorted(pattern_set(X)), oracle.block_norms(X)) if nn > eps}
    assert pattern_set(Y) == keepset
    D = to_dense(X) * block_mask(Y)
    np.testing.assert_array_equal(to_dense(Y), D)


def test_mcweeny_spectral_identity(oracle):
    # dense symmetric X0 with spectrum in [0, 1]: X_k = V f^k(L) V^T, f = 3x^2 - 2x^3
    bs = np.array([1, 2, 1, 2, 2], np.int32)
    nb = len(bs)
    rows, cols = np.divmod(np.arange(nb * nb), nb)
    rng = np.random.default_rng(2)
    n = int(bs.sum())
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = rng.uniform(0, 1, n)
    D = (Q * lam) @ Q.T
    X0 = I.assemble(bs, bs, rows, cols, None, seed=0, values="zeros")
    ro = np.concatenate([[0], np.cumsum(bs)])
    for b in range(X0.nnzb):
        i, j = int(rows[b]), int(cols[b])
        X0.data[X0.blk_off[b]:X0.blk_off[b] + bs[i] * bs[j]] = D[ro[i]:ro[i] + bs[i], ro[j]:ro[j] + bs[j]].ravel()
    lam0 = np.linalg.eigvalsh(to_dense(X0))
    V = np.linalg.eigh(to_dense(X0))[1]
    xs = oracle.mcweeny(X0, 6, eps=0.0)
    f = lam0.copy()
    for k in range(1, 7):
        f = 3 * f ** 2 - 2 * f ** 3
        exp = (V * f) @ V.T
        assert rel_fro(to_dense(xs[k]), exp) <= 1e-12
    idem = [np.linalg.norm(to_dense(x) @ to_dense(x) - to_dense(x)) for x in xs]
    assert all(idem[q + 1] <= idem[q] + 1e-14 for q in range(len(idem) - 1))
