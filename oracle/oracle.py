"""CPU FP64 oracle for the local block-sparse multiply of the DBCSR method.

TEST INFRASTRUCTURE ONLY: this module (and the C library it loads) may be
used by ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py``, never by the product path.  It imports
nothing from the CUDA package; matrices are accepted by duck typing (any
object with ``row_bs, col_bs, row_ptr, col_idx, blk_off, data``).

What it computes (Bethune et al. 2017, §2 "DBCSR Library"; Gustavson's
row-by-row SpGEMM, §1.1):

* ``block_norms``: Frobenius norm of every block, FP64, fma chain in
  row-major order from +0.0, then sqrt (the quantity the on-the-fly filter
  of §2 compares);
* ``multiply``: C = alpha*A.B + beta*C as pairwise products of small dense
  blocks, A's row-blocks outermost, a block product kept iff
  nA*nB > eps (eps <= 0 keeps all);
* ``stacks``: the kept products ("batches" of §2) as (a_off, b_off, c_off)
  triples bucketed by block shape (m, n, k) in lexicographic shape order and,
  inside a shape, in (i, j, k) order;
* ``multiply_backward``: the adjoint of C = alpha*A.B at fixed
  keep-decisions, dA on A's pattern and dB on B's pattern;
* ``add``: Z = a*X + b*Y over the union of patterns, blocks with norm
  <= eps dropped when eps > 0;
* ``post_filter``: drop C blocks with norm <= eps;
* ``mcweeny``: X_{k+1} = 3 X_k^2 - 2 X_k^3 with the multiplies and the add
  filtered at eps.

Parity pins for every function live in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from types import SimpleNamespace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bsm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the C oracle (plain gcc, -O2, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Bcsr(C.Structure):
    _fields_ = [("nbr", C.c_int32), ("nbc", C.c_int32),
                ("row_bs", C.c_void_p), ("col_bs", C.c_void_p),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p),
                ("blk_off", C.c_void_p), ("data", C.c_void_p)]


class _Result(C.Structure):
    _fields_ = [("nnzb", C.c_int64), ("row_ptr", C.POINTER(C.c_int64)),
                ("col_idx", C.POINTER(C.c_int32)), ("blk_off", C.POINTER(C.c_int64)),
                ("data", C.POINTER(C.c_double)), ("data_len", C.c_int64),
                ("nprod", C.c_int64), ("prod_a", C.POINTER(C.c_int32)),
                ("prod_b", C.POINTER(C.c_int32)), ("prod_c", C.POINTER(C.c_int32)),
                ("nfiltered", C.c_int64), ("useful_flop", C.c_double)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        lib.or_block_norms.argtypes = [C.POINTER(_Bcsr), C.c_void_p]
        lib.or_multiply.argtypes = [C.c_double, C.POINTER(_Bcsr), C.POINTER(_Bcsr), C.c_double,
                                    C.POINTER(_Bcsr), C.c_double, C.c_void_p, C.c_int32, C.c_int,
                                    C.POINTER(_Result)]
        lib.or_multiply.restype = C.c_int
        lib.or_result_free.argtypes = [C.POINTER(_Result)]
        lib.or_multiply_backward.argtypes = [C.c_double, C.POINTER(_Bcsr), C.POINTER(_Bcsr),
                                             C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                             C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                             C.c_void_p, C.c_int64]
        lib.or_multiply_backward.restype = C.c_int
        lib.or_add.argtypes = [C.c_double, C.POINTER(_Bcsr), C.c_double, C.POINTER(_Bcsr),
                               C.c_double, C.POINTER(_Result)]
        lib.or_add.restype = C.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a.size else None


def _view(X, keep: list):
    """ctypes view of a matrix; FP32 data is widened to FP64 (exact)."""
    arrs = dict(row_bs=np.ascontiguousarray(X.row_bs, dtype=np.int32),
                col_bs=np.ascontiguousarray(X.col_bs, dtype=np.int32),
                row_ptr=np.ascontiguousarray(X.row_ptr, dtype=np.int64),
                col_idx=np.ascontiguousarray(X.col_idx, dtype=np.int32),
                blk_off=np.ascontiguousarray(X.blk_off, dtype=np.int64),
                data=np.ascontiguousarray(X.data, dtype=np.float64))
    keep.append(arrs)
    return _Bcsr(arrs["row_bs"].shape[0], arrs["col_bs"].shape[0],
                 *(_ptr(arrs[k]) for k in ("row_bs", "col_bs", "row_ptr", "col_idx", "blk_off", "data")))


def _take(res: _Result, nbr: int, row_bs, col_bs, want_values: bool):
    def arr(p, n, dt):
        if n == 0 or not p:
            return np.zeros(0, dtype=dt)
        return np.ctypeslib.as_array(p, shape=(n,)).copy()
    out = SimpleNamespace(
        row_bs=np.asarray(row_bs, dtype=np.int32), col_bs=np.asarray(col_bs, dtype=np.int32),
        row_ptr=arr(res.row_ptr, nbr + 1, np.int64), col_idx=arr(res.col_idx, res.nnzb, np.int32),
        blk_off=arr(res.blk_off, res.nnzb, np.int64),
        data=arr(res.data, res.data_len, np.float64) if want_values else None,
        data_len=int(res.data_len), nnzb=int(res.nnzb))
    prods = SimpleNamespace(a=arr(res.prod_a, res.nprod, np.int32), b=arr(res.prod_b, res.nprod, np.int32),
                            c=arr(res.prod_c, res.nprod, np.int32))
    return out, prods


def block_norms(X) -> np.ndarray:
    keep: list = []
    v = _view(X, keep)
    out = np.zeros(int(np.asarray(X.row_ptr)[-1]), dtype=np.float64)
    _load().or_block_norms(C.byref(v), _ptr(out))
    return out


def multiply(alpha, A, B, beta=0.0, Cold=None, eps=0.0, rows=None, values=True):
    """C = alpha*A.B + beta*Cold with on-the-fly filtering at ``eps``.

    ``rows``: optional ascending list of block rows to produce (others empty).
    Returns a namespace with ``C`` (pattern, data), ``prods`` (a, b, c block
    indices in canonical (i, j, k) order), ``nfiltered`` and ``useful_flop``."""
    keep: list = []
    va, vb = _view(A, keep), _view(B, keep)
    vc = _view(Cold, keep) if Cold is not None else None
    r = None
    nrows = -1
    if rows is not None:
        r = np.ascontiguousarray(np.unique(np.asarray(rows, dtype=np.int32)))
        nrows = int(r.shape[0])
        if nrows == 0:
            r = np.full(1, -1, dtype=np.int32)   # non-NULL list, no row selected
        keep.append(r)
    res = _Result()
    rc = _load().or_multiply(float(alpha), C.byref(va), C.byref(vb), float(beta),
                             C.byref(vc) if vc is not None else None, float(eps),
                             _ptr(r) if r is not None else None, max(nrows, 0) if r is not None else -1, 1 if values else 0, C.byref(res))
    if rc == -2:
        raise ValueError("blocking mismatch")
    if rc != 0:
        raise MemoryError("oracle multiply failed")
    try:
        Cm, prods = _take(res, len(A.row_bs), A.row_bs, B.col_bs, values)
        return SimpleNamespace(C=Cm, prods=prods, nfiltered=int(res.nfiltered),
                               useful_flop=float(res.useful_flop))
    finally:
        _load().or_result_free(C.byref(res))


def stacks(A, B, Cm, prods):
    """Bucket the kept products by shape (m, n, k).

    Returns (shapes int32[S,3] lexicographic, stack_ptr int64[S+1],
    triples int64[P,3] = (a_off, b_off, c_off)); inside a shape the products
    keep the canonical (i, j, k) order."""
    a, b, c = (np.asarray(x, dtype=np.int64) for x in (prods.a, prods.b, prods.c))
    arow = np.repeat(np.arange(len(A.row_bs)), np.diff(np.asarray(A.row_ptr)))
    m = np.asarray(A.row_bs)[arow[a]].astype(np.int64)
    k = np.asarray(A.col_bs)[np.asarray(A.col_idx)[a]].astype(np.int64)
    n = np.asarray(B.col_bs)[np.asarray(B.col_idx)[b]].astype(np.int64)
    key = (m * 65536 + n) * 65536 + k
    order = np.argsort(key, kind="stable")
    uniq, counts = np.unique(key, return_counts=True)
    shapes = np.stack([uniq // (65536 * 65536), (uniq // 65536) % 65536, uniq % 65536], axis=1).astype(np.int32)
    ptr = np.zeros(len(uniq) + 1, dtype=np.int64)
    np.cumsum(counts, out=ptr[1:])
    trip = np.stack([np.asarray(A.blk_off)[a[order]], np.asarray(B.blk_off)[b[order]],
                     np.asarray(Cm.blk_off)[c[order]]], axis=1).astype(np.int64)
    return shapes.reshape(-1, 3), ptr, trip.reshape(-1, 3)


def multiply_backward(alpha, A, B, Cm, dC, prods, want_dA=True, want_dB=True):
    """Adjoint of C = alpha*A.B at the forward's kept products.

    dC is laid out with C's blk_off.  Returns (dA, dB) data arrays in A's and
    B's layouts (None where not wanted)."""
    keep: list = []
    va, vb = _view(A, keep), _view(B, keep)
    cof = np.ascontiguousarray(Cm.blk_off, dtype=np.int64)
    g = np.ascontiguousarray(dC, dtype=np.float64)
    pa, pb, pc = (np.ascontiguousarray(x, dtype=np.int32) for x in (prods.a, prods.b, prods.c))
    dA = np.zeros(len(A.data)) if want_dA else None
    dB = np.zeros(len(B.data)) if want_dB else None
    rc = _load().or_multiply_backward(float(alpha), C.byref(va), C.byref(vb), _ptr(cof), _ptr(g),
                                      int(pa.shape[0]), _ptr(pa), _ptr(pb), _ptr(pc),
                                      _ptr(dA) if dA is not None else None, len(A.data),
                                      _ptr(dB) if dB is not None else None, len(B.data))
    if rc != 0:
        raise MemoryError("oracle backward failed")
    return dA, dB


def add(a, X, b, Y, eps=0.0):
    keep: list = []
    vx, vy = _view(X, keep), _view(Y, keep)
    res = _Result()
    rc = _load().or_add(float(a), C.byref(vx), float(b), C.byref(vy), float(eps), C.byref(res))
    if rc == -2:
        raise ValueError("blocking mismatch")
    if rc != 0:
        raise MemoryError("oracle add failed")
    try:
        Z, _ = _take(res, len(X.row_bs), X.row_bs, X.col_bs, True)
        return Z
    finally:
        _load().or_result_free(C.byref(res))


def post_filter(Cm, eps):
    """Drop blocks whose Frobenius norm is <= eps (blocks re-laid contiguously)."""
    if eps <= 0:
        return Cm
    nrm = block_norms(Cm)
    keepb = nrm > eps
    brow = np.repeat(np.arange(len(Cm.row_bs)), np.diff(Cm.row_ptr))
    m = np.asarray(Cm.row_bs)[brow].astype(np.int64)
    n = np.asarray(Cm.col_bs)[np.asarray(Cm.col_idx)].astype(np.int64)
    sizes = (m * n)[keepb]
    new_off = np.zeros(int(keepb.sum()), dtype=np.int64)
    if new_off.size > 1:
        np.cumsum(sizes[:-1], out=new_off[1:])
    data = np.concatenate([Cm.data[o:o + s] for o, s in zip(np.asarray(Cm.blk_off)[keepb], sizes)]) \
        if new_off.size else np.zeros(0)
    counts = np.bincount(brow[keepb], minlength=len(Cm.row_bs))
    row_ptr = np.zeros(len(Cm.row_bs) + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return SimpleNamespace(row_bs=Cm.row_bs, col_bs=Cm.col_bs, row_ptr=row_ptr,
                           col_idx=np.asarray(Cm.col_idx)[keepb], blk_off=new_off, data=data,
                           data_len=int(sizes.sum()), nnzb=int(keepb.sum()))


def mcweeny(X0, steps, eps):
    """McWeeny purification X <- 3 X^2 - 2 X^3, every multiply and the add
    filtered at eps.  Returns the list [X_0, X_1, ..., X_steps]."""
    xs = [X0]
    X = X0
    for _ in range(steps):
        X2 = multiply(1.0, X, X, eps=eps).C
        X3 = multiply(1.0, X2, X, eps=eps).C
        X = add(3.0, X2, -2.0, X3, eps=eps)
        xs.append(X)
    return xs
