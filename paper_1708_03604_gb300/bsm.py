"""Thin Python binding of libbsm (the C ABI declared in include/bsm.h).

Only argument marshalling lives here: every step of the multiply runs in the
library's CUDA kernels.  The raw entry points keep the C names
(``bsm_create``, ``bsm_multiply``, ...); ``Matrix`` and the functions
``multiply`` / ``multiply_backward`` / ``add`` wrap handles for convenience.
PyTorch provides device memory and the current CUDA stream; there is no CPU
fallback: if libbsm.so is missing the first call raises.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
from types import SimpleNamespace

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# BSM_DEBUG=1 in the environment loads the debug build (device-side bounds
# checks in the numeric kernels; built with build.build(debug=True))
LIB_PATH = os.path.join(_PKG, "libbsm_debug.so" if os.environ.get("BSM_DEBUG") == "1" else "libbsm.so")

# bsm_status
BSM_OK, BSM_ERR_ARG, BSM_ERR_BLOCKING, BSM_ERR_CAPACITY, BSM_ERR_ALLOC, BSM_ERR_CUDA, BSM_ERR_TIMEOUT, \
    BSM_ERR_UNSUPPORTED = range(8)
STATUS_NAMES = ["OK", "ERR_ARG", "ERR_BLOCKING", "ERR_CAPACITY", "ERR_ALLOC", "ERR_CUDA", "ERR_TIMEOUT",
                "ERR_UNSUPPORTED"]
BSM_FP64, BSM_FP32 = 0, 1
BSM_P_FP64, BSM_P_FP64_DMMA, BSM_P_TF32x3, BSM_P_BF16x3, BSM_P_BF16x6, BSM_P_OZAKI, BSM_P_TF32x3_PANEL = range(7)
PREC = {"fp64": BSM_P_FP64, "fp64_dmma": BSM_P_FP64_DMMA, "tf32x3": BSM_P_TF32x3, "bf16x3": BSM_P_BF16x3,
        "bf16x6": BSM_P_BF16x6, "ozaki": BSM_P_OZAKI, "tf32x3_panel": BSM_P_TF32x3_PANEL}
# bsm_engine
BSM_E_NONE, BSM_E_FP64_CORES, BSM_E_SPLIT_MMA, BSM_E_OZAKI_MMA, BSM_E_PANEL_TCGEN05 = -1, 0, 1, 2, 3
ENGINE_NAMES = {-1: "none", 0: "fp64_cores", 1: "split_mma", 2: "ozaki_mma", 3: "panel_tcgen05"}
BSM_DATA_COPY, BSM_DATA_BORROW = 0, 1
TIMING_PHASES = ["norms", "symbolic", "fill", "stacks", "numeric", "post", "total"]

EXPORTS = ["bsm_last_error", "bsm_set_stream", "bsm_set_profiling", "bsm_get_launch_count", "bsm_opts_default", "bsm_create",
           "bsm_create_empty", "bsm_create_like", "bsm_destroy", "bsm_get_info", "bsm_copy_pattern",
           "bsm_copy_data", "bsm_set_data", "bsm_data_ptr", "bsm_block_norms", "bsm_multiply",
           "bsm_multiply_backward", "bsm_get_counts", "bsm_get_timings", "bsm_get_products",
           "bsm_get_stacks", "bsm_add", "bsm_count_products_static", "bsm_borrow_data", "bsm_add_backward",
           "bsm_get_status", "bsm_set_variant", "bsm_get_variant", "bsm_get_engine", "bsm_set_allocator",
           "bsm_get_allocator_stats", "bsm_measure_peak",
           "bsm_set_wait_limit", "bsm_set_tuning", "bsm_get_tuning", "bsm_get_launch_config",
           "bsm_set_product_limit"]


class BsmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"bsm {STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class Opts(C.Structure):
    _fields_ = [("prec", C.c_int32), ("post_filter", C.c_int32), ("build_stacks", C.c_int32),
                ("flush_every", C.c_int32), ("no_sync", C.c_int32), ("reserved", C.c_int32 * 3)]


_lib = None
_vp, _i32, _i64, _f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double
_P = C.POINTER
# device-memory hooks of bsm_set_allocator
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
# Every hook pair ever installed stays referenced here: the library returns
# each block to the hooks that made it, even after another pair is installed,
# so a released ctypes thunk would be called after it is gone.
_hooks_alive: list = []


def lib() -> C.CDLL:
    """Load libbsm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libbsm.so not found at {LIB_PATH}; build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(LIB_PATH)
    sig = {
        "bsm_last_error": ([], C.c_char_p),
        "bsm_set_stream": ([_vp], _i32),
        "bsm_set_profiling": ([_i32], _i32),
        "bsm_get_launch_count": ([_P(_i64)], _i32),
        "bsm_opts_default": ([_P(Opts)], _i32),
        "bsm_create": ([_P(_vp), _i32, _i32, _vp, _vp, _vp, _vp, _vp, _i32, _vp, _i64, _i32], _i32),
        "bsm_create_empty": ([_P(_vp), _i32, _i32, _vp, _vp, _i32], _i32),
        "bsm_create_like": ([_P(_vp), _vp], _i32),
        "bsm_destroy": ([_vp], _i32),
        "bsm_get_info": ([_vp, _P(_i32), _P(_i32), _P(_i64), _P(_i64), _P(_i32)], _i32),
        "bsm_copy_pattern": ([_vp, _vp, _vp, _vp], _i32),
        "bsm_copy_data": ([_vp, _vp], _i32),
        "bsm_set_data": ([_vp, _vp], _i32),
        "bsm_data_ptr": ([_vp, _P(_vp)], _i32),
        "bsm_block_norms": ([_vp, _vp], _i32),
        "bsm_multiply": ([_f64, _vp, _vp, _f64, _vp, _f64, _P(Opts)], _i32),
        "bsm_multiply_backward": ([_f64, _vp, _vp, _vp, _vp, _vp, _vp, _P(Opts)], _i32),
        "bsm_get_counts": ([_vp, _P(_i64), _P(_i64), _P(_f64)], _i32),
        "bsm_get_timings": ([_vp, _P(_f64)], _i32),
        "bsm_get_products": ([_vp, _P(_i64), _vp, _vp, _vp], _i32),
        "bsm_get_stacks": ([_vp, _P(_i32), _P(_i64), _vp, _vp, _vp], _i32),
        "bsm_add": ([_f64, _vp, _f64, _vp, _vp, _f64, _P(Opts)], _i32),
        "bsm_get_status": ([_vp, _P(_i32)], _i32),
        "bsm_get_engine": ([_vp, _P(_i32)], _i32),
        "bsm_set_variant": ([_i32, _i32, _i32, _i32], _i32),
        "bsm_get_variant": ([_i32, _i32, _i32, _P(_i32)], _i32),
        "bsm_count_products_static": ([_vp, _vp, _f64, _vp, _vp, _vp], _i32),
        "bsm_borrow_data": ([_vp, _vp], _i32),
        "bsm_add_backward": ([_vp, _vp, _vp, _vp, _vp, _vp], _i32),
        "bsm_set_allocator": ([ALLOC_FN, FREE_FN, _vp], _i32),
        "bsm_get_allocator_stats": ([_P(_i64)], _i32),
        "bsm_measure_peak": ([_i32, _i32, _P(_f64)], _i32),
        "bsm_set_wait_limit": ([_f64], _i32),
        "bsm_set_product_limit": ([_i64], _i32),
        "bsm_set_tuning": ([_i32, _i32, _i32], _i32),
        "bsm_get_tuning": ([_i32, _i32, _P(_i32)], _i32),
        "bsm_get_launch_config": ([_vp, _P(_i32)], _i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    if os.environ.get("BSM_ALLOCATOR", "torch") == "torch":
        use_torch_allocator()
    return L


_exiting = False


def _at_exit():
    # handles destroyed while the interpreter shuts down leave their memory to
    # the process exit instead of calling into a half-finalised torch
    global _exiting
    _exiting = True


atexit.register(_at_exit)


def _torch_alloc(nbytes, stream, ctx):
    import torch
    try:
        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))
    except Exception:   # out of memory: the library reports BSM_ERR_ALLOC
        return None


def _torch_free(ptr, nbytes, stream, ctx):
    if _exiting:
        return
    import torch
    torch.cuda.caching_allocator_delete(int(ptr))


def set_allocator(alloc=None, free=None):
    """Install Python callables as the library's device-memory provider
    (``alloc(nbytes, stream) -> int | None``, ``free(ptr, nbytes, stream)``);
    no arguments restore the library's own stream-ordered pool."""
    L = lib() if _lib is None else _lib
    if alloc is None and free is None:
        _check(L.bsm_set_allocator(ALLOC_FN(), FREE_FN(), None))
        return
    a = ALLOC_FN(lambda n, s, c: alloc(n, s))
    f = FREE_FN(lambda p, n, s, c: free(p, n, s))
    _hooks_alive.append((a, f, alloc, free))
    _check(L.bsm_set_allocator(a, f, None))


_torch_hooks = None


def use_torch_allocator():
    """Route every library allocation through PyTorch's caching allocator on
    the library's stream (the default of this binding; BSM_ALLOCATOR=pool in
    the environment keeps the library's own pool instead)."""
    global _torch_hooks
    if _torch_hooks is None:
        _torch_hooks = (ALLOC_FN(_torch_alloc), FREE_FN(_torch_free))
        _hooks_alive.append(_torch_hooks)
    _check(_lib.bsm_set_allocator(_torch_hooks[0], _torch_hooks[1], None))


def allocator_outstanding() -> int:
    """Blocks the library holds from the installed hooks."""
    n = _i64()
    _check(lib().bsm_get_allocator_stats(C.byref(n)))
    return n.value


PEAK_UNITS = {"fp64_fma": 0, "fp64_mma": 1, "tf32_mma": 2, "bf16_mma": 3, "fp32_fma": 4}


def measure_peak(unit: str, reps: int = 5) -> float:
    """Measured FLOP/s of one arithmetic unit (PEAK_UNITS) on the current GPU."""
    _sync_stream()
    v = _f64()
    _check(lib().bsm_measure_peak(PEAK_UNITS[unit], int(reps), C.byref(v)))
    return v.value


def set_product_limit(max_products: int = 2**31 - 1):
    """Most kept products one pass of a multiply holds; above it the multiply
    runs row panel by row panel of C (no product list is kept)."""
    _check(lib().bsm_set_product_limit(int(max_products)))


def _check(st: int):
    if st != BSM_OK:
        raise BsmError(st, lib().bsm_last_error().decode())


def _ptr(a) -> int | None:
    """Address of a numpy array or torch tensor (None for empty arrays)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data if a.size else None
    return a.data_ptr() if a.numel() else None


def _sync_stream():
    """Route library work onto torch's current CUDA stream."""
    import torch
    _check(lib().bsm_set_stream(C.c_void_p(torch.cuda.current_stream().cuda_stream)))


def make_opts(prec="fp64", post_filter=False, build_stacks=True, flush_every=0, no_sync=False) -> Opts:
    o = Opts()
    _check(lib().bsm_opts_default(C.byref(o)))
    o.prec = PREC[prec] if isinstance(prec, str) else int(prec)
    o.post_filter = int(bool(post_filter))
    o.build_stacks = int(bool(build_stacks))
    o.flush_every = int(flush_every)
    o.no_sync = int(bool(no_sync))
    return o


# ---------------------------------------------------------------------------
# raw entry points with the C names
# ---------------------------------------------------------------------------
def bsm_set_profiling(on: bool):
    _check(lib().bsm_set_profiling(1 if on else 0))


def bsm_get_launch_count() -> int:
    n = _i64()
    _check(lib().bsm_get_launch_count(C.byref(n)))
    return n.value


def bsm_create(row_bs, col_bs, row_ptr, col_idx, blk_off, dtype, data_ptr, data_len, data_mode) -> int:
    h = C.c_void_p()
    row_bs = np.ascontiguousarray(row_bs, np.int32)
    col_bs = np.ascontiguousarray(col_bs, np.int32)
    row_ptr = np.ascontiguousarray(row_ptr, np.int64)
    col_idx = np.ascontiguousarray(col_idx, np.int32)
    blk_off = np.ascontiguousarray(blk_off, np.int64)
    _check(lib().bsm_create(C.byref(h), len(row_bs), len(col_bs), _ptr(row_bs), _ptr(col_bs), _ptr(row_ptr),
                            _ptr(col_idx), _ptr(blk_off), dtype, data_ptr, int(data_len), data_mode))
    return h.value


def bsm_create_empty(row_bs, col_bs, dtype) -> int:
    h = C.c_void_p()
    row_bs = np.ascontiguousarray(row_bs, np.int32)
    col_bs = np.ascontiguousarray(col_bs, np.int32)
    _check(lib().bsm_create_empty(C.byref(h), len(row_bs), len(col_bs), _ptr(row_bs), _ptr(col_bs), dtype))
    return h.value


def bsm_create_like(X: int) -> int:
    h = C.c_void_p()
    _check(lib().bsm_create_like(C.byref(h), X))
    return h.value


def bsm_destroy(X: int):
    _check(lib().bsm_destroy(X))


def bsm_get_info(X: int):
    nbr, nbc, dt = _i32(), _i32(), _i32()
    nnzb, dlen = _i64(), _i64()
    _check(lib().bsm_get_info(X, C.byref(nbr), C.byref(nbc), C.byref(nnzb), C.byref(dlen), C.byref(dt)))
    return SimpleNamespace(nbr=nbr.value, nbc=nbc.value, nnzb=nnzb.value, data_len=dlen.value, dtype=dt.value)


def bsm_multiply(alpha, A: int, B: int, beta, Cm: int, filter_eps, opts: Opts | None = None):
    _check(lib().bsm_multiply(float(alpha), A, B, float(beta), Cm, float(filter_eps),
                              C.byref(opts) if opts is not None else None))


def bsm_multiply_backward(alpha, Cm: int, dC_ptr, A: int, B: int, dA_ptr, dB_ptr, opts: Opts | None = None):
    _check(lib().bsm_multiply_backward(float(alpha), Cm, dC_ptr, A, B, dA_ptr, dB_ptr,
                                       C.byref(opts) if opts is not None else None))


def bsm_add(a, X: int, b, Y: int, Z: int, filter_eps, opts: Opts | None = None):
    _check(lib().bsm_add(float(a), X, float(b), Y, Z, float(filter_eps), C.byref(opts) if opts is not None else None))


def bsm_set_variant(prec, m: int, n: int, variant: int):
    _check(lib().bsm_set_variant(PREC[prec] if isinstance(prec, str) else int(prec), int(m), int(n), int(variant)))


def bsm_get_variant(prec, m: int, n: int) -> int:
    v = _i32()
    _check(lib().bsm_get_variant(PREC[prec] if isinstance(prec, str) else int(prec), int(m), int(n), C.byref(v)))
    return v.value


TUNE_PARAMS = {"cta_warps": 0, "ctas_per_sm": 1, "pass_mt": 2, "pass_nt": 3, "fp64_build": 4, "sched_tile": 5, "engine": 6,
               "panel_steps": 7}
KERNEL_NAMES = {-1: "none", 0: "fp64_cores", 1: "fp64_mma", 2: "split_mma", 3: "ozaki_mma", 4: "panel_tcgen05"}


def bsm_set_tuning(prec, param: str, value: int):
    _check(lib().bsm_set_tuning(PREC[prec] if isinstance(prec, str) else int(prec), TUNE_PARAMS[param], int(value)))


def bsm_get_tuning(prec, param: str) -> int:
    v = _i32()
    _check(lib().bsm_get_tuning(PREC[prec] if isinstance(prec, str) else int(prec), TUNE_PARAMS[param], C.byref(v)))
    return v.value


def bsm_get_launch_config(Cm: int) -> dict:
    """What the last numeric launch into Cm ran."""
    cfg = (C.c_int32 * 6)()
    _check(lib().bsm_get_launch_config(Cm, cfg))
    return {"kernel": KERNEL_NAMES.get(cfg[0], str(cfg[0])), "fp64_build": cfg[1], "cta_threads": cfg[2],
            "grid": cfg[3], "pass_mt": cfg[4], "pass_nt": cfg[5]}


def bsm_get_status(X: int) -> int:
    s = _i32()
    st = lib().bsm_get_status(X, C.byref(s))
    if st not in (BSM_OK, BSM_ERR_CAPACITY):
        _check(st)
    return s.value


def bsm_get_engine(Cm: int) -> str:
    """Numeric engine of the last multiply into Cm (ENGINE_NAMES)."""
    v = _i32()
    _check(lib().bsm_get_engine(Cm, C.byref(v)))
    return ENGINE_NAMES.get(v.value, str(v.value))


def bsm_get_counts(Cm: int):
    p, f, fl = _i64(), _i64(), _f64()
    _check(lib().bsm_get_counts(Cm, C.byref(p), C.byref(f), C.byref(fl)))
    return SimpleNamespace(products=p.value, filtered=f.value, useful_flop=fl.value)


def bsm_get_timings(Cm: int) -> dict:
    arr = (C.c_double * len(TIMING_PHASES))()
    _check(lib().bsm_get_timings(Cm, arr))
    return dict(zip(TIMING_PHASES, list(arr)))


# ---------------------------------------------------------------------------
# handle wrapper
# ---------------------------------------------------------------------------
_DT = {BSM_FP64: np.float64, BSM_FP32: np.float32}


class Matrix:
    """Owns one bsm_t handle.  ``keep`` holds a torch tensor whose memory the
    handle borrows."""

    def __init__(self, handle: int, row_bs, col_bs, keep=None):
        self.h = handle
        self.row_bs = np.ascontiguousarray(row_bs, np.int32)
        self.col_bs = np.ascontiguousarray(col_bs, np.int32)
        self._keep = keep

    # -- construction
    @classmethod
    def from_host(cls, X, dtype=None) -> "Matrix":
        """Copy a host block-CSR matrix (any object with row_bs, col_bs,
        row_ptr, col_idx, blk_off, data) into library-owned device memory."""
        _sync_stream()
        data = np.ascontiguousarray(X.data, dtype=dtype or X.data.dtype)
        dt = BSM_FP64 if data.dtype == np.float64 else BSM_FP32
        h = bsm_create(X.row_bs, X.col_bs, X.row_ptr, X.col_idx, X.blk_off, dt, _ptr(data), data.size, BSM_DATA_COPY)
        return cls(h, X.row_bs, X.col_bs)

    @classmethod
    def from_device(cls, X, data, borrow: bool = True) -> "Matrix":
        """Pattern from a host BCSR, data from a CUDA tensor (borrowed or copied)."""
        import torch
        assert data.is_cuda and data.is_contiguous()
        _sync_stream()
        dt = BSM_FP64 if data.dtype == torch.float64 else BSM_FP32
        h = bsm_create(X.row_bs, X.col_bs, X.row_ptr, X.col_idx, X.blk_off, dt, _ptr(data), data.numel(),
                       BSM_DATA_BORROW if borrow else BSM_DATA_COPY)
        return cls(h, X.row_bs, X.col_bs, keep=data if borrow else None)

    @classmethod
    def empty(cls, row_bs, col_bs, dtype=np.float64) -> "Matrix":
        _sync_stream()
        dt = BSM_FP64 if np.dtype(dtype) == np.float64 else BSM_FP32
        return cls(bsm_create_empty(row_bs, col_bs, dt), row_bs, col_bs)

    def like(self) -> "Matrix":
        _sync_stream()
        return Matrix(bsm_create_like(self.h), self.row_bs, self.col_bs)

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _lib is not None:
            try:
                _lib.bsm_destroy(h)
            except Exception:
                pass
            self.h = None

    # -- queries
    def info(self):
        return bsm_get_info(self.h)

    @property
    def nnzb(self) -> int:
        return self.info().nnzb

    def pattern(self):
        inf = self.info()
        rp = np.zeros(inf.nbr + 1, np.int64)
        ci = np.zeros(inf.nnzb, np.int32)
        bo = np.zeros(inf.nnzb, np.int64)
        _sync_stream()
        _check(lib().bsm_copy_pattern(self.h, _ptr(rp), _ptr(ci), _ptr(bo)))
        return rp, ci, bo

    def data_host(self) -> np.ndarray:
        inf = self.info()
        out = np.zeros(inf.data_len, _DT[inf.dtype])
        _sync_stream()
        _check(lib().bsm_copy_data(self.h, _ptr(out)))
        return out

    def data_tensor(self):
        """Copy of the data as a new CUDA tensor."""
        import torch
        inf = self.info()
        t = torch.empty(inf.data_len, dtype=torch.float64 if inf.dtype == BSM_FP64 else torch.float32,
                        device="cuda")
        _sync_stream()
        _check(lib().bsm_copy_data(self.h, _ptr(t)))
        return t

    def data_tensor_view(self):
        """The handle's device data as a CUDA tensor without a copy (valid
        while the handle keeps this storage: until its pattern is replaced or
        it is destroyed)."""
        import torch
        inf = self.info()
        if inf.data_len == 0:
            return torch.empty(0, dtype=torch.float64 if inf.dtype == BSM_FP64 else torch.float32, device="cuda")

        class _View:
            pass
        v = _View()
        v.__cuda_array_interface__ = {"shape": (inf.data_len,), "typestr": "<f8" if inf.dtype == BSM_FP64 else "<f4",
                                      "data": (self.data_ptr(), False), "version": 3, "strides": None}
        return torch.as_tensor(v, device="cuda")

    def set_data(self, src):
        _sync_stream()
        _check(lib().bsm_set_data(self.h, _ptr(src)))

    def borrow(self, t):
        """Make the handle's data the CUDA tensor t (kept alive by the handle)."""
        _sync_stream()
        _check(lib().bsm_borrow_data(self.h, _ptr(t)))
        self._keep = t

    def data_ptr(self) -> int:
        p = C.c_void_p()
        _check(lib().bsm_data_ptr(self.h, C.byref(p)))
        return p.value or 0

    def to_host(self):
        rp, ci, bo = self.pattern()
        return SimpleNamespace(row_bs=self.row_bs, col_bs=self.col_bs, row_ptr=rp, col_idx=ci, blk_off=bo,
                               data=self.data_host())

    def block_norms(self) -> np.ndarray:
        out = np.zeros(self.nnzb, np.float64)
        _sync_stream()
        _check(lib().bsm_block_norms(self.h, _ptr(out)))
        return out

    # -- results of the last multiply into this matrix
    def counts(self):
        return bsm_get_counts(self.h)

    def timings(self) -> dict:
        return bsm_get_timings(self.h)

    def engine(self) -> str:
        return bsm_get_engine(self.h)

    def launch_config(self) -> dict:
        return bsm_get_launch_config(self.h)

    def products(self):
        n = _i64()
        _check(lib().bsm_get_products(self.h, C.byref(n), None, None, None))
        a = np.zeros(n.value, np.int32)
        b = np.zeros(n.value, np.int32)
        c = np.zeros(n.value, np.int32)
        if n.value:
            _sync_stream()
            _check(lib().bsm_get_products(self.h, C.byref(n), _ptr(a), _ptr(b), _ptr(c)))
        return SimpleNamespace(a=a, b=b, c=c)

    def stack_shapes(self):
        """Shapes (m, n, k) of the last multiply's stacks and the number of
        products in each (the triples stay on the device)."""
        ns, npr = _i32(), _i64()
        _check(lib().bsm_get_stacks(self.h, C.byref(ns), C.byref(npr), None, None, None))
        shapes = np.zeros((ns.value, 3), np.int32)
        ptr = np.zeros(ns.value + 1, np.int64)
        if ns.value:
            _sync_stream()
            _check(lib().bsm_get_stacks(self.h, C.byref(ns), C.byref(npr), _ptr(shapes), _ptr(ptr), None))
        return shapes, np.diff(ptr)

    def stacks(self):
        ns, npr = _i32(), _i64()
        _check(lib().bsm_get_stacks(self.h, C.byref(ns), C.byref(npr), None, None, None))
        shapes = np.zeros((ns.value, 3), np.int32)
        ptr = np.zeros(ns.value + 1, np.int64)
        trip = np.zeros((npr.value, 3), np.int64)
        if ns.value:
            _sync_stream()
            _check(lib().bsm_get_stacks(self.h, C.byref(ns), C.byref(npr), _ptr(shapes), _ptr(ptr), _ptr(trip)))
        return shapes, ptr, trip


def multiply(alpha, A: Matrix, B: Matrix, beta=0.0, Cm: Matrix | None = None, eps=0.0, prec="fp64",
             post_filter=False, build_stacks=True, flush_every=0, no_sync=False) -> Matrix:
    """C = alpha * A.B + beta * C with on-the-fly filtering at eps."""
    _sync_stream()
    if Cm is None:
        Cm = Matrix.empty(A.row_bs, B.col_bs, np.float64 if A.info().dtype == BSM_FP64 else np.float32)
    bsm_multiply(alpha, A.h, B.h, beta, Cm.h, eps, make_opts(prec, post_filter, build_stacks, flush_every, no_sync))
    return Cm


def multiply_backward(alpha, Cm: Matrix, dC, A: Matrix, B: Matrix, dA=None, dB=None, prec="fp64",
                      flush_every=0):
    """Adjoint of the last multiply into Cm; dC/dA/dB are CUDA tensors laid
    out like C's/A's/B's data (dA, dB overwritten)."""
    _sync_stream()
    bsm_multiply_backward(alpha, Cm.h, _ptr(dC), A.h, B.h, _ptr(dA), _ptr(dB),
                          make_opts(prec, False, False, flush_every))


def add_backward(Z: Matrix, dZ, X: Matrix, Y: Matrix, dX=None, dY=None):
    """Adjoint of the last add into Z; tensors laid out like Z's/X's/Y's data."""
    _sync_stream()
    _check(lib().bsm_add_backward(Z.h, _ptr(dZ), X.h, Y.h, _ptr(dX), _ptr(dY)))


def add(a, X: Matrix, b, Y: Matrix, Z: Matrix | None = None, eps=0.0, no_sync=False) -> Matrix:
    """Z = a*X + b*Y over the union pattern, blocks with norm <= eps dropped."""
    _sync_stream()
    if Z is None:
        Z = Matrix.empty(X.row_bs, X.col_bs, np.float64 if X.info().dtype == BSM_FP64 else np.float32)
    bsm_add(a, X.h, b, Y.h, Z.h, eps, make_opts(no_sync=no_sync))
    return Z
