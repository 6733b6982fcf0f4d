"""libtsqr: the R factor of A = QR for tall-and-skinny matrices on one GB300 (sm_103a).

A thin ctypes binding of the C ABI in ``include/tsqr.h``.  Every function marshals arguments
and calls the library; all computation runs in libtsqr's CUDA kernels.  There is no CPU
fallback: the first call raises ImportError if ``_build/libtsqr.so`` is missing (build it
with ``__graft_entry__.build()`` or ``python paper_1002_4250_gb300/_build.py``).

Two layers:

* ``capi`` -- the C functions themselves (``capi.tsqr_r(A_ptr, m, n, lda, R_ptr, ldr, stream)``
  and so on), taking raw device pointers and sizes;
* functions of the same names taking torch CUDA tensors: a column-major m x n matrix is a
  tensor of logical shape (m, n) with strides (1, lda) -- e.g. ``At.T`` for a contiguous
  (n, m) tensor ``At`` -- and R comes back as a logical (n, n) FP64 tensor with column-major
  storage.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtsqr.so")

SUCCESS, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_CUDA, ERR_ALLOC, ERR_TIMEOUT, STATUS_NONFINITE = range(7)
F64, F32, BF16 = 0, 1, 2
PREC_F64, PREC_MIXED = 0, 1
TREE_AUTO, TREE_BINARY, TREE_FLAT, TREE_HYBRID, TREE_PANELS = 0, 1, 2, 3, 4
LEAF_AUTO, LEAF_FOLD, LEAF_PANELS = 0, 1, 2
MAX_N = 128
_TREES = {"auto": TREE_AUTO, "binary": TREE_BINARY, "flat": TREE_FLAT, "hybrid": TREE_HYBRID,
          "panels": TREE_PANELS}


class Plan(ctypes.Structure):
    """tsqr_plan_t: tree, tile_rows, ctas, warps, arity, leaf (zeros mean "choose")."""
    _fields_ = [("tree", ctypes.c_int32), ("tile_rows", ctypes.c_int32),
                ("ctas", ctypes.c_int32), ("warps", ctypes.c_int32), ("arity", ctypes.c_int32),
                ("leaf", ctypes.c_int32)]


class BatchPlan(ctypes.Structure):
    """tsqr_batch_plan_t: warps, ctas_per_sm, leaves_per_cta, arity[4] (zeros mean "choose")."""
    _fields_ = [("warps", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("leaves_per_cta", ctypes.c_int32), ("arity", ctypes.c_int32 * 4),
                ("leaf", ctypes.c_int32)]

    def as_tuple(self):
        return (self.warps, self.ctas_per_sm, self.leaves_per_cta, tuple(self.arity), self.leaf)


def make_batch_plan(warps=0, ctas_per_sm=0, leaves_per_cta=0, arity=(0, 0, 0, 0),
                    leaf="auto") -> BatchPlan:
    """Knobs of a varlen batch call; arity per width bucket (n <= 8, <= 16, <= 32, > 32); leaf
    "auto", "fold" or "panels" (mixed precision)."""
    lf = {"auto": LEAF_AUTO, "fold": LEAF_FOLD, "panels": LEAF_PANELS}[leaf] \
        if isinstance(leaf, str) else int(leaf)
    return BatchPlan(int(warps), int(ctas_per_sm), int(leaves_per_cta),
                     (ctypes.c_int32 * 4)(*[int(a) for a in arity]), lf)


_capi = None


def _load():
    """Load and bind libtsqr.so.  Raises ImportError when the library has not been built:
    there is no CPU fallback."""
    global _capi
    if _capi is not None:
        return _capi
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"libtsqr is not built ({LIB_PATH} missing); run `python -c \"import __graft_entry__ "
            "as g; g.build()\"` -- there is no CPU fallback")
    capi = ctypes.CDLL(LIB_PATH)
    _p, _i64, _i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    capi.tsqr_r.argtypes = [_p, _i64, _i64, _i64, _p, _i64, _p]
    capi.tsqr_r.restype = _i32
    capi.tsqr_r_ex.argtypes = [_p, _i32, _i32, _i64, _i64, _i64, _p, _i64, ctypes.POINTER(Plan), _p]
    capi.tsqr_r_ex.restype = _i32
    capi.tsqr_qr_uppers.argtypes = [_i64, _p, _i64, _p, _i64, _p, _i64, _i32, _p]
    capi.tsqr_qr_uppers.restype = _i32
    capi.tsqr_r_batched.argtypes = [ctypes.POINTER(_p), ctypes.POINTER(_i64), ctypes.POINTER(_i32),
                                    ctypes.POINTER(_i64), _i32, _p, _i32, _i32, _p]
    capi.tsqr_r_batched.restype = _i32
    capi.tsqr_r_batched_ex.argtypes = [ctypes.POINTER(_p), ctypes.POINTER(_i64),
                                       ctypes.POINTER(_i32), ctypes.POINTER(_i64), _i32, _p, _i32,
                                       _i32, ctypes.POINTER(BatchPlan), _p]
    capi.tsqr_r_batched_ex.restype = _i32
    capi.tsqr_autotune_batched.argtypes = [ctypes.POINTER(_p), ctypes.POINTER(_i64),
                                           ctypes.POINTER(_i32), ctypes.POINTER(_i64), _i32, _p,
                                           _i32, _i32, ctypes.POINTER(BatchPlan), _p]
    capi.tsqr_autotune_batched.restype = _i32
    capi.tsqr_last_batch_plan.argtypes = [ctypes.POINTER(BatchPlan)]
    capi.tsqr_last_batch_plan.restype = _i32
    capi.tsqr_get_device_status.argtypes = [_p]
    capi.tsqr_get_device_status.restype = _i32
    capi.tsqr_release_workspace.argtypes = []
    capi.tsqr_release_workspace.restype = None
    capi.tsqr_status_string.argtypes = [_i32]
    capi.tsqr_status_string.restype = ctypes.c_char_p
    capi.tsqr_resolve_plan.argtypes = [_i64, _i64, _i32, _i32, ctypes.POINTER(Plan), ctypes.POINTER(Plan)]
    capi.tsqr_resolve_plan.restype = _i32
    capi.tsqr_r_noalloc.argtypes = [_p, _i64, _i64, _i64, _p, _i64, _p]
    capi.tsqr_qr.argtypes = [_p, _i64, _i64, _i64, _p, _i64, _p, _i64, ctypes.POINTER(Plan), _p]
    capi.tsqr_qr.restype = _i32
    capi.tsqr_autotune.argtypes = [_p, _i32, _i32, _i64, _i64, _i64, _p, _i64,
                                   ctypes.POINTER(Plan), _p]
    capi.tsqr_autotune.restype = _i32
    capi.tsqr_autotune_reset.argtypes = []
    capi.tsqr_autotune_reset.restype = None
    capi.tsqr_r_host.argtypes = [_p, _i64, _i64, _i64, _p, _i64, _p]
    capi.tsqr_r_host.restype = _i32
    capi.tsqr_lstsq.argtypes = [_p, _i64, _i64, _i64, _p, _i64, _i64, _p, _i64, _p, _i64,
                                ctypes.POINTER(Plan), _p]
    capi.tsqr_lstsq.restype = _i32
    capi.tsqr_caqr_r.argtypes = [_p, _i64, _i64, _i64, _p, _i64, _i64, ctypes.POINTER(Plan), _p]
    capi.tsqr_caqr_r.restype = _i32
    capi.tsqr_last_plan.argtypes = [ctypes.POINTER(Plan)]
    capi.tsqr_last_plan.restype = _i32
    capi.tsqr_r_noalloc.restype = _i32
    capi.tsqr_last_launch_count.argtypes = []
    capi.tsqr_last_launch_count.restype = _i32
    # measurement and self-test hooks (not part of include/tsqr.h)
    capi.tsqr_internal_measure_peaks.argtypes = [ctypes.POINTER(ctypes.c_double), _i32]
    capi.tsqr_internal_measure_peaks.restype = _i32
    capi.tsqr_internal_tc_layout_selftest.argtypes = [_p, _i32, _i32]
    capi.tsqr_internal_tc_layout_selftest.restype = _i32

    _capi = capi
    return capi


def __getattr__(name):
    if name == "capi":
        return _load()
    raise AttributeError(name)


#: every symbol include/tsqr.h declares
ABI_SYMBOLS = ("tsqr_r", "tsqr_r_ex", "tsqr_qr_uppers", "tsqr_r_batched", "tsqr_get_device_status",
               "tsqr_release_workspace", "tsqr_status_string", "tsqr_resolve_plan",
               "tsqr_last_launch_count", "tsqr_r_noalloc", "tsqr_qr", "tsqr_autotune",
               "tsqr_autotune_reset", "tsqr_r_host", "tsqr_lstsq", "tsqr_caqr_r", "tsqr_last_plan",
               "tsqr_r_batched_ex", "tsqr_autotune_batched", "tsqr_last_batch_plan")


class TsqrError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        msg = _load().tsqr_status_string(int(status)).decode()
        super().__init__(f"{what}: {msg} (status {status})" if what else msg)


def check(status: int, what: str = "") -> None:
    if status != SUCCESS:
        raise TsqrError(status, what)


def _stream_ptr(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _colmajor_dims(A, what="A"):
    """(m, n, lda) of a logical (m, n) CUDA tensor stored column-major (strides (1, lda))."""
    if A.dim() != 2 or not A.is_cuda:
        raise ValueError(f"{what} must be a 2-D CUDA tensor")
    m, n = A.shape
    s0, s1 = A.stride()
    if n > 1 and m > 1 and s0 != 1:
        raise ValueError(f"{what} must be column-major (strides (1, lda)); got strides {A.stride()}")
    lda = s1 if n > 1 else max(m, 1)
    return m, n, max(lda, m, 1)


def colmajor(A):
    """Column-major copy of a logical (m, n) tensor (for callers holding row-major data)."""
    return A.T.contiguous().T


def empty_r(n: int, device=None):
    """A logical (n, n) FP64 tensor with column-major storage, for R."""
    import torch
    return torch.empty((n, n), dtype=torch.float64, device=device).T


_LEAVES = {"auto": LEAF_AUTO, "fold": LEAF_FOLD, "panels": LEAF_PANELS}


def make_plan(tree="auto", tile_rows=0, ctas=0, warps=0, arity=0, leaf="auto") -> Plan:
    return Plan(_TREES[tree] if isinstance(tree, str) else int(tree), int(tile_rows), int(ctas),
                int(warps), int(arity), _LEAVES[leaf] if isinstance(leaf, str) else int(leaf))


def tsqr_r(A, R=None, stream=None):
    """R factor (logical (n, n), diag >= 0) of the column-major FP64 CUDA tensor A (m, n)."""
    import torch
    if A.dtype != torch.float64:
        raise ValueError("tsqr_r takes FP64 input; use tsqr_r_ex for FP32/BF16")
    m, n, lda = _colmajor_dims(A)
    if R is None:
        R = empty_r(n, A.device)
    check(_load().tsqr_r(A.data_ptr(), m, n, lda, R.data_ptr(), max(R.stride(1), n, 1),
                      _stream_ptr(stream)), "tsqr_r")
    return R


_DT = {}


def _dtype_code(t):
    import torch
    if not _DT:
        _DT.update({torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16})
    if t not in _DT:
        raise ValueError(f"unsupported dtype {t}")
    return _DT[t]


def tsqr_r_ex(A, prec=None, plan: Plan | None = None, R=None, stream=None):
    """tsqr_r for FP64 / FP32 / BF16 input with an optional plan (see ``make_plan``)."""
    m, n, lda = _colmajor_dims(A)
    dt = _dtype_code(A.dtype)
    if prec is None:
        prec = PREC_F64 if dt == F64 else PREC_MIXED
    if R is None:
        R = empty_r(n, A.device)
    pp = ctypes.byref(plan) if plan is not None else None
    check(_load().tsqr_r_ex(A.data_ptr(), dt, int(prec), m, n, lda, R.data_ptr(),
                         max(R.stride(1), n, 1), pp, _stream_ptr(stream)), "tsqr_r_ex")
    return R


def tsqr_qr(A, Q=None, R=None, plan: Plan | None = None, stream=None):
    """Thin QR of a logical (m, n) column-major FP64 tensor: returns (Q, R) with Q (m, n)
    column-major (orthonormal columns) and R (n, n), diag(R) >= 0, A = Q R."""
    m, n, lda = _colmajor_dims(A)
    if Q is None:
        import torch
        Q = torch.empty(n, m, dtype=torch.float64, device=A.device).T
    _, _, ldq = _colmajor_dims(Q, "Q")
    if R is None:
        R = empty_r(n, A.device)
    pp = ctypes.byref(plan) if plan is not None else None
    check(_load().tsqr_qr(A.data_ptr(), m, n, lda, Q.data_ptr(), ldq, R.data_ptr(),
                          max(R.stride(1), n, 1), pp, _stream_ptr(stream)), "tsqr_qr")
    return Q, R


def tsqr_lstsq(A, B, X=None, R=None, plan: Plan | None = None, stream=None):
    """Least squares min ||A X - B||_F for logical (m, n) A and (m, k) B, column-major FP64
    CUDA tensors (B may also be a vector of length m).  Returns (X, R): X (n, k) (or (n,)),
    R (n, n) as from tsqr_r."""
    import torch
    m, n, lda = _colmajor_dims(A)
    vec = B.dim() == 1
    B2 = B[:, None] if vec else B
    mb, k, ldb = _colmajor_dims(B2, "B")
    if mb != m:
        raise ValueError("A and B must have the same number of rows")
    if X is None:
        X = torch.empty(k, n, dtype=torch.float64, device=A.device).T
    _, _, ldx = _colmajor_dims(X, "X")
    if R is None:
        R = empty_r(n, A.device)
    pp = ctypes.byref(plan) if plan is not None else None
    check(_load().tsqr_lstsq(A.data_ptr(), m, n, lda, B2.data_ptr(), ldb, k, X.data_ptr(),
                             max(ldx, n), R.data_ptr(), max(R.stride(1), n, 1), pp,
                             _stream_ptr(stream)), "tsqr_lstsq")
    return (X[:, 0] if vec else X), R


def tsqr_caqr_r(A, panel: int = 0, R=None, plan: Plan | None = None, stream=None):
    """R (n, n), diag(R) >= 0, of a logical (m, n) column-major FP64 CUDA tensor of any width
    n <= m, by panels of `panel` columns (0 = the default width): each panel factorized by TSQR,
    then its Q^T applied to the columns right of it (Section 5)."""
    m, n, lda = _colmajor_dims(A)
    if R is None:
        R = empty_r(n, A.device)
    pp = ctypes.byref(plan) if plan is not None else None
    check(_load().tsqr_caqr_r(A.data_ptr(), m, n, lda, R.data_ptr(), max(R.stride(1), n, 1),
                              int(panel), pp, _stream_ptr(stream)), "tsqr_caqr_r")
    return R


def tsqr_r_host(A, R=None, stream=None, sync=True):
    """tsqr_r for a CPU FP64 tensor A (logical (m, n), column-major): page-locked A (``pin_memory``)
    is read in place by the device, other memory is copied to the device first.  Returns R as
    a CPU (n, n) column-major tensor.  With ``sync`` (the default) the stream is synchronized
    and the device status read before returning: R is then ready, and a device-side error
    raises TsqrError (non-finite values in R only warn, as R still holds them).  With
    ``sync=False`` synchronize the stream before reading R."""
    import torch
    if A.dim() != 2 or A.is_cuda or A.dtype != torch.float64:
        raise ValueError("A must be a 2-D CPU float64 tensor")
    m, n = A.shape
    if n > 1 and m > 1 and A.stride(0) != 1:
        raise ValueError(f"A must be column-major (strides (1, lda)); got strides {A.stride()}")
    lda = max(A.stride(1) if n > 1 else m, m, 1)
    if R is None:
        R = torch.empty(n, n, dtype=torch.float64).T
    ldr = max(R.stride(1) if n > 1 else n, n, 1)
    check(_load().tsqr_r_host(A.data_ptr(), m, n, lda, R.data_ptr(), ldr, _stream_ptr(stream)),
          "tsqr_r_host")
    if sync:
        st = int(_load().tsqr_get_device_status(_stream_ptr(stream)))
        if st == STATUS_NONFINITE:
            import warnings
            warnings.warn("tsqr_r_host: R holds NaN or Inf", RuntimeWarning, stacklevel=2)
        elif st != SUCCESS:
            raise TsqrError(st, "tsqr_r_host")
    return R


def tsqr_autotune(A, prec=None, R=None, stream=None) -> Plan:
    """Time candidate plans on A (FP64 / FP32 / BF16, logical (m, n) column-major), cache the
    fastest for AUTO calls of the same (n, leaf precision, floor(log2 m)), and return it."""
    m, n, lda = _colmajor_dims(A)
    dt = _dtype_code(A.dtype)
    if prec is None:
        prec = PREC_F64 if dt == F64 else PREC_MIXED
    if R is None:
        R = empty_r(n, A.device)
    best = Plan()
    check(_load().tsqr_autotune(A.data_ptr(), dt, int(prec), m, n, lda, R.data_ptr(),
                                max(R.stride(1), n, 1), ctypes.byref(best), _stream_ptr(stream)),
          "tsqr_autotune")
    return best


def tsqr_autotune_reset() -> None:
    _load().tsqr_autotune_reset()


def tsqr_qr_uppers(R1, R2, normalize=False, R=None, stream=None):
    """The tree operator qr(R1, R2) (Table 3) on two logical (n, n) column-major FP64 tensors."""
    n = R1.shape[0]
    _, _, ld1 = _colmajor_dims(R1, "R1")
    _, _, ld2 = _colmajor_dims(R2, "R2")
    if R is None:
        R = empty_r(n, R1.device)
    check(_load().tsqr_qr_uppers(n, R1.data_ptr(), ld1, R2.data_ptr(), ld2, R.data_ptr(),
                              max(R.stride(1), n, 1), 1 if normalize else 0, _stream_ptr(stream)),
          "tsqr_qr_uppers")
    return R


def _batch_arrays(ptrs, ms, ns, offsets):
    count = len(ms)
    P = (ctypes.c_void_p * max(count, 1))(*[int(p) for p in ptrs])
    M = (ctypes.c_int64 * max(count, 1))(*[int(x) for x in ms])
    N = (ctypes.c_int32 * max(count, 1))(*[int(x) for x in ns])
    O = (ctypes.c_int64 * (count + 1))(*[int(x) for x in offsets])
    return P, M, N, O, count


def tsqr_r_batched(ptrs, ms, ns, offsets, R_packed, dtype=F64, prec=PREC_F64, stream=None,
                   plan=None):
    """Varlen batch through one launch; ptrs/ms/ns/offsets are host sequences (see tsqr.h).
    plan: None (AUTO: the tuned knobs of the batch's bucket, else the built-in rules) or a
    BatchPlan."""
    P, M, N, O, count = _batch_arrays(ptrs, ms, ns, offsets)
    if plan is None:
        check(_load().tsqr_r_batched(P, M, N, O, count, R_packed.data_ptr(), int(dtype),
                                     int(prec), _stream_ptr(stream)), "tsqr_r_batched")
    else:
        check(_load().tsqr_r_batched_ex(P, M, N, O, count, R_packed.data_ptr(), int(dtype),
                                        int(prec), ctypes.byref(plan), _stream_ptr(stream)),
              "tsqr_r_batched_ex")
    return R_packed


def tsqr_autotune_batched(ptrs, ms, ns, offsets, R_packed, dtype=F64, prec=PREC_F64,
                          stream=None) -> BatchPlan:
    """Time knob settings on this batch, cache the fastest for its shape bucket, return it."""
    P, M, N, O, count = _batch_arrays(ptrs, ms, ns, offsets)
    best = BatchPlan()
    check(_load().tsqr_autotune_batched(P, M, N, O, count, R_packed.data_ptr(), int(dtype),
                                        int(prec), ctypes.byref(best), _stream_ptr(stream)),
          "tsqr_autotune_batched")
    return best


def last_batch_plan() -> BatchPlan:
    """The knobs of the last batched call on this thread (tsqr_last_batch_plan)."""
    out = BatchPlan()
    check(_load().tsqr_last_batch_plan(ctypes.byref(out)), "tsqr_last_batch_plan")
    return out


def tsqr_get_device_status(stream=None) -> int:
    return int(_load().tsqr_get_device_status(_stream_ptr(stream)))


def tsqr_release_workspace() -> None:
    _load().tsqr_release_workspace()


def last_plan() -> Plan:
    """The plan of the factorization the last call on this thread ran (tsqr_last_plan)."""
    out = Plan()
    check(_load().tsqr_last_plan(ctypes.byref(out)), "tsqr_last_plan")
    return out


def tsqr_resolve_plan(m, n, dtype=F64, prec=PREC_F64, plan: Plan | None = None) -> Plan:
    out = Plan()
    check(_load().tsqr_resolve_plan(int(m), int(n), int(dtype), int(prec),
                                 ctypes.byref(plan) if plan is not None else None,
                                 ctypes.byref(out)), "tsqr_resolve_plan")
    return out


def tsqr_last_launch_count() -> int:
    return int(_load().tsqr_last_launch_count())


PEAK_NAMES = ("fp64_dfma", "fp32_ffma", "tf32_mma_sync", "tf32_tcgen05", "bf16_tcgen05")


def measure_peaks() -> dict:
    """Pipe peaks of the current GPU in TFLOP/s, measured by libtsqr's microbenchmarks (dense;
    2 flops per FMA): FP64 DFMA, FP32 FFMA, TF32 through the warp-level mma and through
    tcgen05.mma, BF16 through tcgen05.mma.  Synchronizes the device (about a second)."""
    out = (ctypes.c_double * len(PEAK_NAMES))()
    check(_load().tsqr_internal_measure_peaks(out, len(PEAK_NAMES)), "measure_peaks")
    return dict(zip(PEAK_NAMES, list(out)))
