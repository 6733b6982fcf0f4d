"""TEST INFRASTRUCTURE ONLY -- the plain FP64 CPU oracle for the R (and thin Q) factor of A = QR.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The GPU library (``paper_1002_4250_gb300``) never imports it, and it
imports nothing of the GPU library: the two share no code.

Python side of ``oracle.c`` (ctypes + numpy).  Every matrix crosses the boundary as a
column-major (Fortran-order) float64 numpy array; a torch tensor of shape (n, m) in
row-major order is the same memory as a column-major m x n matrix, see ``as_colmajor``.

Functions and the passages of Langou, "Computing the R of the QR factorization of tall and
skinny matrices using MPI_Reduce" (arXiv:1002.4250) they follow:

* ``householder_r``  -- Section 3 / Table 1 (the local Householder QR) applied to all of A,
  then the diag(R) >= 0 sign convention of Section 2;
* ``householder_qr`` -- the same factorization plus the thin Q factor, formed by applying the
  reflectors to the identity (Section 3, the remark on computing Q);
* ``lstsq``          -- least squares through that thin QR: X = R^-1 (Q^T B) (Section 3, the
  remark on applying the Householder transformations to a matrix);
* ``qr_uppers``      -- Section 2 / Table 3, the reduction operator qr(R1, R2);
* ``tsqr_r``         -- Section 2 (local QR per tile, then the reduction) with the binary,
  flat and hybrid trees of Section 1 and Fig. 1;
* ``cholesky_r_ld``  -- closed form: R is the unique upper Cholesky factor of A^T A;
* ``gram_dot2`` / ``gram_residual`` -- checker: ||R^T R - A^T A||_F / ||A||_F^2 with
  compensated (Dot2) sums.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

TREE_BINARY, TREE_FLAT, TREE_HYBRID = 0, 1, 2
_TREES = {"binary": TREE_BINARY, "flat": TREE_FLAT, "hybrid": TREE_HYBRID}


def compile_command(src: str = _SRC, out: str = _LIB_PATH) -> list[str]:
    """gcc command that builds the oracle library (portable flags: x86-64 and aarch64)."""
    return ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
            "-o", out, src, "-lm"]


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``oracle/_build/liboracle.so`` (if stale or forced)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(compile_command(_SRC, tmp), check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    d, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.oracle_householder_r.argtypes = [d, i64, i64, i64, d, i64, i32]
    lib.oracle_householder_r.restype = i32
    lib.oracle_householder_qr.argtypes = [d, i64, i64, i64, d, i64, d, i64, i32]
    lib.oracle_householder_qr.restype = i32
    lib.oracle_qr_uppers.argtypes = [i64, d, i64, d, i64, d, d]
    lib.oracle_qr_uppers.restype = None
    lib.oracle_tsqr_r.argtypes = [d, i64, i64, i64, i64, i32, i64, d, i64]
    lib.oracle_tsqr_r.restype = i32
    lib.oracle_cholesky_r_ld.argtypes = [d, i64, i64, i64, d, i64]
    lib.oracle_cholesky_r_ld.restype = i32
    lib.oracle_gram_dot2.argtypes = [d, i64, i64, i64, d, i64, i32]
    lib.oracle_gram_dot2.restype = i32
    lib.oracle_gram_residual.argtypes = [i64, d, i64, d, i64]
    lib.oracle_gram_residual.restype = ctypes.c_double
    lib.oracle_reflector.argtypes = [i64, d, d, i64, d]
    lib.oracle_reflector.restype = None
    lib.oracle_sign_fix.argtypes = [i64, d, i64]
    lib.oracle_sign_fix.restype = None
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


def load_variant(path: str):
    """Bind another build of ``oracle.c`` (the mutation tests use this); pass the result as
    ``lib=`` to any function here."""
    return _bind(ctypes.CDLL(path))


def as_colmajor(A) -> np.ndarray:
    """A float64 column-major (Fortran-order) copy or view of the m x n numpy matrix A.
    For a column-major matrix held by an (n, m) torch tensor use ``from_torch_colmajor``."""
    A = np.asarray(A, dtype=np.float64)
    if A.ndim != 2:
        raise ValueError("expected a 2-D matrix")
    return np.asfortranarray(A)


def from_torch_colmajor(t) -> np.ndarray:
    """The m x n column-major matrix held by a CPU torch tensor of shape (n, m)."""
    a = t.detach().cpu().numpy()
    if a.dtype != np.float64:
        a = a.astype(np.float64)
    return a.T  # (m, n), Fortran-contiguous view of the same memory


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc == 3:
        raise np.linalg.LinAlgError(f"{what}: matrix is not numerically full rank")
    if rc != 0:
        raise RuntimeError(f"{what} failed with code {rc}")


def householder_r(A, nthreads: int = 1, lib=None) -> np.ndarray:
    """R (n x n, diag >= 0) of one unblocked Householder QR of all of A, in FP64."""
    A = as_colmajor(A)
    m, n = A.shape
    R = np.zeros((n, n), dtype=np.float64, order="F")
    _check((lib or _load()).oracle_householder_r(_ptr(A), m, n, max(m, 1), _ptr(R), max(n, 1),
                                        int(nthreads)), "householder_r")
    return R


def householder_qr(A, nthreads: int = 1, lib=None):
    """(Q, R) of one unblocked Householder QR of all of A (m >= n), in FP64: Q m x n with
    orthonormal columns, R n x n with diag(R) >= 0, A = Q R."""
    A = as_colmajor(A)
    m, n = A.shape
    Q = np.zeros((m, n), dtype=np.float64, order="F")
    R = np.zeros((n, n), dtype=np.float64, order="F")
    _check((lib or _load()).oracle_householder_qr(_ptr(A), m, n, max(m, 1), _ptr(Q), max(m, 1),
                                                  _ptr(R), max(n, 1), int(nthreads)),
           "householder_qr")
    return Q, R


def back_substitute(R, C) -> np.ndarray:
    """X with R X = C for R upper triangular (n x n, nonzero diagonal), C (n, k): the rows
    solved last to first, each from the already solved rows below it."""
    R = np.asarray(R, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    n = R.shape[0]
    X = np.zeros_like(C)
    for i in range(n - 1, -1, -1):
        X[i] = (C[i] - R[i, i + 1:] @ X[i + 1:]) / R[i, i]
    return X


def lstsq(A, B, nthreads: int = 1, lib=None) -> np.ndarray:
    """X minimizing ||A X - B||_F for A (m x n, m >= n) of full column rank and B (m x k): the
    thin QR of A (householder_qr, Q formed from the Householder reflectors), then
    X = R^-1 (Q^T B) by back substitution (Section 3: the stored Householder transformations
    applied to a matrix instead of to the identity)."""
    Q, R = householder_qr(A, nthreads=nthreads, lib=lib)
    B = np.asarray(B, dtype=np.float64)
    vec = B.ndim == 1
    C = Q.T @ (B[:, None] if vec else B)
    X = back_substitute(R, C)
    return X[:, 0] if vec else X


def qr_uppers(R1, R2, count_flops: bool = False, lib=None):
    """The reduction operator of Table 3 on two n x n upper triangles.

    Returns (R, V, tau[, flops]): R is the raw R factor of [R1; R2] (diagonal signs as the
    reflectors leave them), V the reflector tails stored in place of R2, tau the scalars."""
    R1 = np.array(R1, dtype=np.float64, order="F", copy=True)
    R2 = np.array(R2, dtype=np.float64, order="F", copy=True)
    n = R1.shape[0]
    if R1.shape != (n, n) or R2.shape != (n, n):
        raise ValueError("qr_uppers needs two n x n matrices")
    tau = np.zeros(n, dtype=np.float64)
    fl = ctypes.c_int64(0)
    (lib or _load()).oracle_qr_uppers(n, _ptr(R1), n, _ptr(R2), n, _ptr(tau),
                             ctypes.cast(ctypes.pointer(fl), ctypes.c_void_p))
    if count_flops:
        return R1, R2, tau, int(fl.value)
    return R1, R2, tau


def tsqr_r(A, b: int, tree: str = "binary", group: int = 8, lib=None) -> np.ndarray:
    """TSQR on the CPU: per-tile Householder QR (tile height b) reduced with qr(R_i, R_j)
    along a binary, flat or hybrid (flat within groups of ``group`` tiles) tree; diag >= 0."""
    A = as_colmajor(A)
    m, n = A.shape
    R = np.zeros((n, n), dtype=np.float64, order="F")
    _check((lib or _load()).oracle_tsqr_r(_ptr(A), m, n, max(m, 1), int(b), _TREES[tree], int(group),
                                 _ptr(R), max(n, 1)), "tsqr_r")
    return R


def reflector(alpha: float, x, lib=None):
    """(beta, v, tau) of the Householder reflector mapping [alpha; x] to [beta; 0]."""
    x = np.array(x, dtype=np.float64, copy=True)
    a = ctypes.c_double(alpha)
    tau = ctypes.c_double(0.0)
    (lib or _load()).oracle_reflector(len(x) + 1, ctypes.cast(ctypes.pointer(a), ctypes.c_void_p),
                             _ptr(x), 1, ctypes.cast(ctypes.pointer(tau), ctypes.c_void_p))
    return a.value, x, tau.value


def sign_fix(R, lib=None) -> np.ndarray:
    """Rows flipped so that diag(R) >= 0; strict lower triangle zeroed."""
    R = np.array(R, dtype=np.float64, order="F", copy=True)
    n = R.shape[0]
    (lib or _load()).oracle_sign_fix(n, _ptr(R), n)
    return R


def cholesky_r_ld(A, lib=None) -> np.ndarray:
    """Upper Cholesky factor of A^T A, Gram matrix and factorization in long double."""
    A = as_colmajor(A)
    m, n = A.shape
    R = np.zeros((n, n), dtype=np.float64, order="F")
    _check((lib or _load()).oracle_cholesky_r_ld(_ptr(A), m, n, m, _ptr(R), n), "cholesky_r_ld")
    return R


def gram_dot2(A, nthreads: int = 1, lib=None) -> np.ndarray:
    """A^T A with every entry a compensated (Dot2) dot product."""
    A = as_colmajor(A)
    m, n = A.shape
    G = np.zeros((n, n), dtype=np.float64, order="F")
    _check((lib or _load()).oracle_gram_dot2(_ptr(A), m, n, max(m, 1), _ptr(G), max(n, 1),
                                    int(nthreads)), "gram_dot2")
    return G


def gram_residual(A=None, R=None, G=None, nthreads: int = 1, lib=None) -> float:
    """||R^T R - A^T A||_F / ||A||_F^2 (pass G = gram_dot2(A) to reuse a Gram matrix)."""
    if G is None:
        G = gram_dot2(A, nthreads, lib=lib)
    G = np.asfortranarray(G, dtype=np.float64)
    R = np.asfortranarray(R, dtype=np.float64)
    n = R.shape[0]
    return float((lib or _load()).oracle_gram_residual(n, _ptr(G), n, _ptr(R), n))


def rel_err(R, R_ref) -> float:
    """||R - R_ref||_F / ||R_ref||_F."""
    R = np.asarray(R, dtype=np.float64)
    R_ref = np.asarray(R_ref, dtype=np.float64)
    den = np.linalg.norm(R_ref)
    return float(np.linalg.norm(R - R_ref) / den) if den > 0 else float(np.linalg.norm(R))


def kappa_from_r(R) -> float:
    """2-norm condition number of A from its R factor (kappa(A) = kappa(R))."""
    s = np.linalg.svd(np.asarray(R, dtype=np.float64), compute_uv=False)
    return float(s[0] / s[-1]) if s[-1] > 0 else float("inf")
