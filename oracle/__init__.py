"""FP64 CPU oracle for Flip-Flop SRQR (arXiv 1803.01982) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it and
the two share no code: the oracle is plain C (``ffsrqr_oracle.c``) compiled
with gcc, wrapped here with ctypes over numpy arrays.

Functions (row-major float64 arrays):

* ``philox(ctr, key)``            -- Philox4x32-10 block (Salmon et al., SC'11)
* ``normal(seed, stream, idx)``   -- Gaussian stream element (Box-Muller)
* ``omega(seed, s, m)``           -- Omega in N(0,1)^{s x m} (Alg. 2)
* ``qrcp(B, k)``                  -- Alg. 1 on B, returns (perm, factored B)
* ``house_qr(X)``                 -- Householder QR, explicit Q, diag(R) >= 0
* ``srqr(A, B, k, g, max_swaps)`` -- Alg. 4 initialised by Alg. 2 (b = k)
* ``jacobi_svd(M)``               -- one-sided Jacobi SVD of a square matrix
* ``ffsrqr(A, k, p, seed, ...)``  -- Alg. 9, returns U, S, V, piv, info, trace
* ``residual_fro(A, U, S, V)``    -- ||A - U diag(S) V^T||_F

The SRQR swap loop has no printed worked example; it is pinned through the
invariants the mathematics fixes (factorisation identity and orthonormal Q
after the swaps, |det R11| growing by more than g per swap, termination with
g2 <= g or the cap status).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ffsrqr_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, OpenMP). Returns the .so path."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _SrqrInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("swaps", ctypes.c_int32),
                ("g2_first", ctypes.c_double), ("g2_final", ctypes.c_double),
                ("cand_first", ctypes.c_int32), ("alpha_first", ctypes.c_double)]


class _Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("swaps", ctypes.c_int32),
                ("g2_first", ctypes.c_double), ("g2_final", ctypes.c_double),
                ("cand_first", ctypes.c_int32), ("alpha_first", ctypes.c_double),
                ("jacobi_sweeps", ctypes.c_int32)]


class _Trace(ctypes.Structure):
    _fields_ = [("B", ctypes.c_void_p), ("perm0", ctypes.c_void_p),
                ("r0", ctypes.c_void_p), ("Q1", ctypes.c_void_p),
                ("R", ctypes.c_void_p), ("Vp", ctypes.c_void_p),
                ("Rhat", ctypes.c_void_p), ("tmp", ctypes.c_void_p)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, u64, u32 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32
            P, D = ctypes.c_void_p, ctypes.c_double
            lib.oracle_philox4x32_10.argtypes = [P, P, P]
            lib.oracle_normal.argtypes = [u64, u32, u64]
            lib.oracle_normal.restype = D
            lib.oracle_omega.argtypes = [u64, i64, i64, P]
            lib.oracle_qrcp.argtypes = [P, i64, i64, i32, P]
            lib.oracle_qrcp.restype = ctypes.c_int
            lib.oracle_house_qr.argtypes = [P, i64, i64, i64, P, P]
            lib.oracle_srqr.argtypes = [P, i64, i64, i64, P, i64, i32, D, i32, P, P, P, P, P, P]
            lib.oracle_srqr.restype = ctypes.c_int
            lib.oracle_srqr_x.argtypes = [P, i64, i64, i64, P, i64, i32, i32, D, i32, i32, u64,
                                          P, P, P, P, P, P]
            lib.oracle_srqr_x.restype = ctypes.c_int
            lib.oracle_jacobi_svd.argtypes = [P, i64, P, P, P]
            lib.oracle_jacobi_svd.restype = ctypes.c_int
            lib.oracle_ffsrqr.argtypes = [P, i64, i64, i64, i32, i32, u64, D, i32,
                                          P, P, P, P, P, P]
            lib.oracle_ffsrqr.restype = ctypes.c_int
            lib.oracle_ffsrqr_x.argtypes = [P, i64, i64, i64, i32, i32, i32, u64, D, i32, i32,
                                            P, P, P, P, P, P]
            lib.oracle_ffsrqr_x.restype = ctypes.c_int
            lib.oracle_residual_fro.argtypes = [P, i64, i64, i64, P, P, P, i32]
            lib.oracle_residual_fro.restype = D
            _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def philox(ctr, key) -> np.ndarray:
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib.oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def normal(seed: int, stream: int, idx: int) -> float:
    return _load().oracle_normal(seed, stream, idx)


def omega(seed: int, s: int, m: int) -> np.ndarray:
    out = np.empty((s, m), dtype=np.float64)
    _load().oracle_omega(seed, s, m, _ptr(out))
    return out


def qrcp(B, k: int):
    """Alg. 1 for k steps on a copy of B. Returns (perm, factored B, status)."""
    W = _f64(B).copy()
    s, n = W.shape
    perm = np.zeros(n, dtype=np.int32)
    st = _load().oracle_qrcp(_ptr(W), s, n, k, _ptr(perm))
    return perm, W, st


def house_qr(X):
    X = _f64(X)
    m, k = X.shape
    Q = np.empty((m, k))
    R = np.empty((k, k))
    _load().oracle_house_qr(_ptr(X), m, k, k, _ptr(Q), _ptr(R))
    return Q, R


@dataclass
class SrqrResult:
    perm: np.ndarray
    Q1: np.ndarray
    R: np.ndarray
    perm0: np.ndarray
    r0: np.ndarray
    status: int
    swaps: int
    g2_first: float
    g2_final: float
    cand_first: int
    alpha_first: float


def srqr(A, B, k: int, g: float = 2.0, max_swaps: int | None = None, g2_rows: int = 0,
         seed: int = 0, b: int | None = None) -> SrqrResult:
    """Alg. 4 initialised by TRQRCP with block size b (None: b = k, one block;
    B then has b + p rows).  g2_rows = d >= 1 replaces the exact g2 by Alg. 4's
    d-row random estimate, its Omega_t drawn from Philox stream 1 under
    `seed`."""
    A = _f64(A)
    B = _f64(B)
    m, n = A.shape
    s = B.shape[0]
    if max_swaps is None:
        max_swaps = 4 * k
    perm = np.zeros(n, dtype=np.int32)
    perm0 = np.zeros(n, dtype=np.int32)
    Q1 = np.zeros((m, k))
    R = np.zeros((k, n))
    r0 = np.zeros(n)
    info = _SrqrInfo()
    _load().oracle_srqr_x(_ptr(A), m, n, n, _ptr(B), s, k, k if b is None else b, g, max_swaps,
                          g2_rows, seed, _ptr(perm), _ptr(Q1), _ptr(R), _ptr(perm0), _ptr(r0),
                          ctypes.byref(info))
    return SrqrResult(perm, Q1, R, perm0, r0, info.status, info.swaps, info.g2_first,
                      info.g2_final, info.cand_first, info.alpha_first)


def jacobi_svd(M):
    M = _f64(M)
    k = M.shape[0]
    assert M.shape == (k, k)
    U = np.empty((k, k))
    S = np.empty(k)
    V = np.empty((k, k))
    sweeps = _load().oracle_jacobi_svd(_ptr(M), k, _ptr(U), _ptr(S), _ptr(V))
    return U, S, V, sweeps


@dataclass
class FfsrqrResult:
    U: np.ndarray
    S: np.ndarray
    V: np.ndarray
    piv: np.ndarray
    status: int
    swaps: int
    g2_first: float
    g2_final: float
    cand_first: int
    alpha_first: float
    jacobi_sweeps: int
    trace: dict


def ffsrqr(A, k: int, p: int, seed: int = 0, g: float = 2.0, max_swaps: int | None = None,
           trace: bool = False, l: int | None = None, g2_rows: int = 0,
           b: int | None = None) -> FfsrqrResult:
    """Alg. 9 in FP64 on A (any float array, upcast to float64).  l (>= k) is
    the SRQR depth: SRQR and the SVD of A Pi Qhat_1 run at depth l, and the
    leading k singular triplets are returned (Alg. 9's U_k, Sigma_k, V_k).
    g2_rows = d >= 1 uses Alg. 4's d-row random g2 estimate instead of the
    exact g2.  b (< the depth) is TRQRCP's block size (Alg. 2): the sketch has
    b + p rows and the pivots are chosen block by block; None: one block."""
    if l is not None and l != k:
        assert l > k
        r = ffsrqr(A, l, p, seed, g, max_swaps, trace, g2_rows=g2_rows, b=b)
        r.U, r.S, r.V = r.U[:, :k].copy(), r.S[:k].copy(), r.V[:, :k].copy()
        return r
    A = _f64(A)
    m, n = A.shape
    bs = k if b is None else b
    s = bs + p
    if max_swaps is None:
        max_swaps = 4 * k
    U = np.zeros((m, k))
    S = np.zeros(k)
    V = np.zeros((n, k))
    piv = np.zeros(n, dtype=np.int32)
    info = _Info()
    tr = {}
    tstruct = None
    if trace:
        tr = {"B": np.zeros((s, n)), "perm0": np.zeros(n, dtype=np.int32), "r0": np.zeros(n),
              "Q1": np.zeros((m, k)), "R": np.zeros((k, n)), "Vp": np.zeros((n, k)),
              "Rhat": np.zeros((k, k)), "tmp": np.zeros((m, k))}
        tstruct = _Trace(*(_ptr(tr[f]) for f, _ in _Trace._fields_))
    st = _load().oracle_ffsrqr_x(_ptr(A), m, n, n, k, bs, p, seed, g, max_swaps, g2_rows, _ptr(U),
                                 _ptr(S), _ptr(V), _ptr(piv), ctypes.byref(info),
                               ctypes.byref(tstruct) if tstruct is not None else None)
    if st < 0:
        raise ValueError(f"oracle_ffsrqr rejected its arguments (code {st})")
    return FfsrqrResult(U, S, V, piv, info.status, info.swaps, info.g2_first, info.g2_final,
                        info.cand_first, info.alpha_first, info.jacobi_sweeps, tr)


def residual_fro(A, U, S, V) -> float:
    A, U, S, V = _f64(A), _f64(U), _f64(S), _f64(V)
    m, n = A.shape
    k = S.shape[0]
    return _load().oracle_residual_fro(_ptr(A), m, n, n, _ptr(U), _ptr(S), _ptr(V), k)
