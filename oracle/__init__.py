"""FP64 CPU oracle for NIPALS-PCA and GS-PCA (Andrecut, arXiv:0811.1081).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use it; the library itself never does.
The arithmetic lives in ``oracle.c`` (plain C, FP64, no BLAS); this module
only compiles it with gcc, loads it with ctypes and marshals numpy arrays.

Parity pins for every function: ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NIPALS, GS = 0, 1
CENTER_NONE, CENTER_COLUMNS, CENTER_ROWS = 0, 1, 2
STATUS = {0: "ok", 1: "invalid argument", 4: "not converged", 5: "degenerate"}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2 as in the paper's Sec. 3 build line)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", _SO + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            lib.oracle_fit.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_int, ctypes.c_int, ip, ctypes.c_int,
                                       dp, dp, dp, ip, dp, ip]
            lib.oracle_round_bf16.argtypes = [ctypes.c_double]
            lib.oracle_round_bf16.restype = ctypes.c_double
            lib.oracle_fit.restype = ctypes.c_int
            lib.oracle_center.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.oracle_center.restype = ctypes.c_int
            lib.oracle_jacobi_eigh.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                               dp, dp]
            lib.oracle_jacobi_eigh.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a: np.ndarray | None):
    if a is None:
        return ctypes.POINTER(ctypes.c_int)()
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


@dataclass
class Fit:
    T: np.ndarray        # M×K scores (GS: V·Λ; NIPALS: unnormalised t)
    P: np.ndarray        # N×K loadings
    lam: np.ndarray      # K values λ_k
    iters: np.ndarray    # K iteration counts
    R: np.ndarray        # M×N final residual
    found: int           # components extracted
    status: int          # 0 ok, 4 not converged, 5 degenerate


STORAGE = {"f64": 0, "bf16": 1}


def fit(X: np.ndarray, K: int, tol: float = 1e-6, max_iter: int = 1000, algo: int | str = GS,
        center: int = CENTER_NONE, iters_lock=None, storage: str = "f64") -> Fit:
    """Run NIPALS-PCA (algo=0/'nipals') or GS-PCA (algo=1/'gs') on X (M×N) in FP64.

    storage="bf16": the residual R is rounded to bfloat16 after centring and after
    every deflation (Eq. 3); all arithmetic stays FP64."""
    if isinstance(algo, str):
        algo = {"nipals": NIPALS, "gs": GS}[algo.lower()]
    X = np.asfortranarray(np.asarray(X, dtype=np.float64))
    M, N = X.shape
    T = np.zeros((M, K), dtype=np.float64, order="F")
    P = np.zeros((N, K), dtype=np.float64, order="F")
    R = np.zeros((M, N), dtype=np.float64, order="F")
    lam = np.zeros(K, dtype=np.float64)
    iters = np.zeros(K, dtype=np.int32)
    found = np.zeros(1, dtype=np.int32)
    lock = None
    if iters_lock is not None:
        lock = np.ascontiguousarray(np.asarray(iters_lock, dtype=np.int32))
        if lock.shape != (K,):
            raise ValueError("iters_lock must have K entries")
    st = _load().oracle_fit(algo, _dptr(X), M, N, K, float(tol), int(max_iter), int(center),
                            _iptr(lock), STORAGE[storage], _dptr(T), _dptr(P), _dptr(lam), _iptr(iters),
                            _dptr(R), _iptr(found))
    if st == 1:
        raise ValueError("oracle_fit: invalid argument")
    return Fit(T=T, P=P, lam=lam, iters=iters, R=R, found=int(found[0]), status=int(st))


def round_bf16(x) -> np.ndarray:
    """Every entry of x rounded to the nearest bfloat16 (ties to even), as float64."""
    lib = _load()
    a = np.asarray(x, dtype=np.float64)
    return np.vectorize(lib.oracle_round_bf16, otypes=[np.float64])(a) if a.size else a.copy()


def center(X: np.ndarray, mode: int) -> np.ndarray:
    """mode 1: subtract column means; mode 2: subtract the average column (Eq. 1 as printed)."""
    R = np.array(X, dtype=np.float64, order="F", copy=True)
    M, N = R.shape
    if _load().oracle_center(_dptr(R), M, N, int(mode)) != 0:
        raise ValueError("oracle_center: invalid argument")
    return R


def jacobi_eigh(A: np.ndarray, tol: float = 1e-15, max_sweeps: int = 100):
    """Cyclic Jacobi eigen-decomposition of a symmetric matrix: (evals desc, evecs, sweeps)."""
    A = np.array(A, dtype=np.float64, order="F", copy=True)
    n = A.shape[0]
    if A.shape != (n, n):
        raise ValueError("square matrix required")
    w = np.zeros(n)
    V = np.zeros((n, n), order="F")
    sweeps = _load().oracle_jacobi_eigh(_dptr(A), n, float(tol), int(max_sweeps), _dptr(w), _dptr(V))
    if sweeps == -1:
        raise ValueError("oracle_jacobi_eigh: invalid argument")
    return w, V, sweeps
