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
_SRCS = [_SRC, os.path.join(_HERE, "warmstart.c")]
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NIPALS, GS = 0, 1
CENTER_NONE, CENTER_COLUMNS, CENTER_ROWS = 0, 1, 2
STATUS = {0: "ok", 1: "invalid argument", 4: "not converged", 5: "degenerate"}


# Builds of the same sources.  "O2" (the paper's optimisation level, Sec. 3,
# single-threaded) is the checker every test uses; the others exist only to time
# the oracle on the host cores: "O3", and "O2-omp" / "O3-omp" with OpenMP, whose
# loops split over independent outputs so the results are the same bits.
FLAVORS = {"O2": ["-O2"], "O3": ["-O3"], "O2-omp": ["-O2", "-fopenmp"], "O3-omp": ["-O3", "-fopenmp"]}


def _so_path(flavor: str) -> str:
    return _SO if flavor == "O2" else os.path.join(_HERE, f"liboracle_{flavor.replace('-', '_')}.so")


def build(force: bool = False, flavor: str = "O2") -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2 as in the paper's Sec. 3 build line), or
    one of the timing builds of FLAVORS."""
    so = _so_path(flavor)
    if force or not os.path.exists(so) or any(os.path.getmtime(so) < os.path.getmtime(f) for f in _SRCS):
        cmd = ["gcc", *FLAVORS[flavor], "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
               *_SRCS, "-o", so + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(so + ".tmp", so)
    return so


_flavors: dict = {}


def _load(flavor: str = "O2"):
    global _lib
    with _lock:
        if flavor != "O2":
            if flavor not in _flavors:
                _flavors[flavor] = _bind(ctypes.CDLL(build(flavor=flavor)))
            return _flavors[flavor]
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_SO))
    return _lib


def _bind(lib):
    """Declare the argument and result types of the exported functions."""
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.oracle_fit.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_double, ctypes.c_int, ctypes.c_int, ip, ctypes.c_int,
                               ctypes.c_int, dp, dp, ip, dp, dp, dp, dp, ip, dp, ip]
    lib.oracle_cgs.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int]
    lib.oracle_cgs.restype = ctypes.c_int
    lib.oracle_block_fit.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_int, ip, dp, dp, dp, ip, dp, ip]
    lib.oracle_block_fit.restype = ctypes.c_int
    lib.oracle_ws_nparams.restype = ctypes.c_int
    lib.oracle_ws_features.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, dp]
    lib.oracle_ws_features.restype = ctypes.c_int
    lib.oracle_ws_forward.argtypes = [dp, dp, ctypes.c_int, dp]
    lib.oracle_ws_forward.restype = None
    lib.oracle_ws_loss_grad.argtypes = [dp, dp, dp, ip, ctypes.c_int, dp]
    lib.oracle_ws_loss_grad.restype = ctypes.c_double
    lib.oracle_ws_adam.argtypes = [dp, dp, dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_int]
    lib.oracle_ws_adam.restype = None
    lib.oracle_round_bf16.argtypes = [ctypes.c_double]
    lib.oracle_round_bf16.restype = ctypes.c_double
    lib.oracle_fit.restype = ctypes.c_int
    lib.oracle_center.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.oracle_center.restype = ctypes.c_int
    lib.oracle_jacobi_eigh.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                       dp, dp]
    lib.oracle_jacobi_eigh.restype = ctypes.c_int
    return lib


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
    ws_choice: np.ndarray | None = None  # per component: 1 if the learned start was used
    ws_rho: np.ndarray | None = None     # per component: (rho_plain, rho_learned)


STORAGE = {"f64": 0, "bf16": 1}


def fit(X: np.ndarray, K: int, tol: float = 1e-6, max_iter: int = 1000, algo: int | str = GS,
        center: int = CENTER_NONE, iters_lock=None, storage: str = "f64", ws_net=None, ws_G=None,
        gs_passes: int = 1, flavor: str = "O2") -> Fit:
    """Run NIPALS-PCA (algo=0/'nipals') or GS-PCA (algo=1/'gs') on X (M×N) in FP64.

    gs_passes (GS-PCA): classical Gram-Schmidt passes per half-iteration, 1 as in the
    Sec. 2.3 pseudo-code, 2 for the iterated form (CGS2).

    storage="bf16": the residual R is rounded to bfloat16 after centring and after
    every deflation (Eq. 3); all arithmetic stays FP64.
    ws_net (5377 parameters) and ws_G (M×16 sketch): GS-PCA with the learned warm start
    (warmstart.c).
    flavor: which build runs the fit (FLAVORS; the results do not depend on it)."""
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
    net = G = choice = rho = None
    if ws_net is not None:
        net = np.ascontiguousarray(np.asarray(ws_net, dtype=np.float64))
        G = np.ascontiguousarray(np.asarray(ws_G, dtype=np.float64)[:M])
        if net.shape != (ws_nparams(),) or G.shape != (M, 16):
            raise ValueError("ws_net must hold 5377 parameters and ws_G at least M x 16 values")
        choice = np.zeros(K, dtype=np.int32)
        rho = np.zeros(2 * K, dtype=np.float64)
    nul = ctypes.POINTER(ctypes.c_double)()
    st = _load(flavor).oracle_fit(algo, _dptr(X), M, N, K, float(tol), int(max_iter), int(center),
                            _iptr(lock), STORAGE[storage], int(gs_passes), _dptr(net) if net is not None else nul,
                            _dptr(G) if G is not None else nul, _iptr(choice), _dptr(rho) if rho is not None else nul,
                            _dptr(T), _dptr(P), _dptr(lam), _iptr(iters), _dptr(R), _iptr(found))
    if st == 1:
        raise ValueError("oracle_fit: invalid argument")
    return Fit(T=T, P=P, lam=lam, iters=iters, R=R, found=int(found[0]), status=int(st), ws_choice=choice,
               ws_rho=None if rho is None else rho.reshape(K, 2))


def block_fit(X: np.ndarray, K: int, b: int, tol: float = 1e-6, max_iter: int = 1000, iters_lock=None,
              flavor: str = "O2") -> Fit:
    """Block power iteration (oracle.c, oracle_block_fit): components b at a time, FP64."""
    X = np.asfortranarray(np.asarray(X, dtype=np.float64))
    M, N = X.shape
    T = np.zeros((M, K), order="F")
    P = np.zeros((N, K), order="F")
    R = np.zeros((M, N), order="F")
    lam = np.zeros(K)
    iters = np.zeros(K, dtype=np.int32)
    found = np.zeros(1, dtype=np.int32)
    lock = None
    if iters_lock is not None:
        lock = np.ascontiguousarray(np.asarray(iters_lock, dtype=np.int32))
    st = _load(flavor).oracle_block_fit(_dptr(X), M, N, K, int(b), float(tol), int(max_iter), _iptr(lock), _dptr(T),
                                        _dptr(P), _dptr(lam), _iptr(iters), _dptr(R), _iptr(found))
    if st == 1:
        raise ValueError("oracle_block_fit: invalid argument")
    return Fit(T=T, P=P, lam=lam, iters=iters, R=R, found=int(found[0]), status=int(st))


# ------------------------------------------------------------ learned warm start

def ws_nparams() -> int:
    return int(_load().oracle_ws_nparams())


def ws_features(R: np.ndarray, G: np.ndarray) -> np.ndarray:
    """Features (N×17) of every column of the residual R (M×N) with sketch G (M×16)."""
    R = np.asfortranarray(np.asarray(R, dtype=np.float64))
    M, N = R.shape
    G = np.ascontiguousarray(np.asarray(G, dtype=np.float64)[:M])
    out = np.zeros((N, 17), dtype=np.float64)
    if _load().oracle_ws_features(_dptr(R), M, N, _dptr(G), _dptr(out)) != 0:
        raise ValueError("oracle_ws_features: invalid argument")
    return out


def ws_forward(net: np.ndarray, feat: np.ndarray) -> np.ndarray:
    """Network output w (one value per feature row)."""
    net = np.ascontiguousarray(np.asarray(net, dtype=np.float64))
    feat = np.ascontiguousarray(np.asarray(feat, dtype=np.float64))
    w = np.zeros(feat.shape[0], dtype=np.float64)
    _load().oracle_ws_forward(_dptr(net), _dptr(feat), feat.shape[0], _dptr(w))
    return w


def ws_loss_grad(net, feat, target, offsets):
    """(mean loss, gradient) over instances; instance i owns rows offsets[i]:offsets[i+1]."""
    net = np.ascontiguousarray(np.asarray(net, dtype=np.float64))
    feat = np.ascontiguousarray(np.asarray(feat, dtype=np.float64))
    target = np.ascontiguousarray(np.asarray(target, dtype=np.float64))
    offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    g = np.zeros(ws_nparams(), dtype=np.float64)
    loss = _load().oracle_ws_loss_grad(_dptr(net), _dptr(feat), _dptr(target), _iptr(offs), len(offs) - 1,
                                       _dptr(g))
    return float(loss), g


def ws_adam(net, m, v, grad, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in place on float64 arrays net, m, v."""
    _load().oracle_ws_adam(_dptr(net), _dptr(m), _dptr(v), _dptr(np.ascontiguousarray(grad, dtype=np.float64)),
                           int(t), float(lr), float(b1), float(b2), float(eps), len(net))


def cgs(Q: np.ndarray, x: np.ndarray, passes: int = 1):
    """`passes` classical Gram-Schmidt passes of x against the columns of Q: (x', last coefficients)."""
    Q = np.asfortranarray(np.asarray(Q, dtype=np.float64))
    rows, k = Q.shape
    xx = np.array(x, dtype=np.float64, copy=True)
    coef = np.zeros(k)
    if _load().oracle_cgs(_dptr(Q), rows, k, _dptr(xx), _dptr(coef), int(passes)) != 0:
        raise ValueError("oracle_cgs: invalid argument")
    return xx, coef


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
