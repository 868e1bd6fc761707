"""Python binding of the C ABI in ``include/gspca.h``.

Argument marshalling only: every step of NIPALS-PCA / GS-PCA runs in the
CUDA library ``_lib/libgspca.so`` (built by ``build.py``).  PyTorch supplies
device memory and the current CUDA stream.  There is no CPU fallback: when
the library is missing, importing the entry points raises.

Thin wrappers keep the C names (``gspca_create``, ``gspca_fit``,
``gspca_fit_host``, ``gspca_fit_batched``, ``gspca_get_info``,
``gspca_destroy``, ``gspca_status_string``); ``Handle`` bundles them.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

from .buildlib import LIB, build

GSPCA_NIPALS, GSPCA_GS = 0, 1
GSPCA_F32, GSPCA_BF16, GSPCA_F64 = 0, 1, 2
GSPCA_COL_MAJOR, GSPCA_ROW_MAJOR = 0, 1
GSPCA_CENTER_NONE, GSPCA_CENTER_COLUMNS, GSPCA_CENTER_ROWS = 0, 1, 2
GSPCA_OK = 0
GSPCA_ERR_INVALID_ARG = 1
GSPCA_ERR_CUDA = 2
GSPCA_ERR_OOM = 3
GSPCA_WARN_NOT_CONVERGED = 4
GSPCA_ERR_DEGENERATE = 5
GSPCA_ERR_TIMEOUT = 6
GSPCA_ERR_NOT_SUPPORTED = 7

EXPORTS = ["gspca_create", "gspca_fit", "gspca_fit_host", "gspca_fit_batched", "gspca_fit_batched_async",
           "gspca_get_info", "gspca_destroy", "gspca_status_string", "gspca_last_cuda_error",
           "gspca_fit_noalloc", "gspca_ws_features", "gspca_ws_forward", "gspca_ws_train_step", "gspca_fit_f64",
           "gspca_fit_block"]

WS_SKETCH, WS_FEATURES, WS_PARAMS = 16, 17, 5377

_ALGOS = {"nipals": GSPCA_NIPALS, "gs": GSPCA_GS, GSPCA_NIPALS: GSPCA_NIPALS, GSPCA_GS: GSPCA_GS}
_DTYPES = {"f32": GSPCA_F32, "bf16": GSPCA_BF16, "f64": GSPCA_F64, GSPCA_F32: GSPCA_F32, GSPCA_BF16: GSPCA_BF16,
           GSPCA_F64: GSPCA_F64}


class GspcaError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = f"{where}: {status_string(status)}"
        if status == GSPCA_ERR_CUDA:
            msg += f" ({last_cuda_error()})"
        super().__init__(msg)


class WarmStartC(ctypes.Structure):
    _fields_ = [("net", ctypes.c_void_p), ("G", ctypes.c_void_p), ("G_rows", ctypes.c_long),
                ("choice", ctypes.c_void_p)]


class Opts(ctypes.Structure):
    _fields_ = [("center", ctypes.c_int), ("iters_lock", ctypes.POINTER(ctypes.c_int)),
                ("grid_ctas", ctypes.c_int), ("timeout_s", ctypes.c_double),
                ("cluster_ctas", ctypes.c_int), ("batch_pass", ctypes.c_int), ("test_stall", ctypes.c_int),
                ("warm", ctypes.POINTER(WarmStartC)), ("resident", ctypes.c_int), ("load_path", ctypes.c_int),
                ("gs_step", ctypes.c_int), ("gs_passes", ctypes.c_int), ("svd_form", ctypes.c_int),
                ("coef_trace", ctypes.c_void_p)]


class Info(ctypes.Structure):
    _fields_ = [("found", ctypes.c_int), ("total_iters", ctypes.c_longlong),
                ("kernel_launches", ctypes.c_int), ("grid_ctas", ctypes.c_int),
                ("block_threads", ctypes.c_int), ("alg_bytes", ctypes.c_double),
                ("kernel_ms", ctypes.c_double), ("team_ctas", ctypes.c_int), ("batch_pass", ctypes.c_int)]


class Problem(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("ldx", ctypes.c_long), ("M", ctypes.c_int),
                ("N", ctypes.c_int), ("K", ctypes.c_int), ("T", ctypes.c_void_p),
                ("P", ctypes.c_void_p), ("lambda_", ctypes.c_void_p), ("iters", ctypes.c_void_p),
                ("status", ctypes.c_void_p), ("ws_choice", ctypes.c_void_p)]


_lib = None


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libgspca.so; raise when it is absent (never fall back to anything)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built: {LIB} is missing (run build())")
        build()
    lib = ctypes.CDLL(LIB)
    vp, i, l, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_long, ctypes.c_double
    lib.gspca_create.argtypes = [ctypes.POINTER(vp), i, l, l, i, i]
    fit_args = [vp, vp, vp, i, l, i, i, i, d, i, i, vp, vp, vp, vp, vp, ctypes.POINTER(Opts)]
    lib.gspca_fit.argtypes = fit_args
    lib.gspca_fit_host.argtypes = fit_args
    lib.gspca_fit_batched.argtypes = [vp, vp, ctypes.POINTER(Problem), i, d, i, i, ctypes.POINTER(Opts)]
    lib.gspca_fit_batched_async.argtypes = [vp, vp, ctypes.POINTER(Problem), i, d, i, i, ctypes.POINTER(Opts), vp]
    lib.gspca_fit_f64.argtypes = fit_args
    lib.gspca_fit_block.argtypes = [vp, vp, vp, i, l, i, i, i, i, d, i, vp, vp, vp, vp, vp, ctypes.POINTER(Opts)]
    lib.gspca_fit_block.restype = i
    lib.gspca_fit_noalloc.argtypes = fit_args[1:]
    lib.gspca_fit_noalloc.restype = i
    lib.gspca_ws_features.argtypes = [vp, vp, l, i, i, vp, vp, i, vp, vp]
    lib.gspca_ws_forward.argtypes = [vp, vp, vp, l, vp]
    lib.gspca_ws_train_step.argtypes = [vp, vp, vp, vp, vp, i, ctypes.c_float, vp, vp, vp, i, l, vp, vp]
    lib.gspca_get_info.argtypes = [vp, ctypes.POINTER(Info)]
    lib.gspca_destroy.argtypes = [vp]
    lib.gspca_status_string.argtypes = [i]
    lib.gspca_status_string.restype = ctypes.c_char_p
    lib.gspca_last_cuda_error.argtypes = []
    lib.gspca_last_cuda_error.restype = ctypes.c_char_p
    for name in ("gspca_create", "gspca_fit", "gspca_fit_host", "gspca_fit_batched",
                 "gspca_fit_batched_async", "gspca_get_info", "gspca_destroy", "gspca_ws_features", "gspca_fit_f64",
                 "gspca_ws_forward", "gspca_ws_train_step"):
        getattr(lib, name).restype = i
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().gspca_status_string(int(status)).decode()


gspca_status_string = status_string


def last_cuda_error() -> str:
    return load().gspca_last_cuda_error().decode()


gspca_last_cuda_error = last_cuda_error


class WarmStart:
    """Learned warm start: network parameters (GSPCA_WS_PARAMS float32 CUDA values) and the
    sketch G (rows x 16 float32 CUDA, row-major; a problem of M rows uses the first M)."""

    def __init__(self, net, G):
        import torch

        if not (isinstance(net, torch.Tensor) and net.is_cuda and net.dtype == torch.float32
                and net.numel() == WS_PARAMS and net.is_contiguous()):
            raise TypeError("net must be a contiguous float32 CUDA tensor of 5377 values")
        if not (isinstance(G, torch.Tensor) and G.is_cuda and G.dtype == torch.float32 and G.dim() == 2
                and G.shape[1] == WS_SKETCH and G.is_contiguous()):
            raise TypeError("G must be a contiguous float32 CUDA tensor of shape (rows, 16)")
        self.net, self.G = net, G

    def c_struct(self, choice=None):
        return WarmStartC(self.net.data_ptr(), self.G.data_ptr(), self.G.shape[0],
                          choice.data_ptr() if choice is not None else None)


def _opts(center=0, iters_lock=None, grid_ctas=0, timeout_s=0.0, cluster_ctas=0, test_stall=0, batch_pass=0,
          warm=None, resident=0, load_path=0, gs_step=0, gs_passes=0, svd_form=0, coef_trace=None):
    o = Opts()
    o.coef_trace = coef_trace.data_ptr() if coef_trace is not None else None
    o.gs_passes = int(gs_passes)
    o.svd_form = int(svd_form)
    o.resident = int(resident)
    o.load_path = int(load_path)
    o.gs_step = int(gs_step)
    o.batch_pass = int(batch_pass)
    o.test_stall = int(test_stall)
    o.center = int(center)
    o.grid_ctas = int(grid_ctas)
    o.timeout_s = float(timeout_s)
    o.cluster_ctas = int(cluster_ctas)
    keep = None
    if iters_lock is not None:
        keep = (ctypes.c_int * len(iters_lock))(*[int(v) for v in iters_lock])
        o.iters_lock = ctypes.cast(keep, ctypes.POINTER(ctypes.c_int))
    if warm is not None:
        o.warm = ctypes.pointer(warm)
        keep = (keep, warm)
    return o, keep


def gspca_create(device: int, max_M: int, max_N: int, max_K: int, dtype="f32") -> int:
    h = ctypes.c_void_p()
    st = load().gspca_create(ctypes.byref(h), int(device), int(max_M), int(max_N), int(max_K),
                             _DTYPES[dtype])
    if st != GSPCA_OK:
        raise GspcaError(st, "gspca_create")
    return h.value


def gspca_destroy(h: int) -> int:
    return load().gspca_destroy(ctypes.c_void_p(h))


def gspca_get_info(h: int) -> dict:
    info = Info()
    st = load().gspca_get_info(ctypes.c_void_p(h), ctypes.byref(info))
    if st != GSPCA_OK:
        raise GspcaError(st, "gspca_get_info")
    return {f: getattr(info, f) for f, _ in Info._fields_}


def _layout_of(X):
    """(layout, ldx) of a 2-D tensor/array given its strides in elements."""
    M, N = X.shape
    s0, s1 = (X.stride() if hasattr(X, "stride") and callable(X.stride)
              else tuple(s // X.itemsize for s in X.strides))
    if s1 == 1 and s0 >= N:
        return GSPCA_ROW_MAJOR, s0
    if s0 == 1 and s1 >= M:
        return GSPCA_COL_MAJOR, s1
    return None, None


@dataclass
class FitResult:
    T: object
    P: object
    lam: object
    iters: object
    R: object
    status: int
    info: dict
    ws_choice: object = None


def gspca_fit(h: int, X, K: int, tol: float = 1e-6, max_iter: int = 1000, algo="gs",
              center: int = 0, iters_lock=None, want_R: bool = False, grid_ctas: int = 0,
              timeout_s: float = 0.0, stream=None, check: bool = True, test_stall: int = 0,
              warm: WarmStart | None = None, resident: int = 0, load_path: int = 0,
              gs_step: int = 0, gs_passes: int = 0, svd_form: int = 0, coef_trace=None) -> FitResult:
    """Fit K components of X (a float32 CUDA tensor, any 2-D strided layout).  `warm`: the
    learned warm start (GS-PCA); the result's ws_choice marks the components that used it.
    `gs_passes=2`: two classical Gram-Schmidt passes per half-iteration (CGS2).
    `svd_form=1`: T receives the unit score directions (X = T diag(lam) P^T + R).
    `coef_trace` (testing aid): a float32 CUDA tensor of K * (2K + M + N) values, see gspca.h."""
    import torch

    if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.float32 and X.dim() == 2):
        raise TypeError("X must be a 2-D float32 CUDA tensor")
    layout, ldx = _layout_of(X)
    if layout is None:
        X = X.contiguous()
        layout, ldx = GSPCA_ROW_MAJOR, X.shape[1]
    M, N = X.shape
    dev = X.device
    T = torch.empty((K, M), device=dev, dtype=torch.float32).t()
    P = torch.empty((K, N), device=dev, dtype=torch.float32).t()
    lam = torch.empty(K, device=dev, dtype=torch.float64)
    iters = torch.empty(K, device=dev, dtype=torch.int32)
    R = torch.empty((N, M), device=dev, dtype=torch.float32).t() if want_R else None
    if stream is None:
        stream = torch.cuda.current_stream(dev).cuda_stream
    choice = torch.zeros(K, device=dev, dtype=torch.int32) if warm is not None else None
    o, keep = _opts(center, iters_lock, grid_ctas, timeout_s, 0, test_stall,
                    warm=warm.c_struct(choice) if warm is not None else None, resident=resident,
                    load_path=load_path, gs_step=gs_step, gs_passes=gs_passes, svd_form=svd_form,
                    coef_trace=coef_trace)
    st = load().gspca_fit(ctypes.c_void_p(h), ctypes.c_void_p(stream), ctypes.c_void_p(X.data_ptr()),
                          layout, int(ldx), M, N, int(K), float(tol), int(max_iter), _ALGOS[algo],
                          ctypes.c_void_p(T.data_ptr()), ctypes.c_void_p(P.data_ptr()),
                          ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(iters.data_ptr()),
                          ctypes.c_void_p(R.data_ptr()) if R is not None else None, ctypes.byref(o))
    del keep
    if check and st not in (GSPCA_OK, GSPCA_WARN_NOT_CONVERGED, GSPCA_ERR_DEGENERATE):
        raise GspcaError(st, "gspca_fit")
    return FitResult(T, P, lam, iters, R, st, gspca_get_info(h), choice)


def gspca_fit_f64(h: int, X, K: int, tol: float = 1e-6, max_iter: int = 1000, algo="gs", center: int = 0,
                  iters_lock=None, want_R: bool = False, grid_ctas: int = 0, timeout_s: float = 0.0, stream=None,
                  check: bool = True, svd_form: int = 0) -> FitResult:
    """FP64 fit on a handle created with dtype="f64": X a 2-D float64 CUDA tensor (any row- or
    column-major strides); T, P, lam and R are float64."""
    import torch

    if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.float64 and X.dim() == 2):
        raise TypeError("X must be a 2-D float64 CUDA tensor")
    layout, ldx = _layout_of(X)
    if layout is None:
        X = X.contiguous()
        layout, ldx = GSPCA_ROW_MAJOR, X.shape[1]
    M, N = X.shape
    dev = X.device
    T = torch.empty((K, M), device=dev, dtype=torch.float64).t()
    P = torch.empty((K, N), device=dev, dtype=torch.float64).t()
    lam = torch.empty(K, device=dev, dtype=torch.float64)
    iters = torch.empty(K, device=dev, dtype=torch.int32)
    R = torch.empty((N, M), device=dev, dtype=torch.float64).t() if want_R else None
    if stream is None:
        stream = torch.cuda.current_stream(dev).cuda_stream
    o, keep = _opts(center, iters_lock, grid_ctas, timeout_s, svd_form=svd_form)
    st = load().gspca_fit_f64(ctypes.c_void_p(h), ctypes.c_void_p(stream), ctypes.c_void_p(X.data_ptr()), layout,
                              int(ldx), M, N, int(K), float(tol), int(max_iter), _ALGOS[algo],
                              ctypes.c_void_p(T.data_ptr()), ctypes.c_void_p(P.data_ptr()),
                              ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(iters.data_ptr()),
                              ctypes.c_void_p(R.data_ptr()) if R is not None else None, ctypes.byref(o))
    del keep
    if check and st not in (GSPCA_OK, GSPCA_WARN_NOT_CONVERGED, GSPCA_ERR_DEGENERATE):
        raise GspcaError(st, "gspca_fit_f64")
    return FitResult(T, P, lam, iters, R, st, gspca_get_info(h))


def gspca_fit_block(h: int, X, K: int, block: int = 16, tol: float = 1e-6, max_iter: int = 1000, center: int = 0,
                    iters_lock=None, want_R: bool = False, stream=None, check: bool = True,
                    svd_form: int = 0) -> FitResult:
    """Block power iteration (components `block` at a time) on a float32 handle; X a 2-D float32
    CUDA tensor.  iters_lock: K counts, entry k0 fixes the iterations of the block starting at k0."""
    import torch

    if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.float32 and X.dim() == 2):
        raise TypeError("X must be a 2-D float32 CUDA tensor")
    layout, ldx = _layout_of(X)
    if layout is None:
        X = X.contiguous()
        layout, ldx = GSPCA_ROW_MAJOR, X.shape[1]
    M, N = X.shape
    dev = X.device
    T = torch.empty((K, M), device=dev, dtype=torch.float32).t()
    P = torch.empty((K, N), device=dev, dtype=torch.float32).t()
    lam = torch.empty(K, device=dev, dtype=torch.float64)
    iters = torch.empty(K, device=dev, dtype=torch.int32)
    R = torch.empty((N, M), device=dev, dtype=torch.float32).t() if want_R else None
    if stream is None:
        stream = torch.cuda.current_stream(dev).cuda_stream
    o, keep = _opts(center, iters_lock, svd_form=svd_form)
    st = load().gspca_fit_block(ctypes.c_void_p(h), ctypes.c_void_p(stream), ctypes.c_void_p(X.data_ptr()), layout,
                                int(ldx), M, N, int(K), int(block), float(tol), int(max_iter),
                                ctypes.c_void_p(T.data_ptr()), ctypes.c_void_p(P.data_ptr()),
                                ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(iters.data_ptr()),
                                ctypes.c_void_p(R.data_ptr()) if R is not None else None, ctypes.byref(o))
    del keep
    if check and st not in (GSPCA_OK, GSPCA_WARN_NOT_CONVERGED, GSPCA_ERR_DEGENERATE):
        raise GspcaError(st, "gspca_fit_block")
    return FitResult(T, P, lam, iters, R, st, gspca_get_info(h))


def gspca_fit_host(h: int, X, K: int, tol: float = 1e-6, max_iter: int = 1000, algo="gs",
                   center: int = 0, iters_lock=None, want_R: bool = False, stream=None,
                   out=None, check: bool = True, gs_passes: int = 0, svd_form: int = 0) -> FitResult:
    """Same as gspca_fit with host memory: X a float32 numpy array or CPU tensor (pinned is
    fastest); outputs are host arrays (reused from `out` when given)."""
    import numpy as np

    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(X, torch.Tensor):
        if X.is_cuda or X.dtype != torch.float32:
            raise TypeError("X must be a float32 host tensor")
        xp = X.data_ptr()
        layout, ldx = _layout_of(X)
    else:
        X = np.asarray(X)
        if X.dtype != np.float32:
            raise TypeError("X must be float32")
        layout, ldx = _layout_of(X)
        xp = X.ctypes.data
    if layout is None:
        raise ValueError("X must be row- or column-major")
    M, N = X.shape
    if out is None:
        out = {"T": np.empty((K, M), np.float32), "P": np.empty((K, N), np.float32),
               "lam": np.empty(K, np.float64), "iters": np.empty(K, np.int32),
               "R": np.empty((N, M), np.float32) if want_R else None}
    if stream is None and torch is not None and torch.cuda.is_available():
        stream = torch.cuda.current_stream().cuda_stream
    o, keep = _opts(center, iters_lock, gs_passes=gs_passes, svd_form=svd_form)
    st = load().gspca_fit_host(ctypes.c_void_p(h), ctypes.c_void_p(stream), ctypes.c_void_p(xp), layout,
                               int(ldx), M, N, int(K), float(tol), int(max_iter), _ALGOS[algo],
                               ctypes.c_void_p(out["T"].ctypes.data), ctypes.c_void_p(out["P"].ctypes.data),
                               ctypes.c_void_p(out["lam"].ctypes.data),
                               ctypes.c_void_p(out["iters"].ctypes.data),
                               ctypes.c_void_p(out["R"].ctypes.data) if out["R"] is not None else None,
                               ctypes.byref(o))
    del keep
    if check and st not in (GSPCA_OK, GSPCA_WARN_NOT_CONVERGED, GSPCA_ERR_DEGENERATE):
        raise GspcaError(st, "gspca_fit_host")
    R = out["R"].T if out["R"] is not None else None
    return FitResult(out["T"].T, out["P"].T, out["lam"], out["iters"], R, st, gspca_get_info(h))


class Handle:
    """Owns one gspca handle (device workspace for problems up to max_M x max_N x max_K)."""

    def __init__(self, max_M: int, max_N: int, max_K: int, device: int = 0, dtype="f32"):
        self.h = gspca_create(device, max_M, max_N, max_K, dtype)

    def fit(self, X, K, **kw) -> FitResult:
        return gspca_fit(self.h, X, K, **kw)

    def fit_host(self, X, K, **kw) -> FitResult:
        return gspca_fit_host(self.h, X, K, **kw)

    def fit64(self, X, K, **kw) -> FitResult:
        return gspca_fit_f64(self.h, X, K, **kw)

    def fit_block(self, X, K, **kw) -> FitResult:
        return gspca_fit_block(self.h, X, K, **kw)

    def info(self) -> dict:
        return gspca_get_info(self.h)

    def close(self):
        if self.h:
            gspca_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Descriptors and output tensors of a batch of independent problems.

    `problems` is a list of dicts with a float32 CUDA tensor "X" (a row-major X is copied
    to column-major here) and "K".  `results` holds, per problem, a FitResult whose T, P,
    lam, iters and status (a 1-element int32 tensor) the library writes."""

    def __init__(self, problems):
        import torch

        self.descs = (Problem * len(problems))()
        self.keep = []
        self.outs = []
        for i, pr in enumerate(problems):
            X = pr["X"]
            if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.float32
                    and X.dim() == 2):
                raise TypeError("each X must be a 2-D float32 CUDA tensor")
            layout, ldx = _layout_of(X)
            if layout != GSPCA_COL_MAJOR:
                X = X.t().contiguous().t()
                ldx = X.shape[0]
            self.keep.append(X)
            M, N = X.shape
            K = int(pr["K"])
            dev = X.device
            T = torch.zeros((K, M), device=dev, dtype=torch.float32).t()
            P = torch.zeros((K, N), device=dev, dtype=torch.float32).t()
            lam = torch.zeros(K, device=dev, dtype=torch.float64)
            iters = torch.zeros(K, device=dev, dtype=torch.int32)
            st = torch.full((1,), -1, device=dev, dtype=torch.int32)
            ch = torch.zeros(K, device=dev, dtype=torch.int32)
            d = self.descs[i]
            d.X, d.ldx, d.M, d.N, d.K = X.data_ptr(), int(ldx), M, N, K
            d.T, d.P, d.lambda_, d.iters, d.status = (T.data_ptr(), P.data_ptr(), lam.data_ptr(),
                                                      iters.data_ptr(), st.data_ptr())
            d.ws_choice = ch.data_ptr()
            self.outs.append(FitResult(T, P, lam, iters, None, st, {}, ch))

    def __len__(self):
        return len(self.outs)

    @property
    def results(self):
        return self.outs


def gspca_fit_batched(h: int, problems, tol: float = 1e-6, max_iter: int = 1000, algo="gs",
                      cluster_ctas: int = 0, timeout_s: float = 0.0, stream=None, check: bool = True,
                      test_stall: int = 0, batch_pass: int = 0, warm: WarmStart | None = None):
    """Fit independent problems in one persistent launch (per 256 problems) and wait.
    `problems` is a Batch or a list accepted by Batch; returns (Batch, worst status)."""
    import torch

    b = problems if isinstance(problems, Batch) else Batch(problems)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    o, _keep = _opts(0, None, 0, timeout_s, cluster_ctas, test_stall, batch_pass,
                     warm=warm.c_struct() if warm is not None else None)
    st = load().gspca_fit_batched(ctypes.c_void_p(h), ctypes.c_void_p(stream), b.descs, len(b),
                                  float(tol), int(max_iter), _ALGOS[algo], ctypes.byref(o))
    if check and st not in (GSPCA_OK, GSPCA_WARN_NOT_CONVERGED, GSPCA_ERR_DEGENERATE):
        raise GspcaError(st, "gspca_fit_batched")
    info = gspca_get_info(h)
    for r in b.outs:
        r.info = info
    return b, st


def gspca_fit_batched_async(h: int, batch: Batch, tol: float = 1e-6, max_iter: int = 1000, algo="gs",
                            cluster_ctas: int = 0, timeout_s: float = 0.0, worst=None, stream=None,
                            batch_pass: int = 0, warm: WarmStart | None = None) -> int:
    """Enqueue a batch without waiting (usable inside CUDA stream capture after one uncaptured
    call on the same shapes).  `worst` is an optional 1-element int32 CUDA tensor that receives
    the worst per-problem status.  Returns the enqueue status."""
    import torch

    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    o, _keep = _opts(0, None, 0, timeout_s, cluster_ctas, 0, batch_pass,
                     warm=warm.c_struct() if warm is not None else None)
    return load().gspca_fit_batched_async(ctypes.c_void_p(h), ctypes.c_void_p(stream), batch.descs, len(batch),
                                          float(tol), int(max_iter), _ALGOS[algo], ctypes.byref(o),
                                          ctypes.c_void_p(worst.data_ptr()) if worst is not None else None)


NOALLOC_SCRATCH_BYTES = 64 << 20


def gspca_fit_noalloc(X, K: int, tol: float = 1e-6, max_iter: int = 1000, algo="gs", center: int = 0,
                      iters_lock=None, want_R: bool = False, stream=None, check: bool = True,
                      timeout_s: float = 0.0, test_stall: int = 0, gs_passes: int = 0) -> FitResult:
    """gspca_fit without a handle and without any device allocation inside the library: the
    workspace is the library's fixed scratch array (NOALLOC_SCRATCH_BYTES per device).  For
    callers that must not allocate device memory.  Output tensors are the caller's (allocated
    here by PyTorch, outside the library)."""
    import torch

    if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.float32 and X.dim() == 2):
        raise TypeError("X must be a 2-D float32 CUDA tensor")
    layout, ldx = _layout_of(X)
    if layout is None:
        X = X.contiguous()
        layout, ldx = GSPCA_ROW_MAJOR, X.shape[1]
    M, N = X.shape
    dev = X.device
    T = torch.empty((K, M), device=dev, dtype=torch.float32).t()
    P = torch.empty((K, N), device=dev, dtype=torch.float32).t()
    lam = torch.empty(K, device=dev, dtype=torch.float64)
    iters = torch.empty(K, device=dev, dtype=torch.int32)
    R = torch.empty((N, M), device=dev, dtype=torch.float32).t() if want_R else None
    if stream is None:
        stream = torch.cuda.current_stream(dev).cuda_stream
    o, keep = _opts(center, iters_lock, timeout_s=timeout_s, test_stall=test_stall, gs_passes=gs_passes)
    with torch.cuda.device(dev):
        st = load().gspca_fit_noalloc(ctypes.c_void_p(stream), ctypes.c_void_p(X.data_ptr()), layout, int(ldx),
                                      M, N, int(K), float(tol), int(max_iter), _ALGOS[algo],
                                      ctypes.c_void_p(T.data_ptr()), ctypes.c_void_p(P.data_ptr()),
                                      ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(iters.data_ptr()),
                                      ctypes.c_void_p(R.data_ptr()) if R is not None else None,
                                      ctypes.byref(o))
    del keep
    if check and st not in (GSPCA_OK, GSPCA_WARN_NOT_CONVERGED, GSPCA_ERR_DEGENERATE):
        raise GspcaError(st, "gspca_fit_noalloc")
    return FitResult(T, P, lam, iters, R, st, {})


# ------------------------------------------------------------------ learned warm start

def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream, dev=None):
    import torch

    return stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream


def gspca_ws_features(X, G, T=None, P=None, k: int = 0, out=None, stream=None):
    """Features (N x 17 float32 CUDA) of the columns of R_k = X - T[:, :k] P[:, :k]^T; X column-major
    float32 CUDA (a transposed contiguous tensor), T and P as gspca_fit returns them."""
    import torch

    M, N = X.shape
    if X.stride(0) != 1:
        raise TypeError("X must be column-major")
    for t in (T, P):
        if t is not None and not (t.stride(0) == 1 and t.stride(1) == t.shape[0]):
            raise TypeError("T and P must be column-major with leading dimension = rows")
    feat = out if out is not None else torch.empty((N, WS_FEATURES), device=X.device, dtype=torch.float32)
    st = load().gspca_ws_features(ctypes.c_void_p(_stream(stream, X.device)), _ptr(X), int(X.stride(1)), M, N,
                                  _ptr(T) if k > 0 else None, _ptr(P) if k > 0 else None, int(k), _ptr(G),
                                  _ptr(feat))
    if st != GSPCA_OK:
        raise GspcaError(st, "gspca_ws_features")
    return feat


def gspca_ws_forward(net, feat, out=None, stream=None):
    """Network output for every feature row (float32 CUDA)."""
    import torch

    w = out if out is not None else torch.empty(feat.shape[0], device=feat.device, dtype=torch.float32)
    st = load().gspca_ws_forward(ctypes.c_void_p(_stream(stream, feat.device)), _ptr(net), _ptr(feat),
                                 int(feat.shape[0]), _ptr(w))
    if st != GSPCA_OK:
        raise GspcaError(st, "gspca_ws_forward")
    return w


def gspca_ws_train_step(h: int, net, m, v, step: int, lr: float, feat, target, offsets, loss=None, grad=None,
                        stream=None):
    """One Adam step of the network on the instances delimited by `offsets` (int32 CUDA)."""
    st = load().gspca_ws_train_step(ctypes.c_void_p(h), ctypes.c_void_p(_stream(stream, feat.device)), _ptr(net),
                                    _ptr(m), _ptr(v), int(step), float(lr), _ptr(feat), _ptr(target),
                                    _ptr(offsets), int(offsets.numel() - 1), int(feat.shape[0]), _ptr(loss),
                                    _ptr(grad))
    if st != GSPCA_OK:
        raise GspcaError(st, "gspca_ws_train_step")
