"""Seeded synthetic inputs for the iterative-PCA workloads.

This module only *draws* input matrices.  It contains none of the PCA
arithmetic (no power iteration, no Gram-Schmidt, no deflation), so both the
FP64 oracle and the CUDA path can consume its output without sharing any of
the method's code.

Every generator is a pure function of its arguments and a seed: numpy's
PCG64 stream seeded through ``SeedSequence`` (platform independent).

Workloads (shapes follow the paper's experiment, Sec. 4, and the planted
spectra used to pin accuracy):

* ``planted``      X = L diag(s) Rᵀ + noise·N(0,1), column-centred.  L (M×r) is
                   the Q factor of a column-centred Gaussian, so 1ᵀL = 0 and the
                   noise-free part is exactly column-centred; Rt (N×r) is the
                   Q factor of a Gaussian.  r = min(M, N).  s_i = s0·ratio**i.
* ``collinear``    B ~ N(0,1) (M×N0), X = [B | B + eps·E], column-centred
                   (the high-collinearity case where NIPALS loses
                   orthogonality, Sec. 1 and Sec. 2.3).
* ``uniform``      X_mn ~ U[0,1) as in the paper's own test matrices (Sec. 4,
                   Appendices), N = M/2.
* ``batch_shapes`` 256 (M_i, N_i) pairs, log-uniform in [256, 8192]×[64, 1024].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "rng",
    "planted",
    "collinear",
    "uniform",
    "batch_shapes",
    "batch_problem",
    "gaussian_sketch",
    "Workload",
    "WORKLOADS",
]


def rng(*key: int) -> np.random.Generator:
    """A PCG64 generator keyed by a tuple of non-negative ints."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(list(key))))


def _orthonormal(g: np.random.Generator, rows: int, cols: int, centre: bool) -> np.ndarray:
    a = g.standard_normal((rows, cols))
    if centre:
        a -= a.mean(axis=0, keepdims=True)
    q, r = np.linalg.qr(a)
    # Fix the sign ambiguity of the QR factor so the draw is reproducible
    # independently of the LAPACK build.
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d


@dataclass
class Planted:
    X: np.ndarray          # M×N float64, C order
    left: np.ndarray       # M×r orthonormal score directions of the noise-free part
    right: np.ndarray      # N×r orthonormal loadings of the noise-free part
    s: np.ndarray          # r planted singular values (descending)


def planted(M: int, N: int, s0: float, ratio: float, noise: float, seed,
            centre: bool = True) -> Planted:
    """X = L·diag(s)·Rᵀ + noise·N(0,1), then column-centred (each column zero mean)."""
    key = seed if isinstance(seed, tuple) else (seed,)
    g = rng(*key)
    r = min(M, N)
    # With r == M a column-centred M×M basis cannot exist (rank M-1): centre
    # the left factor only when there is room for it.
    left = _orthonormal(g, M, r, centre=centre and r < M)
    right = _orthonormal(g, N, r, centre=False)
    s = s0 * ratio ** np.arange(r, dtype=np.float64)
    X = (left * s) @ right.T
    if noise > 0:
        X = X + noise * g.standard_normal((M, N))
    if centre:
        X = X - X.mean(axis=0, keepdims=True)
    return Planted(X=np.ascontiguousarray(X), left=left, right=right, s=s)


def collinear(M: int = 4096, N0: int = 512, eps: float = 1e-3, seed: int = 2) -> np.ndarray:
    """X = [B | B + eps·E], B, E ~ N(0,1) (M×N0 each), column-centred."""
    g = rng(seed)
    B = g.standard_normal((M, N0))
    E = g.standard_normal((M, N0))
    X = np.concatenate([B, B + eps * E], axis=1)
    X -= X.mean(axis=0, keepdims=True)
    return np.ascontiguousarray(X)


def uniform(M: int, N: int | None = None, seed: int = 7) -> np.ndarray:
    """The paper's test matrix: entries uniform in [0, 1), N = M/2 by default."""
    if N is None:
        N = M // 2
    return rng(seed).random((M, N))


def batch_shapes(count: int = 256, seed: int = 3,
                 m_range=(256, 8192), n_range=(64, 1024)) -> list[tuple[int, int]]:
    """(M_i, N_i) log-uniform in the given closed ranges."""
    g = rng(seed, 1_000_000)
    lm = g.uniform(math.log(m_range[0]), math.log(m_range[1]), size=count)
    ln = g.uniform(math.log(n_range[0]), math.log(n_range[1]), size=count)
    Ms = np.clip(np.rint(np.exp(lm)).astype(int), *m_range)
    Ns = np.clip(np.rint(np.exp(ln)).astype(int), *n_range)
    return [(int(m), int(n)) for m, n in zip(Ms, Ns)]


def batch_problem(i: int, M: int, N: int, seed: int = 3, s0: float = 10.0,
                  ratio: float = 0.9, noise: float = 0.01) -> Planted:
    """Problem i of a batch: planted spectrum drawn from stream (seed, i)."""
    return planted(M, N, s0, ratio, noise, (seed, i))


def gaussian_sketch(M: int, width: int = 16, seed: int = 11) -> np.ndarray:
    """G (M×width) with N(0, 1/width) entries, for column sketches GᵀR."""
    return rng(seed, M).standard_normal((M, width)) / math.sqrt(width)


@dataclass(frozen=True)
class Workload:
    """One named workload: the generator call plus the fit parameters."""
    name: str
    M: int
    N: int
    K: int
    tol: float
    max_iter: int
    kind: str                     # "planted" | "collinear" | "uniform"
    s0: float = 0.0
    ratio: float = 0.0
    noise: float = 0.0
    seed: int = 0
    extra: dict = field(default_factory=dict, hash=False, compare=False)

    def make(self) -> np.ndarray:
        if self.kind == "planted":
            return planted(self.M, self.N, self.s0, self.ratio, self.noise, self.seed).X
        if self.kind == "collinear":
            return collinear(self.M, self.N // 2, self.extra.get("eps", 1e-3), self.seed)
        if self.kind == "uniform":
            return uniform(self.M, self.N, self.seed)
        raise ValueError(self.kind)


WORKLOADS = {
    # 500×200 planted spectrum s_i = 10·0.85^i, noise 0.01, K = 10 (small case)
    "planted_500x200": Workload("planted_500x200", 500, 200, 10, 1e-6, 1000, "planted",
                                10.0, 0.85, 0.01, 0),
    # 10000×2000 planted spectrum s_i = 100·0.95^i, noise 0.05, K = 50 (80 MB FP32)
    "planted_10000x2000": Workload("planted_10000x2000", 10000, 2000, 50, 1e-6, 1000,
                                   "planted", 100.0, 0.95, 0.05, 1),
    # 4096×1024 duplicated-column matrix, K = N = 1024 (full spectrum)
    "collinear_4096x1024": Workload("collinear_4096x1024", 4096, 1024, 1024, 1e-6, 1000,
                                    "collinear", seed=2, extra={"eps": 1e-3}),
    # paper-shaped uniform matrix at the largest size of its Figure 1 sweep
    "uniform_15000x7500": Workload("uniform_15000x7500", 15000, 7500, 10, 1e-7, 10000,
                                   "uniform", seed=7),
}
