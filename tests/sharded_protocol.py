"""Row-sharded NIPALS-PCA / GS-PCA exchange protocol, in FP64 on CPU ranks.

Test infrastructure: it checks the multi-GPU design of the power-iteration
loop (Sec. 2.2 / 2.3 pseudo-code) without a second GPU.  It imports neither
the oracle nor the CUDA library.

Partitioning.  Rank p holds rows [r_p, r_{p+1}) of the residual R and of the
score factors V; the loadings U, W = R^T V and the k x k Gram matrix V^T V are
replicated.  One pass over the local rows forms v'_p = R_p u and, from the
same rows, s'_p = R_p^T v'_p, b'_p = V_p^T v'_p and ||v'_p||^2.

Exchange.  Exactly one reduction per power iteration, of N + k + 1 FP64 words
(s', b', ||v'||^2); everything else is replicated arithmetic:
  * R^T (v' - V b') = s' - W b' (W follows every deflation, Eq. 3, by a
    rank-1 update), so the loading needs no second pass over R;
  * ||v' - V b'||^2 = ||v'||^2 - 2 b'.b' + b'^T (V^T V) b';
  * a' = U^T (s' - W b') with U replicated.
The start of a component exchanges N + k + 1 words too (R^T R(k), the Gram row
V^T v_{k-1} for the W and V^T V updates, ||R(k)||^2); the zero-start-column
rule adds one exchange of the N column norms, and ||X||_F^2 is one word at the
start.  NIPALS exchanges N + 1 words per iteration.

Reduction order.  The reduction is an all-gather of the per-rank payloads
followed by a sum in rank order, so a run on P processes gives the same bits
as one process holding P virtual shards.
"""
from __future__ import annotations

import numpy as np


class LocalReduce:
    """All shards in this process: the ordered sum of their payloads."""

    def __init__(self):
        self.log: list[int] = []

    def __call__(self, payloads: list[np.ndarray]) -> np.ndarray:
        self.log.append(int(payloads[0].size))
        out = payloads[0].copy()
        for p in payloads[1:]:
            out = out + p
        return out


class GlooReduce:
    """One shard per process: all_gather over torch.distributed, then the ordered sum."""

    def __init__(self, world: int):
        self.world = world
        self.log: list[int] = []

    def __call__(self, payloads: list[np.ndarray]) -> np.ndarray:
        import torch
        import torch.distributed as dist

        assert len(payloads) == 1
        t = torch.from_numpy(np.ascontiguousarray(payloads[0]))
        parts = [torch.empty_like(t) for _ in range(self.world)]
        dist.all_gather(parts, t)
        self.log.append(int(t.numel()))
        out = parts[0].numpy().copy()
        for p in parts[1:]:
            out = out + p.numpy()
        return out


def row_bounds(M: int, P: int) -> list[int]:
    return [(p * M) // P for p in range(P + 1)]


def fit(shards: list[np.ndarray], N: int, K: int, tol: float, max_iter: int, algo: str, reduce,
        iters_lock=None) -> dict:
    """shards: this process's row blocks of X (FP64, each rows x N).  Returns this
    process's rows of T, the replicated P, lambda, iters, found and status.
    iters_lock: run exactly iters_lock[k] iterations for component k."""
    R = [np.array(x, dtype=np.float64, copy=True) for x in shards]
    rows = [r.shape[0] for r in R]
    V = [np.zeros((m, K)) for m in rows]
    U = np.zeros((N, K))
    W = np.zeros((N, K))
    GV = np.zeros((K, K))
    lam = np.zeros(K)
    iters = np.zeros(K, dtype=np.int64)
    gs = algo == "gs"
    xx = reduce([np.array([float(np.sum(r * r))]) for r in R])[0]
    thresh = 64.0 * np.finfo(np.float64).eps * np.sqrt(xx)
    not_converged = False
    lam_prev, upre_last = 0.0, None
    for k in range(K):
        if k > 0:  # deflation of component k-1 (Eq. 3) on the local rows
            for p in range(len(R)):
                if gs:
                    R[p] -= lam_prev * np.outer(V[p][:, k - 1], U[:, k - 1])
                else:
                    R[p] -= np.outer(V[p][:, k - 1], U[:, k - 1])
        col = k
        v = [r[:, col].copy() for r in R]

        def start_payload(v):
            parts = []
            for p in range(len(R)):
                g = V[p][:, :k].T @ V[p][:, k - 1] if (gs and k > 0) else np.zeros(0)
                parts.append(np.concatenate([R[p].T @ v[p], g, [v[p] @ v[p]]]))
            return reduce(parts)

        red = start_payload(v)
        if red[-1] == 0.0:  # zero start column: the residual column of largest norm
            cn = reduce([np.sum(r * r, axis=0) for r in R])
            if not np.any(cn > 0.0):
                return _result(V, U, lam, iters, k, K, gs, 5)
            col = int(np.argmax(cn))  # lowest index on ties
            v = [r[:, col].copy() for r in R]
            red = start_payload(v)
        s0 = red[:N]
        if gs and k > 0:
            g = red[N:N + k]
            # W_j = R_k^T v_j = R_{k-1}^T v_j - lam u_{k-1} (v_{k-1} . v_j); new column from
            # R_{k-1}^T v_{k-1} = u_pre / lambda of component k-1's last iteration
            W[:, :k - 1] -= lam_prev * np.outer(U[:, k - 1], g[:k - 1])
            W[:, k - 1] = upre_last / lam_prev - lam_prev * U[:, k - 1] * g[k - 1]
            GV[k - 1, :k] = g
            GV[:k, k - 1] = g
        u = s0.copy()
        if gs and k > 0:
            a = U[:, :k].T @ u
            u -= U[:, :k] @ a
        nu = np.sqrt(u @ u)
        if nu == 0.0:
            return _result(V, U, lam, iters, k, K, gs, 5)
        u /= nu
        mu, j = 0.0, 0
        while True:
            vp = [r @ u for r in R]
            parts = []
            for p in range(len(R)):
                b = V[p][:, :k].T @ vp[p] if gs else np.zeros(0)
                parts.append(np.concatenate([R[p].T @ vp[p], b, [vp[p] @ vp[p]]]))
            red = reduce(parts)
            s, q = red[:N], red[-1]
            if gs:
                b = red[N:N + k]
                lam2 = q - 2.0 * (b @ b) + b @ (GV[:k, :k] @ b)
                cur = np.sqrt(lam2) if lam2 > 0.0 else 0.0
            else:
                cur = np.sqrt(q)
            if cur <= thresh:
                return _result(V, U, lam, iters, k, K, gs, 5)
            j += 1
            if iters_lock is not None:
                stop = j >= iters_lock[k]
            else:
                stop = abs(mu - cur) < tol * cur
                if not stop and j >= max_iter:
                    stop, not_converged = True, True
            if gs:
                upre = s - W[:, :k] @ b
            if stop:
                for p in range(len(R)):
                    V[p][:, k] = (vp[p] - V[p][:, :k] @ b) / cur if gs else vp[p]
                U[:, k] = u
                lam[k], iters[k] = cur, j
                lam_prev = cur
                if gs:
                    upre_last = upre
                break
            mu = cur
            if gs:
                a = U[:, :k].T @ upre
                u = upre - U[:, :k] @ a
            else:
                u = s.copy()
            u /= np.sqrt(u @ u)
    return _result(V, U, lam, iters, K, K, gs, 4 if not_converged else 0)


def _result(V, U, lam, iters, found, K, gs, status):
    T = [v.copy() for v in V]
    for t in T:
        t[:, found:] = 0.0
        if gs:
            t[:, :found] *= lam[:found]
    P = U.copy()
    P[:, found:] = 0.0
    lam = lam.copy()
    lam[found:] = 0.0
    iters = iters.copy()
    iters[found:] = 0
    return {"T": T, "P": P, "lam": lam, "iters": iters, "found": found, "status": status}
