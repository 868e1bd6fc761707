"""Training of the learned warm start through the library's own kernels.

Argument marshalling and data arrangement only: the features come from
``gspca_ws_features``, the converged loadings from the library's GS-PCA fits,
and every forward, backward and Adam step from ``gspca_ws_train_step``.
PyTorch holds the device buffers.

An instance is one residual R_k of one problem: its N feature rows (one per
column) and the target loading p* = P[:, k] of the converged fit (unit norm).
Instances are stored back to back; ``offsets`` delimits them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import (WS_FEATURES, WS_PARAMS, Batch, gspca_fit_batched, gspca_ws_features, gspca_ws_forward,
               gspca_ws_train_step)

# parameter offsets (see include/gspca.h)
W1, B1, W2, B2, W3, B3 = 0, 1088, 1152, 5248, 5312, 5376


def init_params(rng: np.random.Generator) -> np.ndarray:
    """Glorot-normal weights, zero biases (float32, WS_PARAMS values) from the caller's generator."""
    p = np.zeros(WS_PARAMS, dtype=np.float32)
    p[W1:B1] = rng.standard_normal(64 * 17) * math.sqrt(2.0 / (17 + 64))
    p[W2:B2] = rng.standard_normal(64 * 64) * math.sqrt(2.0 / (64 + 64))
    p[W3:B3] = rng.standard_normal(64) * math.sqrt(2.0 / (64 + 1))
    return p


@dataclass
class TrainingSet:
    feat: object      # (rows, 17) float32 CUDA
    target: object    # (rows,) float32 CUDA
    offsets: object   # (ninst + 1,) int32 CUDA
    offsets_host: np.ndarray
    ninst: int


def make_training_set(h: int, problems, K: int, G, tol: float = 1e-6, max_iter: int = 1000,
                      components=None) -> TrainingSet:
    """Fit `problems` (float32 CUDA matrices) with the plain GS-PCA batched form and take, for
    every problem and component k (all K, or those listed in `components`), the features of
    R_k and the converged loading P[:, k] as one instance."""
    import torch

    ks = list(range(K)) if components is None else list(components)
    feats, tgts, sizes = [], [], []
    for c0 in range(0, len(problems), 256):
        chunk = problems[c0:c0 + 256]
        b = Batch([{"X": X.t().contiguous().t() if X.stride(0) != 1 else X, "K": K} for X in chunk])
        gspca_fit_batched(h, b, tol=tol, max_iter=max_iter, algo="gs")
        for X, r in zip(b.keep, b.results):
            found = int((r.lam > 0).sum().item())
            for k in ks:
                if k >= found:
                    continue
                feats.append(gspca_ws_features(X, G, r.T, r.P, k))
                tgts.append(r.P[:, k].clone())
                sizes.append(X.shape[1])
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    dev = problems[0].device
    return TrainingSet(torch.cat(feats), torch.cat(tgts), torch.from_numpy(offs).to(dev), offs, len(sizes))


def _minibatches(ts: TrainingSet, per_batch: int):
    """Contiguous instance ranges (so every minibatch is a contiguous block of rows)."""
    return [(i, min(i + per_batch, ts.ninst)) for i in range(0, ts.ninst, per_batch)]


def train(h: int, net, ts: TrainingSet, epochs: int, per_batch: int = 64, lr: float = 1e-3,
          rng: np.random.Generator | None = None, log=None):
    """Adam on the mean instance loss, minibatches of `per_batch` consecutive instances visited in
    a fresh random order every epoch.  `net` (float32 CUDA, WS_PARAMS) is updated in place.
    Returns the mean training loss of every epoch."""
    import torch

    dev = net.device
    m = torch.zeros_like(net)
    v = torch.zeros_like(net)
    loss = torch.zeros(1, device=dev, dtype=torch.float32)
    rng = rng if rng is not None else np.random.default_rng(0)
    mbs = _minibatches(ts, per_batch)
    offs = ts.offsets_host
    step = 0
    history = []
    for ep in range(epochs):
        tot = torch.zeros(1, device=dev, dtype=torch.float64)
        for bi in rng.permutation(len(mbs)):
            i0, i1 = mbs[bi]
            r0, r1 = int(offs[i0]), int(offs[i1])
            o = ts.offsets[i0:i1 + 1] - r0
            step += 1
            gspca_ws_train_step(h, net, m, v, step, lr, ts.feat[r0:r1], ts.target[r0:r1], o.contiguous(), loss=loss)
            tot += loss.double() * (i1 - i0)
        history.append(float(tot.item()) / ts.ninst)
        if log:
            log(ep, history[-1])
    return history


def mean_loss(h: int, net, ts: TrainingSet) -> float:
    """Mean instance loss of `net` on a set (no update)."""
    import torch

    loss = torch.zeros(1, device=net.device, dtype=torch.float32)
    gspca_ws_train_step(h, net, None, None, 1, 0.0, ts.feat, ts.target, ts.offsets, loss=loss)
    return float(loss.item())


def forward(net, feat):
    return gspca_ws_forward(net, feat)
