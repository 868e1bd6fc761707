"""Comparison helpers shared by the GPU parity tests (test infrastructure only).

* ``angle``: sign-invariant angle between two vectors (readings A10 of the
  paper's sign ambiguity).
* ``subspace_angle``: largest principal angle between two column spaces,
  arccos of the smallest singular value of QaᵀQb (Qa, Qb orthonormal bases).
* ``clusters``: groups of components whose reference singular values lie within
  a relative gap of each other.  Inside such a group the individual singular
  vectors are ill-conditioned (a perturbation of the residual of size d turns
  them by about d / gap), so only the group's subspace is compared.
* ``sigma_ok``: the singular-value rule for spectra with a long tail: relative
  error for sigma >= floor * sigma_1, absolute error (relative to sigma_1)
  below it, since FP32 storage of R bounds the absolute error of every sigma
  by a few FP32 ulps of sigma_1.
* ``oracle_many``: several oracle fits at once.  The oracle is C called through
  ctypes, which releases the GIL, so threads run the fits on separate cores;
  no process is forked after CUDA was initialised.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle


def angle(a, b) -> float:
    na, nb = np.linalg.norm(a), np.linalg.norm(b)
    if na == 0 or nb == 0:
        return 0.0 if na == nb else math.pi / 2
    return math.acos(min(1.0, abs(float(a @ b)) / (na * nb)))


def subspace_angle(A: np.ndarray, B: np.ndarray) -> float:
    qa, _ = np.linalg.qr(A)
    qb, _ = np.linalg.qr(B)
    s = np.linalg.svd(qa.T @ qb, compute_uv=False)
    return math.acos(min(1.0, float(s.min())))


def clusters(lam_ref: np.ndarray, gap_rel: float, floor: float = 0.0) -> list[list[int]]:
    """Components grouped by their reference singular values: sorted descending,
    neighbours closer than gap_rel (relative to the larger) share a group.  With
    floor > 0 only components with sigma >= floor * sigma_1 are grouped (the rest
    are left out)."""
    s1 = float(np.max(lam_ref)) if len(lam_ref) else 0.0
    order = [int(i) for i in np.argsort(-lam_ref) if lam_ref[i] >= floor * s1]
    groups: list[list[int]] = []
    for i in order:
        if groups and (lam_ref[groups[-1][-1]] - lam_ref[i]) < gap_rel * lam_ref[groups[-1][-1]]:
            groups[-1].append(i)
        else:
            groups.append([i])
    return groups


def sigma_ok(lam, lam_ref, rel=1e-4, floor=1e-2, abs_rel=1e-4):
    """Per component: True where the singular value meets the tail-aware bar."""
    s1 = float(np.max(lam_ref))
    err = np.abs(np.asarray(lam) - np.asarray(lam_ref))
    big = lam_ref >= floor * s1
    return np.where(big, err <= rel * lam_ref, err <= abs_rel * s1)


def oracle_many(jobs, workers: int | None = None):
    """jobs: list of (args, kwargs) for oracle.fit; results in the same order."""
    oracle.build()
    n = workers or max(1, min(len(jobs), os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=n) as ex:
        futs = [ex.submit(oracle.fit, *a, **kw) for a, kw in jobs]
        return [f.result() for f in futs]
