"""Train the learned warm start on the GPU and write its parameters.

    python -m paper_0811_1081_gb300.train_warm_start [--instances 20000] [--epochs 40]
           [--out paper_0811_1081_gb300/warm_start_net.f32]

Training data: problems of the batched workload's generator (256 <= M <= 8192,
64 <= N <= 1024 log-uniform, planted spectrum 10 * 0.9^i, noise 0.01), seed
stream 5, K = 16; every (problem, component) pair is one instance: the features
of the residual R_k and the converged GS-PCA loading P[:, k] of the library's
plain FP32 fit at tol 1e-6.  The sketch G is the first M rows of one 8192 x 16
Gaussian draw (N(0, 1/16), seed 11).  Every forward, backward and Adam step runs
in the library's kernels (gspca_ws_train_step); the problems are drawn on the
host cores in a spawned process pool.

Writes the parameters (5377 little-endian float32 values) and, beside them, a
JSON record of the run (data, seeds, loss per epoch).
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

DEFAULT_OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "warm_start_net.f32")
SKETCH_ROWS = 8192
K = 16


def _draw(args):
    import synth

    i, M, N, seed = args
    return synth.batch_problem(i, M, N, seed=seed).X.astype(np.float32)


_BLAS_THREADS = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")


def draw_problems(count: int, seed: int, workers: int):
    """The problems, drawn in `workers` spawned processes with one BLAS thread each (many
    processes that each start a full-width BLAS thread pool oversubscribe the cores badly)."""
    import synth

    shapes = synth.batch_shapes(count, seed=seed)
    jobs = [(i, M, N, seed) for i, (M, N) in enumerate(shapes)]
    if workers <= 1:
        return [_draw(j) for j in jobs]
    saved = {v: os.environ.get(v) for v in _BLAS_THREADS}
    try:
        for v in _BLAS_THREADS:
            os.environ[v] = "1"  # inherited by the spawned workers only
        with mp.get_context("spawn").Pool(workers) as pool:
            return pool.map(_draw, jobs, chunksize=2)
    finally:
        for v, old in saved.items():
            if old is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = old


def sketch():
    import synth

    return synth.gaussian_sketch(SKETCH_ROWS).astype(np.float32)


def load_net(path: str = DEFAULT_OUT) -> np.ndarray:
    a = np.fromfile(path, dtype="<f4")
    if a.size != 5377:
        raise ValueError(f"{path}: expected 5377 parameters, found {a.size}")
    return a


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--instances", type=int, default=20000)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--per-batch", type=int, default=64)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--workers", type=int, default=max(1, min(16, os.cpu_count() or 1)))
    ap.add_argument("--out", default=DEFAULT_OUT)
    args = ap.parse_args()

    nprob = math.ceil(args.instances / K)
    t0 = time.time()
    Xs = draw_problems(nprob, args.seed, args.workers)  # before the first GPU call
    t_draw = time.time() - t0

    import torch

    import synth
    import paper_0811_1081_gb300 as gp
    from paper_0811_1081_gb300 import warmstart as ws

    gp.load()
    G = torch.from_numpy(sketch()).cuda()
    probs = [torch.from_numpy(np.ascontiguousarray(X.T)).cuda().t() for X in Xs]
    with gp.Handle(8192, 1024, K) as h:
        t1 = time.time()
        ts = ws.make_training_set(h.h, probs, K, G)
        del probs
        torch.cuda.synchronize()
        t_data = time.time() - t1
        net = torch.from_numpy(ws.init_params(synth.rng(args.seed, 7))).cuda()
        l0 = ws.mean_loss(h.h, net, ts)
        t2 = time.time()
        hist = ws.train(h.h, net, ts, args.epochs, args.per_batch, args.lr, rng=synth.rng(args.seed, 8),
                        log=lambda ep, l: print(f"epoch {ep:3d} loss {l:.4f}", flush=True))
        torch.cuda.synchronize()
        t_train = time.time() - t2
        out = net.cpu().numpy().astype("<f4")
    out.tofile(args.out)
    rec = {"instances": ts.ninst, "problems": nprob, "K": K, "seed_stream": args.seed, "sketch_seed": 11,
           "sketch_rows": SKETCH_ROWS, "rows_total": int(ts.offsets_host[-1]), "epochs": args.epochs,
           "per_batch": args.per_batch, "lr": args.lr, "loss_init": l0, "loss_per_epoch": hist,
           "seconds": {"draw_host": t_draw, "fits_and_features_gpu": t_data, "train_gpu": t_train}}
    with open(os.path.splitext(args.out)[0] + ".json", "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps({k: v for k, v in rec.items() if k != "loss_per_epoch"}))


if __name__ == "__main__":
    main()
