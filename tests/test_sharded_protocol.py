"""The row-sharded exchange protocol of the power-iteration loop (multi-GPU
design, tests/sharded_protocol.py) on CPU ranks: FP64, gloo, world size 2
and 4.  Not measured on hardware (every run of this build has one GPU).

* P virtual shards in one process vs the FP64 oracle: the loop of Sec. 2.2 /
  2.3 with the exchange in place of the global products, the same singular
  values to 1e-12 relative and loadings to 1e-9 rad (iteration-locked),
  iteration counts within one of the oracle's free run;
* exactly one exchange of N + k + 1 words per GS-PCA iteration (N + 1 for
  NIPALS-PCA);
* P gloo processes give the same bits as one process with P virtual shards
  (all-gather, then a sum in rank order).
"""
import os
import socket

import numpy as np
import pytest

import oracle
import sharded_protocol as sp
import synth


def angle(a, b):
    """Sign-invariant angle, resolved below 1e-8 rad: min ||a^ -+ b^|| (= 2 sin(theta/2));
    arccos of the cosine cannot resolve angles under sqrt(2 eps) ~ 1.5e-8 in FP64."""
    a = a / np.linalg.norm(a)
    b = b / np.linalg.norm(b)
    return min(float(np.linalg.norm(a - b)), float(np.linalg.norm(a + b)))


def shards_of(X, P):
    b = sp.row_bounds(X.shape[0], P)
    return [X[b[p]:b[p + 1]] for p in range(P)]


def run_local(X, P, K, algo, tol=1e-8, max_iter=2000, iters_lock=None):
    red = sp.LocalReduce()
    out = sp.fit(shards_of(X, P), X.shape[1], K, tol, max_iter, algo, red, iters_lock=iters_lock)
    out["T"] = np.concatenate(out["T"], axis=0)
    out["log"] = red.log
    return out


CASES = [("planted", 240, 90, 8), ("planted", 97, 130, 6), ("collinear", 300, 80, 30)]


def make(kind, M, N):
    if kind == "planted":
        return synth.planted(M, N, 10.0, 0.8, 0.01, (91, M, N)).X
    return synth.collinear(M, N // 2, 1e-3, 92)


@pytest.mark.parametrize("P", [1, 3, 4])
@pytest.mark.parametrize("algo", ["gs", "nipals"])
@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}{c[1]}x{c[2]}" for c in CASES])
def test_sharded_protocol_matches_the_oracle(oracle_mod, case, algo, P):
    kind, M, N, K = case
    X = make(kind, M, N)
    tol = 1e-8
    free = run_local(X, P, K, algo, tol)
    ref_free = oracle.fit(X, K, tol=tol, max_iter=2000, algo=algo)
    assert free["status"] == ref_free.status
    assert np.abs(free["iters"] - ref_free.iters).max() <= 1
    got = run_local(X, P, K, algo, tol, iters_lock=ref_free.iters)
    ref = oracle.fit(X, K, tol=tol, max_iter=2000, algo=algo, iters_lock=ref_free.iters)
    np.testing.assert_allclose(got["lam"], ref.lam, rtol=1e-12)
    for k in range(K):
        if kind == "collinear" and ref.lam[k] < 1e-2 * ref.lam[0]:
            continue
        assert angle(got["P"][:, k], ref.P[:, k]) <= 1e-9, k
        assert angle(got["T"][:, k], ref.T[:, k]) <= 1e-9, k
    if algo == "gs":
        assert np.abs(got["P"].T @ got["P"] - np.eye(K)).max() <= 1e-12


@pytest.mark.parametrize("algo", ["gs", "nipals"])
def test_one_exchange_per_iteration(oracle_mod, algo):
    X = make("planted", 240, 90)
    N, K, P = 90, 6, 3
    out = run_local(X, P, K, algo)
    log = out["log"]
    assert log[0] == 1  # ||X||_F^2
    i = 1
    for k in range(K):
        kk = k if (algo == "gs" and k > 0) else 0
        assert log[i] == N + kk + 1, (k, "start")
        i += 1
        for _ in range(int(out["iters"][k])):
            assert log[i] == N + (k if algo == "gs" else 0) + 1, (k, "iteration")
            i += 1
    assert i == len(log)


def test_zero_start_column_and_rank_exhaustion(oracle_mod):
    X = synth.planted(120, 40, 5.0, 0.7, 0.01, 8).X
    X[:, 0] = 0.0
    got = run_local(X, 3, 4, "gs")
    ref = oracle.fit(X, 4, tol=1e-8, max_iter=2000, algo="gs")
    np.testing.assert_allclose(got["lam"], ref.lam, rtol=1e-12)
    g0 = synth.rng(12, 1)
    X = g0.standard_normal((60, 3)) @ g0.standard_normal((3, 20))
    got = run_local(X, 4, 5, "gs")
    ref = oracle.fit(X, 5, tol=1e-8, max_iter=2000, algo="gs")
    assert got["status"] == ref.status == 5 and got["found"] == ref.found == 3
    np.testing.assert_allclose(got["lam"][:3], ref.lam[:3], rtol=1e-12)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, kind, M, N, K, algo, outdir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X = make(kind, M, N)
        b = sp.row_bounds(M, world)
        red = sp.GlooReduce(world)
        out = sp.fit([X[b[rank]:b[rank + 1]]], N, K, 1e-8, 2000, algo, red)
        np.savez(os.path.join(outdir, f"r{rank}.npz"), T=out["T"][0], P=out["P"], lam=out["lam"],
                 iters=out["iters"], log=np.array(red.log))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("algo", ["gs", "nipals"])
def test_gloo_ranks_give_the_bits_of_virtual_shards(tmp_path, world, algo):
    import torch.multiprocessing as mp

    kind, M, N, K = "planted", 240, 90, 8
    mp.start_processes(_rank_main, args=(world, _free_port(), kind, M, N, K, algo, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    local = run_local(make(kind, M, N), world, K, algo)
    b = sp.row_bounds(M, world)
    for r in range(world):
        d = np.load(tmp_path / f"r{r}.npz")
        assert np.array_equal(d["P"], local["P"])
        assert np.array_equal(d["lam"], local["lam"])
        assert np.array_equal(d["iters"], local["iters"])
        assert np.array_equal(d["T"], local["T"][b[r]:b[r + 1]])
        assert list(d["log"]) == local["log"]
