"""Pins of the oracle's block power iteration (oracle_block_fit): components b at
a time (the block form of the Sec. 2.3 loop, a variant the paper does not have).

What fixes it, independently of its code:
  * a noise-free planted spectrum: the planted singular values and right factor;
  * one block holding every component: numpy's SVD (a third opinion);
  * b = 1: the singular triplets of the one-vector GS-PCA loop (same start R(k));
  * Eq. 4 (X = T P^T + R), P^T P = I and T^T T = diag(lambda^2) on random data;
  * a ragged last block, the iteration lock replaying the free run, a rank-deficient
    X stopping as degenerate once a block's start has dependent columns.
"""
import numpy as np
import pytest

import oracle
import synth


def cos1(a, b):
    return 1.0 - abs(float(a @ b)) / (np.linalg.norm(a) * np.linalg.norm(b))


@pytest.mark.parametrize("b", [1, 3, 4, 12])
def test_noise_free_planted_spectrum(oracle_mod, b):
    p = synth.planted(90, 40, 10.0, 0.75, 0.0, 5)
    f = oracle.block_fit(p.X, 12, b, tol=1e-13, max_iter=100000)
    assert f.status == 0 and f.found == 12
    np.testing.assert_allclose(f.lam, p.s[:12], rtol=1e-10)
    for k in range(12):
        assert cos1(f.P[:, k], p.right[:, k]) < 1e-12


def test_single_block_matches_numpy_svd(oracle_mod):
    X = synth.rng(31, 7).standard_normal((60, 25))
    f = oracle.block_fit(X, 6, 6, tol=1e-14, max_iter=100000)
    s = np.linalg.svd(X, compute_uv=False)
    # a block of 6 converges at the rate sigma_7 / sigma_6
    np.testing.assert_allclose(f.lam, s[:6], rtol=1e-9)


def test_width_one_is_the_gs_pca_loop(oracle_mod):
    X = synth.planted(120, 50, 5.0, 0.8, 0.01, 9).X
    a = oracle.block_fit(X, 6, 1, tol=1e-13, max_iter=100000)
    g = oracle.fit(X, 6, tol=1e-13, max_iter=100000, algo="gs")
    np.testing.assert_allclose(a.lam, g.lam, rtol=1e-10)
    for k in range(6):
        assert cos1(a.P[:, k], g.P[:, k]) < 1e-10


@pytest.mark.parametrize("b", [2, 4, 7])
def test_invariants_and_ragged_blocks(oracle_mod, b):
    X = synth.planted(150, 60, 5.0, 0.85, 0.01, 11).X
    K = 10
    f = oracle.block_fit(X, K, b, tol=1e-8, max_iter=5000)
    assert f.found == K
    assert np.linalg.norm(X - f.T @ f.P.T - f.R) <= 1e-12 * np.linalg.norm(X)
    assert np.abs(f.P.T @ f.P - np.eye(K)).max() <= 1e-12
    assert np.abs(f.T.T @ f.T - np.diag(f.lam ** 2)).max() <= 1e-10 * f.lam[0] ** 2
    # every component of a block reports the block's count
    for k0 in range(0, K, b):
        assert len(set(f.iters[k0:k0 + b].tolist())) == 1
    s = np.linalg.svd(X, compute_uv=False)
    np.testing.assert_allclose(np.sort(f.lam)[::-1], s[:K], rtol=1e-6)


def test_iteration_lock_replays_the_free_run(oracle_mod):
    X = synth.planted(100, 40, 5.0, 0.8, 0.01, 12).X
    a = oracle.block_fit(X, 8, 3, tol=1e-8, max_iter=5000)
    b = oracle.block_fit(X, 8, 3, tol=1e-8, max_iter=5000, iters_lock=a.iters)
    for key in ("T", "P", "lam", "iters", "R"):
        assert np.array_equal(getattr(a, key), getattr(b, key)), key


def test_rank_deficient_stops_as_degenerate(oracle_mod):
    g0 = synth.rng(12, 1)
    X = g0.standard_normal((60, 3)) @ g0.standard_normal((3, 20))
    f = oracle.block_fit(X, 6, 2, tol=1e-10, max_iter=5000)
    assert f.status == 5 and f.found == 2
    s = np.linalg.svd(X, compute_uv=False)
    np.testing.assert_allclose(f.lam[:2], s[:2], rtol=1e-8)
    assert np.all(f.lam[2:] == 0) and np.all(f.P[:, 2:] == 0)


def test_invalid_arguments(oracle_mod):
    with pytest.raises(ValueError):
        oracle.block_fit(np.eye(4), 2, 0)
    with pytest.raises(ValueError):
        oracle.block_fit(np.eye(4), 5, 2)
