"""Pins of the oracle's iterated classical Gram-Schmidt (CGS2).

Sec. 2.3 remarks, before the GS-PCA pseudo-code, that the classical
Gram-Schmidt step can be applied iteratively for stability; the pseudo-code
and the appendix programs apply it once per half-iteration.  The oracle's
``gs_passes = 2`` applies it twice, each pass taking its coefficients from
the vector the previous pass left.  What fixes it, independently of the code:
  * with an exactly orthonormal basis (Hadamard columns / 2, binary exact) one
    pass leaves x exactly orthogonal, so the second pass has zero coefficients;
  * with a basis that is orthonormal only to delta, one pass leaves Q^T x of
    order delta and the second of order delta^2 ("twice is enough"); a second
    pass that reused the first pass's coefficients, or subtracted with the
    wrong sign, would not contract;
  * in a fit: the noise-free planted spectrum and the rational closed forms
    are returned exactly by both forms, gs_passes = 1 is the pseudo-code's
    fit bit for bit, and orthogonality on duplicated columns is no worse.
"""
import numpy as np
import pytest

import oracle
import synth


def hadamard4():
    return np.array([[1, 1, 1, 1], [1, -1, 1, -1], [1, 1, -1, -1], [1, -1, -1, 1]], dtype=np.float64) / 2.0


def test_cgs_exact_on_orthonormal_basis(oracle_mod):
    Q = hadamard4()[:, :3]
    x = np.array([3.0, -1.0, 4.0, 2.0])
    x1, c1 = oracle.cgs(Q, x, passes=1)
    # coefficients Q^T x (half-integers, exact), and x1 spans only the 4th Hadamard column
    assert np.array_equal(c1, np.array([4.0, 3.0, -2.0]))
    h4 = hadamard4()[:, 3]
    assert np.array_equal(Q.T @ x1, np.zeros(3))
    assert np.array_equal(x1, (h4 @ x) * h4)
    x2, c2 = oracle.cgs(Q, x, passes=2)
    assert np.array_equal(c2, np.zeros(3))
    assert np.array_equal(x2, x1)


@pytest.mark.parametrize("delta", [1e-4, 1e-6])
def test_twice_is_enough_on_a_perturbed_basis(oracle_mod, delta):
    g = synth.rng(5, 17)
    Q0, _ = np.linalg.qr(g.standard_normal((60, 6)))
    Q = Q0 + delta * g.standard_normal((60, 6))
    x = g.standard_normal(60)
    x1, _ = oracle.cgs(Q, x, passes=1)
    x2, c2 = oracle.cgs(Q, x, passes=2)
    r1 = np.linalg.norm(Q.T @ x1) / np.linalg.norm(x)
    r2 = np.linalg.norm(Q.T @ x2) / np.linalg.norm(x)
    assert delta / 100 < r1 < 100 * delta
    assert r2 < 100 * delta * delta + 1e-14
    # the second pass's coefficients are those of x1, not of x
    assert np.linalg.norm(c2) < 100 * delta * np.linalg.norm(x)


def test_cgs_rejects_bad_arguments(oracle_mod):
    with pytest.raises(ValueError):
        oracle.cgs(np.eye(3), np.ones(3), passes=0)
    with pytest.raises(ValueError):
        oracle.fit(np.eye(3), 2, gs_passes=3)


@pytest.mark.parametrize("algo", ["gs", "nipals"])
def test_one_pass_is_the_pseudo_code(oracle_mod, algo):
    X = synth.planted(120, 50, 5.0, 0.8, 0.01, 3).X
    a = oracle.fit(X, 6, algo=algo)
    b = oracle.fit(X, 6, algo=algo, gs_passes=1)
    for key in ("T", "P", "lam", "iters", "R"):
        assert np.array_equal(getattr(a, key), getattr(b, key)), key


def test_two_passes_recover_the_noise_free_spectrum(oracle_mod):
    p = synth.planted(80, 40, 10.0, 0.7, 0.0, 9)
    f = oracle.fit(p.X, 8, tol=1e-13, max_iter=100000, algo="gs", gs_passes=2)
    np.testing.assert_allclose(f.lam, p.s[:8], rtol=1e-10)
    for k in range(8):
        c = abs(f.P[:, k] @ p.right[:, k])
        assert 1.0 - c < 1e-12
    assert np.abs(f.P.T @ f.P - np.eye(8)).max() < 1e-13


def test_two_passes_on_duplicated_columns(oracle_mod):
    X = synth.collinear(200, 30, 1e-3, 4)
    K = 50
    one = oracle.fit(X, K, tol=1e-5, max_iter=200, algo="gs")
    two = oracle.fit(X, K, tol=1e-5, max_iter=200, algo="gs", gs_passes=2)
    o1 = np.abs(one.P.T @ one.P - np.eye(K)).max()
    o2 = np.abs(two.P.T @ two.P - np.eye(K)).max()
    assert o2 <= max(o1, 1e-14)
    assert o2 < 1e-12
    # Eq. 4 and T^T T = diag(lambda^2) hold for the iterated form as well
    assert np.linalg.norm(X - two.T @ two.P.T - two.R) <= 1e-12 * np.linalg.norm(X)
    G = two.T.T @ two.T
    assert np.abs(G - np.diag(two.lam ** 2)).max() <= 1e-10 * two.lam[0] ** 2


def test_two_passes_on_the_closed_forms(oracle_mod):
    """The rational closed-form fixtures of tests/golden (X = Q diag(sigma) Z^T) are
    returned by the iterated form too."""
    import test_golden as tg

    for name in tg.CASES:
        fx = tg.load(name)
        K = fx["K"]
        f = oracle.fit(fx["X"], K, tol=1e-14, max_iter=100000, algo="gs", gs_passes=2)
        np.testing.assert_allclose(f.lam, fx["lambda"], rtol=1e-12)
        for k in range(K):
            assert 1.0 - abs(f.P[:, k] @ fx["P"][:, k]) < 1e-12
