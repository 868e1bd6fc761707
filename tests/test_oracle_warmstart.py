"""Pins of the learned-warm-start oracle (oracle/warmstart.c) against facts that do not
come from its code: library routines (numpy's norms and products, scipy's normal CDF),
closed forms (an exactly affine regime of the network, Adam's first step), central
finite differences of the loss, and special cases of the start rule with a known answer.
"""
import math

import numpy as np
import pytest

import synth

NPAR = 5377
W1, B1, W2, B2, W3, B3 = 0, 1088, 1152, 5248, 5312, 5376


def zeros():
    return np.zeros(NPAR)


def affine_net(g):
    """A network whose pre-activations all stay above 40, where Phi(z) == 1 exactly in
    FP64, so gelu(z) == z and the network is the affine map W3 (W2 (W1 x + b1) + b2) + b3."""
    net = zeros()
    net[W1:B1] = 0.1 * g.standard_normal(64 * 17)
    net[B1:W2] = 50.0
    net[W2:B2] = 0.01 * g.standard_normal(64 * 64)
    net[B2:W3] = 50.0
    net[W3:B3] = g.standard_normal(64)
    net[B3] = 0.3
    return net


def test_forward_affine_regime_matches_matrix_products(oracle_mod):
    g = synth.rng(61)
    net = affine_net(g)
    x = g.uniform(-3, 3, size=(40, 17))
    A1 = net[W1:B1].reshape(64, 17)
    A2 = net[W2:B2].reshape(64, 64)
    ref = (A2 @ (A1 @ x.T + net[B1:W2, None]) + net[B2:W3, None]).T @ net[W3:B3] + net[B3]
    np.testing.assert_allclose(oracle_mod.ws_forward(net, x), ref, rtol=1e-12, atol=1e-9)


def test_forward_gelu_against_normal_cdf(oracle_mod):
    """One path through the network: w = gelu(gelu(a x_f)), gelu(z) = z Phi(z)."""
    stats = pytest.importorskip("scipy.stats")
    net = zeros()
    f, a = 5, 1.7
    net[W1 + 0 * 17 + f] = a
    net[W2 + 0 * 64 + 0] = 1.0
    net[W3 + 0] = 1.0
    x = np.zeros((9, 17))
    x[:, f] = np.linspace(-3, 3, 9)
    z = a * x[:, f]
    h = z * stats.norm.cdf(z)
    ref = h * stats.norm.cdf(h)
    np.testing.assert_allclose(oracle_mod.ws_forward(net, x), ref, rtol=1e-13, atol=1e-15)


def test_features_against_numpy_and_scale_invariance(oracle_mod):
    g = synth.rng(62)
    R = g.standard_normal((70, 23))
    G = g.standard_normal((70, 16)) / 4
    f = oracle_mod.ws_features(R, G)
    c = np.linalg.norm(R, axis=0)
    rho = math.sqrt(np.mean(c**2))
    np.testing.assert_allclose(f[:, 0], c / rho, rtol=1e-13)
    np.testing.assert_allclose(f[:, 1:], (G.T @ R).T / rho, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(oracle_mod.ws_features(7.5 * R, G), f, rtol=1e-12, atol=1e-14)
    assert np.all(oracle_mod.ws_features(np.zeros((5, 4)), G[:5]) == 0)


def _instances(g, sizes):
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    feat = g.standard_normal((offs[-1], 17))
    tgt = np.zeros(offs[-1])
    for i in range(len(sizes)):
        t = g.standard_normal(sizes[i])
        tgt[offs[i]:offs[i + 1]] = t / np.linalg.norm(t)
    return feat, tgt, offs


def test_gradient_against_central_differences(oracle_mod):
    g = synth.rng(63)
    net = 0.3 * g.standard_normal(NPAR)
    feat, tgt, offs = _instances(g, [17, 31, 9])
    loss, grad = oracle_mod.ws_loss_grad(net, feat, tgt, offs)
    assert 0.0 <= loss <= 1.0
    idx = np.concatenate([g.choice(np.arange(s, e), 12, replace=False)
                          for s, e in [(W1, B1), (B1, W2), (W2, B2), (B2, W3), (W3, B3)]] + [[B3]])
    for i in idx:
        h = 1e-6 * max(1.0, abs(net[i]))
        up, dn = net.copy(), net.copy()
        up[i] += h
        dn[i] -= h
        fd = (oracle_mod.ws_loss_grad(up, feat, tgt, offs)[0] - oracle_mod.ws_loss_grad(dn, feat, tgt, offs)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1e-3, abs(grad[i])) + 1e-10, (i, fd, grad[i])


def test_loss_closed_cases(oracle_mod):
    """w = x_0 exactly (affine regime): loss 0 when the target is x_0 / ||x_0||, 1 when it
    is orthogonal to x_0; negating the output leaves the loss unchanged."""
    net = zeros()
    net[W1 + 0] = 1.0           # hidden 0 <- x_0
    net[B1:W2] = 50.0
    net[W2:B2] = np.eye(64).ravel()
    net[W3 + 0] = 1.0
    net[B3] = -50.0             # w = (x_0 + 50) - 50
    g = synth.rng(64)
    feat = g.standard_normal((12, 17))
    x0 = feat[:, 0]
    offs = np.array([0, 12], dtype=np.int32)
    assert oracle_mod.ws_loss_grad(net, feat, x0 / np.linalg.norm(x0), offs)[0] <= 1e-12
    ortho = g.standard_normal(12)
    ortho -= (ortho @ x0) / (x0 @ x0) * x0
    assert abs(oracle_mod.ws_loss_grad(net, feat, ortho / np.linalg.norm(ortho), offs)[0] - 1.0) <= 1e-12
    t = g.standard_normal(12)
    t /= np.linalg.norm(t)
    neg = net.copy()
    neg[W3:] *= -1
    assert abs(oracle_mod.ws_loss_grad(net, feat, t, offs)[0] - oracle_mod.ws_loss_grad(neg, feat, t, offs)[0]) <= 1e-12
    # a zero output counts as the worst loss, with no gradient
    l0, g0 = oracle_mod.ws_loss_grad(zeros(), feat, t, offs)
    assert l0 == 1.0 and not np.any(g0)


def test_adam_first_step_closed_form(oracle_mod):
    """From m = v = 0 the bias-corrected first step moves each parameter by lr g / (|g| + eps)."""
    g = synth.rng(65)
    net = g.standard_normal(50)
    grad = g.standard_normal(50)
    m, v = np.zeros(50), np.zeros(50)
    new = net.copy()
    oracle_mod.ws_adam(new, m, v, grad, 1, lr=1e-2, eps=1e-8)
    np.testing.assert_allclose(new, net - 1e-2 * grad / (np.abs(grad) + 1e-8), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * grad, rtol=1e-15)
    np.testing.assert_allclose(v, 0.001 * grad**2, rtol=1e-14)


def test_zero_network_keeps_the_papers_start(oracle_mod):
    """w == 0: no learned candidate, the fit is the paper's, bit for bit."""
    X = synth.planted(90, 40, 10.0, 0.85, 0.01, 66).X
    G = synth.rng(66, 1).standard_normal((90, 16)) / 4
    a = oracle_mod.fit(X, 5, algo="gs", ws_net=zeros(), ws_G=G)
    b = oracle_mod.fit(X, 5, algo="gs")
    assert not np.any(a.ws_choice)
    for key in ("T", "P", "lam", "iters", "R"):
        assert np.array_equal(getattr(a, key), getattr(b, key)), key


def test_exact_candidate_is_chosen_and_converges_at_once(oracle_mod):
    """X = s1 a 1^T / sqrt(N) + s2 c d^T with d orthogonal to 1 and a to c.  A constant
    network (w = b3) proposes p0 = 1 / sqrt(N), the exact first loading: it beats the
    paper's start R(0) (the largest Rayleigh quotient there is, s1^2), and the first
    component then converges in two iterations to lambda = s1."""
    g = synth.rng(67)
    M, N = 60, 30
    a = g.standard_normal(M)
    a /= np.linalg.norm(a)
    c = g.standard_normal(M)
    c -= (c @ a) * a
    c /= np.linalg.norm(c)
    d = g.standard_normal(N)
    d -= d.mean()
    d /= np.linalg.norm(d)
    X = 5.0 * np.outer(a, np.ones(N) / math.sqrt(N)) + 2.0 * np.outer(c, d)
    net = zeros()
    net[B3] = 1.0
    G = g.standard_normal((M, 16)) / 4
    f = oracle_mod.fit(X, 2, tol=1e-12, max_iter=100, algo="gs", ws_net=net, ws_G=G)
    plain = oracle_mod.fit(X, 2, tol=1e-12, max_iter=100, algo="gs")
    assert f.ws_choice[0] == 1
    assert abs(f.ws_rho[0, 1] - 25.0) <= 1e-12 * 25.0 and f.ws_rho[0, 0] < 25.0
    assert f.iters[0] == 2 and plain.iters[0] > 2
    assert abs(f.lam[0] - 5.0) <= 1e-13 * 5.0
    assert abs(abs(f.P[:, 0] @ np.ones(N)) / math.sqrt(N) - 1.0) <= 1e-13


def test_learned_start_finds_the_same_components(oracle_mod):
    """With any network the loop converges to the same singular triplets (Eq. 5): a start
    changes the trajectory, not the answer; GS orthogonality and Eq. 4 hold."""
    X = synth.planted(120, 50, 10.0, 0.8, 0.01, 68).X
    G = synth.rng(68, 1).standard_normal((120, 16)) / 4
    net = 0.3 * synth.rng(68, 2).standard_normal(NPAR)
    K = 6
    f = oracle_mod.fit(X, K, tol=1e-13, max_iter=20000, algo="gs", ws_net=net, ws_G=G)
    p = oracle_mod.fit(X, K, tol=1e-13, max_iter=20000, algo="gs")
    np.testing.assert_allclose(f.lam, p.lam, rtol=1e-9)
    for k in range(K):
        assert abs(abs(f.P[:, k] @ p.P[:, k]) - 1.0) <= 1e-9
    assert np.abs(f.P.T @ f.P - np.eye(K)).max() <= 1e-12
    assert np.linalg.norm(X - f.T @ f.P.T - f.R) <= 1e-12 * np.linalg.norm(X)
    assert f.ws_choice.sum() >= 1  # the candidate is really in play on this data
