"""The SVD form of GS-PCA (Eq. 5, Sec. 2.3) and K = N at scale, through the C ABI.

With svd_form = 1 the library returns the unit score directions V instead of
the scores T = V Lambda, so X = V Lambda P^T + R (Eq. 4 / Eq. 5); Sec. 2.3
states that for K = N GS-PCA gives the full SVD, V and P orthogonal, R = 0
once every component has converged.
  * a rank-64 planted 300 x 64 matrix, K = N = 64, run to FP32 convergence: the
    planted singular values and right factor, ||R||_F <= 1e-5 ||X||_F, the
    oracle (iteration-locked) on every component, V^T V = P^T P = I;
  * a full-rank planted 1024 x 1024 matrix, K = N = 1024, 40 iterations per
    component (not converged; orthogonality and Eq. 4 do not need it):
    ||P^T P - I||_max <= 1e-5, ||V^T V - I||_max <= 1e-4,
    ||X - V Lambda P^T - R||_F <= 1e-5 ||X||_F;
  * svd_form = 1 and 0 give the same fit (T = V lambda within FP32 rounding),
    for NIPALS-PCA too (t_k / lambda_k).
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    import paper_0811_1081_gb300 as m

    m.load()
    return m


def angle(a, b):
    c = abs(float(a @ b)) / (np.linalg.norm(a) * np.linalg.norm(b))
    return math.acos(min(1.0, c))


def fit(gp, X32, K, tol, max_iter, algo="gs", **kw):
    import torch

    M, N = X32.shape
    with gp.Handle(M, N, K) as h:
        r = h.fit(torch.from_numpy(X32).cuda(), K, tol=tol, max_iter=max_iter, algo=algo, want_R=True, **kw)
        torch.cuda.synchronize()
        return dict(T=r.T.cpu().numpy().astype(np.float64), P=r.P.cpu().numpy().astype(np.float64),
                    lam=r.lam.cpu().numpy(), iters=r.iters.cpu().numpy(), status=r.status, info=r.info,
                    R=r.R.cpu().numpy().astype(np.float64))


def test_full_svd_k_equals_n_converged(gp):
    p = synth.planted(300, 64, 10.0, 0.9, 0.0, 101)
    X32 = p.X.astype(np.float32)
    K = 64
    # converged to FP32 rounding: the test (tol 1e-12) never fires, every component runs
    # 400 iterations, 0.9^400 of the start remains (a tolerance on lambda leaves loading
    # errors of about sqrt(2 tol / (1 - r^2)), and R keeps what they leave)
    g = fit(gp, X32, K, 1e-12, 400, svd_form=1)
    assert g["status"] in (0, 4) and g["info"]["found"] == K
    V, P, lam = g["T"], g["P"], g["lam"]
    xn = np.linalg.norm(X32)
    assert np.abs(V.T @ V - np.eye(K)).max() <= 1e-5
    assert np.abs(P.T @ P - np.eye(K)).max() <= 1e-5
    assert np.linalg.norm(X32 - (V * lam) @ P.T - g["R"]) <= 1e-5 * xn
    assert np.linalg.norm(g["R"]) <= 1e-5 * xn
    s = np.linalg.svd(X32.astype(np.float64), compute_uv=False)
    big = s >= 1e-2 * s[0]
    np.testing.assert_allclose(np.sort(lam)[::-1][big], s[big], rtol=1e-4)
    ref = oracle.fit(X32.astype(np.float64), K, tol=1e-12, max_iter=400, algo="gs", iters_lock=g["iters"])
    for k in range(K):
        if ref.lam[k] >= 1e-2 * ref.lam[0]:
            assert abs(lam[k] - ref.lam[k]) <= 1e-4 * ref.lam[k], k
            assert angle(P[:, k], ref.P[:, k]) <= 1e-3, k
            assert angle(V[:, k], ref.T[:, k]) <= 1e-3, k


def test_k_equals_n_1024_orthogonality_and_eq4(gp):
    p = synth.planted(1024, 1024, 10.0, 0.995, 0.0, 102, centre=False)
    X32 = p.X.astype(np.float32)
    K = 1024
    g = fit(gp, X32, K, 1e-6, 40, svd_form=1)
    assert g["status"] in (0, 4) and g["info"]["found"] == K
    V, P, lam = g["T"], g["P"], g["lam"]
    o_p = np.abs(P.T @ P - np.eye(K)).max()
    o_v = np.abs(V.T @ V - np.eye(K)).max()
    e4 = np.linalg.norm(X32 - (V * lam) @ P.T - g["R"]) / np.linalg.norm(X32)
    print(f"1024x1024 K=N: ||PtP-I|| {o_p:.2e} ||VtV-I|| {o_v:.2e} Eq.4 {e4:.2e} "
          f"iters {int(g['iters'].sum())}")
    assert o_p <= 1e-5
    assert o_v <= 1e-4
    assert e4 <= 1e-5


@pytest.mark.parametrize("algo", ["gs", "nipals"])
def test_svd_form_is_the_same_fit(gp, algo):
    X32 = synth.planted(700, 300, 10.0, 0.85, 0.01, 103).X.astype(np.float32)
    a = fit(gp, X32, 8, 1e-6, 1000, algo=algo, svd_form=0)
    b = fit(gp, X32, 8, 1e-6, 1000, algo=algo, svd_form=1)
    for key in ("P", "lam", "iters", "R"):
        assert np.array_equal(a[key], b[key]), key
    np.testing.assert_allclose(b["T"] * b["lam"], a["T"], rtol=2e-6, atol=2e-6 * np.abs(a["T"]).max())
    np.testing.assert_allclose(np.linalg.norm(b["T"], axis=0), 1.0, rtol=1e-5)
