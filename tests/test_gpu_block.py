"""Block power iteration on the GPU (gspca_fit_block) vs the FP64 oracle's
block_fit, through the C ABI.

Mode L: the oracle replays the GPU's per-block iteration counts on the same
FP32-rounded X.  Bars of the FP32 path: singular values 1e-4 relative
(tail-aware rule below 1e-2 sigma_1), loadings and scores within 1e-3 rad per
component, or per cluster of reference singular values closer than 1e-3
relative (subspace angle), ||P^T P - I||_max <= 1e-5, ||V^T V - I||_max <= 1e-4,
||R_gpu - R_or||_F <= 1e-5 ||X||_F.  Also: the exact singular values of a
noise-free planted spectrum, K = N = 1024 orthogonality and Eq. 4, a
rank-deficient X stopping as degenerate.
"""
import numpy as np
import pytest

import oracle
import synth
from parity_helpers import angle, clusters, sigma_ok, subspace_angle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    import paper_0811_1081_gb300 as m

    m.load()
    return m


def fit_block(gp, X32, K, b, tol=1e-6, max_iter=1000, **kw):
    import torch

    M, N = X32.shape
    with gp.Handle(M, N, K) as h:
        r = h.fit_block(torch.from_numpy(X32).cuda(), K, block=b, tol=tol, max_iter=max_iter, want_R=True, **kw)
        torch.cuda.synchronize()
        return dict(T=r.T.cpu().numpy().astype(np.float64), P=r.P.cpu().numpy().astype(np.float64),
                    lam=r.lam.cpu().numpy(), iters=r.iters.cpu().numpy(), R=r.R.cpu().numpy().astype(np.float64),
                    status=r.status, info=r.info)


CASES = [(500, 200, 10, 4, 10.0, 0.85), (1003, 517, 12, 5, 10.0, 0.9), (3000, 800, 24, 8, 10.0, 0.93),
         (200, 2049, 6, 3, 5.0, 0.8)]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}k{c[2]}b{c[3]}" for c in CASES])
def test_block_vs_oracle(gp, case):
    M, N, K, b, s0, ratio = case
    X32 = synth.planted(M, N, s0, ratio, 0.01, (97, M, N)).X.astype(np.float32)
    g = fit_block(gp, X32, K, b)
    assert g["status"] in (0, 4) and g["info"]["found"] == K
    ref = oracle.block_fit(X32.astype(np.float64), K, b, tol=1e-6, max_iter=1000, iters_lock=g["iters"])
    assert ref.found == K
    ok = sigma_ok(g["lam"], ref.lam)
    assert ok.all(), (np.nonzero(~ok), g["lam"], ref.lam)
    for grp in clusters(ref.lam, 1e-3, floor=1e-2):
        if len(grp) == 1:
            assert angle(g["P"][:, grp[0]], ref.P[:, grp[0]]) <= 1e-3, grp
            assert angle(g["T"][:, grp[0]], ref.T[:, grp[0]]) <= 1e-3, grp
        else:
            assert subspace_angle(g["P"][:, grp], ref.P[:, grp]) <= 1e-3, grp
    assert np.abs(g["P"].T @ g["P"] - np.eye(K)).max() <= 1e-5
    V = g["T"] / g["lam"]
    assert np.abs(V.T @ V - np.eye(K)).max() <= 1e-4
    assert np.linalg.norm(g["R"] - ref.R) <= 1e-5 * np.linalg.norm(X32)
    assert np.linalg.norm(X32 - g["T"] @ g["P"].T - g["R"]) <= 1e-5 * np.linalg.norm(X32)


def test_block_recovers_a_noise_free_spectrum(gp):
    p = synth.planted(2000, 400, 10.0, 0.8, 0.0, 98)
    X32 = p.X.astype(np.float32)
    g = fit_block(gp, X32, 16, 8, tol=1e-7, max_iter=2000)
    s = np.linalg.svd(X32.astype(np.float64), compute_uv=False)
    np.testing.assert_allclose(g["lam"], s[:16], rtol=1e-5)
    for k in range(16):
        assert angle(g["P"][:, k], p.right[:, k]) <= 1e-3


def test_block_k_equals_n_1024(gp):
    p = synth.planted(1024, 1024, 10.0, 0.995, 0.0, 102, centre=False)
    X32 = p.X.astype(np.float32)
    K = 1024
    g = fit_block(gp, X32, K, 32, tol=1e-6, max_iter=40, svd_form=1)
    assert g["status"] in (0, 4) and g["info"]["found"] == K
    V, P, lam = g["T"], g["P"], g["lam"]
    o_p = np.abs(P.T @ P - np.eye(K)).max()
    o_v = np.abs(V.T @ V - np.eye(K)).max()
    e4 = np.linalg.norm(X32 - (V * lam) @ P.T - g["R"]) / np.linalg.norm(X32)
    print(f"block 1024x1024 K=N b=32: ||PtP-I|| {o_p:.2e} ||VtV-I|| {o_v:.2e} Eq.4 {e4:.2e}, "
          f"{g['info']['kernel_ms']:.0f} ms")
    assert o_p <= 1e-5 and o_v <= 1e-4 and e4 <= 1e-5


def test_block_rank_deficient_stops_as_degenerate(gp):
    """A rank-3 X in blocks of 2: the second block's start has one independent direction
    (FP32 rounding of X is far below the Gram-pivot threshold), so the fit ends there as
    degenerate with the first block kept.  (The FP64 oracle, on the same FP32-rounded X,
    sees the rounding directions as independent: the thresholds scale with the precision,
    as for the one-vector loop, so the singular values are compared with numpy's SVD.)"""
    g0 = synth.rng(12, 1)
    X32 = (g0.standard_normal((60, 3)) @ g0.standard_normal((3, 20))).astype(np.float32)
    g = fit_block(gp, X32, 6, 2, tol=1e-7)
    assert g["status"] == 5 and g["info"]["found"] == 2
    s = np.linalg.svd(X32.astype(np.float64), compute_uv=False)
    np.testing.assert_allclose(g["lam"][:2], s[:2], rtol=1e-4)
    assert np.all(g["lam"][2:] == 0) and np.all(g["P"][:, 2:] == 0)
