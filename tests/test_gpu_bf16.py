"""bfloat16 storage of the residual R (the precision variant of Sec. 3's remark that the
programs change precision through their types) vs the FP64 oracle, through the C ABI.

Two comparisons, both iteration-locked (the oracle replays the GPU's iteration counts):

* Parity: the oracle with storage="bf16" on the same X, which rounds R to bfloat16 after
  centring and after every deflation exactly where the library stores it.  The two sides
  differ by the FP32 arithmetic of the GPU and by the rare deflated entry whose FP32 and
  FP64 values round to neighbouring bfloat16 numbers, so the FP32-storage bars apply:
  singular value 1e-4 relative, loading and score angle 1e-3 rad, GS ||P^T P - I|| 1e-5.
  Residual: R = X - sum_k lambda_k v_k u_k^T (Eq. 4) moves by at most
  sum_k (|d lambda_k| + lambda_k (|du_k| + |dv_k|)) when the components move, plus the
  storage rounding (2^-9 ||R||_F if every entry flipped to its neighbour) and the FP32
  arithmetic (1e-5 ||X||_F); the bound is evaluated from the measured differences.  (With
  bfloat16 storage a flip in one deflation nudges the later components, whose deflations
  then differ by more than one spacing, so no bound of the FP32 kind holds.)
* Stated error against the FP64 oracle on the unrounded X (what bfloat16 storage costs):
  singular value 2e-3 relative; loading angle within 1e-2 rad on the planted 500 x 200
  workload, where rounding X perturbs it by ~2^-9/sqrt(3) of each entry.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SIG_REL = 1e-4
ANGLE = 1e-3
ORTHO = 1e-5


@pytest.fixture(scope="module")
def gp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    import paper_0811_1081_gb300 as m

    m.load()
    return m


def angle(a, b):
    na, nb = np.linalg.norm(a), np.linalg.norm(b)
    if na == 0 or nb == 0:
        return 0.0 if na == nb else math.pi / 2
    return math.acos(min(1.0, abs(float(a @ b)) / (na * nb)))


def run_bf16(gp, X32, K, algo="gs", tol=1e-6, max_iter=1000, want_R=True, **kw):
    import torch

    M, N = X32.shape
    with gp.Handle(M, N, K, dtype="bf16") as h:
        r = h.fit(torch.from_numpy(X32).cuda(), K, tol=tol, max_iter=max_iter, algo=algo, want_R=want_R, **kw)
        torch.cuda.synchronize()
        return dict(T=r.T.cpu().numpy().astype(np.float64), P=r.P.cpu().numpy().astype(np.float64),
                    lam=r.lam.cpu().numpy(), iters=r.iters.cpu().numpy(), status=r.status, info=r.info,
                    R=None if r.R is None else r.R.cpu().numpy().astype(np.float64))


def check_bf16_locked(g, X32, K, algo, tol=1e-6, max_iter=1000, center=0):
    ref = oracle.fit(X32.astype(np.float64), K, tol=tol, max_iter=max_iter, algo=algo, center=center,
                     iters_lock=np.maximum(g["iters"], 1), storage="bf16")
    drift = 0.0  # bound on ||sum_k lambda_k v_k u_k^T - (same for the oracle)||_F
    for k in range(ref.found):
        lam_o = np.linalg.norm(ref.T[:, k])  # ||T(k)|| = lambda_k (GS) or ||t_k|| (NIPALS)
        du = 2 * math.sin(angle(g["P"][:, k], ref.P[:, k]) / 2)
        dv = 2 * math.sin(angle(g["T"][:, k], ref.T[:, k]) / 2)
        drift += abs(np.linalg.norm(g["T"][:, k]) - lam_o) + lam_o * (du + dv)
        assert abs(g["lam"][k] - ref.lam[k]) <= SIG_REL * ref.lam[k], (k, g["lam"][k], ref.lam[k])
        assert angle(g["P"][:, k], ref.P[:, k]) <= ANGLE, (k, angle(g["P"][:, k], ref.P[:, k]))
        assert angle(g["T"][:, k], ref.T[:, k]) <= ANGLE, k
    if algo == "gs" and ref.found:
        P = g["P"][:, :ref.found]
        assert np.abs(P.T @ P - np.eye(ref.found)).max() <= ORTHO
    if g["R"] is not None:
        xn = np.linalg.norm(X32.astype(np.float64))
        assert np.linalg.norm(g["R"] - ref.R) <= 1e-5 * xn + 2.0**-9 * np.linalg.norm(ref.R) + drift
        # the residual the library hands back is made of bfloat16 values
        np.testing.assert_array_equal(oracle.round_bf16(g["R"]), g["R"])
    return ref


@pytest.mark.parametrize("algo", ["gs", "nipals"])
def test_bf16_planted_500x200_locked(gp, algo):
    w = synth.WORKLOADS["planted_500x200"]
    X32 = w.make().astype(np.float32)
    g = run_bf16(gp, X32, w.K, algo, w.tol, w.max_iter)
    assert g["status"] == 0 and g["info"]["found"] == w.K
    check_bf16_locked(g, X32, w.K, algo, w.tol, w.max_iter)


@pytest.mark.parametrize("algo", ["gs", "nipals"])
def test_bf16_error_against_fp64_oracle(gp, algo):
    """What storing R in bfloat16 costs against the FP64 oracle on the unrounded X."""
    w = synth.WORKLOADS["planted_500x200"]
    X32 = w.make().astype(np.float32)
    g = run_bf16(gp, X32, w.K, algo, w.tol, w.max_iter, want_R=False)
    ref = oracle.fit(X32.astype(np.float64), w.K, tol=w.tol, max_iter=w.max_iter, algo=algo,
                     iters_lock=np.maximum(g["iters"], 1))
    rel = np.abs(g["lam"] - ref.lam) / ref.lam
    ang = [angle(g["P"][:, k], ref.P[:, k]) for k in range(w.K)]
    assert rel.max() <= 2e-3, rel
    assert max(ang) <= 1e-2, ang
    assert rel.max() > 1e-6  # the storage is really bfloat16


SHAPES = [(1, 1, 1), (2, 3, 2), (3, 2, 2), (5, 7, 3), (31, 33, 5), (33, 31, 5), (257, 31, 7), (31, 257, 7),
          (1003, 517, 6), (130, 1025, 4), (200, 2049, 3), (64, 4097, 3), (40, 8191, 2)]


@pytest.mark.parametrize("algo", ["gs", "nipals"])
@pytest.mark.parametrize("shape", SHAPES, ids=[f"{m}x{n}k{k}" for m, n, k in SHAPES])
def test_bf16_shapes_locked(gp, algo, shape):
    """Odd column counts (panels padded to an even number of cells), tiny and wide shapes:
    every column template."""
    M, N, K = shape
    if min(M, N) >= 8:
        X = synth.planted(M, N, 5.0, 0.8, 0.01, (23, M, N)).X
    else:
        X = synth.rng(23, M, N).standard_normal((M, N))
    X32 = X.astype(np.float32)
    g = run_bf16(gp, X32, K, algo, 1e-6, 500)
    assert g["status"] in (0, 4)
    check_bf16_locked(g, X32, K, algo, 1e-6, 500)


@pytest.mark.parametrize("center", [1, 2])
def test_bf16_centering(gp, center):
    """Centring before the rounding to bfloat16.  The planted part keeps clear spectral gaps
    (a near-degenerate spectrum, such as uniform noise, turns the rare FP32-vs-FP64 tie of a
    rounding into angle differences above the bar)."""
    p = synth.planted(400, 151, 5.0, 0.8, 0.01, 3, centre=False)
    offs = 1.0 + synth.rng(3, 1).random(151)[None, :] + 0.5 * synth.rng(3, 2).random(400)[:, None]
    X32 = (p.X + offs).astype(np.float32)
    g = run_bf16(gp, X32, 4, "gs", center=center, want_R=False)
    check_bf16_locked(g, X32, 4, "gs", center=center)


@pytest.mark.parametrize("team", [1, 4, 16])
@pytest.mark.parametrize("bpass", [1, 2])
def test_bf16_batched_locked(gp, team, bpass):
    """The batched form with bfloat16 storage, every problem against the bf16 oracle."""
    import torch

    shapes = [(5, 3, 3), (37, 61, 4), (300, 65, 6), (257, 513, 5), (1001, 1023, 4), (640, 201, 8), (96, 700, 1)]
    probs = []
    for i, (M, N, K) in enumerate(shapes):
        probs.append((synth.batch_problem(i, M, N, seed=9).X.astype(np.float32), K))
    with gp.Handle(1001, 1024, 16, dtype="bf16") as h:
        b = gp.Batch([{"X": torch.from_numpy(X).cuda().t().contiguous().t(), "K": K} for X, K in probs])
        try:
            _, st = gp.gspca_fit_batched(h.h, b, tol=1e-6, max_iter=1000, algo="gs", cluster_ctas=team,
                                         batch_pass=bpass)
        except gp.GspcaError as e:
            if team == 16:
                pytest.skip(f"team of 16 CTAs not launchable here: {e}")
            raise
        torch.cuda.synchronize()
        assert st in (gp.GSPCA_OK, gp.GSPCA_WARN_NOT_CONVERGED)
        outs = [dict(T=r.T.cpu().numpy().astype(np.float64), P=r.P.cpu().numpy().astype(np.float64),
                     lam=r.lam.cpu().numpy(), iters=r.iters.cpu().numpy(), R=None) for r in b.results]
    for (X, K), g in zip(probs, outs):
        check_bf16_locked(g, X, K, "gs")


def test_bf16_alg_bytes_halve_the_residual_stream(gp):
    """The persistent kernel's algorithmic byte count charges 2 bytes per element of R."""
    import torch

    X32 = synth.planted(800, 300, 5.0, 0.85, 0.01, 3).X.astype(np.float32)
    Xd = torch.from_numpy(X32).cuda()
    lock = [6, 5, 4]
    with gp.Handle(800, 300, 3) as h32, gp.Handle(800, 300, 3, dtype="bf16") as h16:
        a = h32.fit(Xd, 3, iters_lock=lock, algo="nipals").info["alg_bytes"]
        b = h16.fit(Xd, 3, iters_lock=lock, algo="nipals").info["alg_bytes"]
    assert b == pytest.approx(a / 2)
