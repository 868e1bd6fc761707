"""GPU vs FP64 oracle parity through the C ABI.

Mode L (iteration-locked): the oracle replays the GPU's iteration count per
component on the same FP32-rounded X, so both follow one trajectory and the
comparison has no stopping jitter.  Bars (FP32 storage of R):
  singular value   |lambda_gpu - lambda_or| / lambda_or <= 1e-4
  loading angle    angle(P_gpu(k), P_or(k))              <= 1e-3 rad
  GS orthogonality ||P^T P - I||_max                     <= 1e-5
  scores           angle(T(k)) <= 1e-3 rad, ||T(k)|| within 1e-4 relative
  residual         ||R_gpu - R_or||_F                    <= 1e-5 ||X||_F
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
RESID = 1e-5


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
    c = abs(float(a @ b)) / (na * nb)
    return math.acos(min(1.0, c))


def to_dev(X32, layout="row", pad=0):
    import torch

    M, N = X32.shape
    if layout == "row":
        base = torch.zeros((M, N + pad), dtype=torch.float32)
        base[:, :N] = torch.from_numpy(X32)
        return base.cuda()[:, :N]
    base = torch.zeros((N, M + pad), dtype=torch.float32)
    base[:, :M] = torch.from_numpy(np.ascontiguousarray(X32.T))
    return base.cuda()[:, :M].t()


def run_gpu(gp, X32, K, algo="gs", tol=1e-6, max_iter=1000, want_R=True, layout="row", pad=0, **kw):
    import torch

    M, N = X32.shape
    Xd = to_dev(X32, layout, pad)
    with gp.Handle(M, N, K) as h:
        r = h.fit(Xd, K, tol=tol, max_iter=max_iter, algo=algo, want_R=want_R, **kw)
        torch.cuda.synchronize()
        out = dict(T=r.T.cpu().numpy().astype(np.float64), P=r.P.cpu().numpy().astype(np.float64),
                   lam=r.lam.cpu().numpy(), iters=r.iters.cpu().numpy(), status=r.status, info=r.info,
                   R=r.R.cpu().numpy().astype(np.float64) if r.R is not None else None)
    return out


def check_locked(g, X32, K, algo, tol=1e-6, max_iter=1000, center=0, kmax=None, resid=True):
    X64 = X32.astype(np.float64)
    ref = oracle.fit(X64, K, tol=tol, max_iter=max_iter, algo=algo, center=center,
                     iters_lock=np.maximum(g["iters"], 1))
    found = ref.found
    kk = found if kmax is None else min(found, kmax)
    for k in range(kk):
        assert abs(g["lam"][k] - ref.lam[k]) <= SIG_REL * ref.lam[k], (k, g["lam"][k], ref.lam[k])
        assert angle(g["P"][:, k], ref.P[:, k]) <= ANGLE, (k, angle(g["P"][:, k], ref.P[:, k]))
        assert angle(g["T"][:, k], ref.T[:, k]) <= ANGLE, k
        tn, rn = np.linalg.norm(g["T"][:, k]), np.linalg.norm(ref.T[:, k])
        assert abs(tn - rn) <= SIG_REL * rn, k
    if algo == "gs":
        P = g["P"][:, :kk]
        assert np.abs(P.T @ P - np.eye(kk)).max() <= ORTHO
    if resid and g["R"] is not None and kmax is None:
        xn = np.linalg.norm(ref.R + ref.T @ ref.P.T)
        assert np.linalg.norm(g["R"] - ref.R) <= RESID * xn
    return ref


@pytest.mark.parametrize("algo", ["gs", "nipals"])
def test_planted_500x200_locked(gp, algo):
    w = synth.WORKLOADS["planted_500x200"]
    X32 = w.make().astype(np.float32)
    g = run_gpu(gp, X32, w.K, algo, w.tol, w.max_iter)
    assert g["status"] == 0
    assert g["info"]["found"] == w.K
    check_locked(g, X32, w.K, algo, w.tol, w.max_iter)
    # Eq. 4 on the GPU's own outputs
    assert np.linalg.norm(X32 - g["T"] @ g["P"].T - g["R"]) <= 1e-5 * np.linalg.norm(X32)


@pytest.mark.parametrize("algo", ["gs", "nipals"])
def test_planted_500x200_free_running(gp, algo):
    """Free-running: iteration counts within a few of the oracle's own free run."""
    w = synth.WORKLOADS["planted_500x200"]
    X32 = w.make().astype(np.float32)
    g = run_gpu(gp, X32, w.K, algo, w.tol, w.max_iter)
    ref = oracle.fit(X32.astype(np.float64), w.K, tol=w.tol, max_iter=w.max_iter, algo=algo)
    assert np.abs(g["iters"] - ref.iters).max() <= 3, (g["iters"], ref.iters)
    for k in range(w.K):
        assert abs(g["lam"][k] - ref.lam[k]) <= SIG_REL * ref.lam[k]


SHAPES = [(1, 1, 1), (2, 3, 2), (3, 2, 2), (4, 1, 1), (1, 5, 1), (31, 33, 5), (33, 31, 5),
          (257, 31, 7), (31, 257, 7), (1003, 517, 6), (130, 1025, 4), (200, 2049, 3), (64, 4097, 3)]


@pytest.mark.parametrize("algo", ["gs", "nipals"])
@pytest.mark.parametrize("shape", SHAPES, ids=[f"{m}x{n}k{k}" for m, n, k in SHAPES])
def test_shapes_locked(gp, algo, shape):
    """Tiny, ragged and wide shapes: every column template (N up to 512, 1024, 2048, 4096, 8192)."""
    M, N, K = shape
    if min(M, N) >= 8:
        X = synth.planted(M, N, 5.0, 0.8, 0.01, (17, M, N)).X
    else:
        X = synth.rng(17, M, N).standard_normal((M, N))
    X32 = X.astype(np.float32)
    g = run_gpu(gp, X32, K, algo, 1e-6, 500)
    assert g["status"] in (0, 4)
    check_locked(g, X32, K, algo, 1e-6, 500)


@pytest.mark.parametrize("layout,pad", [("row", 0), ("row", 7), ("col", 0), ("col", 5)])
def test_input_layouts(gp, layout, pad):
    X32 = synth.planted(301, 97, 5.0, 0.8, 0.01, 5).X.astype(np.float32)
    g = run_gpu(gp, X32, 5, "gs", layout=layout, pad=pad)
    check_locked(g, X32, 5, "gs")


@pytest.mark.parametrize("center", [1, 2])
def test_centering(gp, center):
    X32 = (synth.uniform(400, 150, 3) + 1.0).astype(np.float32)
    g = run_gpu(gp, X32, 4, "gs", tol=1e-6, center=center, want_R=False)
    check_locked(g, X32, 4, "gs", center=center)


@pytest.mark.parametrize("algo", ["gs", "nipals"])
def test_zero_start_column(gp, algo):
    X = synth.planted(120, 40, 5.0, 0.7, 0.01, 8).X
    X[:, 0] = 0.0
    X32 = X.astype(np.float32)
    g = run_gpu(gp, X32, 4, algo)
    assert g["status"] == 0 and g["info"]["found"] == 4
    check_locked(g, X32, 4, algo)


@pytest.mark.parametrize("algo", ["gs", "nipals"])
def test_rank_exhausted(gp, algo):
    g0 = synth.rng(12, 1)
    X32 = (g0.standard_normal((60, 3)) @ g0.standard_normal((3, 20))).astype(np.float32)
    g = run_gpu(gp, X32, 5, algo, tol=1e-7)
    assert g["status"] == 5 and g["info"]["found"] == 3
    assert np.all(g["lam"][3:] == 0) and np.all(g["P"][:, 3:] == 0) and np.all(g["T"][:, 3:] == 0)
    s = np.linalg.svd(X32.astype(np.float64), compute_uv=False)
    np.testing.assert_allclose(g["lam"][:3], s[:3], rtol=1e-4)


@pytest.mark.parametrize("algo", ["gs", "nipals"])
def test_max_iter_one(gp, algo):
    X32 = synth.WORKLOADS["planted_500x200"].make().astype(np.float32)
    g = run_gpu(gp, X32, 3, algo, tol=1e-12, max_iter=1)
    assert g["status"] == 4 and np.all(g["iters"] == 1)
    check_locked(g, X32, 3, algo, tol=1e-12, max_iter=1)


def test_device_iteration_lock(gp):
    X32 = synth.WORKLOADS["planted_500x200"].make().astype(np.float32)
    lock = [3, 5, 2, 7]
    g = run_gpu(gp, X32, 4, "gs", iters_lock=lock)
    assert list(g["iters"]) == lock
    check_locked(g, X32, 4, "gs")


def test_deterministic_and_host_path(gp):
    """Two device fits are bit-identical, and the host-buffer entry point gives the same bits."""
    import torch

    X32 = synth.planted(777, 333, 5.0, 0.85, 0.01, 9).X.astype(np.float32)
    a = run_gpu(gp, X32, 6, "gs")
    b = run_gpu(gp, X32, 6, "gs")
    for key in ("T", "P", "lam", "iters", "R"):
        assert np.array_equal(a[key], b[key]), key
    with gp.Handle(777, 333, 6) as h:
        r = h.fit_host(np.ascontiguousarray(X32), 6, tol=1e-6, max_iter=1000, algo="gs", want_R=True)
        torch.cuda.synchronize()
        assert np.array_equal(r.lam, a["lam"])
        assert np.array_equal(r.P.astype(np.float64), a["P"])
        assert np.array_equal(r.T.astype(np.float64), a["T"])
        assert np.array_equal(r.R.astype(np.float64), a["R"])


def test_collinear_orthogonality(gp):
    """Sec. 1/2.3 on duplicated columns: GS keeps PᵀP = I on the GPU; NIPALS's loss is reported."""
    X32 = synth.collinear(400, 64, 1e-3, 4).astype(np.float32)
    K = 100
    gg = run_gpu(gp, X32, K, "gs", tol=1e-5, max_iter=300, want_R=False)
    gn = run_gpu(gp, X32, K, "nipals", tol=1e-5, max_iter=300, want_R=False)
    og = np.abs(gg["P"].T @ gg["P"] - np.eye(K)).max()
    on = np.abs(gn["P"].T @ gn["P"] - np.eye(K)).max()
    print(f"collinear 400x128 K={K}: ||PtP-I||max GS {og:.2e}  NIPALS {on:.2e}")
    assert og <= ORTHO
    assert on > og


def test_wait_limit_returns_timeout_status(gp):
    """The testing hook makes the first ring wait of every pass wait first for a device
    word that nothing sets: its 20 ms limit runs out in every CTA, the CTAs leave through
    the abort word (the grid barrier waits are bounded too), the kernel returns
    GSPCA_ERR_TIMEOUT, and the context stays usable for the next fit."""
    import torch

    X32 = synth.planted(4000, 300, 5.0, 0.8, 0.01, 3).X.astype(np.float32)
    Xd = to_dev(X32)
    with gp.Handle(4000, 300, 3) as h:
        r = h.fit(Xd, 3, tol=1e-6, max_iter=100, algo="gs", timeout_s=0.02, test_stall=1, check=False)
        torch.cuda.synchronize()
        assert r.status == gp.GSPCA_ERR_TIMEOUT
        r2 = h.fit(Xd, 3, tol=1e-6, max_iter=100, algo="gs")
        torch.cuda.synchronize()
        assert r2.status in (0, 4)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("shape", [(1003, 517, 6), (700, 2000, 4), (500, 3000, 3), (64, 4097, 3), (300, 7500, 3)])
def test_load_path_gives_the_same_fit(gp, shape, storage):
    """Reading R through the TMA ring or straight into registers: the same fit (the two-group
    ring pass sums in another order, so the second run replays the first's iteration counts and
    the results agree to FP32 rounding)."""
    import torch

    M, N, K = shape
    X32 = synth.planted(M, N, 5.0, 0.85, 0.01, (37, M, N)).X.astype(np.float32)
    Xd = torch.from_numpy(X32).cuda()
    with gp.Handle(M, N, K, dtype=storage) as h:
        a = h.fit(Xd, K, tol=1e-6, max_iter=1000, algo="gs", load_path=1)
        lock = [int(v) for v in a.iters.cpu().numpy()]
        b = h.fit(Xd, K, tol=1e-6, max_iter=1000, algo="gs", load_path=2, iters_lock=lock)
        torch.cuda.synchronize()
        la, lb = a.lam.cpu().numpy(), b.lam.cpu().numpy()
        Pa, Pb = a.P.cpu().numpy().astype(np.float64), b.P.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(la - lb) <= 1e-5 * la)
    for k in range(K):
        assert angle(Pa[:, k], Pb[:, k]) <= 1e-4


@pytest.mark.parametrize("shape", [(1003, 517, 6), (10000, 2000, 4), (64, 4097, 3)])
def test_resident_factors_do_not_change_results(gp, shape):
    """Keeping the factor rows/slices in shared memory or in global memory is a placement
    choice only: with the same Gram-Schmidt step (the three-reduction one, which both
    placements have) the two fits are bit-identical."""
    import torch

    M, N, K = shape
    X32 = synth.planted(M, N, 5.0, 0.85, 0.01, (31, M, N)).X.astype(np.float32)
    Xd = torch.from_numpy(X32).cuda()
    outs = []
    with gp.Handle(M, N, K) as h:
        for mode in (1, 2):
            r = h.fit(Xd, K, tol=1e-6, max_iter=1000, algo="gs", want_R=True, resident=mode, gs_step=1)
            torch.cuda.synchronize()
            outs.append([t.cpu().numpy() for t in (r.T, r.P, r.lam, r.iters, r.R)])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("shape", [(1003, 517, 6), (10000, 2000, 12), (700, 2000, 40), (64, 4097, 3), (5000, 300, 64)])
def test_two_reduction_gs_step_matches_three(gp, shape, storage):
    """The Gram-Schmidt step from maintained Q = R U, Z = U^T W and V^T V (two grid-wide
    reductions per iteration) against the three-reduction step of Sec. 2.3: the same fit to
    FP32 rounding (the second run replays the first's iteration counts), and GS-PCA's
    orthogonality kept.  The planted spectrum decays by 0.85 per component, so the larger K
    also crosses the 64x range beyond which the step falls back to three reductions.  With
    bfloat16 storage (Q's rows recomputed from the stored residual per component) a different
    rounding of v' or u' can round a deflated entry to the neighbouring bfloat16 value, so the
    bars are the bfloat16 parity bars (1e-4 relative in lambda, 1e-3 rad)."""
    import torch

    M, N, K = shape
    X32 = synth.planted(M, N, 5.0, 0.85, 0.01, (43, M, N)).X.astype(np.float32)
    Xd = torch.from_numpy(X32).cuda()
    sig, ang = (1e-5, 1e-4) if storage == "f32" else (1e-4, 1e-3)
    with gp.Handle(M, N, K, dtype=storage) as h:
        a = h.fit(Xd, K, tol=1e-6, max_iter=1000, algo="gs", gs_step=1)
        lock = [int(v) for v in a.iters.cpu().numpy()]
        b = h.fit(Xd, K, tol=1e-6, max_iter=1000, algo="gs", gs_step=0, iters_lock=lock)
        torch.cuda.synchronize()
        la, lb = a.lam.cpu().numpy(), b.lam.cpu().numpy()
        Pa, Pb = a.P.cpu().numpy().astype(np.float64), b.P.cpu().numpy().astype(np.float64)
        Ta, Tb = a.T.cpu().numpy().astype(np.float64), b.T.cpu().numpy().astype(np.float64)
    if storage == "f32":
        assert a.status == 0 and b.status == 0
        assert np.all(np.abs(la - lb) <= sig * la)
        for k in range(K):
            assert angle(Pa[:, k], Pb[:, k]) <= ang
            assert angle(Ta[:, k], Tb[:, k]) <= ang
    else:
        # the second run stops on the replayed counts (status 0) where the first hit max_iter;
        # near the noise floor of the planted spectrum (the largest singular value of the 0.01
        # noise is about 0.01 (sqrt(M) + sqrt(N))) the singular values form a bulk whose members
        # bfloat16 rounding mixes, so the components above twice that are compared
        assert a.status in (0, 4) and b.status in (0, 4)
        kk = int(np.sum(la >= 2 * 0.01 * (math.sqrt(M) + math.sqrt(N))))
        assert kk >= min(3, K)
        assert np.all(np.abs(la[:kk] - lb[:kk]) <= sig * la[:kk])
        for k in range(kk):
            assert angle(Pa[:, k], Pb[:, k]) <= ang
            assert angle(Ta[:, k], Tb[:, k]) <= ang
    assert np.abs(Pb.T @ Pb - np.eye(K)).max() <= ORTHO
    assert np.abs(Pb.T @ Pb - np.eye(K)).max() <= ORTHO
