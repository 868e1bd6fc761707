"""FP64 storage path (gspca_fit_f64 on a GSPCA_F64 handle) vs the FP64 oracle.

The paper's programs run in double (Sec. 3); this path keeps X, R, the factors,
every product and the test in IEEE double, so it is compared with the oracle
at FP64 rounding, not at the FP32 bars: the two sum in different orders (the
GPU per CTA, then across CTAs in CTA order), so bit equality is not expected,
but singular values agree to 1e-12 relative, loadings and scores to 1e-9
(sign-aligned distance of unit vectors), the residual to 1e-12 ||X||_F, and
free-running iteration counts to within one of the oracle's.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SIG = 1e-12
ANG = 1e-9
RES = 1e-12


@pytest.fixture(scope="module")
def gp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    import paper_0811_1081_gb300 as m

    m.load()
    return m


def dist(a, b):
    """Sign-aligned distance of the unit vectors along a and b (about the angle between them)."""
    na, nb = np.linalg.norm(a), np.linalg.norm(b)
    if na == 0 or nb == 0:
        return 0.0 if na == nb else 2.0
    a, b = a / na, b / nb
    return min(float(np.linalg.norm(a - b)), float(np.linalg.norm(a + b)))


def fit64(gp, X, K, algo="gs", tol=1e-10, max_iter=2000, layout="row", **kw):
    import torch

    M, N = X.shape
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    if layout == "col":
        Xd = Xd.t().contiguous().t()
    with gp.Handle(M, N, K, dtype="f64") as h:
        r = h.fit64(Xd, K, tol=tol, max_iter=max_iter, algo=algo, want_R=True, **kw)
        torch.cuda.synchronize()
        return dict(T=r.T.cpu().numpy(), P=r.P.cpu().numpy(), lam=r.lam.cpu().numpy(), iters=r.iters.cpu().numpy(),
                    R=r.R.cpu().numpy(), status=r.status, info=r.info)


def check(g, X, K, algo, tol=1e-10, max_iter=2000, center=0):
    ref = oracle.fit(X, K, tol=tol, max_iter=max_iter, algo=algo, center=center, iters_lock=np.maximum(g["iters"], 1))
    assert g["info"]["found"] == ref.found
    for k in range(ref.found):
        assert abs(g["lam"][k] - ref.lam[k]) <= SIG * ref.lam[k], (k, g["lam"][k], ref.lam[k])
        assert dist(g["P"][:, k], ref.P[:, k]) <= ANG, k
        assert dist(g["T"][:, k], ref.T[:, k]) <= ANG, k
    assert np.linalg.norm(g["R"] - ref.R) <= RES * np.linalg.norm(X)
    return ref


@pytest.mark.parametrize("algo", ["gs", "nipals"])
def test_planted_500x200(gp, algo):
    X = synth.WORKLOADS["planted_500x200"].make()
    g = fit64(gp, X, 10, algo)
    assert g["status"] == 0
    check(g, X, 10, algo)
    free = oracle.fit(X, 10, tol=1e-10, max_iter=2000, algo=algo)
    assert np.abs(g["iters"] - free.iters).max() <= 1, (g["iters"], free.iters)
    if algo == "gs":
        assert np.abs(g["P"].T @ g["P"] - np.eye(10)).max() <= 1e-13


SHAPES = [(1, 1, 1), (2, 3, 2), (3, 2, 2), (33, 31, 5), (31, 33, 5), (257, 31, 7), (31, 257, 7), (1003, 517, 6),
          (130, 1025, 4), (200, 2049, 3), (64, 4097, 3), (40, 8192, 2), (3000, 800, 20)]


@pytest.mark.parametrize("algo", ["gs", "nipals"])
@pytest.mark.parametrize("shape", SHAPES, ids=[f"{m}x{n}k{k}" for m, n, k in SHAPES])
def test_shapes_locked(gp, algo, shape):
    M, N, K = shape
    X = synth.planted(M, N, 5.0, 0.8, 0.01, (23, M, N)).X if min(M, N) >= 8 else synth.rng(23, M, N).standard_normal((M, N))
    g = fit64(gp, X, K, algo, tol=1e-9, max_iter=500)
    assert g["status"] in (0, 4)
    check(g, X, K, algo, tol=1e-9, max_iter=500)


@pytest.mark.parametrize("layout", ["row", "col"])
@pytest.mark.parametrize("center", [0, 1, 2])
def test_layouts_and_centring(gp, layout, center):
    X = synth.uniform(400, 150, 3) + 1.0
    g = fit64(gp, X, 4, "gs", layout=layout, center=center)
    check(g, X, 4, "gs", center=center)


@pytest.mark.parametrize("algo", ["gs", "nipals"])
def test_zero_start_column_and_rank_exhausted(gp, algo):
    X = synth.planted(120, 40, 5.0, 0.7, 0.01, 8).X
    X[:, 0] = 0.0
    g = fit64(gp, X, 4, algo)
    assert g["status"] == 0 and g["info"]["found"] == 4
    check(g, X, 4, algo)
    g0 = synth.rng(12, 1)
    X = g0.standard_normal((60, 3)) @ g0.standard_normal((3, 20))
    g = fit64(gp, X, 5, algo)
    ref = oracle.fit(X, 5, tol=1e-10, max_iter=2000, algo=algo)
    assert g["status"] == 5 and g["info"]["found"] == ref.found == 3
    np.testing.assert_allclose(g["lam"][:3], ref.lam[:3], rtol=SIG)
    assert np.all(g["lam"][3:] == 0) and np.all(g["P"][:, 3:] == 0)


def test_closed_forms_and_determinism(gp):
    """The rational closed-form fixtures (X = Q diag(sigma) Z^T) are returned to FP64 rounding,
    and two runs give the same bits."""
    import test_golden as tg

    for name in tg.CASES:
        fx = tg.load(name)
        K = fx["K"]
        a = fit64(gp, fx["X"], K, "gs", tol=1e-14, max_iter=100000)
        b = fit64(gp, fx["X"], K, "gs", tol=1e-14, max_iter=100000)
        for key in ("T", "P", "lam", "iters", "R"):
            assert np.array_equal(a[key], b[key]), key
        np.testing.assert_allclose(a["lam"], fx["lambda"], rtol=1e-13)
        # a stop on |d lambda| < 1e-14 lambda leaves angles of about its square root (lambda
        # converges quadratically in the angle): the oracle's own pin, 1 - |cos| < 1e-12
        for k in range(K):
            c = abs(a["P"][:, k] @ fx["P"][:, k]) / np.linalg.norm(a["P"][:, k])
            assert 1.0 - c < 1e-12


def test_svd_form_and_iteration_lock(gp):
    X = synth.planted(700, 300, 10.0, 0.85, 0.01, 31).X
    lock = [3, 5, 2, 7, 4]
    g = fit64(gp, X, 5, "gs", iters_lock=lock, svd_form=1)
    assert list(g["iters"]) == lock
    ref = oracle.fit(X, 5, tol=1e-10, max_iter=2000, algo="gs", iters_lock=lock)
    np.testing.assert_allclose(g["lam"], ref.lam, rtol=SIG)
    np.testing.assert_allclose(np.linalg.norm(g["T"], axis=0), 1.0, rtol=1e-13)
    for k in range(5):
        assert dist(g["T"][:, k], ref.T[:, k]) <= ANG


def test_dtype_mismatch_is_refused(gp):
    import ctypes

    import torch

    X64 = torch.ones((20, 10), dtype=torch.float64, device="cuda")
    with gp.Handle(20, 10, 2, dtype="f32") as h:
        with pytest.raises(gp.GspcaError) as e:
            gp.gspca_fit_f64(h.h, X64, 2)
        assert e.value.status == gp.GSPCA_ERR_INVALID_ARG
    with gp.Handle(20, 10, 2, dtype="f64") as h:
        with pytest.raises(gp.GspcaError) as e:
            h.fit(X64.float(), 2)
        assert e.value.status == gp.GSPCA_ERR_INVALID_ARG
        o, _ = gp._opts(gs_passes=2)
        T = torch.empty((2, 20), dtype=torch.float64, device="cuda").t()
        P = torch.empty((2, 10), dtype=torch.float64, device="cuda").t()
        lam = torch.empty(2, dtype=torch.float64, device="cuda")
        st = gp.load().gspca_fit_f64(ctypes.c_void_p(h.h), None, ctypes.c_void_p(X64.data_ptr()), gp.GSPCA_ROW_MAJOR,
                                     10, 20, 10, 2, 1e-6, 100, gp.GSPCA_GS, ctypes.c_void_p(T.data_ptr()),
                                     ctypes.c_void_p(P.data_ptr()), ctypes.c_void_p(lam.data_ptr()), None, None,
                                     ctypes.byref(o))
        assert st == gp.GSPCA_ERR_NOT_SUPPORTED
