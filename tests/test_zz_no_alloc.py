"""gspca_fit_noalloc: the fit for callers that must not allocate device memory.

Some callers cannot call cudaMalloc: a plug-in inside an application whose own
allocator owns the GPU's memory, or a latency-critical loop that cannot pay
for a cudaMalloc/cudaFree pair.  gspca_fit_noalloc serves them from a fixed
scratch array inside the library.  This test calls it through the C ABI and
checks its results against gspca_fit (the handle-based entry point) on the
same input, twice in a row (the second call reuses the scratch the first one
left behind), with the tolerances of the other parity tests.

Named so that pytest collects it last.
"""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

SIG_REL = 1e-4
ANGLE = 1e-3


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


def host(r):
    return {"T": r.T.cpu().numpy().astype(np.float64), "P": r.P.cpu().numpy().astype(np.float64),
            "lam": r.lam.cpu().numpy(), "iters": r.iters.cpu().numpy(),
            "R": None if r.R is None else r.R.cpu().numpy().astype(np.float64)}


@pytest.mark.parametrize("algo", ["gs", "nipals"])
def test_noalloc_matches_handle_fit_twice(gp, algo):
    import torch

    X32 = synth.planted(700, 260, 10.0, 0.85, 0.01, 41).X.astype(np.float32)
    Xd = torch.from_numpy(X32).cuda()
    K = 8
    with gp.Handle(700, 260, K) as h:
        ref = host(h.fit(Xd, K, tol=1e-6, max_iter=1000, algo=algo, want_R=True))
    for _ in range(2):
        r = gp.gspca_fit_noalloc(Xd, K, tol=1e-6, max_iter=1000, algo=algo, want_R=True)
        torch.cuda.synchronize()
        assert r.status == gp.GSPCA_OK
        got = host(r)
        assert np.array_equal(got["iters"], ref["iters"])
        for k in range(K):
            assert abs(got["lam"][k] - ref["lam"][k]) <= SIG_REL * ref["lam"][k]
            assert angle(got["P"][:, k], ref["P"][:, k]) <= ANGLE
            assert angle(got["T"][:, k], ref["T"][:, k]) <= ANGLE
        assert np.linalg.norm(got["R"] - ref["R"]) <= 1e-5 * np.linalg.norm(X32)


def test_noalloc_rejects_sizes_beyond_its_scratch(gp):
    """A problem whose workspace exceeds the fixed scratch is refused before any launch."""
    import torch

    M, N = 9000, 2000  # the residual alone needs 72 MB > 64 MiB of scratch
    assert M * N * 4 > gp.NOALLOC_SCRATCH_BYTES
    Xd = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    r = gp.gspca_fit_noalloc(Xd, 2, check=False)
    assert r.status == gp.GSPCA_ERR_NOT_SUPPORTED


def _check_against_handle(gp, Xd, X32, K, algo):
    """One no-allocation fit of Xd compared with a handle fit of the same input."""
    import torch

    M, N = X32.shape
    with gp.Handle(M, N, K) as h:
        ref = host(h.fit(Xd, K, tol=1e-6, max_iter=1000, algo=algo, want_R=True))
    r = gp.gspca_fit_noalloc(Xd, K, tol=1e-6, max_iter=1000, algo=algo, want_R=True)
    torch.cuda.synchronize()
    assert r.status == gp.GSPCA_OK
    got = host(r)
    assert np.array_equal(got["iters"], ref["iters"])
    for k in range(K):
        assert abs(got["lam"][k] - ref["lam"][k]) <= SIG_REL * ref["lam"][k]
        assert angle(got["P"][:, k], ref["P"][:, k]) <= ANGLE
        assert angle(got["T"][:, k], ref["T"][:, k]) <= ANGLE
    assert np.linalg.norm(got["R"] - ref["R"]) <= 1e-5 * np.linalg.norm(X32)


def test_noalloc_after_calls_of_other_shapes(gp):
    """The scratch keeps whatever the previous call left, laid out for another shape: the
    partial sums, reductions and flags of the next call sit on stale residual and factor
    bytes.  A large fit, then a small one, then NIPALS and GS with other K (so the factor
    leading dimension and every offset move): each matches a handle fit of the same input."""
    import torch

    cases = [((4000, 2000, 16), "gs"), ((700, 260, 8), "gs"), ((900, 333, 3), "nipals"),
             ((640, 500, 40), "gs"), ((700, 260, 8), "nipals")]
    for i, ((M, N, K), algo) in enumerate(cases):
        X32 = synth.planted(M, N, 10.0, 0.85, 0.01, (53, i)).X.astype(np.float32)
        _check_against_handle(gp, torch.from_numpy(X32).cuda(), X32, K, algo)


def test_noalloc_wait_limit_after_other_shape(gp):
    """The testing hook's stall word is cleared by the call's own first kernel, so the
    bounded wait runs out (GSPCA_ERR_TIMEOUT) even after a call of another shape left data
    under it; the next call on the same scratch is normal."""
    import torch

    big = synth.planted(3000, 1500, 10.0, 0.85, 0.01, 61).X.astype(np.float32)
    r0 = gp.gspca_fit_noalloc(torch.from_numpy(big).cuda(), 6, tol=1e-6, max_iter=200, algo="gs")
    torch.cuda.synchronize()
    assert r0.status in (gp.GSPCA_OK, gp.GSPCA_WARN_NOT_CONVERGED)
    X32 = synth.planted(4000, 300, 5.0, 0.8, 0.01, 3).X.astype(np.float32)
    Xd = torch.from_numpy(X32).cuda()
    r = gp.gspca_fit_noalloc(Xd, 3, tol=1e-6, max_iter=100, algo="gs", timeout_s=0.02, test_stall=1, check=False)
    torch.cuda.synchronize()
    assert r.status == gp.GSPCA_ERR_TIMEOUT
    r2 = gp.gspca_fit_noalloc(Xd, 3, tol=1e-6, max_iter=100, algo="gs")
    torch.cuda.synchronize()
    assert r2.status in (gp.GSPCA_OK, gp.GSPCA_WARN_NOT_CONVERGED)


def test_noalloc_rejects_bad_options(gp):
    """Out-of-range option values are refused before any launch, as gspca_fit refuses them."""
    import ctypes

    import torch

    Xd = torch.zeros((50, 20), dtype=torch.float32, device="cuda") + 1.0
    for field, value in (("resident", 3), ("load_path", 7), ("gs_step", 2), ("center", 5)):
        o, _ = gp._opts()
        setattr(o, field, value)
        T = torch.empty((2, 50), device="cuda").t()
        P = torch.empty((2, 20), device="cuda").t()
        lam = torch.empty(2, device="cuda", dtype=torch.float64)
        st = gp.load().gspca_fit_noalloc(None, ctypes.c_void_p(Xd.data_ptr()), gp.GSPCA_ROW_MAJOR, 20, 50, 20, 2,
                                         1e-6, 100, gp.GSPCA_GS, ctypes.c_void_p(T.data_ptr()),
                                         ctypes.c_void_p(P.data_ptr()), ctypes.c_void_p(lam.data_ptr()), None, None,
                                         ctypes.byref(o))
        assert st == gp.GSPCA_ERR_INVALID_ARG, field
