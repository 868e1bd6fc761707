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
