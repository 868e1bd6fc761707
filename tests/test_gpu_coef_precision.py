"""Precision of the GS-PCA Gram-Schmidt coefficients on the GPU against FP64.

Sec. 2.3 forms, every half-iteration, the coefficients b' = V_(k)^T v' and
a' = U_(k)^T u_pre' of the classical Gram-Schmidt step (the paper computes
them in FP64).  The library stores R and the factors in FP32 and combines the
per-CTA FP32 partial sums in float-float (k <= 128) or in 64-bit fixed point
(k > 128); with the two-reduction step a' is formed as Q^T v' - Z b' from
factors kept up to date per component.  The reading of the precision
requirement: every coefficient within one FP32 ulp of the norm of the vector
it is taken from (plus the FP64 computation's own error, ~1e-16 relative).

The fit writes, through the testing aid opts->coef_trace, the last iteration's
b', a', v' and u_pre' of every component; the test recomputes V_(k)^T v' and
U_(k)^T u_pre' in FP64 from the GPU's own FP32 vectors (V from the SVD-form
output, U = P) and measures |coefficient - FP64| in ulps of ||v'|| and
||u_pre'||.  Cases: the 10000 x 2000, K = 50 workload (two-reduction step where
its range guard allows), the same with the three-reduction step forced, and
a 200-component fit (fixed-point sums past 128 components).
"""
import numpy as np
import pytest

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


def ulp32(x):
    """Spacing of FP32 numbers at |x| (x > 0): 2^(floor(log2 x) - 23)."""
    return 2.0 ** (np.floor(np.log2(x)) - 23)


def coefficient_errors(gp, X32, K, tol, max_iter, **kw):
    import torch

    M, N = X32.shape
    tr = torch.full((K * (2 * K + M + N),), float("nan"), dtype=torch.float32, device="cuda")
    with gp.Handle(M, N, K) as h:
        r = h.fit(torch.from_numpy(X32).cuda(), K, tol=tol, max_iter=max_iter, algo="gs", svd_form=1,
                  coef_trace=tr, **kw)
        torch.cuda.synchronize()
        V = r.T.cpu().numpy().astype(np.float64)
        U = r.P.cpu().numpy().astype(np.float64)
        found = r.info["found"]
    t = tr.cpu().numpy().astype(np.float64).reshape(K, 2 * K + M + N)
    eb, ea = [], []
    for k in range(1, found):
        b, a = t[k, :k], t[k, K:K + k]
        v, u = t[k, 2 * K:2 * K + M], t[k, 2 * K + M:]
        b64 = V[:, :k].T @ v
        a64 = U[:, :k].T @ u
        eb.append(np.abs(b - b64).max() / ulp32(np.linalg.norm(v)))
        ea.append(np.abs(a - a64).max() / ulp32(np.linalg.norm(u)))
    return np.array(eb), np.array(ea)


CASES = {
    "10000x2000_k50_two_reduction": (lambda: synth.WORKLOADS["planted_10000x2000"].make(), 50, 1e-6, 1000, {}),
    "10000x2000_k50_three_reduction": (lambda: synth.WORKLOADS["planted_10000x2000"].make(), 50, 1e-6, 1000,
                                       {"gs_step": 1}),
    "1024x512_k200_fixed_point": (lambda: synth.planted(1024, 512, 10.0, 0.98, 1e-3, 73).X, 200, 1e-6, 300, {}),
}


@pytest.mark.parametrize("name", list(CASES))
def test_gram_schmidt_coefficients_within_one_ulp(gp, name):
    make, K, tol, max_iter, kw = CASES[name]
    X32 = make().astype(np.float32)
    eb, ea = coefficient_errors(gp, X32, K, tol, max_iter, **kw)
    print(f"{name}: b' error max {eb.max():.3f} ulp (median {np.median(eb):.3f}), "
          f"a' error max {ea.max():.3f} ulp (median {np.median(ea):.3f})")
    assert np.isfinite(eb).all() and np.isfinite(ea).all()
    assert eb.max() <= 1.0
    assert ea.max() <= 1.0
