"""Closed-form fixtures (tests/golden/*.txt, written by make_closed_forms.py with
exact rational arithmetic): X = Q diag(sigma) Z^T with orthonormal rational Q, Z.
By Eq. 5 every correct run returns lambda_k = sigma_k, P(k) = +-Z(k) and
T(k) = +-sigma_k Q(k).  The oracle is held to FP64 rounding; the CUDA path (FP32
arithmetic, X exact in FP32) to the FP32 parity bars."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
CASES = ["closed_form_4x3", "closed_form_8x4_zero_rows"]
ALGOS = ["nipals", "gs"]


def load(name):
    """Parse a fixture: header lines M/N/K, then blocks X, lambda, P, T of rationals."""
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, name + ".txt")) if ln.strip() and not ln.startswith("#")]
    d, key, blocks = {}, None, {}
    for r in rows:
        if len(r) == 2 and r[0] in ("M", "N", "K"):
            d[r[0]] = int(r[1])
        elif len(r) == 1 and r[0] in ("X", "lambda", "P", "T"):
            key = r[0]
            blocks[key] = []
        else:
            blocks[key].append([float(Fraction(v)) for v in r])
    d.update({k: np.array(v, dtype=np.float64) for k, v in blocks.items()})
    d["lambda"] = d["lambda"].ravel()
    assert d["X"].shape == (d["M"], d["N"]) and d["P"].shape == (d["N"], d["K"]) and d["T"].shape == (d["M"], d["K"])
    return d


def angle(a, b):
    c = abs(float(a @ b)) / (np.linalg.norm(a) * np.linalg.norm(b))
    return math.acos(min(1.0, c))


def check(fx, lam, P, T, sig_rel, ang, t_rel):
    K = fx["K"]
    np.testing.assert_allclose(lam[:K], fx["lambda"], rtol=sig_rel)
    for k in range(K):
        assert angle(P[:, k], fx["P"][:, k]) <= ang
        # T(k) = +-sigma_k Q(k): same direction and norm as the fixture's column
        assert angle(T[:, k], fx["T"][:, k]) <= ang
        assert abs(np.linalg.norm(T[:, k]) - fx["lambda"][k]) <= t_rel * fx["lambda"][k]


def test_fixtures_are_exact_svds():
    """The stored factors multiply back to X exactly and have orthonormal columns."""
    for name in CASES:
        fx = load(name)
        Pn = fx["P"]
        Qn = fx["T"] / fx["lambda"]
        np.testing.assert_allclose(fx["T"] @ Pn.T, fx["X"], atol=1e-14)
        np.testing.assert_allclose(Pn.T @ Pn, np.eye(fx["K"]), atol=1e-15)
        np.testing.assert_allclose(Qn.T @ Qn, np.eye(fx["K"]), atol=1e-15)


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("algo", ALGOS)
def test_oracle_reproduces_closed_form(oracle_mod, name, algo):
    fx = load(name)
    f = oracle_mod.fit(fx["X"], fx["K"], tol=1e-14, max_iter=100000, algo=algo)
    assert f.status == 0 and f.found == fx["K"]
    check(fx, f.lam, f.P, f.T, 1e-12, 1e-7, 1e-12)


@pytest.mark.gpu
@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("algo", ALGOS)
def test_cuda_path_reproduces_closed_form(name, algo, storage):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    import paper_0811_1081_gb300 as gp

    gp.load()
    fx = load(name)
    X = torch.from_numpy(fx["X"].astype(np.float32)).cuda()
    with gp.Handle(fx["M"], fx["N"], fx["K"], dtype=storage) as h:
        r = h.fit(X, fx["K"], tol=1e-7, max_iter=10000, algo=algo)
        torch.cuda.synchronize()
        lam, P, T = r.lam.cpu().numpy(), r.P.cpu().numpy().astype(np.float64), r.T.cpu().numpy().astype(np.float64)
    assert r.status == 0
    # X is exact in both storages; bfloat16 rounds the deflated residuals (2^-9 relative)
    bars = (1e-5, 1e-3, 1e-5) if storage == "f32" else (1e-2, 2e-2, 1e-2)
    check(fx, lam, P, T, *bars)
