"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test ties one part of the oracle to something independent of its code:
a closed form, a textbook routine written separately (cyclic Jacobi), a
library routine (numpy's SVD / eigh) as a third opinion, brute force on tiny
inputs, or an invariant the paper states (Eq. 2-5, Sec. 2.3).  They are
chosen so that a plausible slip in the oracle (a dropped Gram-Schmidt term,
a wrong sign in the deflation, a transposed product, a missing normalisation,
an off-by-one in the iteration count) fails at least one of them.
"""
import math

import numpy as np
import pytest

import synth


def angle(a, b):
    """Sign-invariant angle between two vectors."""
    c = abs(float(np.dot(a, b))) / (np.linalg.norm(a) * np.linalg.norm(b))
    return math.acos(min(1.0, c))


ALGOS = ["nipals", "gs"]


# --------------------------------------------------------------- closed forms

@pytest.mark.parametrize("algo", ALGOS)
def test_planted_noise_free_spectrum(oracle_mod, algo):
    """X = L diag(s) Rᵀ exactly: singular values are s_i and loadings the columns of R (Eq. 5)."""
    p = synth.planted(60, 40, 10.0, 0.8, 0.0, 123)
    K = 6
    f = oracle_mod.fit(p.X, K, tol=1e-14, max_iter=100000, algo=algo)
    assert f.status == 0 and f.found == K
    np.testing.assert_allclose(f.lam, p.s[:K], rtol=1e-10)
    for k in range(K):
        assert angle(f.P[:, k], p.right[:, k]) < 1e-6
        t_dir = f.T[:, k] / np.linalg.norm(f.T[:, k])
        assert angle(t_dir, p.left[:, k]) < 1e-6
        # T = V Λ (GS) and T = R p (NIPALS): ‖T(k)‖ = λ_k either way
        assert abs(np.linalg.norm(f.T[:, k]) - f.lam[k]) <= 1e-12 * f.lam[k]


@pytest.mark.parametrize("algo", ALGOS)
def test_rank_one_brute_force(oracle_mod, algo):
    """X = a bᵀ: λ = ‖a‖‖b‖, P = ±b/‖b‖, R = 0, and the test stops after exactly 2 iterations."""
    g = synth.rng(5)
    a = g.standard_normal(7)
    b = g.standard_normal(4)
    X = np.outer(a, b)
    f = oracle_mod.fit(X, 1, tol=1e-12, max_iter=50, algo=algo)
    assert f.iters[0] == 2
    assert abs(f.lam[0] - np.linalg.norm(a) * np.linalg.norm(b)) <= 1e-14 * f.lam[0]
    assert angle(f.P[:, 0], b) < 1e-12
    assert np.abs(f.R).max() <= 1e-14 * np.abs(X).max()
    np.testing.assert_allclose(np.outer(f.T[:, 0], f.P[:, 0]), X, atol=1e-14 * np.abs(X).max())


def two_dim_trajectory(sig, Z, start, tol, max_iter):
    """Closed form of the first-component power iteration on X = Q diag(sig) Zᵀ.

    The start vector is v = X e_start.  Then u_0 ∝ Xᵀv = Z diag(sig²) Zᵀ e_start and
    every later u_j is multiplied by Xᵀ X: in the Z basis its coordinates are
    (sig_i^(2(j+1)) z_i).  λ_j = ‖X u_j‖ = sqrt(Σ sig_i² c_i²) with c = unit coordinates.
    Returns the iteration count at which |λ_j − λ_{j−1}| < tol λ_j first holds, and λ there.
    """
    z = Z.T[:, start]
    prev = 0.0
    for j in range(max_iter):
        w = np.array([s ** (2 * (j + 1)) * zi for s, zi in zip(sig, z)])
        c = w / np.linalg.norm(w)
        lam = math.sqrt(float(np.sum((np.asarray(sig) * c) ** 2)))
        if abs(prev - lam) < tol * lam:
            return j + 1, lam, Z @ c
        prev = lam
    return max_iter, lam, Z @ c


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("M", [2, 3])
@pytest.mark.parametrize("ratio", [0.5, 0.8, 0.95])
def test_two_dim_trajectory(oracle_mod, algo, M, ratio):
    """The iteration count and λ at the stop match the closed-form 2-D power iteration."""
    g = synth.rng(11, M)
    Q, _ = np.linalg.qr(g.standard_normal((M, 2)))
    th = 0.7
    Z = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    sig = [3.0, 3.0 * ratio]
    X = Q @ np.diag(sig) @ Z.T
    tol = 1e-9
    n_pred, lam_pred, u_pred = two_dim_trajectory(sig, Z, 0, tol, 10000)
    f = oracle_mod.fit(X, 1, tol=tol, max_iter=10000, algo=algo)
    assert f.iters[0] == n_pred
    assert abs(f.lam[0] - lam_pred) <= 1e-13 * lam_pred
    assert angle(f.P[:, 0], u_pred) < 1e-9


# ------------------------------------------------------------ Jacobi + SVD

def test_jacobi_self_consistency(oracle_mod):
    """Jacobi returns A W = W diag(w) and WᵀW = I; its eigenvalues match numpy's eigh."""
    g = synth.rng(3)
    B = g.standard_normal((50, 30))
    A = B.T @ B
    w, W, sweeps = oracle_mod.jacobi_eigh(A, tol=1e-15)
    assert sweeps > 0
    assert np.abs(A @ W - W * w).max() <= 1e-12 * np.abs(A).max()
    assert np.abs(W.T @ W - np.eye(30)).max() <= 1e-12
    np.testing.assert_allclose(w, np.sort(np.linalg.eigvalsh(A))[::-1], rtol=1e-11)
    assert np.all(np.diff(w) <= 0)


@pytest.mark.parametrize("algo", ALGOS)
def test_matches_jacobi_of_gram(oracle_mod, algo):
    """λ_k² are the eigenvalues of XᵀX and the loadings its eigenvectors (Jacobi, written apart)."""
    p = synth.planted(96, 48, 5.0, 0.75, 1e-3, 17)
    X = p.X
    K = 8
    w, W, _ = oracle_mod.jacobi_eigh(X.T @ X, tol=1e-15)
    f = oracle_mod.fit(X, K, tol=1e-14, max_iter=100000, algo=algo)
    np.testing.assert_allclose(f.lam ** 2, w[:K], rtol=1e-9)
    for k in range(K):
        assert angle(f.P[:, k], W[:, k]) < 1e-6


def test_numpy_svd_third_opinion(oracle_mod):
    """GS-PCA at a tight tolerance reproduces numpy's SVD on the 500×200 planted matrix."""
    w = synth.WORKLOADS["planted_500x200"]
    X = w.make()
    f = oracle_mod.fit(X, w.K, tol=1e-13, max_iter=100000, algo="gs")
    U, s, Vt = np.linalg.svd(X, full_matrices=False)
    np.testing.assert_allclose(f.lam, s[: w.K], rtol=1e-9)
    for k in range(w.K):
        assert angle(f.P[:, k], Vt[k]) < 1e-5
        assert angle(f.T[:, k], U[:, k]) < 1e-5


# --------------------------------------------------------------- invariants

@pytest.mark.parametrize("algo", ALGOS)
def test_reconstruction_identity(oracle_mod, algo):
    """Eq. 4: X = T_(K) P_(K)ᵀ + R to rounding, at a loose tolerance too."""
    p = synth.planted(80, 30, 10.0, 0.85, 0.01, 4)
    for tol in (1e-3, 1e-8):
        f = oracle_mod.fit(p.X, 10, tol=tol, max_iter=1000, algo=algo)
        err = np.linalg.norm(p.X - f.T @ f.P.T - f.R) / np.linalg.norm(p.X)
        assert err <= 1e-13


def test_gs_orthogonality(oracle_mod):
    """Sec. 2.3: GS-PCA keeps PᵀP = I and TᵀT = diag(λ²) even at a loose tolerance."""
    X = synth.collinear(200, 40, 1e-3, 9)
    K = 80
    f = oracle_mod.fit(X, K, tol=1e-4, max_iter=200, algo="gs")
    assert np.abs(f.P.T @ f.P - np.eye(K)).max() <= 1e-12
    G = f.T.T @ f.T
    D = np.diag(f.lam ** 2)
    assert np.abs(G - D).max() <= 1e-11 * f.lam[0] ** 2


def test_nipals_loses_orthogonality_gs_does_not(oracle_mod):
    """Sec. 1 / Sec. 2.3: on collinear data NIPALS loadings drift from orthogonality, GS's do not."""
    X = synth.collinear(200, 40, 1e-5, 9)
    K = 80
    fn = oracle_mod.fit(X, K, tol=1e-4, max_iter=200, algo="nipals")
    fg = oracle_mod.fit(X, K, tol=1e-4, max_iter=200, algo="gs")
    on = np.abs(fn.P.T @ fn.P - np.eye(K)).max()
    og = np.abs(fg.P.T @ fg.P - np.eye(K)).max()
    assert og <= 1e-12
    assert on > 1e3 * og


def test_gs_and_nipals_share_first_component(oracle_mod):
    """For k = 0 the Gram-Schmidt terms vanish, so both algorithms take identical steps."""
    w = synth.WORKLOADS["planted_500x200"]
    X = w.make()
    fn = oracle_mod.fit(X, 1, tol=1e-6, max_iter=1000, algo="nipals")
    fg = oracle_mod.fit(X, 1, tol=1e-6, max_iter=1000, algo="gs")
    assert fn.iters[0] == fg.iters[0]
    assert abs(fn.lam[0] - fg.lam[0]) <= 1e-14 * fg.lam[0]
    np.testing.assert_allclose(fn.P[:, 0], fg.P[:, 0], atol=1e-15)
    np.testing.assert_allclose(fn.T[:, 0], fg.T[:, 0], rtol=1e-12, atol=1e-15)


def test_full_spectrum_k_equals_n(oracle_mod):
    """K = N (Sec. 2.3): U is square orthogonal, λ are the singular values, and
    R·U = [V_(j) V_(j)ᵀ X u_j]_j — what is left in R is only the projection of
    X u_j onto the earlier score directions, which vanishes as the iteration converges."""
    p = synth.planted(40, 12, 4.0, 0.7, 0.0, 21)
    X = p.X
    N = X.shape[1]
    f = oracle_mod.fit(X, N, tol=1e-14, max_iter=100000, algo="gs")
    assert f.status == 0
    assert np.abs(f.P.T @ f.P - np.eye(N)).max() <= 1e-12
    np.testing.assert_allclose(f.lam, p.s[:N], rtol=1e-9)
    V = f.T / f.lam
    RU = f.R @ f.P
    for j in range(N):
        Vj = V[:, :j]
        expect = Vj @ (Vj.T @ (X @ f.P[:, j]))
        assert np.linalg.norm(RU[:, j] - expect) <= 1e-12 * np.linalg.norm(X)
    assert np.linalg.norm(f.R) <= 1e-6 * np.linalg.norm(X)


def test_stopping_rule_loading_error(oracle_mod):
    """At tol the loading error against the exact singular vector stays within 3× the
    two-term power-iteration estimate θ ≈ sqrt(2 tol / ((1 − r²)(1 − r⁴))), r = σ_{k+1}/σ_k."""
    p = synth.planted(300, 100, 10.0, 0.85, 0.0, 31)
    tol = 1e-6
    f = oracle_mod.fit(p.X, 5, tol=tol, max_iter=1000, algo="gs")
    r = 0.85
    bound = 3.0 * math.sqrt(2 * tol / ((1 - r * r) * (1 - r ** 4)))
    for k in range(5):
        assert angle(f.P[:, k], p.right[:, k]) <= bound


# ------------------------------------------------------- edge cases / modes

@pytest.mark.parametrize("algo", ALGOS)
def test_iteration_lock_replays_free_run(oracle_mod, algo):
    """Replaying the free run's iteration counts reproduces it bit for bit."""
    w = synth.WORKLOADS["planted_500x200"]
    X = w.make()
    f = oracle_mod.fit(X, 5, tol=1e-6, max_iter=1000, algo=algo)
    g = oracle_mod.fit(X, 5, tol=1e-6, max_iter=1000, algo=algo, iters_lock=f.iters)
    assert np.array_equal(f.iters, g.iters)
    assert np.array_equal(f.lam, g.lam) and np.array_equal(f.P, g.P) and np.array_equal(f.R, g.R)


@pytest.mark.parametrize("algo", ALGOS)
def test_zero_start_column(oracle_mod, algo):
    """A zero column k: the start moves to the largest residual column and σ_1 is still found."""
    p = synth.planted(50, 20, 5.0, 0.6, 0.0, 8)
    X = p.X.copy()
    X[:, 0] = 0.0
    s = np.linalg.svd(X, compute_uv=False)
    f = oracle_mod.fit(X, 3, tol=1e-13, max_iter=100000, algo=algo)
    assert f.status == 0
    np.testing.assert_allclose(f.lam, s[:3], rtol=1e-9)


@pytest.mark.parametrize("algo", ALGOS)
def test_rank_exhausted_is_degenerate(oracle_mod, algo):
    """Rank 3 with K = 5: three components, then the degenerate status and zero tails."""
    p = synth.planted(30, 10, 3.0, 0.7, 0.0, 12)
    g = synth.rng(12, 1)
    A = g.standard_normal((30, 3))
    B = g.standard_normal((3, 10))
    X = A @ B
    f = oracle_mod.fit(X, 5, tol=1e-12, max_iter=10000, algo=algo)
    assert f.status == 5 and f.found == 3
    assert np.all(f.lam[3:] == 0) and np.all(f.P[:, 3:] == 0) and np.all(f.T[:, 3:] == 0)
    np.testing.assert_allclose(f.lam[:3], np.linalg.svd(X, compute_uv=False)[:3], rtol=1e-9)
    del p


@pytest.mark.parametrize("algo", ALGOS)
def test_max_iter_reports_not_converged(oracle_mod, algo):
    w = synth.WORKLOADS["planted_500x200"]
    X = w.make()
    f = oracle_mod.fit(X, 3, tol=1e-12, max_iter=1, algo=algo)
    assert f.status == 4 and np.all(f.iters == 1)


def test_invalid_arguments(oracle_mod):
    X = np.ones((4, 3))
    for K in (0, 4):
        with pytest.raises(ValueError):
            oracle_mod.fit(X, K)
    with pytest.raises(ValueError):
        oracle_mod.fit(X, 1, tol=0.0)
    with pytest.raises(ValueError):
        oracle_mod.fit(X, 1, max_iter=0)


def test_centering_modes(oracle_mod):
    """Mode 1 zeroes every column mean; mode 2 (Eq. 1 as printed) subtracts the mean column,
    which zeroes every row mean."""
    g = synth.rng(2)
    X = g.random((9, 5)) + 3.0
    C1 = oracle_mod.center(X, 1)
    assert np.abs(C1.mean(axis=0)).max() < 1e-15
    np.testing.assert_allclose(C1, X - X.mean(axis=0), atol=1e-15)
    C2 = oracle_mod.center(X, 2)
    assert np.abs(C2.mean(axis=1)).max() < 1e-15
    np.testing.assert_allclose(C2, X - X.mean(axis=1, keepdims=True), atol=1e-15)
    # fit with centring = fit on the centred matrix
    f = oracle_mod.fit(X, 2, tol=1e-10, max_iter=1000, algo="gs", center=1)
    h = oracle_mod.fit(C1, 2, tol=1e-10, max_iter=1000, algo="gs")
    np.testing.assert_allclose(f.lam, h.lam, rtol=1e-14)


# ------------------------------------------------------- bfloat16 storage of R

def _bf16_by_bits(x32: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even float32 -> bfloat16 by integer arithmetic on the bit
    pattern (add 0x7fff plus the lowest kept bit, drop the low 16 bits), widened back."""
    b = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def test_round_bf16_against_bit_rounding_and_library(oracle_mod):
    """oracle.round_bf16 agrees with two independent routes on float32 inputs (a single
    rounding either way): the bit-pattern rule and torch's float32 -> bfloat16 cast; and
    the halfway cases go to the even neighbour."""
    g = synth.rng(31)
    mags = 10.0 ** g.uniform(-42, 38, size=4000)
    x = (np.where(g.random(4000) < 0.5, -1.0, 1.0) * mags).astype(np.float32)
    x = x[np.isfinite(x)]
    got = oracle_mod.round_bf16(x.astype(np.float64))
    fin = np.abs(x.astype(np.float64)) < 3.38e38  # the bit rule does not saturate to inf
    np.testing.assert_array_equal(got[fin], _bf16_by_bits(x[fin]))
    torch = pytest.importorskip("torch")
    lib = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(got, lib)
    ties = oracle_mod.round_bf16(np.array([1 + 2.0**-8, 1 + 3 * 2.0**-8, -(1 + 2.0**-8), 2.0**-133 * 1.5,
                                           2.0**-133 * 2.5, 0.0, 3.0]))
    np.testing.assert_array_equal(ties, [1.0, 1 + 2.0**-6, -1.0, 2.0**-132, 2.0**-132, 0.0, 3.0])
    big = oracle_mod.round_bf16(np.array([3.3961e38, 3.3962e38]))  # (2 - 2^-8) 2^127 = 3.39615e38
    assert big[0] == float.fromhex("0x1.fep127") and np.isinf(big[1])


@pytest.mark.parametrize("algo", ALGOS)
def test_bf16_storage_rounds_every_residual(oracle_mod, algo):
    """storage="bf16": the returned residual is made of bfloat16 values, and Eq. 4 holds up
    to the rounding of the K deflations (each moves an entry by at most half a bfloat16
    spacing, 2^-9 of its magnitude) but no better than a single rounding would allow."""
    X = synth.planted(90, 50, 10.0, 0.85, 0.01, 44).X
    K = 5
    f = oracle_mod.fit(X, K, tol=1e-12, max_iter=5000, algo=algo, storage="bf16")
    assert f.found == K
    np.testing.assert_array_equal(oracle_mod.round_bf16(f.R), f.R)
    Xb = oracle_mod.round_bf16(X)
    err = np.linalg.norm(Xb - f.T @ f.P.T - f.R)
    assert err <= K * 2.0**-9 * np.linalg.norm(Xb)
    assert err >= 1e-5 * np.linalg.norm(f.R)
    # the FP64 run on the same rounded input keeps Eq. 4 to rounding level: the gap is the storage
    f64 = oracle_mod.fit(Xb, K, tol=1e-12, max_iter=5000, algo=algo)
    assert np.linalg.norm(Xb - f64.T @ f64.P.T - f64.R) <= 1e-12 * np.linalg.norm(Xb)


@pytest.mark.parametrize("algo", ALGOS)
def test_bf16_storage_singular_values_within_weyl_bound(oracle_mod, algo):
    """Rounding the residual after deflation j perturbs it by E_j with ||E_j||_2 <= ||E_j||_F
    <= 2^-9 ||R_j||_F; by Weyl's inequality each singular value of the later residuals moves
    by at most the sum of those, so converged lambdas of the bf16-storage run stay that close
    to the FP64 run on the same rounded X (and do move: the rounding is applied)."""
    X = synth.planted(120, 60, 10.0, 0.8, 0.01, 45).X
    Xb = oracle_mod.round_bf16(X)
    K = 6
    fb = oracle_mod.fit(Xb, K, tol=1e-13, max_iter=20000, algo=algo, storage="bf16")
    f64 = oracle_mod.fit(Xb, K, tol=1e-13, max_iter=20000, algo=algo)
    bound = 0.0
    moved = 0.0
    for k in range(K):
        # ||R_k||_F^2 = ||X||_F^2 - sum_{j<k} lambda_j^2 for the FP64 run (exact deflation of
        # converged singular pairs); the bf16 bound uses its square root at every step
        bound += 2.0**-9 * math.sqrt(max(0.0, np.sum(Xb**2) - np.sum(f64.lam[:k] ** 2)))
        if k > 0:
            assert abs(fb.lam[k] - f64.lam[k]) <= 1.5 * bound, (k, fb.lam[k], f64.lam[k], bound)
        moved = max(moved, abs(fb.lam[k] - f64.lam[k]) / f64.lam[k])
    assert abs(fb.lam[0] - f64.lam[0]) <= 1e-10 * f64.lam[0]  # component 0 sees no deflation
    assert moved > 1e-9


@pytest.mark.parametrize("flavor", ["O3", "O2-omp", "O3-omp"])
@pytest.mark.parametrize("algo", ["gs", "nipals"])
def test_timing_builds_give_the_checkers_bits(oracle_mod, flavor, algo):
    """The builds that only time the oracle on the host (-O3, OpenMP) return the
    single-threaded -O2 checker's results bit for bit: their parallel loops split over
    independent outputs, every sum keeps its index order, and -ffp-contract=off keeps
    one rounding per operation.  Shapes span several row blocks and parallel columns."""
    X = synth.planted(1300, 150, 5.0, 0.85, 0.01, (7, 1300)).X
    a = oracle_mod.fit(X, 6, algo=algo, gs_passes=1)
    b = oracle_mod.fit(X, 6, algo=algo, gs_passes=1, flavor=flavor)
    for key in ("T", "P", "lam", "iters", "R"):
        assert np.array_equal(getattr(a, key), getattr(b, key)), key
