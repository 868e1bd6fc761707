"""The algebra behind the two-reduction Gram-Schmidt step, checked in FP64 numpy
on the GS-PCA iteration of Sec. 2.3 (no oracle or CUDA code involved).

With W = R_k^T V (kept by the rank-1 updates the deflation implies, Eq. 3),
Q = R_k U, Z = U^T W and GV = V^T V, every GS-PCA iteration's
  a'            = U^T (s' - W b')           equals c' - Z b' with c' = Q^T v', and
  ||v' - V b'||^2                           equals ||v'||^2 - 2 b'.b' + b'^T GV b',
and Q, Z, GV follow each deflation by the updates the kernel applies at a
component start:
  Q(:, i<k-1) -= lam v_{k-1} h_i,  Q(:, k-1) = R_{k-1} u_{k-1} - lam v_{k-1} (u.u),
  Z(i<k-1, j<k-1) -= lam h_i g_j,  Z(i, k-1) = vinv a'_last,i - lam h_i g_{k-1},
  Z(k-1, j) = r_j - lam (u.u) g_j, Z(k-1, k-1) = vinv (u.u_pre) - lam (u.u) g_{k-1},
with h = U_old^T u_{k-1}, r = W_old^T u_{k-1}, g the Gram row V^T v_{k-1}, and
R_{k-1} u_{k-1} the last pass's v' / ||u'||.

The first test runs the iteration: there U and V are orthonormal to FP64
rounding, so terms carrying u_i.u_{k-1} or v_i.v_{k-1} (i < k-1) vanish and it
pins the dominant terms, signs and indices.  The second applies the same updates
to random, non-orthogonal factors, where every term counts: a dropped or
mis-indexed term makes the maintained matrices drift from their definitions.
"""
import numpy as np

import synth


def test_maintained_matrices_and_formulas_match_their_definitions():
    X = synth.planted(300, 90, 10.0, 0.8, 0.01, 21).X.astype(np.float64)
    M, N = X.shape
    K, tol = 6, 1e-10
    R = X.copy()
    V = np.zeros((M, K)); U = np.zeros((N, K)); W = np.zeros((N, K))
    Q = np.zeros((M, K)); Z = np.zeros((K, K)); GV = np.zeros((K, K))
    lam_prev = vinv_prev = inv_nu = 0.0
    vraw_last = upre_last = None
    a_last = np.zeros(K)
    checked = 0
    for k in range(K):
        if k > 0:
            km, lam = k - 1, lam_prev
            v, u = V[:, km], U[:, km]
            g = V[:, :k].T @ v
            h = U[:, :k].T @ u                      # h[km] = u.u
            r = W[:, :km].T @ u
            s1, s2 = u @ upre_last, h[km]
            Zn = np.zeros((K, K))
            Zn[:km, :km] = Z[:km, :km] - lam * np.outer(h[:km], g[:km])
            Zn[:km, km] = vinv_prev * a_last[:km] - lam * h[:km] * g[km]
            Zn[km, :km] = r - lam * s2 * g[:km]
            Zn[km, km] = vinv_prev * s1 - lam * s2 * g[km]
            Z = Zn
            GV[km, :k] = g
            GV[:k, km] = g
            Q[:, :km] -= lam * np.outer(v, h[:km])
            Q[:, km] = vraw_last * inv_nu - lam * v * s2
            W[:, :km] -= lam * np.outer(u, g[:km])
            W[:, km] = upre_last * vinv_prev - lam * u * g[km]
            R = R - lam * np.outer(v, u)              # Eq. 3
            np.testing.assert_allclose(W[:, :k], R.T @ V[:, :k], atol=1e-10 * lam)
            np.testing.assert_allclose(Q[:, :k], R @ U[:, :k], atol=1e-10 * lam)
            np.testing.assert_allclose(Z[:k, :k], U[:, :k].T @ W[:, :k], atol=1e-10 * lam)
            np.testing.assert_allclose(GV[:k, :k], V[:, :k].T @ V[:, :k], atol=1e-12)
        # Sec. 2.3 iteration, in the kernel's pass scale
        x = R[:, k].copy()
        s0 = R.T @ x
        a = U[:, :k].T @ s0
        ut = (s0 - U[:, :k] @ a) / (x @ x)
        mu = 0.0
        for j in range(1000):
            nu2 = ut @ ut
            vp = R @ ut
            sp = R.T @ vp
            b = V[:, :k].T @ vp
            vc = vp - V[:, :k] @ b
            up = sp - W[:, :k] @ b
            a_direct = U[:, :k].T @ up
            if k > 0:
                c = Q[:, :k].T @ vp
                np.testing.assert_allclose(c - Z[:k, :k] @ b, a_direct, atol=1e-10 * np.abs(sp).max())
                l2 = vp @ vp - 2 * b @ b + b @ GV[:k, :k] @ b
                assert abs(l2 - vc @ vc) <= 1e-10 * (vp @ vp)
                checked += 1
            l2 = vc @ vc
            lam = np.sqrt(l2 / nu2)
            if abs(mu - lam) < tol * lam:
                vinv = 1.0 / np.sqrt(l2)
                inv_nu = 1.0 / np.sqrt(nu2)
                V[:, k] = vc * vinv
                U[:, k] = ut * inv_nu
                lam_prev, vinv_prev = lam, vinv
                vraw_last, upre_last = vp, up
                a_last = np.zeros(K)
                a_last[:k] = a_direct
                break
            mu = lam
            ut = (up - U[:, :k] @ a_direct) * (np.sqrt(nu2) / l2)
    assert checked > 50
    s = np.linalg.svd(X, compute_uv=False)
    np.testing.assert_allclose([np.linalg.norm(V[:, i]) for i in range(K)], 1.0, rtol=1e-12)
    assert lam_prev > 0 and abs(lam_prev - s[K - 1]) <= 1e-6 * s[0]


def _updates(Rp, Uo, Vo, Wo, Qo, Zo, Go, u, v, lam, Rt_v, R_u):
    """The component-start updates (as the kernel applies them) for the deflation
    R = Rp - lam v u^T, given R_{k-1}^T v (= u_pre vinv) and R_{k-1} u (= v' / ||u'||)."""
    km = Uo.shape[1]
    k = km + 1
    h = np.concatenate([Uo.T @ u, [u @ u]])
    r = Wo.T @ u
    g = np.concatenate([Vo.T @ v, [v @ v]])
    a_vinv = Uo.T @ Rt_v                  # vinv a'_last
    s1_vinv = u @ Rt_v                    # vinv (u . u_pre)
    s2 = h[km]
    W = np.zeros((Rp.shape[1], k)); Q = np.zeros((Rp.shape[0], k)); Z = np.zeros((k, k)); G = np.zeros((k, k))
    W[:, :km] = Wo - lam * np.outer(u, g[:km])
    W[:, km] = Rt_v - lam * u * g[km]
    Q[:, :km] = Qo - lam * np.outer(v, h[:km])
    Q[:, km] = R_u - lam * v * s2
    Z[:km, :km] = Zo - lam * np.outer(h[:km], g[:km])
    Z[:km, km] = a_vinv - lam * h[:km] * g[km]
    Z[km, :km] = r - lam * s2 * g[:km]
    Z[km, km] = s1_vinv - lam * s2 * g[km]
    G[:km, :km] = Go
    G[km, :] = g
    G[:, km] = g
    return W, Q, Z, G


def test_component_start_updates_are_exact_for_any_factors():
    rng = synth.rng(99, 1)
    for M, N, km in [(40, 30, 1), (60, 25, 4), (33, 70, 7)]:
        Rp = rng.standard_normal((M, N))
        Uo, Vo = rng.standard_normal((N, km)), rng.standard_normal((M, km))
        u, v = rng.standard_normal(N), rng.standard_normal(M)
        lam = 1.7
        Wo, Qo = Rp.T @ Vo, Rp @ Uo
        W, Q, Z, G = _updates(Rp, Uo, Vo, Wo, Qo, Uo.T @ Wo, Vo.T @ Vo, u, v, lam, Rp.T @ v, Rp @ u)
        R = Rp - lam * np.outer(v, u)         # Eq. 3
        U, V = np.column_stack([Uo, u]), np.column_stack([Vo, v])
        np.testing.assert_allclose(W, R.T @ V, atol=1e-12 * np.abs(R.T @ V).max())
        np.testing.assert_allclose(Q, R @ U, atol=1e-12 * np.abs(R @ U).max())
        np.testing.assert_allclose(Z, U.T @ (R.T @ V), atol=1e-12 * np.abs(Z).max())
        np.testing.assert_allclose(G, V.T @ V, atol=1e-12 * np.abs(G).max())
        # and the two formulas of the iteration, for any v' and b' = V^T v'
        vp = R @ rng.standard_normal(N)
        b = V.T @ vp
        np.testing.assert_allclose(Q.T @ vp - Z @ b, U.T @ (R.T @ vp - W @ b), atol=1e-10 * np.abs(Q.T @ vp).max())
        lhs = vp @ vp - 2 * b @ b + b @ G @ b
        assert abs(lhs - np.sum((vp - V @ b) ** 2)) <= 1e-10 * (vp @ vp + b @ G @ b)


def _fp32_run(X, K, tol, ratio_guard):
    """GS-PCA in FP32 (numpy) with the two-reduction step as the kernel takes it:
    Q, Z, GV maintained through the deflations (which round in FP32 and are not
    tracked), the step taken when b'.b' <= ||v'||^2 / 4 and lambda_0 <= guard mu."""
    f32 = np.float32
    R = X.astype(f32)
    M, N = R.shape
    V = np.zeros((M, K), f32); U = np.zeros((N, K), f32); W = np.zeros((N, K), f32)
    Q = np.zeros((M, K), f32); Z = np.zeros((K, K), f32); G = np.zeros((K, K), f32)
    lams, a_last = [], np.zeros(K, f32)
    vinv_prev = inv_nu = f32(0)
    vraw_last = upre_last = None
    for k in range(K):
        if k > 0:
            km, lam = k - 1, f32(lams[-1])
            v, u = V[:, km], U[:, km]
            g = V[:, :k].T @ v
            h = U[:, :k].T @ u
            r = W[:, :km].T @ u
            s1, s2 = f32(u @ upre_last), h[km]
            Zn = np.zeros((K, K), f32)
            Zn[:km, :km] = Z[:km, :km] - lam * np.outer(h[:km], g[:km])
            Zn[:km, km] = vinv_prev * a_last[:km] - lam * h[:km] * g[km]
            Zn[km, :km] = r - lam * s2 * g[:km]
            Zn[km, km] = vinv_prev * s1 - lam * s2 * g[km]
            Z = Zn
            G[km, :k] = g
            G[:k, km] = g
            Q[:, :km] -= lam * np.outer(v, h[:km])
            Q[:, km] = vraw_last * inv_nu - lam * v * s2
            W[:, :km] -= lam * np.outer(u, g[:km])
            W[:, km] = upre_last * vinv_prev - lam * u * g[km]
            R = (R - lam * np.outer(v, u)).astype(f32)
        x = R[:, k].copy()
        s0 = R.T @ x
        a = U[:, :k].T @ s0
        ut = ((s0 - U[:, :k] @ a) / (x @ x)).astype(f32)
        mu = 0.0
        for j in range(5000):
            nu2 = float(ut @ ut)
            vp = R @ ut
            sp = R.T @ vp
            b = V[:, :k].T @ vp
            up = sp - W[:, :k] @ b
            bb, vv = float(b @ b), float(vp @ vp)
            vc = vp - V[:, :k] @ b
            if k > 0 and mu > 0 and lams[0] <= ratio_guard * mu and 4 * bb <= vv:
                a_ = Q[:, :k].T @ vp - Z[:k, :k] @ b
                l2 = vv - 2 * bb + float(b @ G[:k, :k] @ b)
            else:
                a_ = U[:, :k].T @ up
                l2 = float(vc @ vc)
            lam = np.sqrt(l2 / nu2)
            if abs(mu - lam) < tol * lam or j == 4999:
                vinv_prev, inv_nu = f32(1 / np.sqrt(l2)), f32(1 / np.sqrt(nu2))
                V[:, k], U[:, k] = vc * vinv_prev, ut * inv_nu
                lams.append(lam)
                vraw_last, upre_last = vp, up
                a_last = np.zeros(K, f32)
                a_last[:k] = a_
                break
            mu = lam
            ut = ((up - U[:, :k] @ a_) * f32(np.sqrt(nu2) / l2)).astype(f32)
    return np.array(lams), U


def test_fp32_model_needs_the_range_guard():
    """In FP32, Q and Z miss the rounding of each deflation; relative to lambda_k that error
    grows with lambda_0 / lambda_k.  On a spectrum spanning ~5000x the step without the
    range guard lets the loadings drift from orthogonality, with the kernel's guard
    (lambda_0 <= 64 mu) they stay at FP32 rounding, and the singular values agree."""
    X = synth.planted(800, 300, 10.0, 0.9, 0.0001, 9).X
    K = 80
    lam_g, U_g = _fp32_run(X, K, 1e-6, 64.0)
    lam_n, U_n = _fp32_run(X, K, 1e-6, np.inf)
    ortho_g = np.abs(U_g.T.astype(np.float64) @ U_g - np.eye(K)).max()
    ortho_n = np.abs(U_n.T.astype(np.float64) @ U_n - np.eye(K)).max()
    assert ortho_g <= 2e-6
    assert ortho_n >= 4 * ortho_g
    s = np.linalg.svd(X, compute_uv=False)
    assert np.abs(lam_g - s[:K]).max() <= 1e-5 * s[0]
