"""Learned warm start on the GPU (through the C ABI) against the FP64 oracle
(oracle/warmstart.c), and what the trained network gains.

Bars (FP32 kernels vs FP64 oracle): features 1e-4 absolute (they are O(1)); network
output 1e-5 relative to its scale; loss 1e-5; gradient 1e-4 relative in norm; the fit
with the learned start iteration-locked against the oracle with the same network: the
FP32 fit bars (singular value 1e-4, angles 1e-3 rad, GS orthogonality 1e-5), and the
same choice of start wherever the oracle's two Rayleigh quotients differ by more than
1e-3 relatively (closer than that, both starts are equally valid and FP32 may pick
either).
"""
import math

import numpy as np
import pytest

import oracle
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


def cuda(a, dtype=None):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype or np.float32)).cuda()


def col_major(X32):
    import torch

    return torch.from_numpy(np.ascontiguousarray(X32.T)).cuda().t()


def angle(a, b):
    na, nb = np.linalg.norm(a), np.linalg.norm(b)
    if na == 0 or nb == 0:
        return 0.0 if na == nb else math.pi / 2
    return math.acos(min(1.0, abs(float(a @ b)) / (na * nb)))


def sketch(M, seed=71):
    return (synth.rng(seed, M).standard_normal((M, 16)) / 4.0).astype(np.float32)


def random_net(seed, scale=0.3):
    return (scale * synth.rng(seed).standard_normal(oracle.ws_nparams())).astype(np.float32)


@pytest.mark.parametrize("k", [0, 3])
def test_features_match_oracle(gp, k):
    X = synth.planted(300, 97, 10.0, 0.8, 0.01, 72).X.astype(np.float32)
    ref = oracle.fit(X.astype(np.float64), 4, tol=1e-10, max_iter=5000, algo="gs")
    T32, P32 = ref.T.astype(np.float32), ref.P.astype(np.float32)
    G = sketch(300)
    Rk = X.astype(np.float64) - T32[:, :k].astype(np.float64) @ P32[:, :k].astype(np.float64).T
    want = oracle.ws_features(Rk, G.astype(np.float64))
    import torch

    Tt = torch.from_numpy(np.ascontiguousarray(T32.T)).cuda().t()
    Pt = torch.from_numpy(np.ascontiguousarray(P32.T)).cuda().t()
    got = gp.gspca_ws_features(col_major(X), cuda(G), Tt, Pt, k).cpu().numpy()
    np.testing.assert_allclose(got, want, atol=1e-4, rtol=0)


def test_forward_matches_oracle(gp):
    feat = synth.rng(73).standard_normal((777, 17)).astype(np.float32)
    net = random_net(74)
    want = oracle.ws_forward(net.astype(np.float64), feat.astype(np.float64))
    got = gp.gspca_ws_forward(cuda(net), cuda(feat)).cpu().numpy()
    np.testing.assert_allclose(got, want, atol=1e-5 * np.abs(want).max(), rtol=0)


def _instances(seed, sizes):
    g = synth.rng(seed)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    feat = g.standard_normal((offs[-1], 17)).astype(np.float32)
    tgt = np.zeros(offs[-1], dtype=np.float32)
    for i in range(len(sizes)):
        t = g.standard_normal(sizes[i])
        tgt[offs[i]:offs[i + 1]] = t / np.linalg.norm(t)
    return feat, tgt, offs


def test_loss_gradient_and_adam_match_oracle(gp):
    import torch

    feat, tgt, offs = _instances(75, [300, 64, 1024, 5, 2500])  # one instance spans two gradient blocks
    net = random_net(76)
    L, gref = oracle.ws_loss_grad(net.astype(np.float64), feat.astype(np.float64), tgt.astype(np.float64), offs)
    with gp.Handle(8, 8, 1) as h:
        dnet = cuda(net)
        loss = torch.zeros(1, device="cuda")
        grad = torch.zeros(oracle.ws_nparams(), device="cuda")
        gp.gspca_ws_train_step(h.h, dnet, None, None, 1, 0.0, cuda(feat), cuda(tgt), cuda(offs, np.int32),
                               loss=loss, grad=grad)
        torch.cuda.synchronize()
        assert abs(loss.item() - L) <= 1e-5
        g = grad.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(g - gref) <= 1e-4 * np.linalg.norm(gref)
        assert np.array_equal(dnet.cpu().numpy(), net)  # lr = 0: no update
        # one Adam step from zero moments: theta - lr g / (|g| + eps) per parameter
        m = torch.zeros_like(dnet)
        v = torch.zeros_like(dnet)
        gp.gspca_ws_train_step(h.h, dnet, m, v, 1, 1e-3, cuda(feat), cuda(tgt), cuda(offs, np.int32))
        torch.cuda.synchronize()
        new = dnet.cpu().numpy().astype(np.float64)
    want = net.astype(np.float64).copy()
    oracle.ws_adam(want, np.zeros_like(want), np.zeros_like(want), gref, 1, lr=1e-3)
    big = np.abs(gref) > 1e-2 * np.sqrt(np.mean(gref**2))
    assert np.abs(new - want)[big].max() <= 1e-6 + 1e-5 * np.abs(want)[big].max()
    assert np.abs(new - want).max() <= 2e-3 + 1e-6 * np.abs(want).max()


def run_warm(gp, X32, K, net, G, tol=1e-6, max_iter=1000, lock=None):
    import torch

    M, N = X32.shape
    with gp.Handle(M, N, K) as h:
        w = gp.WarmStart(cuda(net), cuda(G))
        r = h.fit(torch.from_numpy(X32).cuda(), K, tol=tol, max_iter=max_iter, algo="gs", warm=w,
                  iters_lock=lock, want_R=True)
        torch.cuda.synchronize()
        return dict(T=r.T.cpu().numpy().astype(np.float64), P=r.P.cpu().numpy().astype(np.float64),
                    lam=r.lam.cpu().numpy(), iters=r.iters.cpu().numpy(), status=r.status,
                    choice=r.ws_choice.cpu().numpy(), R=r.R.cpu().numpy().astype(np.float64))


def check_warm_locked(g, X32, K, net, G):
    ref = oracle.fit(X32.astype(np.float64), K, tol=1e-6, max_iter=1000, algo="gs",
                     iters_lock=np.maximum(g["iters"], 1), ws_net=net.astype(np.float64), ws_G=G.astype(np.float64))
    for k in range(ref.found):
        ra, rb = ref.ws_rho[k]
        if abs(rb - ra) > 1e-3 * max(abs(ra), abs(rb)):
            assert g["choice"][k] == ref.ws_choice[k], (k, ra, rb, g["choice"])
        if g["choice"][k] != ref.ws_choice[k]:
            continue  # a near tie: the two sides follow different (equally valid) trajectories
        assert abs(g["lam"][k] - ref.lam[k]) <= 1e-4 * ref.lam[k], (k, g["lam"][k], ref.lam[k])
        assert angle(g["P"][:, k], ref.P[:, k]) <= 1e-3, (k, angle(g["P"][:, k], ref.P[:, k]))
        assert angle(g["T"][:, k], ref.T[:, k]) <= 1e-3, k
    P = g["P"][:, :ref.found]
    assert np.abs(P.T @ P - np.eye(ref.found)).max() <= 1e-5
    return ref


@pytest.mark.parametrize("shape", [(500, 200, 8), (257, 31, 6), (1003, 517, 5), (130, 1025, 4), (64, 2048, 3)])
def test_fit_with_learned_start_locked(gp, shape):
    M, N, K = shape
    X32 = synth.planted(M, N, 10.0, 0.85, 0.01, (77, M, N)).X.astype(np.float32)
    G = sketch(M)
    net = random_net(78)
    g = run_warm(gp, X32, K, net, G)
    assert g["status"] == 0
    ref = check_warm_locked(g, X32, K, net, G)
    assert 0 < ref.ws_choice.sum() or shape != (500, 200, 8)  # the candidate wins somewhere here


def test_zero_network_is_the_papers_fit_bit_for_bit(gp):
    """With w == 0 the warm-start machinery runs but never offers a candidate: the fit is
    bit-identical to the plain one (with the same, three-reduction Gram-Schmidt step)."""
    import torch

    X32 = synth.planted(600, 250, 10.0, 0.85, 0.01, 79).X.astype(np.float32)
    g = run_warm(gp, X32, 6, np.zeros(oracle.ws_nparams(), np.float32), sketch(600))
    with gp.Handle(600, 250, 6) as h:
        r = h.fit(torch.from_numpy(X32).cuda(), 6, algo="gs", want_R=True, gs_step=1)
        torch.cuda.synchronize()
        assert not g["choice"].any()
        assert np.array_equal(g["P"], r.P.cpu().numpy().astype(np.float64))
        assert np.array_equal(g["lam"], r.lam.cpu().numpy())
        assert np.array_equal(g["R"], r.R.cpu().numpy().astype(np.float64))


def test_batched_with_learned_start_locked(gp):
    import torch

    shapes = [(300, 64, 6), (257, 513, 5), (1001, 1000, 4), (640, 201, 8), (96, 700, 3)]
    probs = [(synth.batch_problem(i, M, N, seed=80).X.astype(np.float32), K) for i, (M, N, K) in enumerate(shapes)]
    G = sketch(1024)
    net = random_net(81)
    with gp.Handle(1024, 1024, 8) as h:
        b = gp.Batch([{"X": col_major(X), "K": K} for X, K in probs])
        _, st = gp.gspca_fit_batched(h.h, b, tol=1e-6, max_iter=1000, algo="gs",
                                     warm=gp.WarmStart(cuda(net), cuda(G)))
        torch.cuda.synchronize()
        assert st in (gp.GSPCA_OK, gp.GSPCA_WARN_NOT_CONVERGED)
        outs = [dict(T=r.T.cpu().numpy().astype(np.float64), P=r.P.cpu().numpy().astype(np.float64),
                     lam=r.lam.cpu().numpy(), iters=r.iters.cpu().numpy(), choice=r.ws_choice.cpu().numpy())
                for r in b.results]
    for (X, K), g in zip(probs, outs):
        check_warm_locked(g, X, K, net, G[:X.shape[0]])


def test_warm_start_refusals(gp):
    """NIPALS-PCA has no learned start; the learned start is compiled for up to 2048 columns."""
    import torch

    warm = gp.WarmStart(cuda(np.zeros(oracle.ws_nparams(), np.float32)), cuda(sketch(20)))
    with gp.Handle(20, 3000, 2) as h:
        r = gp.gspca_fit(h.h, torch.zeros((20, 10), device="cuda"), 2, algo="nipals", check=False, warm=warm)
        assert r.status == gp.GSPCA_ERR_NOT_SUPPORTED
        r = gp.gspca_fit(h.h, torch.zeros((20, 2049), device="cuda"), 2, algo="gs", check=False, warm=warm)
        assert r.status == gp.GSPCA_ERR_NOT_SUPPORTED


def test_trained_network_saves_iterations(gp):
    """Train on the GPU (the library's kernels) on converged loadings of problems from the
    batched generator, then fit held-out problems of the same distribution: the learned
    start, with its fallback to the paper's start, needs fewer iterations in total."""
    import torch

    from paper_0811_1081_gb300 import warmstart as ws

    K = 8
    def problems(seed, count):
        shapes = synth.batch_shapes(count, seed=seed, m_range=(256, 2048), n_range=(64, 512))
        return [col_major(synth.batch_problem(i, M, N, seed=seed).X.astype(np.float32))
                for i, (M, N) in enumerate(shapes)]
    G = cuda(sketch(2048, seed=82))
    train_x, test_x = problems(5, 96), problems(6, 48)
    with gp.Handle(2048, 512, K) as h:
        ts = ws.make_training_set(h.h, train_x, K, G)
        net = cuda(ws.init_params(synth.rng(83)))
        l0 = ws.mean_loss(h.h, net, ts)
        hist = ws.train(h.h, net, ts, epochs=25, per_batch=32, lr=2e-3, rng=synth.rng(84))
        assert hist[-1] < l0 - 0.02, (l0, hist)
        plain = gp.Batch([{"X": X, "K": K} for X in test_x])
        learned = gp.Batch([{"X": X, "K": K} for X in test_x])
        gp.gspca_fit_batched(h.h, plain, algo="gs")
        gp.gspca_fit_batched(h.h, learned, algo="gs", warm=gp.WarmStart(net, G))
        torch.cuda.synchronize()
        it_plain = sum(int(r.iters.sum().item()) for r in plain.results)
        it_learned = sum(int(r.iters.sum().item()) for r in learned.results)
        used = sum(int(r.ws_choice.sum().item()) for r in learned.results)
        # same components found: the start changes the path, not the answer
        for a, b in zip(plain.results, learned.results):
            np.testing.assert_allclose(b.lam.cpu().numpy(), a.lam.cpu().numpy(), rtol=1e-3)
    print(f"iterations plain {it_plain}, learned {it_learned} ({it_learned / it_plain:.3f}); "
          f"learned start used for {used} of {len(test_x) * K} components; loss {l0:.3f} -> {hist[-1]:.3f}")
    assert it_learned < it_plain
