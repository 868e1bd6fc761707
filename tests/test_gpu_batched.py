"""Batched form (many independent problems per persistent launch) vs the FP64
oracle and vs the single-problem form, through the C ABI.

Every problem of a batch is checked in Mode L: the oracle replays that
problem's GPU iteration counts on the same FP32-rounded X.  Bars as for the
single-problem form (FP32 storage): singular value 1e-4 relative, loading
and score angle 1e-3 rad, GS ||P^T P - I||_max 1e-5.
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

# (M, N, K): ragged M, both column classes (N <= 512 and N > 512), K = 1,
# K = N (M = N + 1: a column-centred X has rank <= M - 1), rows fewer than
# 4 x team size (CTAs without panels), N = 1024.
SHAPES = [(5, 3, 3), (37, 61, 4), (300, 64, 6), (257, 513, 5), (1001, 1024, 4), (640, 200, 8),
          (96, 700, 1), (13, 12, 12), (2048, 130, 6), (413, 999, 3)]


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


def make_problems(shapes, seed=3):
    out = []
    for i, (M, N, K) in enumerate(shapes):
        X = synth.batch_problem(i, M, N, seed=seed).X.astype(np.float32)
        out.append((X, K))
    return out


def to_batch(gp, probs, col_major=True):
    import torch

    lst = []
    for X, K in probs:
        t = torch.from_numpy(X).cuda()
        if col_major:
            t = t.t().contiguous().t()
        lst.append({"X": t, "K": K})
    return gp.Batch(lst)


def results(b):
    import torch

    torch.cuda.synchronize()
    out = []
    for r in b.results:
        out.append(dict(T=r.T.cpu().numpy().astype(np.float64), P=r.P.cpu().numpy().astype(np.float64),
                        lam=r.lam.cpu().numpy(), iters=r.iters.cpu().numpy(), status=int(r.status.item())))
    return out


def check_locked(g, X32, K, algo, tol=1e-6, max_iter=1000):
    ref = oracle.fit(X32.astype(np.float64), K, tol=tol, max_iter=max_iter, algo=algo,
                     iters_lock=np.maximum(g["iters"], 1))
    found = ref.found
    for k in range(found):
        assert abs(g["lam"][k] - ref.lam[k]) <= SIG_REL * ref.lam[k], (k, g["lam"][k], ref.lam[k])
        assert angle(g["P"][:, k], ref.P[:, k]) <= ANGLE, (k, angle(g["P"][:, k], ref.P[:, k]))
        assert angle(g["T"][:, k], ref.T[:, k]) <= ANGLE, k
        tn, rn = np.linalg.norm(g["T"][:, k]), np.linalg.norm(ref.T[:, k])
        assert abs(tn - rn) <= SIG_REL * rn, k
    if algo == "gs" and found > 0:
        P = g["P"][:, :found]
        assert np.abs(P.T @ P - np.eye(found)).max() <= ORTHO
    return ref


@pytest.mark.parametrize("team", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("bpass", [1, 2])
def test_batched_locked_parity_gs(gp, team, bpass):
    """Both loading passes (independent warp groups; CTA-wide rounds through the TMA
    ring) at every team size."""
    probs = make_problems(SHAPES)
    with gp.Handle(2048, 1024, 16) as h:
        b = to_batch(gp, probs)
        try:
            _, st = gp.gspca_fit_batched(h.h, b, tol=1e-6, max_iter=1000, algo="gs", cluster_ctas=team,
                                         batch_pass=bpass)
        except gp.GspcaError as e:
            if team == 16:
                pytest.skip(f"team of 16 CTAs not launchable here: {e}")
            raise
        info = h.info()
        assert info["team_ctas"] == team and info["batch_pass"] == bpass
        outs = results(b)
        assert st in (gp.GSPCA_OK, gp.GSPCA_WARN_NOT_CONVERGED), [(s, g["status"]) for s, g in zip(SHAPES, outs)]
    for (X, K), g in zip(probs, outs):
        assert g["status"] in (0, 4)
        check_locked(g, X, K, "gs")


@pytest.mark.parametrize("bpass", [1, 2])
def test_batched_locked_parity_nipals(gp, bpass):
    probs = make_problems(SHAPES)
    with gp.Handle(2048, 1024, 16) as h:
        b = to_batch(gp, probs)
        gp.gspca_fit_batched(h.h, b, algo="nipals", cluster_ctas=4, batch_pass=bpass)
        outs = results(b)
    for (X, K), g in zip(probs, outs):
        check_locked(g, X, K, "nipals")


def test_batched_matches_single_problem_form(gp):
    """Same problems through gspca_fit one at a time: same lambda to FP32 rounding."""
    probs = make_problems(SHAPES[:6])
    with gp.Handle(2048, 1024, 16) as h:
        b = to_batch(gp, probs)
        gp.gspca_fit_batched(h.h, b, cluster_ctas=2)
        outs = results(b)
        import torch

        for (X, K), g in zip(probs, outs):
            r = h.fit(torch.from_numpy(X).cuda(), K, iters_lock=[int(v) for v in np.maximum(g["iters"], 1)])
            lam = r.lam.cpu().numpy()
            assert np.all(np.abs(lam - g["lam"]) <= SIG_REL * lam)
            P = r.P.cpu().numpy().astype(np.float64)
            for k in range(K):
                assert angle(P[:, k], g["P"][:, k]) <= ANGLE


def test_batched_zero_problem_and_zero_start_column(gp):
    """A zero X reports GSPCA_ERR_DEGENERATE with zero outputs; a zero first
    column restarts from the largest residual column; the others are unaffected."""
    probs = make_problems([(300, 64, 4), (200, 100, 3), (150, 90, 5)])
    probs[1] = (np.zeros((200, 100), np.float32), 3)
    X2 = probs[2][0].copy()
    X2[:, 0] = 0.0
    probs[2] = (X2, 5)
    with gp.Handle(512, 512, 8) as h:
        b = to_batch(gp, probs)
        _, st = gp.gspca_fit_batched(h.h, b, cluster_ctas=2)
        outs = results(b)
    assert st == gp.GSPCA_ERR_DEGENERATE
    assert outs[1]["status"] == gp.GSPCA_ERR_DEGENERATE
    assert not outs[1]["T"].any() and not outs[1]["P"].any() and not outs[1]["lam"].any()
    assert outs[0]["status"] == 0 and outs[2]["status"] == 0
    check_locked(outs[0], probs[0][0], 4, "gs")
    check_locked(outs[2], X2, 5, "gs")


def test_batched_autotune_then_graph_replay(gp):
    """Uncaptured call picks the team size; a CUDA graph captured from the async form
    replays it and reproduces the uncaptured outputs bit for bit (same team size,
    fixed-order reductions)."""
    import torch

    shapes = [(int(M), int(N), 4) for M, N in synth.batch_shapes(24, seed=9, m_range=(64, 1500),
                                                                   n_range=(16, 900))]
    probs = make_problems(shapes, seed=9)
    with gp.Handle(1500, 1024, 8) as h:
        b = to_batch(gp, probs)
        _, st = gp.gspca_fit_batched(h.h, b)
        team = h.info()["team_ctas"]
        assert team in (1, 2, 4, 8, 16)
        ref = results(b)
        for r in b.results:  # scribble over the outputs
            r.T.fill_(7.0)
            r.P.fill_(7.0)
            r.lam.fill_(7.0)
        worst = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            g.capture_begin()
            rc = gp.gspca_fit_batched_async(h.h, b, worst=worst, stream=s.cuda_stream)
            g.capture_end()
        assert rc == gp.GSPCA_OK
        torch.cuda.synchronize()
        for _ in range(2):
            g.replay()
            torch.cuda.synchronize()
            got = results(b)
            for a, c in zip(ref, got):
                assert np.array_equal(a["T"], c["T"]) and np.array_equal(a["P"], c["P"])
                assert np.array_equal(a["lam"], c["lam"]) and np.array_equal(a["iters"], c["iters"])
                assert a["status"] == c["status"]
            assert int(worst.item()) == max(a["status"] for a in ref)
        del g
    for (X, K), gg in list(zip(probs, ref))[:6]:
        check_locked(gg, X, K, "gs")


def test_batched_capture_without_warmup_is_refused(gp):
    import torch

    probs = make_problems([(100, 50, 3), (80, 40, 2)], seed=4)
    with gp.Handle(128, 64, 4) as h:
        b = to_batch(gp, probs)
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            g.capture_begin()
            rc = gp.gspca_fit_batched_async(h.h, b, stream=s.cuda_stream)
            g.capture_end()
        assert rc == gp.GSPCA_ERR_NOT_SUPPORTED
        del g


def test_batched_invalid_arguments(gp):
    import torch

    with gp.Handle(256, 2048, 4) as h:
        wide = gp.Batch([{"X": torch.zeros((64, 1025), device="cuda").t().contiguous().t(), "K": 2}])
        with pytest.raises(gp.GspcaError) as e:
            gp.gspca_fit_batched(h.h, wide)
        assert e.value.status == gp.GSPCA_ERR_NOT_SUPPORTED
        bad_k = gp.Batch([{"X": torch.ones((8, 4), device="cuda").t().contiguous().t(), "K": 5}])
        with pytest.raises(gp.GspcaError) as e:
            gp.gspca_fit_batched(h.h, bad_k)
        assert e.value.status == gp.GSPCA_ERR_INVALID_ARG
        ok = gp.Batch([{"X": torch.ones((8, 4), device="cuda").t().contiguous().t(), "K": 1}])
        with pytest.raises(gp.GspcaError) as e:
            gp.gspca_fit_batched(h.h, ok, cluster_ctas=3)
        assert e.value.status == gp.GSPCA_ERR_INVALID_ARG


def test_batched_wait_limit_reports_timeout_and_context_survives(gp):
    """The testing hook makes the first ring wait of every pass wait first for a
    device word that nothing sets; its 20 ms limit runs out, the team reports
    GSPCA_ERR_TIMEOUT, the other teams stop taking work, and the next batch on
    the same context runs normally."""
    probs = make_problems([(2048, 600, 3), (1024, 300, 3), (512, 900, 2), (700, 100, 2)], seed=5)
    with gp.Handle(2048, 1024, 4) as h:
        b = to_batch(gp, probs)
        _, st = gp.gspca_fit_batched(h.h, b, cluster_ctas=2, batch_pass=1, timeout_s=0.02, test_stall=1,
                                     check=False)
        outs = results(b)
        assert st == gp.GSPCA_ERR_TIMEOUT
        assert all(o["status"] == gp.GSPCA_ERR_TIMEOUT for o in outs)
        b2 = to_batch(gp, probs)
        _, st2 = gp.gspca_fit_batched(h.h, b2, cluster_ctas=2)
        assert st2 == gp.GSPCA_OK
        outs2 = results(b2)
    for (X, K), g in zip(probs, outs2):
        check_locked(g, X, K, "gs")


def test_batched_full_workload_properties(gp):
    """The 256-problem workload (M log-uniform in [256, 8192], N in [64, 1024],
    K = 16) in the launch configuration the benchmark times: every problem
    converges or reports max_iter, GS loadings orthonormal to 1e-5, and two
    sampled problems (the largest and a median one) match the oracle locked."""
    shapes = synth.batch_shapes()
    probs = [(synth.batch_problem(i, M, N).X.astype(np.float32), 16) for i, (M, N) in enumerate(shapes)]
    with gp.Handle(8192, 1024, 16) as h:
        b = to_batch(gp, probs)
        _, st = gp.gspca_fit_batched(h.h, b)
        assert st in (gp.GSPCA_OK, gp.GSPCA_WARN_NOT_CONVERGED)
        outs = results(b)
        assert h.info()["found"] == 16 * len(probs)
    for g in outs:
        assert g["status"] in (0, 4)
        P = g["P"]
        assert np.abs(P.T @ P - np.eye(16)).max() <= ORTHO
    sizes = [M * N for M, N in shapes]
    order = np.argsort(sizes)
    for i in (int(order[-1]), int(order[len(order) // 2])):
        check_locked(outs[i], probs[i][0], 16, "gs")
