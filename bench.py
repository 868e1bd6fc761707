#!/usr/bin/env python3
"""Benchmark: GS-PCA components/s (and HBM GB/s of the persistent kernel) on
the 10000 x 2000 planted-spectrum workload, K = 50, tol = 1e-6, FP32.

One step = one complete fit (all K components) through the C ABI with X
already resident in device memory.  L2 is flushed (a 512 MB device write)
before every timed step, outside the timed interval.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--algo gs|nipals]

--impl reference times the FP64 CPU oracle on the host cores: every step is
one whole fit of the same workload by the multi-threaded build of the oracle
(same bits as the single-threaded checker, all host cores).
Under torchrun (N > 1) every rank fits its own replica of the workload; the
value is the sum over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "GS-PCA components/s (10000x2000 planted spectrum, K=50, tol 1e-6, FP32)"


def metric_name(w, algo, storage):
    """The metric string of the main line: the default is the headline metric."""
    if w.name == "planted_10000x2000" and algo == "gs" and storage == "f32":
        return METRIC
    return (f"{'GS' if algo == 'gs' else 'NIPALS'}-PCA components/s ({w.name}, K={w.K}, tol {w.tol:g}, "
            f"{storage.upper()} storage)")
UNIT = "components/s"
FALLBACK_HBM_GBS = 6800.0


def kernel_name(N, storage="f32", K=1, gs_passes=1):
    """The instantiation of the persistent fit kernel for N columns (columns per thread),
    the storage type of R, without the learned warm start; CG2 for two Gram-Schmidt
    passes, WIDE for more than 128 components."""
    cpt = 1
    while cpt * 512 < N:
        cpt *= 2
    cg2 = gs_passes == 2
    wide = cg2 or K > 128
    return (f"fit_kernel<{cpt}, {'float' if storage == 'f32' else '__nv_bfloat16'}, false, "
            f"{'true' if cg2 else 'false'}, {'true' if wide else 'false'}>")


def profile_stem(kernel):
    """File-name form of a kernel name: fit_kernel<4, float, false> -> fit_kernel_4_float_false."""
    return kernel.replace("<", "_").replace(">", "").replace(", ", "_")


def source_sha():
    """SHA-256 over the CUDA sources, to tell whether profile counters still apply."""
    import hashlib

    d = os.path.join(ROOT, "paper_0811_1081_gb300", "csrc")
    hsh = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(d, name), "rb") as f:
                hsh.update(name.encode() + b"\0" + f.read())
    return hsh.hexdigest()


def profile_values(kernel, workload):
    """The "- key: value" figures of the committed ncu summary profiles/<kernel>_<workload>.md
    ({} when absent), and whether it was taken on the current sources."""
    p = os.path.join(ROOT, "profiles", f"{profile_stem(kernel)}_{workload}.md")
    if not os.path.exists(p):
        return {}, False, None
    vals = {}
    with open(p) as f:
        for ln in f:
            if ":" in ln and ln.strip().startswith("- "):
                k, v = ln.strip()[2:].split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
    return vals, vals.get("source_sha256") == source_sha(), p


def profiled_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu summary, or None
    when it is absent or was taken on other sources."""
    vals, fresh, p = profile_values(kernel, workload)
    if not fresh:
        return None, p
    try:
        return float(vals["dram_bytes_per_launch"]), p
    except (KeyError, ValueError):
        return None, p


def l2_read_peak(kernel, workload):
    """Peak L2 -> SM read bandwidth (GB/s) of this GPU from an ncu capture: the bytes read by the
    SMs from L2 per second divided by ncu's percentage of their sustained peak (a property of the
    hardware and its clocks, so it is used whatever the sources); None without a capture."""
    vals, _, p = profile_values(kernel, workload)
    try:
        return float(vals["l2_read_peak_gbs"]), p
    except (KeyError, ValueError):
        return None, p


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", FALLBACK_HBM_GBS)), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        return rank, world, local, dist
    return 0, 1, 0, None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value, device):
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle_sample(X64, w, algo, n_comp, flavor="O2"):
    """Time the oracle (one of its builds) on the first n_comp components of the workload."""
    import oracle

    oracle.build(flavor=flavor)
    t0 = time.perf_counter()
    f = oracle.fit(X64, n_comp, tol=w.tol, max_iter=w.max_iter, algo=algo, flavor=flavor)
    dt = time.perf_counter() - t0
    return dt, f


def host_identity():
    """nproc and the CPU model (lscpu), for the CPU baseline."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": os.uname().machine}


def cpu_baseline(X64, w, algo, sample_comp):
    """The FP64 oracle on the host cores as the CPU baseline: the -O2 and -O3
    builds, single-threaded and with OpenMP on every core.  The multi-threaded builds fit
    the whole workload (every component, measured); the single-threaded ones time the
    first `sample_comp` components and their whole-fit time is the multi-threaded whole
    fit scaled by the single- / multi-threaded time ratio on that same sample (stated as
    an estimate).  All builds return the same bits (tested)."""
    ident = host_identity()
    res = {}
    for opt in ("O2", "O3"):
        t_full, f = cpu_oracle_sample(X64, w, algo, w.K, flavor=f"{opt}-omp")
        t_s_omp, _ = cpu_oracle_sample(X64, w, algo, sample_comp, flavor=f"{opt}-omp")
        t_s_1, _ = cpu_oracle_sample(X64, w, algo, sample_comp, flavor=opt)
        res[f"{opt}_nproc"] = {"value": w.K / t_full, "unit": UNIT, "seconds": t_full, "threads": ident["nproc"],
                               "iters_total": int(f.iters.sum()), "measured": "whole fit"}
        res[f"{opt}_1thread"] = {"value": w.K / (t_full * t_s_1 / t_s_omp), "unit": UNIT,
                                 "sample_seconds": t_s_1, "threads": 1,
                                 "measured": f"first {sample_comp} components; whole fit estimated as the "
                                             f"{opt}-omp whole fit x (1-thread / nproc-thread time on the sample)"}
    best = max(("O2_nproc", "O3_nproc"), key=lambda k: res[k]["value"])
    return {"value": res[best]["value"], "unit": UNIT, "cores": ident["nproc"], "kind": "oracle",
            "sample": f"whole fit of {w.name} (all {w.K} components), FP64 plain C oracle, "
                      f"{best.split('_')[0]} build with OpenMP on {ident['nproc']} threads",
            "host": ident, "variants": res}


def run_reference(args):
    """The oracle as the reference arm: each step is one whole fit of the workload on the
    host cores (the OpenMP build of the oracle, the single-threaded checker's bits)."""
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        if int(os.environ.get("RANK", "0")) != 0:
            return 0
    w = synth.WORKLOADS[args.workload]
    X64 = w.make().astype(np.float32).astype(np.float64)
    n_comp = w.K if args.ref_components <= 0 else min(args.ref_components, w.K)
    ident = host_identity()
    flavor = "O3-omp"
    for _ in range(args.warmup):
        cpu_oracle_sample(X64, w, args.algo, n_comp, flavor=flavor)
    times = []
    for _ in range(args.steps):
        dt, _ = cpu_oracle_sample(X64, w, args.algo, n_comp, flavor=flavor)
        times.append(dt)
    total = sum(times)
    value = n_comp * args.steps / total
    what = "whole fit" if n_comp == w.K else f"first {n_comp} of {w.K} components"
    line = {
        "impl": "reference", "metric": metric_name(w, args.algo, args.storage), "value": value, "unit": UNIT,
        "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config(w, args, l2="host run"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": ident["nproc"], "kind": "oracle",
                         "sample": f"{what} of {w.name} per step, FP64 plain C oracle, -O3 build with OpenMP "
                                   f"on {ident['nproc']} threads", "host": ident},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def config(w, args, l2):
    return {"workload": w.name, "M": w.M, "N": w.N, "K": w.K, "algo": args.algo, "tol": w.tol,
            "max_iter": w.max_iter, "storage": args.storage, "l2": l2, "parallelism": "replicas"}


EQUAL_ERROR_TOLS = [1e-4, 3e-5, 1e-5, 3e-6, 1e-6, 3e-7, 1e-7]


def _exact_loadings(Xs, K):
    """Per problem: the leading K + 4 singular values and right singular vectors of X from
    LAPACK (numpy's eigh of X^T X in FP64), the exact loadings that GS-PCA converges to
    (Eq. 5).  Independent of this library and of the oracle."""
    out = []
    for X in Xs:
        X64 = X.astype(np.float64)
        w, V = np.linalg.eigh(X64.T @ X64)
        idx = np.argsort(-w)[:K + 4]
        out.append((np.sqrt(np.maximum(w[idx], 0.0)), V[:, idx]))
    return out


def _loading_error_exact(results, exact):
    """Per problem: max over components of sin(angle) between the loading p_k and the exact
    right singular vector whose singular value is nearest lambda_k (the returned order is
    the loop's, Sec. 2.3; it need not be sorted)."""
    errs = []
    for r, (sig, V) in zip(results, exact):
        P = r.P.double().cpu().numpy()
        lam = r.lam.cpu().numpy()
        e = 0.0
        for k in range(P.shape[1]):
            j = int(np.argmin(np.abs(sig - lam[k])))
            c = abs(float(P[:, k] @ V[:, j])) / max(np.linalg.norm(P[:, k]), 1e-300)
            e = max(e, math.sqrt(max(0.0, 1.0 - min(1.0, c) ** 2)))
        errs.append(e)
    return errs


def _value_at_error(curve, e):
    """components/s of a sweep curve at loading error e, interpolated linearly in
    log(error) - log(components/s) between the two sweep points that bracket e."""
    pts = sorted((p["loading_error_median"], p["value"]) for p in curve)
    for (e0, v0), (e1, v1) in zip(pts, pts[1:]):
        if e0 <= e <= e1:
            if e1 == e0:
                return max(v0, v1)
            t = (math.log(e) - math.log(e0)) / (math.log(e1) - math.log(e0))
            return math.exp(math.log(v0) + t * (math.log(v1) - math.log(v0)))
    return None


def _batched_runs(gp, h, batch, reps, flush, warm=None, tol=1e-6):
    """Best of `reps` device-timed batched fits (L2 flushed before each); returns (ms, info, status)."""
    best = None
    for i in range(reps):
        flush.fill_(float(i))
        _, st = gp.gspca_fit_batched(h.h, batch, warm=warm, tol=tol)
        info = h.info()
        if best is None or info["kernel_ms"] < best[0]:
            best = (info["kernel_ms"], info, st)
    return best


def _plain_per_problem(h, probs, K, flush, dev, tol=1e-6):
    """One gspca_fit per problem, back to back on the stream, device-timed as a whole."""
    import torch

    stream = torch.cuda.current_stream(dev)
    for X in probs[:4]:
        h.fit(X, K, tol=tol)
    flush.fill_(0.0)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    found, iters, res = 0, 0, []
    for X in probs:
        r = h.fit(X, K, tol=tol)
        found += r.info["found"]
        iters += r.info["total_iters"]
        res.append(r)
    b.record(stream)
    torch.cuda.synchronize(dev)
    return a.elapsed_time(b), found, iters, res


def bench_hbm(gp, dev, flush, peak):
    """Secondary measurement where R does not fit in L2: the paper's own test matrix shape
    (uniform entries, M = 15000, N = 7500, K = 10, tol 1e-7, Sec. 4), GS-PCA with R stored as FP32
    (450 MB, streamed from HBM every iteration) and as BF16.  Device-timed fit and the persistent
    kernel's algorithmic bytes / its event-timed duration against the measured HBM peak."""
    import torch

    w = synth.WORKLOADS["uniform_15000x7500"]
    X = torch.from_numpy(w.make().astype(np.float32)).to(dev)
    out = {"workload": f"{w.name}: X_mn ~ U[0,1), K={w.K}, tol {w.tol:g}, max_iter {w.max_iter}, GS"}
    for storage in ("f32", "bf16"):
        h = gp.Handle(w.M, w.N, w.K, device=dev.index or 0, dtype=storage)
        h.fit(X, w.K, tol=w.tol, max_iter=w.max_iter)
        best = None
        for i in range(2):
            flush.fill_(float(i))
            r = h.fit(X, w.K, tol=w.tol, max_iter=w.max_iter)
            if best is None or r.info["kernel_ms"] < best.info["kernel_ms"]:
                best = r
        info = best.info
        gbs = info["alg_bytes"] / info["kernel_ms"] / 1e6
        out[storage] = {"value": w.K / (info["kernel_ms"] / 1e3), "unit": UNIT, "kernel_ms": info["kernel_ms"],
                        "iters_total": info["total_iters"], "alg_gbs": gbs, "frac_of_hbm_peak": gbs / peak,
                        "kernel": kernel_name(w.N, storage), "status": gp.status_string(best.status)}
        h.close()
    del X
    return out


def bench_batched(gp, dev, args):
    """Secondary measurements on 256-problem workloads (M log-uniform in [256, 8192], N in
    [64, 1024], K = 16, planted spectra 10 * 0.9^i, noise 0.01, tol 1e-6), device-timed with
    CUDA events, L2 flushed before each timed run:
      - seed stream 3: one batched launch with R stored as FP32 and as BF16, and the plain
        per-problem FP32 form (one gspca_fit per problem);
      - seed stream 6 (held out from the warm start's training data, stream 5): the plain
        per-problem FP32 form, the batched form, and the batched form with the learned warm
        start (parameters from train_warm_start.py), each swept over the tolerances of
        EQUAL_ERROR_TOLS; per point components/s, iterations and the loading error against
        the exact singular vectors (LAPACK), and components/s of every form interpolated at
        equal loading error."""
    import torch

    K = 16
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = {}

    shapes = synth.batch_shapes()
    probs = [torch.from_numpy(synth.batch_problem(i, M, N).X.astype(np.float32)).to(dev)
             for i, (M, N) in enumerate(shapes)]
    cols = [X.t().contiguous().t() for X in probs]
    maxM, maxN = max(m for m, _ in shapes), max(n for _, n in shapes)
    for storage in ("f32", "bf16"):
        h = gp.Handle(maxM, maxN, K, device=dev.index or 0, dtype=storage)
        batch = gp.Batch([{"X": X, "K": K} for X in cols])
        gp.gspca_fit_batched(h.h, batch)  # autotunes
        ms, info, st = _batched_runs(gp, h, batch, 3, flush)
        out[f"batched_{storage}"] = {"value": info["found"] / ms * 1e3, "unit": UNIT, "ms": ms,
                                     "team_ctas": info["team_ctas"], "pass": info["batch_pass"],
                                     "alg_gbs": info["alg_bytes"] / ms / 1e6, "iters_total": info["total_iters"],
                                     "status": gp.status_string(st)}
        if storage == "f32":
            p_ms, p_found, p_iters, _ = _plain_per_problem(h, probs, K, flush, dev)
            out["plain_per_problem_f32"] = {"value": p_found / p_ms * 1e3, "unit": UNIT, "ms": p_ms,
                                            "iters_total": p_iters}
        h.close()
    out["workload"] = "256 planted problems (stream 3), M in [256, 8192], N in [64, 1024] log-uniform, K=16"
    out["speedup_batched_f32_vs_plain"] = out["batched_f32"]["value"] / out["plain_per_problem_f32"]["value"]
    del probs, cols

    net_path = os.path.join(ROOT, "paper_0811_1081_gb300", "warm_start_net.f32")
    if not os.path.exists(net_path):
        out["learned_start"] = {"unavailable": "no trained parameters (run train_warm_start.py)"}
        return out
    from paper_0811_1081_gb300 import train_warm_start as tws

    shapes = synth.batch_shapes(seed=6)
    X_host = [synth.batch_problem(i, M, N, seed=6).X.astype(np.float32) for i, (M, N) in enumerate(shapes)]
    probs = [torch.from_numpy(X).to(dev) for X in X_host]
    cols = [X.t().contiguous().t() for X in probs]
    exact = _exact_loadings(X_host, K)
    warm = gp.WarmStart(torch.from_numpy(tws.load_net(net_path)).to(dev),
                        torch.from_numpy(tws.sketch()).to(dev))
    maxM, maxN = max(m for m, _ in shapes), max(n for _, n in shapes)
    h = gp.Handle(maxM, maxN, K, device=dev.index or 0)
    plain_b = gp.Batch([{"X": X, "K": K} for X in cols])
    warm_b = gp.Batch([{"X": X, "K": K} for X in cols])
    gp.gspca_fit_batched(h.h, plain_b)  # autotunes once for this shape list
    gp.gspca_fit_batched(h.h, warm_b, warm=warm)
    curves = {"plain_per_problem_f32": [], "batched_f32": [], "batched_f32_learned_start": []}
    med = statistics.median
    for tol in EQUAL_ERROR_TOLS:
        p_ms, p_found, p_iters, p_res = _plain_per_problem(h, probs, K, flush, dev, tol=tol)
        b_ms, b_info, _ = _batched_runs(gp, h, plain_b, 2, flush, tol=tol)
        w_ms, w_info, _ = _batched_runs(gp, h, warm_b, 2, flush, warm=warm, tol=tol)
        used = sum(int(r.ws_choice.sum().item()) for r in warm_b.results)
        for name, ms, found, iters, res, extra in (
                ("plain_per_problem_f32", p_ms, p_found, p_iters, p_res, {}),
                ("batched_f32", b_ms, b_info["found"], b_info["total_iters"], plain_b.results, {}),
                ("batched_f32_learned_start", w_ms, w_info["found"], w_info["total_iters"], warm_b.results,
                 {"learned_start_used": used})):
            e = _loading_error_exact(res, exact)
            curves[name].append({"tol": tol, "value": found / ms * 1e3, "ms": ms, "iters_total": iters,
                                 "loading_error_median": med(e), "loading_error_max": max(e), **extra})
    h.close()
    at = {}
    for pt in curves["plain_per_problem_f32"]:
        e = pt["loading_error_median"]
        row = {"plain_per_problem_f32": pt["value"]}
        for name in ("batched_f32", "batched_f32_learned_start"):
            row[name] = _value_at_error(curves[name], e)
        if row["batched_f32_learned_start"] is not None:
            row["learned_batched_vs_plain_per_problem"] = row["batched_f32_learned_start"] / pt["value"]
            if row["batched_f32"] is not None:
                row["learned_batched_vs_batched"] = row["batched_f32_learned_start"] / row["batched_f32"]
        at[f"{e:.3e}"] = row
    head = at[f"{curves['plain_per_problem_f32'][EQUAL_ERROR_TOLS.index(1e-6)]['loading_error_median']:.3e}"]
    out["learned_start"] = {
        "workload": "256 held-out planted problems (stream 6), same distribution, K=16",
        "loading_error": "per problem: max over the 16 components of sin(angle) between the loading and the "
                         "right singular vector of X whose singular value is nearest lambda_k (LAPACK eigh of "
                         "X^T X in FP64); median over the 256 problems",
        "sweep_tols": EQUAL_ERROR_TOLS,
        "curves": curves,
        "at_equal_error": at,
        "at_plain_tol_1e-6": head,
        "interpolation": "components/s of each form at the plain per-problem form's median error, linear in "
                         "log(error) - log(components/s) between the sweep points (null outside their range)",
    }
    return out


def run_once(gp, args):
    """One fit of --workload (or one launch of the 256-problem batch) on cuda:0 for an ncu
    capture: the library's kernels run exactly as in the timed legs, nothing is timed."""
    import torch

    if args.once_batched:
        shapes = synth.batch_shapes()
        cols = [torch.from_numpy(synth.batch_problem(i, M, N).X.astype(np.float32)).cuda().t().contiguous().t()
                for i, (M, N) in enumerate(shapes)]
        with gp.Handle(max(m for m, _ in shapes), max(n for _, n in shapes), 16) as h:
            _, st = gp.gspca_fit_batched(h.h, gp.Batch([{"X": X, "K": 16} for X in cols]), cluster_ctas=4,
                                         batch_pass=1)
            torch.cuda.synchronize()
            print("batched", len(cols), "problems:", gp.status_string(st), f"{h.info()['kernel_ms']:.2f} ms")
        return 0
    w = synth.WORKLOADS[args.workload]
    K = args.K or w.K
    max_iter = args.max_iter or w.max_iter
    Xd = torch.from_numpy(w.make().astype(np.float32)).cuda()
    with gp.Handle(w.M, w.N, K, dtype=args.storage) as h:
        r = h.fit(Xd, K, tol=w.tol, max_iter=max_iter, algo=args.algo, check=False)
        torch.cuda.synchronize()
        print(f"{w.name} K={K} {args.algo} {args.storage}: {gp.status_string(r.status)}, "
              f"{r.info['kernel_ms']:.2f} ms, {r.info['total_iters']} iterations")
    return 0 if r.status in (gp.GSPCA_OK, gp.GSPCA_WARN_NOT_CONVERGED) else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="planted_10000x2000")
    ap.add_argument("--algo", default="gs", choices=["gs", "nipals"])
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16"],
                    help="storage type of the residual R inside the library")
    ap.add_argument("--ref-components", type=int, default=0,
                    help="reference arm: components per step (0 = the whole fit)")
    ap.add_argument("--cpu-components", type=int, default=3,
                    help="cpu_baseline: components of the single-threaded sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the secondary 256-problem batched measurement")
    ap.add_argument("--no-hbm-leg", action="store_true",
                    help="skip the secondary HBM-streaming measurement (15000 x 7500 uniform, R = 450 MB)")
    ap.add_argument("--no-other-algo", action="store_true",
                    help="skip the secondary measurement of the other algorithm on the same workload")
    ap.add_argument("--once", action="store_true",
                    help="profiling aid: one fit of --workload (no timing, no JSON line), then exit")
    ap.add_argument("--once-batched", action="store_true",
                    help="profiling aid: one launch of the 256-problem FP32 batch (teams of 4 CTAs), then exit")
    ap.add_argument("--K", type=int, default=0, help="with --once: components (default: the workload's)")
    ap.add_argument("--max-iter", type=int, default=0,
                    help="with --once: iteration cap per component (default: the workload's)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch

    import paper_0811_1081_gb300 as gp

    gp.load()
    if args.once or args.once_batched:
        return run_once(gp, args)
    rank, world, local, dist = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    w = synth.WORKLOADS[args.workload]
    X32 = w.make().astype(np.float32)
    M, N, K = X32.shape[0], X32.shape[1], w.K
    Xd = torch.from_numpy(X32).to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    h = gp.Handle(M, N, K, device=local, dtype=args.storage)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        h.fit(Xd, K, tol=w.tol, max_iter=w.max_iter, algo=args.algo)
    torch.cuda.synchronize(dev)

    sampler = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kern_ms, alg_bytes, launches, iters_tot = [], [], 0, []
    barrier(dist)
    torch.cuda.synchronize(dev)
    sampler.start()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        r = h.fit(Xd, K, tol=w.tol, max_iter=w.max_iter, algo=args.algo)
        ev[i][1].record(stream)
        kern_ms.append(r.info["kernel_ms"])
        alg_bytes.append(r.info["alg_bytes"])
        launches += r.info["kernel_launches"]
        iters_tot.append(r.info["total_iters"])
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t_wall
    barrier(dist)
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = max_over_ranks(dist, sum(step_ms) / 1e3, dev)
    value = world * K * args.steps / total_s
    status = r.status

    # roofline of the persistent kernel: algorithmic bytes / its event-timed duration
    peak, peak_src = measured_peaks()
    kname = kernel_name(N, args.storage, K)
    traffic, traffic_src = profiled_traffic(kname, w.name)
    if traffic_src:
        traffic_src = os.path.relpath(traffic_src, ROOT) + (" (sources changed since: null)" if traffic is None else "")
    k_s = sum(kern_ms) / 1e3
    achieved = sum(alg_bytes) / k_s / 1e9
    kernel_share = sum(kern_ms) / sum(step_ms)
    # which memory level binds: the profiled DRAM traffic against the algorithmic bytes
    # when a profile of the current sources exists, else R's size against the L2
    alg_launch = statistics.mean(alg_bytes)
    l2_size = torch.cuda.get_device_properties(dev).L2_cache_size
    r_bytes = M * N * (4 if args.storage == "f32" else 2)
    if traffic is not None:
        ratio = traffic / alg_launch
        bound = "l2" if ratio < 0.1 else "hbm"
        bound_basis = f"profiled DRAM traffic / algorithmic bytes = {ratio:.3f} (l2 below 0.1)"
    else:
        bound = "l2" if r_bytes <= 0.75 * l2_size else "hbm"
        bound_basis = f"R {r_bytes / 1e6:.0f} MB vs L2 {l2_size / 1e6:.0f} MB (l2 up to 75%)"
    l2pk, l2src = l2_read_peak(kname, w.name)
    if bound == "l2" and l2pk is None:
        bound, bound_basis = "hbm", bound_basis + "; no L2 peak recorded, HBM peak used"
    rpeak = l2pk if bound == "l2" else peak

    # end to end through the host-buffer entry point (pinned host memory)
    Xh = torch.from_numpy(X32).pin_memory()
    outs = {"T": torch.empty((K, M), dtype=torch.float32).pin_memory().numpy(),
            "P": torch.empty((K, N), dtype=torch.float32).pin_memory().numpy(),
            "lam": torch.empty(K, dtype=torch.float64).pin_memory().numpy(),
            "iters": torch.empty(K, dtype=torch.int32).pin_memory().numpy(), "R": None}
    h.fit_host(Xh, K, tol=w.tol, max_iter=w.max_iter, algo=args.algo, out=outs)
    e2e_ms = []
    e2e_steps = max(3, min(args.steps, 5))
    for i in range(e2e_steps):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        h.fit_host(Xh, K, tol=w.tol, max_iter=w.max_iter, algo=args.algo, out=outs)
        b.record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms.append(a.elapsed_time(b))
    e2e_s = max_over_ranks(dist, sum(e2e_ms) / 1e3, dev)
    e2e_value = world * K * e2e_steps / e2e_s
    h2d = M * N * 4
    d2h = (M + N) * K * 4 + K * 8 + K * 4

    line = {
        "metric": metric_name(w, args.algo, args.storage), "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config(w, args, l2="flushed before every step (512 MB device write, outside the timed interval)"),
        "status": gp.status_string(status),
        "gpu_launches": launches,
        "clocks": clocks,
        "roofline": {"bound": bound, "achieved": achieved, "peak": rpeak, "unit": "GB/s",
                     "frac": achieved / rpeak, "traffic": traffic, "kernel": kname,
                     "bound_basis": bound_basis,
                     "peak_source": (f"ncu L2->SM read peak (l1tex__m_xbar2l1tex_read_bytes per second / pct of "
                                     f"peak sustained), {os.path.relpath(l2src, ROOT)}") if bound == "l2"
                     else f"MEASURED_PEAKS.json hbm_gbs ({peak_src})",
                     "hbm_peak": peak, "frac_of_hbm_peak": achieved / peak,
                     "traffic_source": traffic_src, "kernel_share_of_step": kernel_share,
                     "kernel_ms_mean": statistics.mean(kern_ms),
                     "alg_bytes_per_launch": alg_launch},
        "iters_total_per_fit": iters_tot[-1],
        "wall_s_timed": wall,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": statistics.mean(e2e_ms)},
    }
    # orthogonality of the loadings (Sec. 2.3: GS keeps P^T P = I, NIPALS loses it)
    Pd = r.P.double()
    eye = torch.eye(K, dtype=torch.float64, device=dev)
    line["orthogonality_max_abs_PtP_minus_I"] = float((Pd.t() @ Pd - eye).abs().max().item())
    if not args.no_other_algo:
        other = "nipals" if args.algo == "gs" else "gs"
        for _ in range(2):
            h.fit(Xd, K, tol=w.tol, max_iter=w.max_iter, algo=other)
        o_ms = []
        for i in range(3):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ro = h.fit(Xd, K, tol=w.tol, max_iter=w.max_iter, algo=other)
            b.record(stream)
            torch.cuda.synchronize(dev)
            o_ms.append(a.elapsed_time(b))
        Po = ro.P.double()
        line["other_algorithm"] = {
            "algo": other, "value": K / (statistics.mean(o_ms) / 1e3), "unit": UNIT, "ms": statistics.mean(o_ms),
            "iters_total_per_fit": ro.info["total_iters"], "status": gp.status_string(ro.status),
            "orthogonality_max_abs_PtP_minus_I": float((Po.t() @ Po - eye).abs().max().item()),
            "alg_gbs": ro.info["alg_bytes"] / ro.info["kernel_ms"] / 1e6}
    if not args.no_hbm_leg and args.workload != "planted_10000x2000":
        args.no_hbm_leg = True
    if not args.no_hbm_leg:
        line["hbm_streaming"] = bench_hbm(gp, dev, flush, peak)
    if not args.no_batched:
        line["batched"] = bench_batched(gp, dev, args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(X32.astype(np.float64), w, args.algo, args.cpu_components)
    h.close()
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
