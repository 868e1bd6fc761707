#!/usr/bin/env python3
"""Benchmark: GS-PCA components/s (and HBM GB/s of the persistent kernel) on
the 10000 x 2000 planted-spectrum workload, K = 50, tol = 1e-6, FP32.

One step = one complete fit (all K components) through the C ABI with X
already resident in device memory.  L2 is flushed (a 512 MB device write)
before every timed step, outside the timed interval.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--algo gs|nipals]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the first components of the fit).
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


def kernel_name(N, storage="f32"):
    """The instantiation of the persistent fit kernel for N columns (columns per thread),
    the storage type of R, without the learned warm start."""
    cpt = 1
    while cpt * 512 < N:
        cpt *= 2
    return f"fit_kernel<{cpt}, {'float' if storage == 'f32' else '__nv_bfloat16'}, false>"


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


def profiled_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu summary
    (profiles/<kernel>_<workload>.md), or None when it is absent or was taken on other sources."""
    p = os.path.join(ROOT, "profiles", f"{profile_stem(kernel)}_{workload}.md")
    if not os.path.exists(p):
        return None, None
    vals = {}
    with open(p) as f:
        for ln in f:
            if ":" in ln and ln.strip().startswith("- "):
                k, v = ln.strip()[2:].split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_sha256") != source_sha():
        return None, p
    try:
        return float(vals["dram_bytes_per_launch"]), p
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


def cpu_oracle_sample(X64, w, algo, n_comp):
    import oracle

    oracle.build()
    t0 = time.perf_counter()
    f = oracle.fit(X64, n_comp, tol=w.tol, max_iter=w.max_iter, algo=algo)
    dt = time.perf_counter() - t0
    return dt, f


def run_reference(args):
    """The oracle as the reference arm: each step fits the first components on the host."""
    rank, world, local, dist = 0, 1, 0, None
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        if int(os.environ.get("RANK", "0")) != 0:
            return 0
    w = synth.WORKLOADS[args.workload]
    X64 = w.make().astype(np.float32).astype(np.float64)
    n_comp = args.ref_components
    for _ in range(args.warmup):
        cpu_oracle_sample(X64, w, args.algo, n_comp)
    times = []
    for _ in range(args.steps):
        dt, _ = cpu_oracle_sample(X64, w, args.algo, n_comp)
        times.append(dt)
    total = sum(times)
    value = n_comp * args.steps / total
    line = {
        "impl": "reference", "metric": metric_name(w, args.algo, args.storage), "value": value, "unit": UNIT,
        "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config(w, args, l2="host run"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"first {n_comp} of {w.K} components of {w.name} per step, "
                                   f"FP64 plain C, 1 thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def config(w, args, l2):
    return {"workload": w.name, "M": w.M, "N": w.N, "K": w.K, "algo": args.algo, "tol": w.tol,
            "max_iter": w.max_iter, "storage": args.storage, "l2": l2, "parallelism": "replicas"}


def _loading_error(results, ref):
    """Per problem: max over components of sin(angle) between a result's loadings and the
    reference's (sign-invariant); returns the list."""
    errs = []
    for r, q in zip(results, ref):
        P, Q = r.P.double(), q.P.double()
        c = (P * Q).sum(0).abs() / (P.norm(dim=0) * Q.norm(dim=0)).clamp_min(1e-300)
        errs.append(float((1 - c.clamp(max=1.0) ** 2).clamp_min(0).sqrt().max().item()))
    return errs


def _batched_runs(gp, h, batch, reps, flush, warm=None):
    """Best of `reps` device-timed batched fits (L2 flushed before each); returns (ms, info, status)."""
    best = None
    for i in range(reps):
        flush.fill_(float(i))
        _, st = gp.gspca_fit_batched(h.h, batch, warm=warm)
        info = h.info()
        if best is None or info["kernel_ms"] < best[0]:
            best = (info["kernel_ms"], info, st)
    return best


def _plain_per_problem(h, probs, K, flush, dev):
    """One gspca_fit per problem, back to back on the stream, device-timed as a whole."""
    import torch

    stream = torch.cuda.current_stream(dev)
    for X in probs[:4]:
        h.fit(X, K)
    flush.fill_(0.0)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    found, iters, res = 0, 0, []
    for X in probs:
        r = h.fit(X, K)
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
        start (parameters from train_warm_start.py), with iterations and the loading error of
        each form against a tight-tolerance fit (tol 1e-10) of the same problems."""
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
    probs = [torch.from_numpy(synth.batch_problem(i, M, N, seed=6).X.astype(np.float32)).to(dev)
             for i, (M, N) in enumerate(shapes)]
    cols = [X.t().contiguous().t() for X in probs]
    warm = gp.WarmStart(torch.from_numpy(tws.load_net(net_path)).to(dev),
                        torch.from_numpy(tws.sketch()).to(dev))
    maxM, maxN = max(m for m, _ in shapes), max(n for _, n in shapes)
    h = gp.Handle(maxM, maxN, K, device=dev.index or 0)
    ref = gp.Batch([{"X": X, "K": K} for X in cols])
    gp.gspca_fit_batched(h.h, ref, tol=1e-10, max_iter=10000)
    plain_b = gp.Batch([{"X": X, "K": K} for X in cols])
    gp.gspca_fit_batched(h.h, plain_b)
    b_ms, b_info, _ = _batched_runs(gp, h, plain_b, 3, flush)
    warm_b = gp.Batch([{"X": X, "K": K} for X in cols])
    gp.gspca_fit_batched(h.h, warm_b, warm=warm)
    w_ms, w_info, w_st = _batched_runs(gp, h, warm_b, 3, flush, warm=warm)
    used = sum(int(r.ws_choice.sum().item()) for r in warm_b.results)
    p_ms, p_found, p_iters, p_res = _plain_per_problem(h, probs, K, flush, dev)
    e_plain = _loading_error(p_res, ref.results)
    e_b = _loading_error(plain_b.results, ref.results)
    e_w = _loading_error(warm_b.results, ref.results)
    h.close()
    med = statistics.median
    out["learned_start"] = {
        "workload": "256 held-out planted problems (stream 6), same distribution, K=16, tol 1e-6",
        "plain_per_problem_f32": {"value": p_found / p_ms * 1e3, "unit": UNIT, "ms": p_ms, "iters_total": p_iters,
                                  "loading_error_median": med(e_plain), "loading_error_max": max(e_plain)},
        "batched_f32": {"value": b_info["found"] / b_ms * 1e3, "unit": UNIT, "ms": b_ms,
                        "iters_total": b_info["total_iters"], "loading_error_median": med(e_b),
                        "loading_error_max": max(e_b)},
        "batched_f32_learned_start": {"value": w_info["found"] / w_ms * 1e3, "unit": UNIT, "ms": w_ms,
                                      "iters_total": w_info["total_iters"], "loading_error_median": med(e_w),
                                      "loading_error_max": max(e_w), "learned_start_used": used,
                                      "components": w_info["found"], "status": gp.status_string(w_st)},
        "loading_error": "max over the 16 components of sin(angle) to a tol 1e-10 fit, per problem",
        "speedup_vs_plain_per_problem": (w_info["found"] / w_ms) / (p_found / p_ms),
        "iteration_ratio_learned_vs_plain_start": w_info["total_iters"] / b_info["total_iters"],
    }
    return out


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
    ap.add_argument("--ref-components", type=int, default=2)
    ap.add_argument("--cpu-components", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the secondary 256-problem batched measurement")
    ap.add_argument("--no-hbm-leg", action="store_true",
                    help="skip the secondary HBM-streaming measurement (15000 x 7500 uniform, R = 450 MB)")
    ap.add_argument("--no-other-algo", action="store_true",
                    help="skip the secondary measurement of the other algorithm on the same workload")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch

    import paper_0811_1081_gb300 as gp

    gp.load()
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
    kname = kernel_name(N, args.storage)
    traffic, traffic_src = profiled_traffic(kname, w.name)
    if traffic_src:
        traffic_src = os.path.relpath(traffic_src, ROOT) + (" (sources changed since: null)" if traffic is None else "")
    k_s = sum(kern_ms) / 1e3
    achieved = sum(alg_bytes) / k_s / 1e9
    kernel_share = sum(kern_ms) / sum(step_ms)

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
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": kname,
                     "traffic_source": traffic_src,
                     "peak_source": peak_src, "kernel_share_of_step": kernel_share,
                     "kernel_ms_mean": statistics.mean(kern_ms),
                     "alg_bytes_per_launch": statistics.mean(alg_bytes)},
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
        X64 = X32.astype(np.float64)
        dt, f = cpu_oracle_sample(X64, w, args.algo, args.cpu_components)
        line["cpu_baseline"] = {"value": args.cpu_components / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"first {args.cpu_components} of {w.K} components of {w.name}, "
                                          f"FP64 plain C oracle, 1 thread, {dt:.1f} s"}
    h.close()
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
