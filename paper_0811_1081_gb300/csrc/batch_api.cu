// Host side of the batched form (gspca_fit_batched, gspca_fit_batched_async):
// team-size plans, the batch workspace, the autotuner and the launches of
// batch_kernel (one per kBatchMax problems, largest M*N*K first).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cfloat>
#include <memory>
#include <numeric>
#include <vector>

#include "../../include/gspca.h"
#include "batch_kernel.cuh"
#include "handle.h"

using namespace gspca;

namespace {

constexpr int kBatchMaxN = 2 * kBlock;  // columns per thread 1 or 2

// The batched kernel for a storage type, with or without the learned warm start.
const void* batch_kernel_for(gspca_dtype dt, bool warm) {
    if (warm) return dt == GSPCA_BF16 ? batch_kernel_ptr<__nv_bfloat16, true>() : batch_kernel_ptr<float, true>();
    return dt == GSPCA_BF16 ? batch_kernel_ptr<__nv_bfloat16, false>() : batch_kernel_ptr<float, false>();
}

cudaError_t plan_batch(int device, gspca_dtype dt, int C, long maxM, int maxN, int maxK, bool warm, BatchPlan* bp) {
    const void* kern = batch_kernel_for(dt, warm);
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    int optin = 0;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device)) != cudaSuccess)
        return e;
    bp->C = C;
    bp->ldk = ws_ld(maxK);
    bp->max_slice = (maxN + C - 1) / C + 1;
    // The same dynamic size for every team size (the kernel attribute is set once
    // per plan and plans are cached): the ring takes what the vectors leave.
    const long dyn = ((long)optin - (long)fa.sharedSizeBytes - 1024) / 128 * 128;
    const long vec = (long)sizeof(float) * (2L * bp->ldk + 2L * bp->max_slice);
    const long ring = (dyn - vec) / 128 * 128;
    if (ring < kLdsBytes) return cudaErrorInvalidConfiguration;  // the warp-group pass needs its stages
    bp->ring_bytes = (int)ring;
    bp->dyn = (size_t)dyn;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bp->dyn)) != cudaSuccess)
        return e;
    if (C > 8 && (e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess)
        return e;
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)((sms + C - 1) / C * C));
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = bp->dyn;
    cudaLaunchAttribute at{};
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = (unsigned)C;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    int n = 0;
    if ((e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg)) != cudaSuccess) return e;
    if (n < 1) return cudaErrorInvalidConfiguration;
    bp->clusters = n;
    bp->dims = WsDims{(maxM + 3) / 4 * 4, maxN, maxK, C, warm};
    bp->stride = align_up(carve(nullptr, bp->dims).bytes, 256);
    return cudaSuccess;
}

// plan_batch through the handle's cache (a captured call finds its plan there
// and makes no attribute or occupancy query).
cudaError_t cached_plan(gspca_t h, int C, long maxM, int maxN, int maxK, bool warm, BatchPlan* bp) {
    const uint64_t key = ((uint64_t)C << 58) ^ ((uint64_t)warm << 57) ^ ((uint64_t)maxM << 24) ^
                         ((uint64_t)maxN << 8) ^ (uint64_t)maxK;
    auto it = h->batch.plans.find(key);
    if (it != h->batch.plans.end() && it->second.C == C && it->second.dims.N == maxN && it->second.dims.K == maxK &&
        it->second.dims.Mp == (maxM + 3) / 4 * 4 && it->second.dims.warm == warm) {
        *bp = it->second;
        return cudaSuccess;
    }
    const cudaError_t e = plan_batch(h->device, h->dtype, C, maxM, maxN, maxK, warm, bp);
    if (e == cudaSuccess) h->batch.plans[key] = *bp;
    return e;
}

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return false;
    return cs != cudaStreamCaptureStatusNone;
}

uint64_t shape_key(const gspca_problem* p, int count, int algo, bool warm) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) {
        h ^= v;
        h *= 1099511628211ull;
    };
    mix((uint64_t)count);
    mix((uint64_t)algo);
    mix((uint64_t)warm);
    for (int i = 0; i < count; ++i) {
        mix((uint64_t)p[i].M);
        mix((uint64_t)p[i].N);
        mix((uint64_t)p[i].K);
    }
    return h;
}

gspca_status check_batch(gspca_t h, const gspca_problem* p, int count, double tol, int max_iter, gspca_algo algo,
                         const gspca_opts* opts) {
    if (!h || !p || count < 1 || !(tol > 0.0) || max_iter < 1) return GSPCA_ERR_INVALID_ARG;
    if (h->dtype == GSPCA_F64) return GSPCA_ERR_NOT_SUPPORTED;  // the batched kernel stores R as FP32 or BF16
    if (algo != GSPCA_NIPALS && algo != GSPCA_GS) return GSPCA_ERR_INVALID_ARG;
    if (count > kBatchMax * kBatchChunks) return GSPCA_ERR_NOT_SUPPORTED;
    if (opts) {
        if (opts->center != GSPCA_CENTER_NONE || opts->iters_lock) return GSPCA_ERR_NOT_SUPPORTED;
        if (opts->gs_passes < 0 || opts->gs_passes > 2) return GSPCA_ERR_INVALID_ARG;
        if (opts->gs_passes == 2) return GSPCA_ERR_NOT_SUPPORTED;  // one Gram-Schmidt pass in the batched kernel
        if (opts->svd_form < 0 || opts->svd_form > 1) return GSPCA_ERR_INVALID_ARG;
        if (opts->svd_form == 1) return GSPCA_ERR_NOT_SUPPORTED;  // the batched epilogue writes scores
        if (opts->timeout_s < 0 || opts->test_stall < 0 || opts->test_stall > 1) return GSPCA_ERR_INVALID_ARG;
        const int c = opts->cluster_ctas;
        if (c != 0 && c != 1 && c != 2 && c != 4 && c != 8 && c != 16) return GSPCA_ERR_INVALID_ARG;
        if (opts->batch_pass < 0 || opts->batch_pass > 2) return GSPCA_ERR_INVALID_ARG;
        if (opts->warm) {
            if (!opts->warm->net || !opts->warm->G) return GSPCA_ERR_INVALID_ARG;
            if (algo != GSPCA_GS) return GSPCA_ERR_NOT_SUPPORTED;
            for (int i = 0; i < count; ++i)
                if (p[i].M > opts->warm->G_rows) return GSPCA_ERR_INVALID_ARG;
        }
    }
    for (int i = 0; i < count; ++i) {
        const gspca_problem& q = p[i];
        if (!q.X || !q.T || !q.P || !q.lambda) return GSPCA_ERR_INVALID_ARG;
        if (q.M < 1 || q.N < 1 || q.K < 1 || q.K > q.M || q.K > q.N || q.ldx < q.M) return GSPCA_ERR_INVALID_ARG;
        if (q.M > h->max_M || q.N > h->max_N || q.K > h->max_K) return GSPCA_ERR_INVALID_ARG;
        if (q.N > kBatchMaxN) return GSPCA_ERR_NOT_SUPPORTED;
    }
    return GSPCA_OK;
}

// Make sure the handle's batch workspace holds bp's teams (only outside capture).
gspca_status ensure_workspace(gspca_t h, const BatchPlan& bp, bool can_alloc) {
    BatchState& b = h->batch;
    const size_t need = bp.stride * (size_t)bp.clusters;
    if (!b.ctl) {
        if (!can_alloc) return GSPCA_ERR_NOT_SUPPORTED;
        GS_CUDA(cudaMalloc((void**)&b.ctl, sizeof(BatchCtl)));
        GS_CUDA(cudaMallocHost((void**)&b.h_ctl, sizeof(BatchCtl)));
        GS_CUDA(cudaEventCreate(&b.e0));
        GS_CUDA(cudaEventCreate(&b.e1));
    }
    if (need <= b.ws_bytes) return GSPCA_OK;
    if (!can_alloc) return GSPCA_ERR_NOT_SUPPORTED;
    if (b.ws) {
        GS_CUDA(cudaFree(b.ws));
        b.ws = nullptr;
        b.ws_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&b.ws, need);
    if (e != cudaSuccess) {
        cuda_ok(e);
        b.ws = nullptr;
        return e == cudaErrorMemoryAllocation ? GSPCA_ERR_OOM : GSPCA_ERR_CUDA;
    }
    b.ws_bytes = need;
    return GSPCA_OK;
}

// Enqueue the launches of one call (no synchronisation).
gspca_status enqueue_batch(gspca_t h, cudaStream_t s, const gspca_problem* p, int count, double tol, int max_iter,
                           gspca_algo algo, const gspca_opts* opts, const BatchPlan& bp, int pass, bool events,
                           int* launches) {
    BatchState& b = h->batch;
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return (double)p[x].M * p[x].N * p[x].K > (double)p[y].M * p[y].N * p[y].K;
    });
    std::unique_ptr<BatchArgs> a(new BatchArgs());
    a->algo = (int)algo;
    a->max_iter = max_iter;
    a->ldk = bp.ldk;
    a->max_slice = bp.max_slice;
    a->ring_bytes = bp.ring_bytes;
    a->redundant_max = kRedundantMaxBatch;
    a->tol = tol;
    a->eps_thresh = 64.0 * (double)FLT_EPSILON;
    const double timeout = (opts && opts->timeout_s > 0) ? opts->timeout_s : 2.0;
    a->timeout_ns = (unsigned long long)(timeout * 1e9);
    a->ctl = b.ctl;
#ifdef GSPCA_PHASE_TIMING
    static unsigned long long* timing_dev = nullptr;  // instrumented builds only
    if (!timing_dev) cudaMalloc(&timing_dev, 16 * sizeof(unsigned long long));
    cudaMemsetAsync(timing_dev, 0, 16 * sizeof(unsigned long long), s);
    a->timing = timing_dev;
    h->batch.timing_dev = timing_dev;
#endif
    a->stall = (opts && opts->test_stall) ? 1 : 0;
    a->ws_net = (opts && opts->warm) ? opts->warm->net : nullptr;
    a->ws_G = (opts && opts->warm) ? opts->warm->G : nullptr;
    a->pass = pass;
    a->ws = carve(b.ws, bp.dims);
    a->ws_stride = bp.stride;
    GS_CUDA(cudaMemsetAsync(b.ctl, 0, sizeof(BatchCtl), s));
    if (events) GS_CUDA(cudaEventRecord(b.e0, s));
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(bp.clusters * bp.C));
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = bp.dyn;
    cfg.stream = s;
    cudaLaunchAttribute at{};
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = (unsigned)bp.C;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    int n = 0;
    for (int c0 = 0, chunk = 0; c0 < count; c0 += kBatchMax, ++chunk) {
        const int cn = std::min(kBatchMax, count - c0);
        a->count = cn;
        a->queue = &b.ctl->queue[chunk];
        for (int j = 0; j < cn; ++j) {
            const gspca_problem& q = p[order[c0 + j]];
            BatchProblem& d = a->prob[j];
            d.X = q.X;
            d.T = q.T;
            d.P = q.P;
            d.lambda = q.lambda;
            d.iters = q.iters;
            d.status = q.status;
            d.ws_choice = q.ws_choice;
            d.ldx = q.ldx;
            d.M = q.M;
            d.N = q.N;
            d.K = q.K;
            d.pad = 0;
        }
        void* args[] = {a.get()};
        GS_CUDA(cudaLaunchKernelExC(&cfg, batch_kernel_for(h->dtype, a->ws_net != nullptr), args));
        ++n;
    }
    if (events) GS_CUDA(cudaEventRecord(b.e1, s));
    *launches = n;
    return GSPCA_OK;
}

// Team size and loading pass for this call: forced by opts, cached, or tuned
// now by timing every candidate on the real batch (uncaptured calls only).
gspca_status choose_team(gspca_t h, cudaStream_t s, const gspca_problem* p, int count, double tol, int max_iter,
                         gspca_algo algo, const gspca_opts* opts, long maxM, int maxN, int maxK, bool cap,
                         BatchPlan* out, int* pass) {
    const int fc = opts ? opts->cluster_ctas : 0, fp = opts ? opts->batch_pass : 0;
    const bool warm = opts && opts->warm;
    if (fc && fp) {
        *pass = fp;
        GS_CUDA(cached_plan(h, fc, maxM, maxN, maxK, warm, out));
        return ensure_workspace(h, *out, !cap);
    }
    const uint64_t key = shape_key(p, count, (int)algo, warm) ^ ((uint64_t)fc << 40) ^ ((uint64_t)fp << 48);
    auto it = h->batch.tuned.find(key);
    if (it != h->batch.tuned.end()) {
        *pass = it->second & 3;
        GS_CUDA(cached_plan(h, it->second >> 2, maxM, maxN, maxK, warm, out));
        return ensure_workspace(h, *out, !cap);
    }
    if (cap) return GSPCA_ERR_NOT_SUPPORTED;
    std::vector<int> teams = fc ? std::vector<int>{fc} : std::vector<int>{1, 2, 4, 8, 16};
    std::vector<int> passes = fp ? std::vector<int>{fp} : std::vector<int>{1, 2};
    float best_ms = 0.f;
    int best = 0;
    for (int C : teams) {
        BatchPlan bp{};
        if (cached_plan(h, C, maxM, maxN, maxK, warm, &bp) != cudaSuccess) {
            cudaGetLastError();  // an infeasible cluster shape is skipped
            continue;
        }
        gspca_status st = ensure_workspace(h, bp, true);
        if (st != GSPCA_OK) return st;
        for (int ps : passes) {
            int n = 0;
            if ((st = enqueue_batch(h, s, p, count, tol, max_iter, algo, opts, bp, ps, true, &n)) != GSPCA_OK)
                return st;
            GS_CUDA(cudaEventSynchronize(h->batch.e1));
            float ms = 0.f;
            GS_CUDA(cudaEventElapsedTime(&ms, h->batch.e0, h->batch.e1));
            if (best == 0 || ms < best_ms) {
                best_ms = ms;
                best = C * 4 + ps;
            }
        }
    }
    if (best == 0) return GSPCA_ERR_NOT_SUPPORTED;
    h->batch.tuned[key] = best;
    *pass = best & 3;
    GS_CUDA(cached_plan(h, best >> 2, maxM, maxN, maxK, warm, out));
    return ensure_workspace(h, *out, true);
}

gspca_status run_batch(gspca_t h, void* stream, const gspca_problem* p, int count, double tol, int max_iter,
                       gspca_algo algo, const gspca_opts* opts, int* worst_status, bool sync) {
    gspca_status st = check_batch(h, p, count, tol, max_iter, algo, opts);
    if (st != GSPCA_OK) return st;
    GS_CUDA(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    const bool cap = capturing(s);
    long maxM = 1;
    int maxN = 1, maxK = 1;
    for (int i = 0; i < count; ++i) {
        maxM = std::max(maxM, (long)p[i].M);
        maxN = std::max(maxN, p[i].N);
        maxK = std::max(maxK, p[i].K);
    }
    BatchPlan bp{};
    int pass = 1;
    if ((st = choose_team(h, s, p, count, tol, max_iter, algo, opts, maxM, maxN, maxK, cap, &bp, &pass)) !=
        GSPCA_OK)
        return st;
    int n = 0;
    const bool events = sync && !cap;
    if ((st = enqueue_batch(h, s, p, count, tol, max_iter, algo, opts, bp, pass, events, &n)) != GSPCA_OK)
        return st;
    h->last.batch_pass = pass;
    if (worst_status)
        GS_CUDA(cudaMemcpyAsync(worst_status, &h->batch.ctl->worst, sizeof(int), cudaMemcpyDeviceToDevice, s));
    h->last.grid_ctas = bp.clusters * bp.C;
    h->last.team_ctas = bp.C;
    h->last.block_threads = kBlock;
    h->last.kernel_launches = n;
    if (!sync) return GSPCA_OK;
    GS_CUDA(cudaMemcpyAsync(h->batch.h_ctl, h->batch.ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    if (events) GS_CUDA(cudaEventElapsedTime(&ms, h->batch.e0, h->batch.e1));
#ifdef GSPCA_PHASE_TIMING
    {
        unsigned long long t[16];
        cudaMemcpy(t, h->batch.timing_dev, sizeof(t), cudaMemcpyDeviceToHost);
        std::fprintf(stderr, "PHASES");
        for (int i = 0; i < 16; ++i) std::fprintf(stderr, " %llu", t[i]);
        std::fprintf(stderr, "\n");
    }
#endif
    const BatchCtl& c = *h->batch.h_ctl;
    h->last.kernel_ms = ms;
    h->last.found = (int)c.found;
    h->last.total_iters = (long long)c.iters;
    h->last.alg_bytes = c.bytes;
    if (c.abort) return GSPCA_ERR_TIMEOUT;
    switch (c.worst) {
        case kStOK: return GSPCA_OK;
        case kStNotConverged: return GSPCA_WARN_NOT_CONVERGED;
        case kStDegenerate: return GSPCA_ERR_DEGENERATE;
        default: return GSPCA_ERR_TIMEOUT;
    }
}

}  // namespace

void gspca::batch_release(BatchState& b) {
    if (b.ws) cudaFree(b.ws);
    if (b.ctl) cudaFree(b.ctl);
    if (b.h_ctl) cudaFreeHost(b.h_ctl);
    if (b.e0) cudaEventDestroy(b.e0);
    if (b.e1) cudaEventDestroy(b.e1);
    b = BatchState{};
}

extern "C" {

gspca_status gspca_fit_batched(gspca_t h, void* stream, const gspca_problem* problems, int count, double tol,
                               int max_iter, gspca_algo algo, const gspca_opts* opts) {
    return run_batch(h, stream, problems, count, tol, max_iter, algo, opts, nullptr, true);
}

gspca_status gspca_fit_batched_async(gspca_t h, void* stream, const gspca_problem* problems, int count, double tol,
                                     int max_iter, gspca_algo algo, const gspca_opts* opts, int* worst_status) {
    return run_batch(h, stream, problems, count, tol, max_iter, algo, opts, worst_status, false);
}

}  // extern "C"
