// Batched form: many independent problems in one persistent launch.
//
// The grid is made of thread-block clusters of C CTAs (C = 1, 2, 4, 8 or 16).
// A cluster is one team: it takes the next problem from a device work queue
// (problems ordered largest first on the host), packs X into its private
// panel workspace, runs the same per-component loop as the single-problem
// kernel (fit_one, Sec. 2.2 / 2.3) with the hardware cluster barrier as its
// team barrier, writes T, P, lambda, iters and the status of that problem,
// and takes the next one.  Nothing here waits on another cluster.
#pragma once

#include "fit_kernel.cuh"
#include "workspace.cuh"

namespace gspca {

constexpr int kBatchMax = 256;
constexpr int kRedundantMaxBatch = 128;  // k up to which every CTA reduces a k-vector itself  // problems per launch (descriptor table in the kernel parameters)

struct BatchProblem {
    const float* X;  // column-major, element (m, n) at X[n*ldx + m]
    float* T;        // M x K column-major
    float* P;        // N x K column-major
    double* lambda;  // K
    int* iters;      // K, nullable
    int* status;     // nullable
    int* ws_choice;  // K, nullable (learned warm start)
    long long ldx;
    int M, N, K;
    int pad;
};

constexpr int kBatchChunks = 64;  // launches (of kBatchMax problems) per call

// Per-call counters (device memory, zeroed before the first launch).
struct BatchCtl {
    int worst;                  // max over problems of the status code
    int abort;                  // a team gave up on a bounded wait
    int never;                  // a word nothing sets (target of the testing stall hook)
    int pad;
    unsigned long long iters;   // total power iterations
    unsigned long long found;   // total components found
    double bytes;               // algorithmic bytes (same count as the single-problem form)
    int queue[kBatchChunks];    // next problem index of each launch
};

struct BatchArgs {
    int count;
    int algo;
    int max_iter;
    int ldk, max_slice, ring_bytes, redundant_max;
    double tol;
    double eps_thresh;
    unsigned long long timeout_ns;
    int stall;  // testing hook: ring waits first wait for ctl->never
    int pass;   // 1: pass_warp (no ring), 2: the CTA-wide ring passes
    unsigned long long* timing;  // phase times of problem 0 (instrumented builds), nullable
    const float* ws_net;  // learned warm start (GS-PCA), nullable: network parameters
    const float* ws_G;    // its sketch (rows >= every problem's M, 16 per row)
    BatchCtl* ctl;
    int* queue;  // this launch's word of ctl->queue
    // cluster 0's workspace; cluster c adds c * ws_stride bytes to every pointer
    Workspace ws;
    size_t ws_stride;
    BatchProblem prob[kBatchMax];
};

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_id() {
    unsigned r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ int ld_rank0(const int* p) {
    unsigned a = smem_addr(p), r;
    int v;
    asm volatile("mapa.shared::cluster.u32 %0, %1, 0;" : "=r"(r) : "r"(a));
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(r) : "memory");
    return v;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <class T>
__device__ __forceinline__ T* shift(T* p, size_t bytes) {
    return p ? reinterpret_cast<T*>(reinterpret_cast<char*>(p) + bytes) : p;
}

// Pack this CTA's panels [p0, p1) of X (column-major, ldx) into the panel
// layout (row 4p+q, column c in element q of cell p*ldp + c, Cell<E> storage)
// through a 16-column x 128-row shared tile (rows past M are zero).  Returns
// this CTA's float-float sum of the stored values squared.
template <class E>
__device__ __forceinline__ ff pack_panels(const float* __restrict__ X, long long ldx, int M, int N, int ldp, int p0,
                                          int p1, void* __restrict__ R, SmemFit& sm) {
    float* tile = &sm.tmpf[0][0];  // 16 x 128, rows XOR-swizzled by column
    const int t = threadIdx.x;
    ff acc = ff_zero();
    for (int pt = p0; pt < p1; pt += 32) {
        const int rows = min(4 * (p1 - pt), 128);
        for (int ct = 0; ct < N; ct += 16) {
            {
                const int rr = t & 127, cc = t >> 7;  // 4 column groups
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int c = cc + 4 * i, col = ct + c, row = 4 * pt + rr;
                    float v = 0.f;
                    if (col < N && rr < rows && row < M) v = Cell<E>::q1(X[(size_t)col * ldx + row]);
                    acc = ff_add(acc, ff_sqr(v));
                    tile[c * 128 + (rr ^ ((c & 7) << 2))] = v;
                }
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int e = t + 512 * i, pl = e >> 6, w = e & 63, c = w >> 2, q = w & 3;
                if (4 * pl < rows && ct + c < N)
                    Cell<E>::st1(R, (size_t)(pt + pl) * ldp + ct + c, q, tile[c * 128 + ((pl * 4 + q) ^ ((c & 7) << 2))]);
            }
            __syncthreads();
        }
    }
    return acc;
}

template <int CPT, class E>
__device__ __forceinline__ void ring_geometry(int ldp, int ring_bytes, int* S, int* groups) {
    constexpr int PPR = PassShape<CPT>::PPR;
    const int stage1 = ldp * Cell<E>::kBytes;
    int s = min(kMaxStages, ring_bytes / stage1) & ~1;
    if (CPT >= 2 && CPT <= 4 && s >= 4) {
        *S = s;
        *groups = 2;
        return;
    }
    s = min(kMaxStages, ring_bytes / (PPR * stage1));
    *S = s < 2 ? 0 : s;
    *groups = 1;
}

template <int CPT, class E, bool WARM>
__device__ __forceinline__ FitOutcome run_problem(FitArgs& fa, const TeamCluster& tm, SmemFit& sm,
                                                  unsigned char* dyn_smem, Ring& rg, float threshf, unsigned& epoch,
                                                  bool narrow) {
    int S = 0, groups = 1;
    if (!narrow) ring_geometry<CPT, E>(fa.ldp, fa.ring_bytes, &S, &groups);
    if (threadIdx.x == 0) {
        fa.tma_stages = S;
        fa.dot_groups = groups;
        fa.narrow = narrow ? 1 : 0;
    }
    __syncthreads();
    ring_setup(rg, sm, dyn_smem, S, groups == 2 ? 1 : PassShape<CPT>::PPR, fa.ldp * Cell<E>::kBytes);
    const FitOutcome r = fit_one<CPT, E, WARM>(fa, tm, sm, dyn_smem, rg, threshf, epoch);
    ring_drain(fa, rg);
    return r;
}

// One launch: clusters of C CTAs take problems from ctl->queue until it runs
// past count.  Columns per thread are 1 (N <= 512) or 2 (N <= 1024).  E is the
// storage type of R (float or __nv_bfloat16); WARM instantiations carry the
// learned warm start.
template <class E, bool WARM>
__global__ void __launch_bounds__(kBlock, 1) batch_kernel(const __grid_constant__ BatchArgs a) {
    __shared__ SmemFit sm;
    __shared__ FitArgs fa;
    __shared__ int s_item, s_fail;
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    const int tid = threadIdx.x;
    const int C = (int)cluster_size(), rank = (int)cluster_rank();
    const size_t off = (size_t)cluster_id() * a.ws_stride;
    int* fail_word = shift(a.ws.abort, off) + 1;  // per-cluster failure word
    const TeamCluster tm{C, rank, fail_word};
    if (tid == 0) {
        sm.mbar_live = 0;
        s_fail = 0;
#ifdef GSPCA_PHASE_TIMING
        for (int i = 0; i < 16; ++i) sm.tacc[i] = 0;
        sm.tcur = 0;
        sm.tmark = 0;
#endif
    }
    Ring rg;
    unsigned epoch = 0;
    bool dead = false;
    for (;;) {
        if (rank == 0 && tid == 0) {
            s_item = atomicAdd(a.queue, 1);
            s_fail = ld_relaxed_s32(&a.ctl->abort) != 0 || dead;
        }
        cluster_sync_all();
        const int item = ld_rank0(&s_item);
        const bool skip = ld_rank0(&s_fail) != 0;
        cluster_sync_all();  // rank 0 may overwrite s_item only after every CTA read it
        if (item >= a.count) break;
        const BatchProblem& pb = a.prob[item];
        const int M = pb.M, N = pb.N, K = pb.K, np = (M + 3) / 4;
        const int p0 = (int)(((long long)rank * np) / C), p1 = (int)(((long long)(rank + 1) * np) / C);
        if (skip) {
            if (rank == 0 && tid == 0) {
                if (pb.status) *pb.status = kStTimeout;
                atomicMax(&a.ctl->worst, kStTimeout);
            }
            continue;
        }
#ifdef GSPCA_PHASE_TIMING
        if (tid == 0) {
            sm.tmark = rank == 0 && item == 0;
            sm.tlast = globaltimer_ns();
            sm.tcur = 14;  // pack
        }
#endif
        if (tid == 0) {
            if (rank == 0) *fail_word = 0;  // read again only after this problem's barriers
            FitArgs f{};
            f.M = M;
            f.N = N;
            f.K = K;
            f.np = np;
            f.algo = a.algo;
            f.max_iter = a.max_iter;
            f.tol = a.tol;
            f.eps_thresh = a.eps_thresh;
            f.R = shift(a.ws.R, off);
            f.ldp = panel_cells(N, Cell<E>::kBytes);
            f.V = shift(a.ws.V, off);
            f.ldv = a.ws.ld;
            f.U = shift(a.ws.U, off);
            f.ldu = a.ws.ld;
            f.W = shift(a.ws.W, off);
            f.ldw = a.ws.ld;
            f.vraw = shift(a.ws.vraw, off);
            f.vcorr = shift(a.ws.vcorr, off);
            f.ut = shift(a.ws.ut, off);
            f.upre = shift(a.ws.upre, off);
            f.partA = shift(a.ws.partA, off);
            f.LA = a.ws.LA;
            f.partB = shift(a.ws.partB, off);
            f.LB = a.ws.LB;
            f.spart = shift(a.ws.spart, off);
            f.red = shift(a.ws.red, off);
            f.lam = shift(a.ws.lam, off);
            f.iters = shift(a.ws.iters, off);
            f.abort = shift(a.ws.abort, off);
            f.timeout_ns = a.timeout_ns;
            f.ring_bytes = a.ring_bytes;
            f.ldk = a.ldk;
            f.max_slice = a.max_slice;
            f.redundant_max = a.redundant_max;
            f.stall_word = a.stall ? &a.ctl->never : nullptr;
            if (a.ws_net) {
                f.ws_net = a.ws_net;
                f.ws_G = a.ws_G;
                f.wsF = shift(a.ws.wsF, off);
                f.wsP0 = shift(a.ws.wsP0, off);
                f.pC = shift(a.ws.pC, off);
                f.wsPart = shift(a.ws.wsPart, off);
                f.wsInit = shift(a.ws.wsInit, off);
                f.ws_choice = pb.ws_choice;
            }
            fa = f;
        }
        __syncthreads();
        // pack, ||X||_F^2 over the team
        ff ss = pack_panels<E>(pb.X, pb.ldx, M, N, fa.ldp, p0, p1, fa.R, sm);
        fence_proxy_async_global();  // the ring reads R through the async proxy
        ss = block_sum_ff(ss, sm);
        write_scalar(fa, rank, 0, ss);
        tm.sync(epoch, nullptr);
        gather_reduce(fa, sm, C, 1, 0, 0, fa.partA, fa.LA, 0, [](int v) { return v; }, nullptr);
        const float threshf =
            (float)(fa.eps_thresh * sqrt(fmax(0.0, ff_to_double(sm.sff[0]))));
        const bool narrow = a.pass == 1;
        FitOutcome r = (N <= kBlock) ? run_problem<1, E, WARM>(fa, tm, sm, dyn_smem, rg, threshf, epoch, narrow)
                                     : run_problem<2, E, WARM>(fa, tm, sm, dyn_smem, rg, threshf, epoch, narrow);
        PHASE_MARK(15);
        tm.sync(epoch, nullptr);  // V, U, lambda of every CTA visible; failure word settled
        if (ldcg(fail_word) != 0) {
            r.status = kStTimeout;
            dead = true;
            if (rank == 0 && tid == 0) atomicExch(&a.ctl->abort, 1);
        }
        // epilogue: T = V Lambda (GS) or V (NIPALS), P = U, zero past `found`
        const bool gs = a.algo == 1;
        const int found = r.status == kStTimeout ? 0 : r.found;
        {
            const int r0 = min(4 * p0, M), r1 = min(4 * p1, M), nr = r1 - r0;
            for (int e = tid; e < nr * K; e += kBlock) {
                const int k = e / nr, row = r0 + e % nr;
                float v = 0.f;
                if (k < found) {
                    v = fa.V[(size_t)row * fa.ldv + k];
                    if (gs) v = (float)((double)v * ldcg(fa.lam + k));
                }
                pb.T[(size_t)k * M + row] = v;
            }
            const int n0 = (int)(((long long)rank * N) / C), n1 = (int)(((long long)(rank + 1) * N) / C);
            const int nn = n1 - n0;
            for (int e = tid; e < nn * K; e += kBlock) {
                const int k = e / nn, n = n0 + e % nn;
                pb.P[(size_t)k * N + n] = k < found ? fa.U[(size_t)n * fa.ldu + k] : 0.f;
            }
        }
#ifdef GSPCA_PHASE_TIMING
        if (tid == 0 && sm.tmark && a.timing) {
            PHASE_MARK(15);
            for (int i = 0; i < 16; ++i) a.timing[i] = sm.tacc[i];
            sm.tmark = 0;
        }
#endif
        if (rank == 0 && tid == 0) {
            double bytes = 0.0;
            long long tot = 0;
            const double mn = (double)M * N * (Cell<E>::kBytes / 4);
            for (int k = 0; k < K; ++k) {
                const int it = k < found ? ldcg(fa.iters + k) : 0;
                pb.lambda[k] = k < found ? ldcg(fa.lam + k) : 0.0;
                if (pb.iters) pb.iters[k] = it;
                if (k < found) {
                    tot += it;
                    bytes += ((double)it + 1.0) * mn + (k > 0 ? mn : 0.0);
                    if (gs && k > 0) bytes += (double)it * (2.0 * M * k + 3.0 * N * k) * 4.0;
                }
            }
            if (pb.status) *pb.status = r.status;
            atomicMax(&a.ctl->worst, r.status);
            atomicAdd(&a.ctl->iters, (unsigned long long)tot);
            atomicAdd(&a.ctl->found, (unsigned long long)found);
            atomicAdd(&a.ctl->bytes, bytes);
        }
    }
    if (tid == 0 && sm.mbar_live > 0)
        for (int s = 0; s < sm.mbar_live; ++s)
            asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(&sm.mbar[s])) : "memory");
}

// The batched kernel of a storage type as a launchable function pointer
// (defined and instantiated with the kernels, see fit_inst.cuh).
template <class E, bool WARM>
const void* batch_kernel_ptr();

}  // namespace gspca
