// Shared device helpers: bounded grid barrier, cache-hinted loads, warp reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gspca {

constexpr unsigned kFull = 0xffffffffu;

// Device status codes (mirror gspca_status).
enum : int { kStOK = 0, kStNotConverged = 4, kStDegenerate = 5, kStTimeout = 6 };

// ---------------------------------------------------------------- memory ops

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned atom_add_acq_rel_u32(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// R panels: 16-byte loads that skip L1 (each CTA streams only its own rows;
// the data is re-read every iteration from L2 / HBM).
__device__ __forceinline__ float4 ld_stream4(const float* p) {
    float4 v;
    asm volatile("ld.global.cg.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ void st_stream4(float* p, float4 v) {
    asm volatile("st.global.cg.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}

// Loads of data written by other CTAs of the same launch (after a barrier):
// L2 only, never a stale L1 line.
template <typename T>
__device__ __forceinline__ T ldcg(const T* p) {
    return __ldcg(p);
}

// ---------------------------------------------------------------- reductions

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Reduce V independent per-lane values over the 32 lanes with a butterfly that
// halves the live values at every level: log2(V) exchange levels move V-1
// values in total, then 5-log2(V) plain levels finish the sum.  On return
// x[0] in lane l holds the warp total of value (l >> (5 - log2 V)); the order
// of additions is fixed, so the result is deterministic.
template <int V>
__device__ __forceinline__ float warp_multi_reduce(float (&x)[V], int lane) {
    static_assert(V >= 1 && V <= 32 && (V & (V - 1)) == 0, "V must be a power of two <= 32");
    int o = 16;
#pragma unroll
    for (int c = V; c > 1; c >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < c / 2; ++i) {
            const float send = upper ? x[i] : x[i + c / 2];
            const float keep = upper ? x[i + c / 2] : x[i];
            x[i] = keep + __shfl_xor_sync(kFull, send, o);
        }
        o >>= 1;
    }
    float r = x[0];
    for (; o >= 1; o >>= 1) r += __shfl_xor_sync(kFull, r, o);
    return r;
}

template <int V>
struct Log2 {
    static constexpr int value = (V <= 1) ? 0 : 1 + Log2<V / 2>::value;
};
template <>
struct Log2<1> {
    static constexpr int value = 0;
};

// ---------------------------------------------------------------- grid barrier

// Barrier over every CTA of a cooperative launch.  Sense is a generation
// counter: a CTA reads the generation, arrives on the counter, and the last
// arrival resets the counter and publishes generation+1.  Every wait is
// bounded by `timeout_ns` of %globaltimer; on expiry (or when another CTA has
// raised `abort`) the barrier sets `abort` and returns false, and the caller
// must leave the kernel.  No CTA ever waits on a flag without a limit.
struct GridBarrier {
    unsigned* count;
    unsigned* gen;
    int* abort;
    uint64_t timeout_ns;

    __device__ __forceinline__ bool sync(int* s_flag) const {
        __syncthreads();
        if (threadIdx.x == 0) {
            int ok = 1;
            const unsigned g = ld_acquire_u32(gen);
            __threadfence();
            const unsigned arrived = atom_add_acq_rel_u32(count, 1u);
            if (arrived == gridDim.x - 1) {
                atomicExch(count, 0u);
                st_release_u32(gen, g + 1u);
            } else {
                const uint64_t t0 = globaltimer_ns();
                while (ld_acquire_u32(gen) == g) {
                    if (ld_relaxed_s32(abort) != 0) {
                        ok = 0;
                        break;
                    }
                    if (globaltimer_ns() - t0 > timeout_ns) {
                        atomicCAS(abort, 0, kStTimeout);
                        ok = 0;
                        break;
                    }
                }
            }
            __threadfence();
            if (ld_relaxed_s32(abort) != 0) ok = 0;
            *s_flag = ok;
        }
        __syncthreads();
        return *s_flag != 0;
    }
};

}  // namespace gspca
