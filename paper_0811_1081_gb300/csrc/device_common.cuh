// Shared device helpers: memory-ordering primitives, float-float arithmetic,
// warp reductions, the bounded grid barrier and the TMA bulk-copy ring.
#pragma once

#include <cuda_bf16.h>
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

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
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

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Orders this thread's earlier generic-proxy global writes before later
// async-proxy (TMA) reads of the same addresses.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// R panels on the register path: 16-byte loads that skip L1.
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

// ---------------------------------------------------------------- float-float

// A value hi + lo carried in two FP32 words (about 44 bits of significand).
// Used for the scalar sums on the latency-critical path: GB300 executes FP64
// at ~1/57 of the FP32 rate, so a chain of FP64 adds costs ~35 ns per step
// while a float-float add is a handful of FP32 operations.
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_zero() { return {0.f, 0.f}; }

// Knuth's two-sum followed by a renormalisation (no multiplications, so no
// FMA contraction can alter it).
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float v = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float hi = __fadd_rn(s, e);
    const float lo = __fsub_rn(e, __fsub_rn(hi, s));
    return {hi, lo};
}

// x*x exactly as hi + lo (the FMA gives the rounding error of the product).
__device__ __forceinline__ ff ff_sqr(float x) {
    const float p = __fmul_rn(x, x);
    return {p, fmaf(x, x, -p)};
}

__device__ __forceinline__ ff ff_from_double(double d) {
    const float hi = __double2float_rn(d);
    return {hi, __double2float_rn(d - (double)hi)};
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// Exact product x*y as hi + lo.
__device__ __forceinline__ ff ff_mul_ff(float x, float y) {
    const float p = __fmul_rn(x, y);
    return {p, fmaf(x, y, -p)};
}

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }

// a / b in float-float: a quotient digit, its exact remainder, a second digit.
__device__ __forceinline__ ff ff_div(ff a, ff b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const ff p = ff_mul_ff(q1, b.hi);
    ff r = ff_add(a, ff_neg(p));
    r = ff_add(r, ff{-__fmul_rn(q1, b.lo), 0.f});
    const float q2 = __fdiv_rn(r.hi, b.hi);
    const float hi = __fadd_rn(q1, q2);
    return {hi, __fsub_rn(q2, __fsub_rn(hi, q1))};
}

// sqrt(a) in float-float: one Newton correction of the FP32 root.
__device__ __forceinline__ ff ff_sqrt(ff a) {
    if (!(a.hi > 0.f)) return ff_zero();
    const float y = __fsqrt_rn(a.hi);
    ff r = ff_add(a, ff_neg(ff_mul_ff(y, y)));
    const float c = __fdiv_rn(r.hi, __fmul_rn(2.f, y));
    const float hi = __fadd_rn(y, c);
    return {hi, __fsub_rn(c, __fsub_rn(hi, y))};
}

__device__ __forceinline__ ff ff_shfl_xor(ff a, int o) {
    return {__shfl_xor_sync(kFull, a.hi, o), __shfl_xor_sync(kFull, a.lo, o)};
}

__device__ __forceinline__ ff warp_sum_ff(ff a) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) a = ff_add(a, ff_shfl_xor(a, o));
    return a;
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

// Split barrier over every CTA of a cooperative launch: one arrival counter.
// arrive(e): after the CTA's work (the caller has passed __syncthreads),
// thread 0 adds 1 to the counter with a release reduction (no round trip).
// wait(e): thread 0 polls the counter with relaxed loads until it reaches
// e * gridDim.x, then an acquire fence and a CTA barrier make the other CTAs'
// writes visible to every thread.  Every wait is bounded by `timeout_ns` of
// %globaltimer; on expiry (or when another CTA has raised `abort`) the wait
// sets `abort` and returns false, and the caller must leave the kernel.
// Epochs only grow within a launch; the counter is zeroed before the launch.
// (Measured on GB300: ~1.3 us per barrier at 152 CTAs; per-CTA flags polled
// by every CTA cost ~2.8 us because of the polling traffic.)
struct GridBarrier {
    unsigned* counter;
    int* abort;
    uint64_t timeout_ns;

    __device__ __forceinline__ void arrive(unsigned epoch) const {
        (void)epoch;
        __syncthreads();
        if (threadIdx.x == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(counter) : "memory");
    }

    __device__ __forceinline__ bool wait(unsigned epoch, int* s_flag) const {
        if (threadIdx.x == 0) {
            const unsigned target = epoch * gridDim.x;
            int ok = 1;
            const uint64_t t0 = globaltimer_ns();
            for (unsigned n = 1;; ++n) {
                if ((int)(ld_relaxed_u32(counter) - target) >= 0) break;
                if (globaltimer_ns() - t0 > timeout_ns) {
                    atomicCAS(abort, 0, kStTimeout);
                    ok = 0;
                    break;
                }
                if ((n & 15u) == 0 && ld_relaxed_s32(abort) != 0) {
                    ok = 0;
                    break;
                }
            }
            fence_acq_rel_gpu();
            // A full count means every CTA arrived; one that gave up elsewhere left
            // without arriving, so the next wait sees its abort flag.
            *s_flag = ok;
        }
        __syncthreads();
        return *s_flag != 0;
    }

    __device__ __forceinline__ bool sync(unsigned& epoch, int* s_flag) const {
        ++epoch;
        arrive(epoch);
        return wait(epoch, s_flag);
    }
};

// ---------------------------------------------------------------- TMA ring

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One 1-D bulk copy global -> shared that completes `bytes` of transaction
// count on `bar` (the arrive and the expected byte count come first).
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    const uint32_t b = smem_addr(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(b)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait for phase `parity` of `bar`; false after `timeout_ns`.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity))
        if (globaltimer_ns() - t0 > timeout_ns) return false;
    return true;
}

__device__ __forceinline__ float4 lds128(const float* p) { return *reinterpret_cast<const float4*>(p); }

// ---------------------------------------------------------------- storage of R

// R is stored in 4-row panels; a cell is the 4 rows of one panel in one column,
// and cell i of the panel array sits at byte offset i * Cell<E>::kBytes.
//   Cell<float>         : 16 bytes, four FP32 values.
//   Cell<__nv_bfloat16> : 8 bytes, four bfloat16 values; a value is rounded to
//                         the nearest bfloat16 (ties to even) when it is stored,
//                         and widened exactly to FP32 when it is loaded.
// quant(v) is the value a store followed by a load gives back, so a pass that
// writes R (the fused deflation) goes on with exactly what later passes read.
// A panel holds ldp cells (panel_cells): N, or N rounded up to even for
// bfloat16 so that every panel starts on a 16-byte boundary (TMA bulk copies).
template <class E>
struct Cell;

template <>
struct Cell<float> {
    static constexpr int kBytes = 16;
    static __device__ __forceinline__ float4 ldg(const void* R, size_t i) {
        return ld_stream4(static_cast<const float*>(R) + i * 4);
    }
    static __device__ __forceinline__ float4 ldg_plain(const void* R, size_t i) {
        return reinterpret_cast<const float4*>(R)[i];
    }
    static __device__ __forceinline__ void stg(void* R, size_t i, float4 v) { st_stream4(static_cast<float*>(R) + i * 4, v); }
    static __device__ __forceinline__ void stg_plain(void* R, size_t i, float4 v) { reinterpret_cast<float4*>(R)[i] = v; }
    static __device__ __forceinline__ void st1(void* R, size_t i, int q, float v) { static_cast<float*>(R)[i * 4 + q] = v; }
    static __device__ __forceinline__ float4 lds(const void* s, size_t i) {
        return *reinterpret_cast<const float4*>(static_cast<const unsigned char*>(s) + i * 16);
    }
    static __device__ __forceinline__ float q1(float v) { return v; }
    static __device__ __forceinline__ float4 quant(float4 v) { return v; }
    static __device__ __forceinline__ void cp_async(void* dst, const void* src) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
    }
};

// Two bfloat16 in one 32-bit word: element 0 in the low half (lower address).
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ uint32_t bf_pack(float lo, float hi) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&b);
}
__device__ __forceinline__ float4 bf_unpack(uint2 w) {
    return make_float4(bf_lo(w.x), bf_hi(w.x), bf_lo(w.y), bf_hi(w.y));
}

template <>
struct Cell<__nv_bfloat16> {
    static constexpr int kBytes = 8;
    static __device__ __forceinline__ float4 ldg(const void* R, size_t i) {
        uint2 w;
        asm volatile("ld.global.cg.v2.u32 {%0,%1}, [%2];"
                     : "=r"(w.x), "=r"(w.y)
                     : "l"(static_cast<const unsigned char*>(R) + i * 8));
        return bf_unpack(w);
    }
    static __device__ __forceinline__ float4 ldg_plain(const void* R, size_t i) {
        return bf_unpack(reinterpret_cast<const uint2*>(R)[i]);
    }
    static __device__ __forceinline__ uint2 pack(float4 v) { return make_uint2(bf_pack(v.x, v.y), bf_pack(v.z, v.w)); }
    static __device__ __forceinline__ void stg(void* R, size_t i, float4 v) {
        const uint2 w = pack(v);
        asm volatile("st.global.cg.v2.u32 [%0], {%1,%2};" ::"l"(static_cast<unsigned char*>(R) + i * 8), "r"(w.x),
                     "r"(w.y)
                     : "memory");
    }
    static __device__ __forceinline__ void stg_plain(void* R, size_t i, float4 v) {
        reinterpret_cast<uint2*>(R)[i] = pack(v);
    }
    static __device__ __forceinline__ void st1(void* R, size_t i, int q, float v) {
        static_cast<__nv_bfloat16*>(R)[i * 4 + q] = __float2bfloat16_rn(v);
    }
    static __device__ __forceinline__ float4 lds(const void* s, size_t i) {
        return bf_unpack(*reinterpret_cast<const uint2*>(static_cast<const unsigned char*>(s) + i * 8));
    }
    static __device__ __forceinline__ float q1(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
    static __device__ __forceinline__ float4 quant(float4 v) { return bf_unpack(pack(v)); }
    static __device__ __forceinline__ void cp_async(void* dst, const void* src) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
    }
};

__host__ __device__ __forceinline__ int panel_cells(int N, int cell_bytes) {
    return cell_bytes == 16 ? N : (N + 1) & ~1;
}

}  // namespace gspca
