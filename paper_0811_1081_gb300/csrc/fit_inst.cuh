// Definitions of the per-(columns per thread, storage type) kernel attribute
// queries and launches declared in launch_common.cuh.  Included only by the
// fit_*.cu translation units, each of which instantiates a few of them, so the
// heavy kernels compile in parallel and once each.
#pragma once

// (launch_common.cuh is deliberately not included: its inline dispatchers name
// every instantiation, which would compile them all in each unit.)
#include "batch_kernel.cuh"
#include "fit_kernel.cuh"
#include "prep_kernels.cuh"

namespace gspca {

template <int CPT, class E, bool WARM, bool CG2, bool WIDE>
cudaError_t fit_attrs(size_t dyn, int* bps, int* static_smem) {
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, fit_kernel<CPT, E, WARM, CG2, WIDE>);
    if (e != cudaSuccess) return e;
    *static_smem = (int)fa.sharedSizeBytes;
    e = cudaFuncSetAttribute(fit_kernel<CPT, E, WARM, CG2, WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, fit_kernel<CPT, E, WARM, CG2, WIDE>, kBlock, dyn);
}

template <int CPT, class E, bool WARM, bool CG2, bool WIDE>
cudaError_t launch_fit_t(const FitArgs& a, int G, size_t dyn, cudaStream_t s) {
    void* args[] = {const_cast<FitArgs*>(&a)};
    return cudaLaunchCooperativeKernel((const void*)fit_kernel<CPT, E, WARM, CG2, WIDE>, dim3(G), dim3(kBlock), args, dyn,
                                       s);
}

template <class E>
void launch_pack(dim3 grid, cudaStream_t s, const float* X, int layout, long ldx, int M, int N, int np, int ldp,
                 int center, const double* cmean, const double* rmean, void* R, double* xpart, unsigned* flags,
                 int nflags, int* abort, int* info, int ninfo) {
    pack_kernel<E><<<grid, kPackThreads, 0, s>>>(X, layout, ldx, M, N, np, ldp, center, cmean, rmean, R, xpart,
                                                 flags, nflags, abort, info, ninfo);
}

template <class E>
void launch_unpack(dim3 grid, cudaStream_t s, const void* R, int M, int N, int np, int ldp, const float* V, int ldv,
                   const float* U, int ldu, const double* lam, const int* info, int K, int gs, float* R_out) {
    unpack_kernel<E><<<grid, kPackThreads, 0, s>>>(R, M, N, np, ldp, V, ldv, U, ldu, lam, info, K, gs, R_out);
}

template <class E, bool WARM>
const void* batch_kernel_ptr() {
    return (const void*)batch_kernel<E, WARM>;
}

}  // namespace gspca

// Explicit instantiation of the fit kernel of one column-block count / storage type
// (WARM: with the learned warm start).
#define GSPCA_INSTANTIATE_FIT(CPT, E, WARM)                                                              \
    template cudaError_t gspca::fit_attrs<CPT, E, WARM, false, false>(size_t, int*, int*);               \
    template cudaError_t gspca::launch_fit_t<CPT, E, WARM, false, false>(const gspca::FitArgs&, int, size_t, \
                                                                         cudaStream_t);

// The fit kernel with two classical Gram-Schmidt passes per half-iteration (CGS2),
// with the factor products for more than 128 components.
#define GSPCA_INSTANTIATE_FIT_CGS2(CPT, E)                                                               \
    template cudaError_t gspca::fit_attrs<CPT, E, false, true, true>(size_t, int*, int*);                \
    template cudaError_t gspca::launch_fit_t<CPT, E, false, true, true>(const gspca::FitArgs&, int, size_t, \
                                                                        cudaStream_t);

// The fit kernel for more than 128 components (wide factor products).
#define GSPCA_INSTANTIATE_FIT_WIDE(CPT, E)                                                                \
    template cudaError_t gspca::fit_attrs<CPT, E, false, false, true>(size_t, int*, int*);               \
    template cudaError_t gspca::launch_fit_t<CPT, E, false, false, true>(const gspca::FitArgs&, int, size_t, \
                                                                         cudaStream_t);

// Explicit instantiation of the pack/unpack kernels and the batched kernel of a storage type.
#define GSPCA_INSTANTIATE_AUX(E)                                                                            \
    template void gspca::launch_pack<E>(dim3, cudaStream_t, const float*, int, long, int, int, int, int, int, \
                                        const double*, const double*, void*, double*, unsigned*, int, int*,   \
                                        int*, int);                                                           \
    template void gspca::launch_unpack<E>(dim3, cudaStream_t, const void*, int, int, int, int, const float*,  \
                                          int, const float*, int, const double*, const int*, int, int,        \
                                          float*);                                                            \
    template const void* gspca::batch_kernel_ptr<E, false>();

// The batched kernel with the learned warm start.
#define GSPCA_INSTANTIATE_BATCH_WARM(E) template const void* gspca::batch_kernel_ptr<E, true>();
