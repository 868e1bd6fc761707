// Kernels for storage type __nv_bfloat16 with two classical Gram-Schmidt passes per
// half-iteration (CGS2): the fit kernel for 4096 and 8192 columns per CTA.
#include "fit_inst.cuh"

GSPCA_INSTANTIATE_FIT_CGS2(8, __nv_bfloat16)
GSPCA_INSTANTIATE_FIT_CGS2(16, __nv_bfloat16)
