// Kernels for storage type __nv_bfloat16 for more than 128 components (the wide factor
// products): the fit kernel for up to 2048 columns per CTA.
#include "fit_inst.cuh"

GSPCA_INSTANTIATE_FIT_WIDE(1, __nv_bfloat16)
GSPCA_INSTANTIATE_FIT_WIDE(2, __nv_bfloat16)
GSPCA_INSTANTIATE_FIT_WIDE(4, __nv_bfloat16)
