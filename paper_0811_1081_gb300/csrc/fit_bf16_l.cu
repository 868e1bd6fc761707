// Kernels for storage type __nv_bfloat16 for more than 128 components (the wide factor
// products): the fit kernel for 4096 and 8192 columns per CTA.
#include "fit_inst.cuh"

GSPCA_INSTANTIATE_FIT_WIDE(8, __nv_bfloat16)
GSPCA_INSTANTIATE_FIT_WIDE(16, __nv_bfloat16)
