// Kernels for storage type __nv_bfloat16: the fit kernel for up to 4096 and 8192 columns
// per CTA.
#include "fit_inst.cuh"

GSPCA_INSTANTIATE_FIT(8, __nv_bfloat16, false)
GSPCA_INSTANTIATE_FIT(16, __nv_bfloat16, false)
