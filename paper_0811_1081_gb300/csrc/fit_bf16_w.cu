// Kernels for storage type __nv_bfloat16 with the learned warm start: the fit kernel for up
// to 2048 columns per CTA.
#include "fit_inst.cuh"

GSPCA_INSTANTIATE_FIT(1, __nv_bfloat16, true)
GSPCA_INSTANTIATE_FIT(2, __nv_bfloat16, true)
GSPCA_INSTANTIATE_FIT(4, __nv_bfloat16, true)
