// Kernels for storage type __nv_bfloat16: the fit kernel for 512 and 1024 columns per CTA.
#include "fit_inst.cuh"

GSPCA_INSTANTIATE_FIT(1, __nv_bfloat16, false)
GSPCA_INSTANTIATE_FIT(2, __nv_bfloat16, false)
