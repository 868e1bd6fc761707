// Kernels for storage type float: the fit kernel for up to 4096 and 8192 columns
// per CTA.
#include "fit_inst.cuh"

GSPCA_INSTANTIATE_FIT(8, float, false)
GSPCA_INSTANTIATE_FIT(16, float, false)
