// Kernels for storage type float: the fit kernel for 512 and 1024 columns per CTA.
#include "fit_inst.cuh"

GSPCA_INSTANTIATE_FIT(1, float, false)
GSPCA_INSTANTIATE_FIT(2, float, false)
