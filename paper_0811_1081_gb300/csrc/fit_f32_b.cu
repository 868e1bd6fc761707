// Kernels for storage type float: the fit kernel for up to 2048 columns per CTA.
#include "fit_inst.cuh"

GSPCA_INSTANTIATE_FIT(4, float, false)
