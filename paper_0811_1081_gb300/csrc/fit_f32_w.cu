// Kernels for storage type float with the learned warm start: the fit kernel for up
// to 2048 columns per CTA.
#include "fit_inst.cuh"

GSPCA_INSTANTIATE_FIT(1, float, true)
GSPCA_INSTANTIATE_FIT(2, float, true)
GSPCA_INSTANTIATE_FIT(4, float, true)
