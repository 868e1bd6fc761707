// Kernels for storage type float with two classical Gram-Schmidt passes per
// half-iteration (CGS2): the fit kernel for up to 2048 columns per CTA.
#include "fit_inst.cuh"

GSPCA_INSTANTIATE_FIT_CGS2(1, float)
GSPCA_INSTANTIATE_FIT_CGS2(2, float)
GSPCA_INSTANTIATE_FIT_CGS2(4, float)
