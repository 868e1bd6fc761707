// Kernels for storage type float with two classical Gram-Schmidt passes per
// half-iteration (CGS2): the fit kernel for 4096 and 8192 columns per CTA.
#include "fit_inst.cuh"

GSPCA_INSTANTIATE_FIT_CGS2(8, float)
GSPCA_INSTANTIATE_FIT_CGS2(16, float)
