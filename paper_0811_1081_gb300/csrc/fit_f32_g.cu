// Kernels for storage type float with two classical Gram-Schmidt passes per
// half-iteration (CGS2): the fit kernel for every column-block count.
#include "fit_inst.cuh"

GSPCA_INSTANTIATE_FIT_CGS2(1, float)
GSPCA_INSTANTIATE_FIT_CGS2(2, float)
GSPCA_INSTANTIATE_FIT_CGS2(4, float)
GSPCA_INSTANTIATE_FIT_CGS2(8, float)
GSPCA_INSTANTIATE_FIT_CGS2(16, float)
