// Kernels for storage type float: the pack/unpack kernels and the batched kernel.
#include "fit_inst.cuh"

GSPCA_INSTANTIATE_AUX(float)
