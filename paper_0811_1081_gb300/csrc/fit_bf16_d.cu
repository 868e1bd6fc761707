// Kernels for storage type __nv_bfloat16: the pack/unpack kernels and the batched kernel.
#include "fit_inst.cuh"

GSPCA_INSTANTIATE_AUX(__nv_bfloat16)
