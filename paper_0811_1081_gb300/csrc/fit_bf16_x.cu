// Kernels for storage type __nv_bfloat16 with the learned warm start: the batched kernel.
#include "fit_inst.cuh"

GSPCA_INSTANTIATE_BATCH_WARM(__nv_bfloat16)
