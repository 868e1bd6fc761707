// Kernels for storage type float with the learned warm start: the batched kernel.
#include "fit_inst.cuh"

GSPCA_INSTANTIATE_BATCH_WARM(float)
