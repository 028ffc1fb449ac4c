// SMPC iteration kernels with a float distance field (see smpc_kernels.cuh).
#include "smpc_dispatch.h"

PM_INSTANTIATE_ITERATION_TABLE(iteration_kernel_f32, float, true, false)
PM_INSTANTIATE_DENSE_TABLE(iteration_kernel_f32_dense, float)
