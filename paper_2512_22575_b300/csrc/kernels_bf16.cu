// SMPC iteration kernels with a __nv_bfloat16 distance field (see smpc_kernels.cuh).
#include "smpc_dispatch.h"

PM_INSTANTIATE_ITERATION_TABLE(iteration_kernel_bf16, __nv_bfloat16, false, false)
PM_INSTANTIATE_DENSE_TABLE(iteration_kernel_bf16_dense, __nv_bfloat16)
