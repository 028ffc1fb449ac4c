// SMPC iteration kernels with a __half distance field (see smpc_kernels.cuh).
#include "smpc_dispatch.h"

PM_INSTANTIATE_ITERATION_TABLE(iteration_kernel_f16, __half, false, false)
