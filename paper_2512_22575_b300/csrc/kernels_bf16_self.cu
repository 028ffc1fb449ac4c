// SMPC iteration kernels with a __nv_bfloat16 distance field and the self-collision
// term compiled in (see smpc_kernels.cuh).
#include "smpc_dispatch.h"

PM_INSTANTIATE_ITERATION_TABLE(iteration_kernel_bf16_self, __nv_bfloat16, false, true)
