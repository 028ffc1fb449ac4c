// SMPC iteration kernels with a float distance field and the self-collision
// term compiled in (see smpc_kernels.cuh).
#include "smpc_dispatch.h"

PM_INSTANTIATE_ITERATION_TABLE(iteration_kernel_f32_self, float, true, true)
