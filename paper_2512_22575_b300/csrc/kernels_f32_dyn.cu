// SMPC iteration kernels with a float distance field that read the call's
// scalars from its device block, for replayed graphs (see smpc_kernels.cuh).
#include "smpc_dispatch.h"

PM_INSTANTIATE_DYN_TABLE(iteration_kernel_f32_dyn)
