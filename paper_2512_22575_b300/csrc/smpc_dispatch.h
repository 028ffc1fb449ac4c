// Instantiation table of the SMPC iteration kernel.  The kernel templates are
// instantiated in one translation unit per distance-field storage type
// (kernels_f32.cu, kernels_f16.cu, kernels_bf16.cu) so they compile in
// parallel; paramap.cu picks one through these lookups.
#pragma once

#include "smpc_kernels.cuh"

namespace pm {

using IterKernel = void (*)(RobotConst, GridConst, IterArgs);

// Tile shape: C steps per lane, L lanes per roll-out (H <= C * L).
struct TileShape { int C, L; };

// Shapes with an instantiated kernel, in order of preference for a horizon.
constexpr TileShape kShapes[] = {{1, 16}, {1, 32}, {3, 16}, {2, 32}, {4, 32}, {8, 32}};

// Kernel for a tile shape and storage type, with its dynamic shared memory
// limit raised to iteration_smem_bytes(C) (done once per kernel).
IterKernel iteration_kernel_f32(int C, int L, bool trace);
IterKernel iteration_kernel_f16(int C, int L, bool trace);
IterKernel iteration_kernel_bf16(int C, int L, bool trace);

} // namespace pm

#define PM_INSTANTIATE_ITERATION_TABLE(NAME, GT)                                        \
    namespace pm {                                                                     \
    IterKernel NAME(int C, int L, bool trace)                                          \
    {                                                                                  \
        if (L == 16 && C == 1) return trace ? smpc_iteration_kernel<1, 16, GT, true>   \
                                            : smpc_iteration_kernel<1, 16, GT, false>; \
        if (L == 16 && C == 3) return trace ? smpc_iteration_kernel<3, 16, GT, true>   \
                                            : smpc_iteration_kernel<3, 16, GT, false>; \
        if (L == 32 && C == 1) return trace ? smpc_iteration_kernel<1, 32, GT, true>   \
                                            : smpc_iteration_kernel<1, 32, GT, false>; \
        if (L == 32 && C == 2) return trace ? smpc_iteration_kernel<2, 32, GT, true>   \
                                            : smpc_iteration_kernel<2, 32, GT, false>; \
        if (L == 32 && C == 4) return trace ? smpc_iteration_kernel<4, 32, GT, true>   \
                                            : smpc_iteration_kernel<4, 32, GT, false>; \
        if (L == 32 && C == 8) return trace ? smpc_iteration_kernel<8, 32, GT, true>   \
                                            : smpc_iteration_kernel<8, 32, GT, false>; \
        return nullptr;                                                                \
    }                                                                                  \
    }
