// Instantiation table of the SMPC iteration kernel.  The kernel templates are
// instantiated in one translation unit per distance-field storage type
// (kernels_f32.cu, kernels_f16.cu, kernels_bf16.cu) so they compile in
// parallel; paramap.cu picks one through these lookups.
#pragma once

#include "smpc_kernels.cuh"

namespace pm {

using IterKernel = void (*)(RobotConst, GridConst, IterArgs);

// Tile shape: C steps per lane, L lanes per roll-out, P warps per roll-out
// (H <= C * L * P).
struct TileShape { int C, L, P; };

// Every instantiated shape.
constexpr TileShape kShapes[] = {{1, 16, 1}, {1, 32, 1}, {3, 16, 1}, {2, 32, 1}, {4, 32, 1},
                                 {8, 32, 1}, {1, 32, 2}, {2, 32, 2}, {4, 32, 2}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

// Default shape for a horizon: the smallest work unit that covers H.
inline TileShape default_shape(int H)
{
    if (H <= 16) return {1, 16, 1};
    if (H <= 32) return {1, 32, 1};
    if (H <= 64) return {1, 32, 2};
    if (H <= 128) return {2, 32, 2};
    return {4, 32, 2};
}

// Kernel for a tile shape and storage type, without or with the
// self-collision term (nullptr if not instantiated; trace kernels exist for
// the float field only).
IterKernel iteration_kernel_f32(int C, int L, int P, bool trace);
IterKernel iteration_kernel_f16(int C, int L, int P, bool trace);
IterKernel iteration_kernel_bf16(int C, int L, int P, bool trace);
IterKernel iteration_kernel_f32_self(int C, int L, int P, bool trace);
IterKernel iteration_kernel_f16_self(int C, int L, int P, bool trace);
IterKernel iteration_kernel_bf16_self(int C, int L, int P, bool trace);
// The kDenseBlocks instantiation of a one-step shape ((1,16,1), (1,32,1),
// (1,32,2)) without tracing or the self term; nullptr for other shapes.
IterKernel iteration_kernel_f32_dense(int C, int L, int P);
// Float-field kernels that read the call's scalars from its device block
// (CallInputs::dyn), for launches captured once in a graph and replayed:
// the default-residency instantiation of a shape, or with dense its
// kDenseBlocks one (one-step shapes only); nullptr if not instantiated.
IterKernel iteration_kernel_f32_dyn(int C, int L, int P, bool dense);
IterKernel iteration_kernel_f16_dense(int C, int L, int P);
IterKernel iteration_kernel_bf16_dense(int C, int L, int P);

} // namespace pm

#define PM_KERNEL_CASE(C_, L_, P_, GT, WITH_TRACE, SELF)                                    \
    if (C == C_ && L == L_ && P == P_)                                                   \
        return trace ? (WITH_TRACE ? smpc_iteration_kernel<C_, L_, P_, GT, WITH_TRACE, SELF> : nullptr) \
                     : smpc_iteration_kernel<C_, L_, P_, GT, false, SELF>;

#define PM_INSTANTIATE_ITERATION_TABLE(NAME, GT, WITH_TRACE, SELF)                         \
    namespace pm {                                                                     \
    IterKernel NAME(int C, int L, int P, bool trace)                                   \
    {                                                                                  \
        PM_KERNEL_CASE(1, 16, 1, GT, WITH_TRACE, SELF)                                     \
        PM_KERNEL_CASE(1, 32, 1, GT, WITH_TRACE, SELF)                                     \
        PM_KERNEL_CASE(3, 16, 1, GT, WITH_TRACE, SELF)                                     \
        PM_KERNEL_CASE(2, 32, 1, GT, WITH_TRACE, SELF)                                     \
        PM_KERNEL_CASE(4, 32, 1, GT, WITH_TRACE, SELF)                                     \
        PM_KERNEL_CASE(8, 32, 1, GT, WITH_TRACE, SELF)                                     \
        PM_KERNEL_CASE(1, 32, 2, GT, WITH_TRACE, SELF)                                     \
        PM_KERNEL_CASE(2, 32, 2, GT, WITH_TRACE, SELF)                                     \
        PM_KERNEL_CASE(4, 32, 2, GT, WITH_TRACE, SELF)                                     \
        return nullptr;                                                                \
    }                                                                                  \
    }

#define PM_INSTANTIATE_DENSE_TABLE(NAME, GT)                                                \
    namespace pm {                                                                     \
    IterKernel NAME(int C, int L, int P)                                               \
    {                                                                                  \
        if (C == 1 && L == 16 && P == 1) return smpc_iteration_kernel<1, 16, 1, GT, false, false, kDenseBlocks>; \
        if (C == 1 && L == 32 && P == 1) return smpc_iteration_kernel<1, 32, 1, GT, false, false, kDenseBlocks>; \
        if (C == 1 && L == 32 && P == 2) return smpc_iteration_kernel<1, 32, 2, GT, false, false, kDenseBlocks>; \
        return nullptr;                                                                \
    }                                                                                  \
    }

#define PM_DYN_CASE(C_, L_, P_)                                                             \
    if (C == C_ && L == L_ && P == P_)                                                   \
        return smpc_iteration_kernel<C_, L_, P_, float, false, false, (C_ == 1 ? 6 : 5), true>;

#define PM_INSTANTIATE_DYN_TABLE(NAME)                                                      \
    namespace pm {                                                                     \
    IterKernel NAME(int C, int L, int P, bool dense)                                   \
    {                                                                                  \
        if (dense) {                                                                   \
            if (C == 1 && L == 16 && P == 1) return smpc_iteration_kernel<1, 16, 1, float, false, false, kDenseBlocks, true>; \
            if (C == 1 && L == 32 && P == 1) return smpc_iteration_kernel<1, 32, 1, float, false, false, kDenseBlocks, true>; \
            if (C == 1 && L == 32 && P == 2) return smpc_iteration_kernel<1, 32, 2, float, false, false, kDenseBlocks, true>; \
            return nullptr;                                                            \
        }                                                                              \
        PM_DYN_CASE(1, 16, 1)                                                          \
        PM_DYN_CASE(1, 32, 1)                                                          \
        PM_DYN_CASE(3, 16, 1)                                                          \
        PM_DYN_CASE(2, 32, 1)                                                          \
        PM_DYN_CASE(4, 32, 1)                                                          \
        PM_DYN_CASE(8, 32, 1)                                                          \
        PM_DYN_CASE(1, 32, 2)                                                          \
        PM_DYN_CASE(2, 32, 2)                                                          \
        PM_DYN_CASE(4, 32, 2)                                                          \
        return nullptr;                                                                \
    }                                                                                  \
    }
