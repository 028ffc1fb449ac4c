// Soft-min merge of the iteration kernel's block partials (Eqs. 29-30),
// shared by the single-instance merge (paramap.cu) and the batched one
// (batch.cu).
#pragma once

#include "smpc_kernels.cuh"

namespace pm {

// One block of kMergeThreads threads produces outputs t0 .. t0+kMergeRows-1
// of U* from an instance's nb block partials (m [nb], z [nb], acc [na][nb]):
//   M = min_b m_b,  f_b = exp((M - m_b) / lambda),  Z = sum_b f_b z_b,
//   U*[t] = Ubar[t] + sum_b f_b acc_b[t] / Z.
// The partials sit in L2 (the iteration kernel has just written them), so
// the merge is bound by load latency: thread i owns partials
// b = i + kMergeThreads r and issues every load of its first kMergeChunk
// partials (m, z and its kMergeRows rows) before the first reduction, so up
// to kMergeThreads * kMergeChunk partials cost one round trip to L2.  Sums
// run over r ascending within a thread, then a fixed butterfly within each
// warp, then the warps in order: every block forms the same M and Z and the
// result does not depend on timing.
constexpr int kMergeThreads = 256;
constexpr int kMergeRows = 4;
constexpr int kMergeChunk = 6;

__device__ __forceinline__ float merge_rows(const float *part, int nb, int na, int t0, float inv_lambda,
                                            const float *Ubar, float *Uout)
{
    __shared__ float s_red[kMergeThreads / 32][kMergeRows + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float *pm_ = part, *pz = part + nb, *pacc = part + 2 * static_cast<size_t>(nb);
    const float *row[kMergeRows];
#pragma unroll
    for (int r = 0; r < kMergeRows; ++r) row[r] = pacc + static_cast<size_t>(min(t0 + r, na - 1)) * nb;

    float mv[kMergeChunk], zv[kMergeChunk], av[kMergeRows][kMergeChunk];
#pragma unroll
    for (int i = 0; i < kMergeChunk; ++i) {
        const int b = tid + i * kMergeThreads;
        const bool in = b < nb;
        mv[i] = in ? __ldg(pm_ + b) : CUDART_INF_F;
        zv[i] = in ? __ldg(pz + b) : 0.f;
#pragma unroll
        for (int r = 0; r < kMergeRows; ++r) av[r][i] = in ? __ldg(row[r] + b) : 0.f;
    }

    // M: the thread's minimum, the warp's, then the block's
    float lm = CUDART_INF_F;
#pragma unroll
    for (int i = 0; i < kMergeChunk; ++i) lm = fminf(lm, mv[i]);
    for (int b = tid + kMergeChunk * kMergeThreads; b < nb; b += kMergeThreads) lm = fminf(lm, __ldg(pm_ + b));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) lm = fminf(lm, __shfl_xor_sync(0xffffffffu, lm, off));
    if (lane == 0) s_red[warp][0] = lm;
    __syncthreads();
    float M = s_red[0][0];
#pragma unroll
    for (int w = 1; w < kMergeThreads / 32; ++w) M = fminf(M, s_red[w][0]);
    __syncthreads();   // s_red is reused for the sums

    float lz = 0.f, la[kMergeRows];
#pragma unroll
    for (int r = 0; r < kMergeRows; ++r) la[r] = 0.f;
#pragma unroll
    for (int i = 0; i < kMergeChunk; ++i) {
        const float f = weight_factor(mv[i], M, inv_lambda);
        lz = fmaf(f, zv[i], lz);
#pragma unroll
        for (int r = 0; r < kMergeRows; ++r) la[r] = fmaf(f, av[r][i], la[r]);
    }
    for (int b = tid + kMergeChunk * kMergeThreads; b < nb; b += kMergeThreads) {
        const float f = weight_factor(__ldg(pm_ + b), M, inv_lambda);
        lz = fmaf(f, __ldg(pz + b), lz);
#pragma unroll
        for (int r = 0; r < kMergeRows; ++r) la[r] = fmaf(f, __ldg(row[r] + b), la[r]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        lz += __shfl_xor_sync(0xffffffffu, lz, off);
#pragma unroll
        for (int r = 0; r < kMergeRows; ++r) la[r] += __shfl_xor_sync(0xffffffffu, la[r], off);
    }
    if (lane == 0) {
        s_red[warp][0] = lz;
#pragma unroll
        for (int r = 0; r < kMergeRows; ++r) s_red[warp][1 + r] = la[r];
    }
    __syncthreads();
    if (tid < kMergeRows && t0 + tid < na) {
        float Z = s_red[0][0], a = s_red[0][1 + tid];
#pragma unroll
        for (int w = 1; w < kMergeThreads / 32; ++w) {
            Z += s_red[w][0];
            a += s_red[w][1 + tid];
        }
        Uout[t0 + tid] = Ubar[t0 + tid] + a / Z;
    }
    return M;
}

} // namespace pm
