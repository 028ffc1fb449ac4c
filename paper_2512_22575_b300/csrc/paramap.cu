// C ABI of the SMPC hot path (include/paramap.h): contexts, argument checks,
// host<->device staging and kernel dispatch.  The arithmetic lives in
// smpc_device.cuh / smpc_kernels.cuh.
#include "ctx_internal.h"
#include "softmin_merge.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <unordered_map>
#include <vector>

using namespace pm;



namespace {

thread_local std::string g_err;

const char *kVersion = "paramap-b300 0.1 (sm_103a)";

pm_status set_err(pm_ctx *ctx, pm_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf; else g_err = buf;
    return st;
}

#define PM_CUDA(ctx, call)                                                                \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return set_err((ctx), e_ == cudaErrorMemoryAllocation ? PM_ENOMEM : PM_ECUDA, \
                           "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,      \
                           __LINE__);                                                     \
    } while (0)

bool finite_all(const float *p, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

IterKernel lookup_kernel(int dtype, TileShape s, bool trace, bool self)
{
    switch (dtype) {
    case PM_F32: return (self ? iteration_kernel_f32_self : iteration_kernel_f32)(s.C, s.L, s.P, trace);
    case PM_F16: return (self ? iteration_kernel_f16_self : iteration_kernel_f16)(s.C, s.L, s.P, trace);
    case PM_BF16: return (self ? iteration_kernel_bf16_self : iteration_kernel_bf16)(s.C, s.L, s.P, trace);
    default: return nullptr;
    }
}

IterKernel lookup_dense_kernel(int dtype, TileShape s)
{
    switch (dtype) {
    case PM_F32: return iteration_kernel_f32_dense(s.C, s.L, s.P);
    case PM_F16: return iteration_kernel_f16_dense(s.C, s.L, s.P);
    case PM_BF16: return iteration_kernel_bf16_dense(s.C, s.L, s.P);
    default: return nullptr;
    }
}

// The iteration kernel of a call, its shared memory and resident blocks.
// A one-step shape without tracing or the self term switches to its
// kDenseBlocks instantiation when that holds more blocks per SM and the
// extra units run the launch in fewer rounds of tiles, and in at most two:
// a short launch is dominated by its partly filled last round, a long one
// by the throughput per round.  (When the instantiations were fitted at 80
// and 72 registers, K = 4096, H = 64 ran 3 rounds of 1776 units or 2 of
// 2072, replan 290 -> 280 us, and K = 16384 862 against 927 us per replan.)
// At equal residency the dense one runs as well on a launch of at most two
// rounds: only it draws its first tile's normals before the wait for the
// previous kernel (replan K = 4096, H = 64 2.3% and K = 1024 5.6% shorter;
// at K = 16384, eight rounds, the default one is 2% faster).
struct KernelPick {
    IterKernel fn = nullptr;
    size_t smem = 0;
    long long resident = 0;
};

pm_status pick_kernel(pm_ctx *c, long long K, TileShape sh, bool trace, KernelPick &out)
{
    const bool self = c->rc.n_self_groups > 0;
    out.fn = lookup_kernel(c->gd.dtype, sh, trace, self);
    if (!out.fn)
        return set_err(c, trace ? PM_EINVAL : PM_EINTERNAL, "no %s kernel for C=%d L=%d P=%d",
                       trace ? "trace" : "iteration", sh.C, sh.L, sh.P);
    out.smem = iteration_smem_bytes(sh.C) + self_smem_bytes(c->rc);
    const int per_sm = resident_blocks_per_sm(reinterpret_cast<const void *>(out.fn), kBlock, out.smem);
    if (per_sm < 1)
        return set_err(c, PM_ECUDA, "cannot give the C=%d kernel %zu bytes of shared memory", sh.C, out.smem);
    out.resident = static_cast<long long>(c->n_sm) * per_sm;
    IterKernel dense = (trace || self) ? nullptr : lookup_dense_kernel(c->gd.dtype, sh);
    if (dense) {
        const int per_sm_d = resident_blocks_per_sm(reinterpret_cast<const void *>(dense), kBlock, out.smem);
        const long long upb = kWarps / sh.P, tiles = (K + 32 / sh.L - 1) / (32 / sh.L);
        const long long units = out.resident * upb, units_d = static_cast<long long>(c->n_sm) * per_sm_d * upb;
        const long long rounds = (tiles + units - 1) / units, rounds_d = (tiles + units_d - 1) / units_d;
        // at equal residency the dense one runs too on a launch of at most
        // two rounds: it draws its first tile's normals before waiting for
        // the previous kernel
        if (rounds_d <= 2 && (per_sm_d == per_sm || (per_sm_d > per_sm && rounds_d < rounds))) {
            out.fn = dense;
            out.resident = static_cast<long long>(c->n_sm) * per_sm_d;
        }
    }
    return PM_OK;
}

bool shape_known(TileShape t)
{
    for (const TileShape &s : kShapes)
        if (s.C == t.C && s.L == t.L && s.P == t.P) return true;
    return false;
}

// The context's shape for horizon H: the forced one if set, else the default.
pm_status pick_shape(pm_ctx *c, int H, TileShape &out)
{
    out = c->forced.C ? c->forced : default_shape(H);
    if (out.C * out.L * out.P < H)
        return set_err(c, PM_EINVAL, "tile shape C=%d L=%d P=%d holds %d steps < H=%d", out.C, out.L,
                       out.P, out.C * out.L * out.P, H);
    return PM_OK;
}

// Blocks of a launch: enough warps for every tile (P warps per tile of R
// roll-outs), at most what stays resident, at most kMaxBlocks.
long long launch_blocks(long long K, TileShape sh, long long resident)
{
    const int R = 32 / sh.L;
    const long long tiles = (K + R - 1) / R;
    const long long need = (tiles * sh.P + kWarps - 1) / kWarps;
    long long nb = std::max(1LL, std::min({need, resident, static_cast<long long>(kMaxBlocks)}));
    // When the tiles divide evenly over the units, the k = 0 pass would
    // follow a unit's last tile; one more block, where it still fits, gives
    // the pass a unit of its own that runs beside the tiles (its partial is
    // empty: m = inf, z = 0).
    if (tiles % (nb * kWarps / sh.P) == 0 && nb < resident && nb < kMaxBlocks) ++nb;
    return nb;
}

size_t dtype_size(int dt) { return dt == PM_F32 ? 4 : 2; }

// ------------------------------------------------------------ small kernels
__global__ void convert_grid_kernel(const float *src, void *dst, size_t n, int dtype)
{
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        if (dtype == PM_F16) static_cast<__half *>(dst)[i] = __float2half_rn(src[i]);
        else static_cast<__nv_bfloat16 *>(dst)[i] = __float2bfloat16_rn(src[i]);
    }
}

// Skip bound of cell (i, j, l): the minimum of the stored field over the
// voxels [max(i-1, 0), i+1] x [max(j-1, 0), j+1] x [max(l-1, 0), l+1],
// i.e. over the 8 corners of the cell and of its lower neighbours.  The
// iteration kernel fetches it through the texture unit at the raw grid
// coordinate: the unit quantises the coordinate to fixed point, and a
// monotone rounding with an error below one texel never lands below the
// point's own cell and at most one cell above it on each axis, so the
// fetched texel's bound covers the point's cell.  Only the
// (nx-1) x (ny-1) x (nz-1) cells are written (the texture holds no others).
// A warp takes 30 cells along x (lanes 1..30; lanes 0 and 31 hold the
// neighbouring voxels), one row j and kBoundZ planes.  Each lane loads its
// voxel column over rows j-1..j+1 on the kBoundZ + 2 planes it needs, all
// before the first minimum (one round trip to memory), takes the row
// minimum per plane, the x window from its neighbours by shuffles and then
// the z window: about 4 loads per cell.
constexpr int kBoundZ = 8;

template <typename T>
__global__ void cell_min_kernel(const T *phi, float *cmin, int nx, int ny, int nz)
{
    const int lane = threadIdx.x & 31;
    const int cx = nx - 1, cy = ny - 1, cz = nz - 1;
    const int nxs = (cx + 29) / 30, nzc = (cz + kBoundZ - 1) / kBoundZ;
    const long long items = static_cast<long long>(nxs) * cy * nzc;
    const size_t sy = nx, sz = static_cast<size_t>(nx) * ny;
    const long long warps = (static_cast<long long>(gridDim.x) * blockDim.x) >> 5;
    for (long long it = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5; it < items;
         it += warps) {
        const int xs = static_cast<int>(it % nxs);
        const long long rest = it / nxs;
        const int j = static_cast<int>(rest % cy), zc = static_cast<int>(rest / cy);
        const int i = xs * 30 + lane - 1;
        const bool in_x = i >= 0 && i < nx;
        const int l_begin = zc * kBoundZ, l_end = min(l_begin + kBoundZ, cz);
        // plane l_begin - 1 + q for q = 0 .. kBoundZ + 1 (planes below 0 or
        // above l_end are not needed and stay +inf); rows max(j-1, 0), j, j+1
        const size_t r0 = static_cast<size_t>(max(j - 1, 0)) * sy, r1 = j * sy, r2 = (j + 1) * sy;
        float v[kBoundZ + 2][3];
#pragma unroll
        for (int q = 0; q < kBoundZ + 2; ++q) {
            const int ll = l_begin - 1 + q;
            const bool in = in_x && ll >= 0 && ll <= l_end;
            const T *col = phi + (in ? ll * sz + i : 0);
            v[q][0] = in ? grid_load(col + r0) : CUDART_INF_F;
            v[q][1] = in ? grid_load(col + r1) : CUDART_INF_F;
            v[q][2] = in ? grid_load(col + r2) : CUDART_INF_F;
        }
        float w[kBoundZ + 2];
#pragma unroll
        for (int q = 0; q < kBoundZ + 2; ++q) {
            const float my = fminf(v[q][0], fminf(v[q][1], v[q][2]));
            const float left = __shfl_up_sync(0xffffffffu, my, 1);
            const float right = __shfl_down_sync(0xffffffffu, my, 1);
            w[q] = fminf(my, fminf(lane > 0 ? left : CUDART_INF_F, lane < 31 ? right : CUDART_INF_F));
        }
        if (lane >= 1 && lane <= 30 && i < cx) {
#pragma unroll
            for (int t = 0; t < kBoundZ; ++t) {
                const int l = l_begin + t;     // planes l-1, l, l+1 are w[t], w[t+1], w[t+2]
                if (l < l_end) cmin[l * sz + j * sy + i] = fminf(w[t], fminf(w[t + 1], w[t + 2]));
            }
        }
    }
}

// FP32 yardstick: 8 independent chains of dependent FMAs per thread.
__global__ void __launch_bounds__(256) fma_peak_kernel(float *sink, int iters, float a, float b)
{
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = static_cast<float>(threadIdx.x + i);
#pragma unroll 4
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, b);
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    if (s == 1.2345e-30f) sink[0] = s;   // never true; keeps the chains live
}

__global__ void philox_words_kernel(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out,
                                    size_t n)
{
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        uint32_t x0 = ctr[4 * i], x1 = ctr[4 * i + 1], x2 = ctr[4 * i + 2], x3 = ctr[4 * i + 3];
        philox4x32_10(x0, x1, x2, x3, k0, k1);
        out[4 * i] = x0; out[4 * i + 1] = x1; out[4 * i + 2] = x2; out[4 * i + 3] = x3;
    }
}

// xi = log(T_g^{-1} T) of each pose pair with the iteration's pose_error
// (Eqs. 11-15): Tg, T row-major 4x4, xi = [v; w].
__global__ void pose_error_kernel(const float *Tg, const float *T, float *xi, size_t n)
{
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const float *g = Tg + 16 * i, *e = T + 16 * i;
        const float Rg[9] = {g[0], g[1], g[2], g[4], g[5], g[6], g[8], g[9], g[10]};
        const float tg[3] = {g[3], g[7], g[11]};
        float x[6];
        pose_error(Rg, tg, mk(e[0], e[4], e[8]), mk(e[1], e[5], e[9]), mk(e[2], e[6], e[10]),
                   mk(e[3], e[7], e[11]), x);
        for (int j = 0; j < 6; ++j) xi[6 * i + j] = x[j];
    }
}

// joint_sincos with the coefficients as the kernels hold them (parameter
// bank), beside CUDA's sincosf of the same argument for comparison

__global__ void joint_sincos_kernel(const float *x, float *sc, float *sc_ref, size_t n, const __grid_constant__ PolyConst kp)
{
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        float s, c;
        joint_sincos(x[i], s, c, kp);
        sc[2 * i] = s;
        sc[2 * i + 1] = c;
        if (sc_ref) {
            sincosf(x[i], &s, &c);
            sc_ref[2 * i] = s;
            sc_ref[2 * i + 1] = c;
        }
    }
}

struct Sigma { float s[8]; };

__global__ void sample_noise_kernel(int K, int H, Sigma sg, uint32_t s_lo, uint32_t s_hi,
                                    uint32_t iter, float *eps, const __grid_constant__ PolyConst kp)
{
    const size_t total = static_cast<size_t>(K) * H;
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const uint32_t m = static_cast<uint32_t>(i / H), k = static_cast<uint32_t>(i % H);
        float z[8];
        step_normals(s_lo, s_hi, iter, m, k, z, kp);
        for (int j = 0; j < kNJ; ++j) eps[i * kNJ + j] = sg.s[j] * z[j];
    }
}

// Soft-min merge (Eqs. 29-30) of the iteration kernel's nb block partials:
// block x produces outputs kMergeRows x .. of U* (merge_rows).  Block 0 also
// writes min S = M + c0, and the k = 0 terms c0 are added to the costs.
__global__ void __launch_bounds__(kMergeThreads)
softmin_merge_kernel(const float *part, int nb, int na, const float *Ubar, float *Uout,
                     float inv_lambda, const float *dyn, float *c0, float *costs, int K)
{
    grid_dependency_prologue();
    if (dyn) inv_lambda = __ldg(dyn + kDynInvLambda);
    const float M = merge_rows(part, nb, na, blockIdx.x * kMergeRows, inv_lambda, Ubar, Uout);
    const float k0 = __ldg(c0);
    if (blockIdx.x == 0 && threadIdx.x == 0) c0[1] = M + k0;
    if (costs)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += gridDim.x * blockDim.x)
            costs[i] += k0;
}

// Receding-horizon step (Sec. IV-C): execute u0* for one integrator step and
// shift U one step left, repeating the last row.  One block.
__global__ void replan_advance_kernel(const float *q0, const float *qd0, float *U, int H, float dt,
                                      const float *dyn, float *q_out, float *qd_out, float *u0_out,
                                      const float *c0, float *best_out)
{
    grid_dependency_prologue();
    if (dyn) dt = __ldg(dyn + kDynDt);
    __shared__ float sU[kMaxHorizon * kNJ];
    const int n = H * kNJ;
    for (int i = threadIdx.x; i < n; i += blockDim.x) sU[i] = U[i];
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) U[i] = (i < n - kNJ) ? sU[i + kNJ] : sU[i];
    if (threadIdx.x < kNJ) {
        const int j = threadIdx.x;
        const float u0 = sU[j];
        const float qd = fmaf(dt, u0, qd0[j]);
        const float q = fmaf(dt, qd, q0[j]);
        q_out[j] = q;
        qd_out[j] = qd;
        if (u0_out) u0_out[j] = u0;
    }
    if (threadIdx.x == 0 && best_out) *best_out = c0[1];
}

// One step of a planning episode (Sec. IV-C receding horizon, Sec. V-A
// metrics), one block: execute u0* (advance q, qd in place), shift U, and
// report [e_pos, e_ori, min S, sum_j |q_{t+1} - q_t|] of the new state
// against the goal.  e_ori is the angle of R_g^T R, which equals
// 2 arccos |q_g . q| of the unit quaternions.
__global__ void episode_step_kernel(const RobotConst rc, const float *Tg, float *q, float *qd, float *U, int H,
                                    float dt, const float *c0, float *metrics)
{
    grid_dependency_prologue();
    __shared__ float sU[kMaxHorizon * kNJ];
    __shared__ float s_dq[kNJ], s_q[kNJ];
    const int n = H * kNJ;
    for (int i = threadIdx.x; i < n; i += blockDim.x) sU[i] = U[i];
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) U[i] = (i < n - kNJ) ? sU[i + kNJ] : sU[i];
    if (threadIdx.x < kNJ) {
        const int j = threadIdx.x;
        const float qd1 = fmaf(dt, sU[j], qd[j]);
        const float q1 = fmaf(dt, qd1, q[j]);
        s_dq[j] = fabsf(q1 - q[j]);
        s_q[j] = q1;
        q[j] = q1;
        qd[j] = qd1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Frame F = base_frame();
        for (int j = 0; j < kNJ; ++j) dh_step(F, rc.ca[j], rc.sa[j], rc.a[j], rc.d[j], s_q[j] + rc.th0[j], rc.poly);
        const f3 t = axpy(rc.flange_d, F.c3, F.t);
        const f3 e = sub(t, mk(Tg[3], Tg[7], Tg[11]));
        // R_d = R_g^T R: entries from the goal's columns and the frame's columns
        const f3 g0 = mk(Tg[0], Tg[4], Tg[8]), g1 = mk(Tg[1], Tg[5], Tg[9]), g2 = mk(Tg[2], Tg[6], Tg[10]);
        const float r00 = dot(g0, F.c1), r11 = dot(g1, F.c2), r22 = dot(g2, F.c3);
        const f3 vee = mk(dot(g2, F.c2) - dot(g1, F.c3), dot(g0, F.c3) - dot(g2, F.c1),
                          dot(g1, F.c1) - dot(g0, F.c2));
        metrics[0] = sqrtf(dot(e, e));
        metrics[1] = atan2f(0.5f * sqrtf(dot(vee, vee)), 0.5f * (r00 + r11 + r22 - 1.0f));
        metrics[2] = c0[1];
        float path = 0.f;
        for (int j = 0; j < kNJ; ++j) path += s_dq[j];
        metrics[3] = path;
    }
}

// ------------------------------------------------------------ helpers
pm_status ensure_capacity(pm_ctx *c, int K, int H, int nb)
{
    const size_t needU = static_cast<size_t>(kMaxHorizon) * kNJ;
    if (!c->d_U) {
        PM_CUDA(c, cudaMalloc(&c->d_U, needU * sizeof(float)));
        c->cap_U = needU;
    }
    if (static_cast<size_t>(K) > c->cap_costs) {
        size_t cap = std::max<size_t>(K, 4096);
        if (c->d_costs) cudaFree(c->d_costs);
        c->d_costs = nullptr;
        c->cap_costs = 0;
        PM_CUDA(c, cudaMalloc(&c->d_costs, cap * sizeof(float)));
        c->cap_costs = cap;
    }
    if (static_cast<size_t>(K) > c->cap_h_out) {
        size_t cap = std::max<size_t>(K, 4096);
        if (c->h_out) cudaFreeHost(c->h_out);
        c->h_out = nullptr;
        c->cap_h_out = 0;
        PM_CUDA(c, cudaMallocHost(&c->h_out, cap * sizeof(float)));
        c->cap_h_out = cap;
    }
    const size_t stride = 2 + static_cast<size_t>(H) * kNJ;
    const size_t needP = static_cast<size_t>(nb) * stride;
    if (needP > c->cap_part) {
        size_t cap = std::max(needP, static_cast<size_t>(1024) * (2 + 64 * kNJ));
        if (c->d_part) cudaFree(c->d_part);
        c->d_part = nullptr;
        c->cap_part = 0;
        PM_CUDA(c, cudaMalloc(&c->d_part, cap * sizeof(float)));
        c->cap_part = cap;
    }
    return PM_OK;
}


// Validate the per-call arguments shared by iterate / replan / trace.
pm_status check_call(pm_ctx *c, const float *q0, const float *qd0, const float *T_goal,
                     const float *U, int K, int H, float dt, float lambda, const float *sigma,
                     bool need_lambda)
{
    if (!c->has_grid) return set_err(c, PM_EINVAL, "no distance field set (pm_set_distance_field)");
    if (!q0 || !qd0 || !T_goal || !U || !sigma) return set_err(c, PM_EINVAL, "NULL argument");
    if (K < 1 || K > PM_MAX_ROLLOUTS) return set_err(c, PM_EINVAL, "K=%d out of [1, %d]", K, PM_MAX_ROLLOUTS);
    if (H < 1 || H > PM_MAX_HORIZON) return set_err(c, PM_EINVAL, "H=%d out of [1, %d]", H, PM_MAX_HORIZON);
    if (!std::isfinite(dt) || dt < 0.f) return set_err(c, PM_EINVAL, "dt must be finite and >= 0");
    if (need_lambda && (!std::isfinite(lambda) || !(lambda > 0.f)))
        return set_err(c, PM_EINVAL, "lambda must be finite and > 0");
    if (is_device_ptr(sigma)) return set_err(c, PM_EINVAL, "sigma must be host memory");
    if (!finite_all(sigma, kNJ)) return set_err(c, PM_EINVAL, "sigma has a non-finite entry");
    for (int j = 0; j < kNJ; ++j)
        if (sigma[j] < 0.f) return set_err(c, PM_EINVAL, "sigma must be >= 0");
    if (!is_device_ptr(q0) && !finite_all(q0, kNJ)) return set_err(c, PM_EINVAL, "q0 has a non-finite entry");
    if (!is_device_ptr(qd0) && !finite_all(qd0, kNJ)) return set_err(c, PM_EINVAL, "qd0 has a non-finite entry");
    if (!is_device_ptr(T_goal) && !finite_all(T_goal, 12)) return set_err(c, PM_EINVAL, "T_goal has a non-finite entry");
    return PM_OK;
}

// Pinned staging slots (host and device mirrors): [0, 32) the inputs q0,
// qd0, T_goal; [32, 64) a call's small outputs; [64, ...) U.  Inputs, and U
// when it is on the host, go to the device in one copy; a replan's outputs
// and U come back in one copy.
constexpr int kSlots = 16;
constexpr int kSlotIn = 32;
constexpr int kSlotOut = 32;
constexpr int kSlotFloats = kSlotIn + kSlotOut + kMaxHorizon * kNJ;

struct SlotIO {
    float *d = nullptr;   // device [kSlotOut] outputs, then U
    float *h = nullptr;   // its pinned host mirror
};

// Resolve q0, qd0, T_goal into device pointers: device inputs are used in
// place, host inputs are copied through the next pinned staging slot.  With
// U_host (nU floats), U is staged too, at io->d + kSlotOut.
pm_status stage_inputs(pm_ctx *c, cudaStream_t s, const float *q0, const float *qd0,
                       const float *T_goal, const float *sigma, CallInputs &in,
                       const float *U_host = nullptr, int nU = 0, SlotIO *io = nullptr)
{
    const int k = c->slot;
    c->slot = (c->slot + 1) % kSlots;
    if (c->slot_pending[k]) {
        PM_CUDA(c, cudaEventSynchronize(c->slot_ev[k]));
        c->slot_pending[k] = false;
    }
    float *h = c->h_stage + k * kSlotFloats;
    float *d = c->d_stage + k * kSlotFloats;
    bool any_host = false;
    auto place = [&](const float *src, int n, int off) -> const float * {
        if (is_device_ptr(src)) return src;
        std::memcpy(h + off, src, n * sizeof(float));
        any_host = true;
        return d + off;
    };
    in.q0 = place(q0, kNJ, 0);
    in.qd0 = place(qd0, kNJ, 8);
    in.Tg = place(T_goal, 16, 16);
    for (int j = 0; j < 8; ++j) in.sigma[j] = j < kNJ ? sigma[j] : 0.f;
    size_t n_copy = kSlotIn;
    if (U_host) {
        std::memcpy(h + kSlotIn + kSlotOut, U_host, nU * sizeof(float));
        n_copy = kSlotIn + kSlotOut + nU;
        any_host = true;
    }
    if (io) {
        io->d = d + kSlotIn;
        io->h = h + kSlotIn;
    }
    if (any_host) {
        PM_CUDA(c, cudaMemcpyAsync(d, h, n_copy * sizeof(float), cudaMemcpyHostToDevice, s));
        PM_CUDA(c, cudaEventRecord(c->slot_ev[k], s));
        c->slot_pending[k] = true;
    }
    return PM_OK;
}

// Enqueue one iteration kernel.  Ubar/Uout device [H][7]; costs device or null.
// Enqueue the iteration kernel on nb blocks and, unless tracing, the merge.
pm_status enqueue_iteration(pm_ctx *c, cudaStream_t s, IterKernel fn, int nb, size_t smem,
                            const CallInputs &in, const float *Ubar, float *Uout, float *costs,
                            float *part, float *c0, int K, int H, float dt, float lambda,
                            uint64_t seed, uint32_t iter, bool trace, float *trace_out,
                            unsigned long long *gathers)
{
    IterArgs a{};
    a.in = in;
    a.Ubar = Ubar;
    a.costs = costs;
    a.part = part;
    a.c0 = c0;
    a.trace = trace_out;
    a.gathers = gathers;
    a.noise_dtype = c->noise_dtype;
    a.K = K;
    a.H = H;
    a.cs.seed_lo = static_cast<uint32_t>(seed & 0xffffffffu);
    a.cs.seed_hi = static_cast<uint32_t>(seed >> 32);
    a.cs.iter = iter;
    a.cs.dt = dt;
    a.cs.inv_lambda = trace ? 1.0f : 1.0f / lambda;
    philox_round_keys(a.cs.seed_lo, a.cs.seed_hi, a.rk);
    const bool prof = c->prof && !trace;
    if (prof) {
        while (c->prof_ev.size() < c->prof_used + 2) {
            cudaEvent_t e;
            PM_CUDA(c, cudaEventCreate(&e));
            c->prof_ev.push_back(e);
        }
        PM_CUDA(c, cudaEventRecord(c->prof_ev[c->prof_used], s));
    }
    PM_CUDA(c, launch_dependent(fn, dim3(nb), dim3(kBlock), smem, s, c->rc, grid_const(c), a));
    PM_CUDA(c, cudaGetLastError());
    if (prof) {
        PM_CUDA(c, cudaEventRecord(c->prof_ev[c->prof_used + 1], s));
        c->prof_used += 2;
        c->prof_stream = s;
    }
    if (!trace) {
        const int na = H * kNJ;
        PM_CUDA(c, launch_dependent(softmin_merge_kernel, dim3((na + kMergeRows - 1) / kMergeRows),
                                    dim3(kMergeThreads), 0, s, static_cast<const float *>(part), nb, na,
                                    Ubar, Uout, a.cs.inv_lambda, in.dyn, c0, costs, K));
        PM_CUDA(c, cudaGetLastError());
    }
    return PM_OK;
}

pm_status launch_iteration(pm_ctx *c, cudaStream_t s, const CallInputs &in, const float *Ubar,
                           float *Uout, float *costs, int K, int H, float dt, float lambda,
                           uint64_t seed, uint32_t iter, bool trace, float *trace_out)
{
    TileShape sh;
    pm_status pst = pick_shape(c, H, sh);
    if (pst != PM_OK) return pst;
    KernelPick kp;
    pst = pick_kernel(c, K, sh, trace, kp);
    if (pst != PM_OK) return pst;
    const int nb = static_cast<int>(launch_blocks(K, sh, kp.resident));
    pm_status st = ensure_capacity(c, K, H, nb);
    if (st != PM_OK) return st;
    return enqueue_iteration(c, s, kp.fn, nb, kp.smem, in, Ubar, Uout, costs, c->d_part, c->d_c0, K, H, dt,
                             lambda, seed, iter, trace, trace_out,
                             (c->count_gathers && !trace) ? c->d_gathers : nullptr);
}

cudaStream_t pick_stream(pm_ctx *c, void *s) { return s ? static_cast<cudaStream_t>(s) : c->stream; }

// ------------------------------------------------------------ call graphs
// A call whose inputs and outputs are all host memory (the usual form for a
// controller) is replayed from a CUDA graph captured once per call shape
// (kind, K, H, n_iters, costs wanted): its launches read the inputs and the
// per-call scalars from one fixed device block (g-slot), which the call
// fills by one copy from its pinned mirror before the graph launch; one
// copy after it brings the outputs back.  A call then costs one graph
// launch and two copies on the host instead of 2 (iterate) or
// 2 n_iters + 1 (replan) kernel launches and two copies, which keeps the
// GPU fed when the host is slow.  The kernels are the
// float-field instantiations that read the scalars from that block (DYN),
// with the same arithmetic, tile shape and blocks as a direct launch, so the
// results are bit-identical.
constexpr int kGraphIterate = 1, kGraphReplan = 2;
constexpr int kGOut = 64;   // replan outputs [q 8][qd 8][u0 8][best]
constexpr int kGU = 96;     // U [H][7]
constexpr size_t kGraphSlotFloats = kGU + static_cast<size_t>(kMaxHorizon) * kNJ;
constexpr size_t kMaxGraphs = 32;
static_assert(kDynFloats <= kGOut, "call scalars overlap the outputs");

bool graph_ok(const pm_ctx *c)
{
    return c->graphs_on && !c->prof && !c->count_gathers && c->gd.dtype == PM_F32 && c->rc.n_self_groups == 0;
}

void graphs_clear(pm_ctx *c)
{
    for (auto &g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
}

pm_status graph_capture(pm_ctx *c, int kind, int K, int H, int n_iters, bool costs, cudaGraphExec_t &exec)
{
    TileShape sh;
    pm_status st = pick_shape(c, H, sh);
    if (st != PM_OK) return st;
    KernelPick kp;
    st = pick_kernel(c, K, sh, false, kp);
    if (st != PM_OK) return st;
    const bool dense = kp.fn == lookup_dense_kernel(c->gd.dtype, sh);
    const IterKernel fn = iteration_kernel_f32_dyn(sh.C, sh.L, sh.P, dense);
    if (!fn) return set_err(c, PM_EINTERNAL, "no graph kernel for C=%d L=%d P=%d", sh.C, sh.L, sh.P);
    if (resident_blocks_per_sm(reinterpret_cast<const void *>(fn), kBlock, kp.smem) < 1)
        return set_err(c, PM_ECUDA, "cannot give the graph kernel %zu bytes of shared memory", kp.smem);
    const int nb = static_cast<int>(launch_blocks(K, sh, kp.resident));
    st = ensure_capacity(c, K, H, nb);
    if (st != PM_OK) return st;
    if (!c->d_gslot) PM_CUDA(c, cudaMalloc(&c->d_gslot, kGraphSlotFloats * sizeof(float)));
    if (!c->h_gslot) PM_CUDA(c, cudaMallocHost(&c->h_gslot, kGraphSlotFloats * sizeof(float)));
    if (!c->cap_stream) PM_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));

    float *d = c->d_gslot;
    CallInputs in{};
    in.q0 = d;
    in.qd0 = d + 8;
    in.Tg = d + 16;
    in.dyn = d;
    float *U = d + kGU;
    const size_t nU = static_cast<size_t>(H) * kNJ;
    cudaStream_t s = c->cap_stream;
    PM_CUDA(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    // nothing may return between here and the end of the capture
    pm_status cst = PM_OK;
    cudaError_t e = cudaSuccess;
    for (int it = 0; it < n_iters && e == cudaSuccess && cst == PM_OK; ++it)
        cst = enqueue_iteration(c, s, fn, nb, kp.smem, in, U, U, costs ? c->d_costs : nullptr, c->d_part, c->d_c0,
                                K, H, 0.f, 1.f, 0, static_cast<uint32_t>(it), false, nullptr, nullptr);
    if (e == cudaSuccess && cst == PM_OK) {
        if (kind == kGraphReplan) {
            e = launch_dependent(replan_advance_kernel, dim3(1), dim3(256), 0, s, in.q0, in.qd0, U, H, 0.f,
                                 in.dyn, d + kGOut, d + kGOut + 8, d + kGOut + 16,
                                 static_cast<const float *>(c->d_c0), d + kGOut + 24);
        }
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(s, &graph);
    if (cst != PM_OK || e != cudaSuccess || ee != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (cst != PM_OK) return cst;
        return set_err(c, PM_ECUDA, "graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : ee));
    }
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, PM_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    return PM_OK;
}

// The graph of a call shape, captured on first use (the least recently used
// graph is dropped beyond kMaxGraphs).  A graph is reused only while the
// scratch it captured is still the context's.
pm_status graph_get(pm_ctx *c, int kind, int K, int H, int n_iters, bool costs, cudaGraphExec_t &exec)
{
    for (size_t i = 0; i < c->graphs.size(); ++i) {
        const pm_ctx::Graph &g = c->graphs[i];
        if (g.kind == kind && g.K == K && g.H == H && g.n_iters == n_iters && g.costs == costs &&
            g.gen == c->graph_gen && g.part == c->d_part && g.costs_d == c->d_costs && g.costs_h == c->h_out &&
            g.c0 == c->d_c0) {
            const pm_ctx::Graph hit = g;
            c->graphs.erase(c->graphs.begin() + static_cast<long>(i));
            c->graphs.push_back(hit);
            exec = hit.exec;
            return PM_OK;
        }
    }
    pm_status st = graph_capture(c, kind, K, H, n_iters, costs, exec);
    if (st != PM_OK) return st;
    // scratch growth inside the capture may have moved buffers that older
    // graphs captured: drop those now
    for (size_t i = 0; i < c->graphs.size();) {
        const pm_ctx::Graph &g = c->graphs[i];
        if (g.gen != c->graph_gen || g.part != c->d_part || g.costs_d != c->d_costs || g.costs_h != c->h_out) {
            cudaGraphExecDestroy(g.exec);
            c->graphs.erase(c->graphs.begin() + static_cast<long>(i));
        } else {
            ++i;
        }
    }
    if (c->graphs.size() >= kMaxGraphs) {
        cudaGraphExecDestroy(c->graphs.front().exec);
        c->graphs.erase(c->graphs.begin());
    }
    c->graphs.push_back({kind, K, H, n_iters, costs, c->graph_gen, c->d_part, c->d_costs, c->h_out, c->d_c0, exec});
    return PM_OK;
}

// Inputs and scalars of a host-buffer call into the pinned g-slot.
void graph_fill(pm_ctx *c, const float *q0, const float *qd0, const float *T_goal, const float *sigma, float dt,
                float lambda, uint64_t seed, uint32_t iter0, const float *U, int H)
{
    float *h = c->h_gslot;
    std::memcpy(h, q0, kNJ * sizeof(float));
    std::memcpy(h + 8, qd0, kNJ * sizeof(float));
    std::memcpy(h + 16, T_goal, 16 * sizeof(float));
    for (int j = 0; j < 8; ++j) h[kDynSigma + j] = j < kNJ ? sigma[j] : 0.f;
    h[kDynDt] = dt;
    h[kDynInvLambda] = 1.0f / lambda;
    const uint32_t w[3] = {static_cast<uint32_t>(seed & 0xffffffffu), static_cast<uint32_t>(seed >> 32), iter0};
    std::memcpy(h + kDynSeedLo, w, sizeof(w));
    std::memcpy(h + kGU, U, static_cast<size_t>(H) * kNJ * sizeof(float));
}

} // namespace

int pm::resident_blocks_per_sm(const void *fn, int block, size_t smem)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, size_t>, int> cache;
    static std::unordered_map<const void *, size_t> attr_set;   // dynamic shared memory limit set so far
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_pair(fn, smem);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    if (smem > attr_set[fn]) {
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
            cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        attr_set[fn] = smem;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, smem) != cudaSuccess) {
        cudaGetLastError();
        n = 1;
    }
    n = std::max(n, 1);
    cache[key] = n;
    return n;
}

pm_status pm::finish_distance_field(pm_ctx *c, cudaStream_t s)
{
    const long long items = static_cast<long long>((c->gd.nx - 1 + 29) / 30) * (c->gd.ny - 1) *
                            ((c->gd.nz - 1 + kBoundZ - 1) / kBoundZ);
    const int threads = 128;
    const unsigned blocks = static_cast<unsigned>(std::min<long long>((items + 3) / 4, 32LL * c->n_sm));
    if (c->gd.dtype == PM_F32)
        cell_min_kernel<<<blocks, threads, 0, s>>>(static_cast<const float *>(c->d_grid), c->d_cmin,
                                                  c->gd.nx, c->gd.ny, c->gd.nz);
    else if (c->gd.dtype == PM_F16)
        cell_min_kernel<<<blocks, threads, 0, s>>>(static_cast<const __half *>(c->d_grid), c->d_cmin,
                                                  c->gd.nx, c->gd.ny, c->gd.nz);
    else
        cell_min_kernel<<<blocks, threads, 0, s>>>(static_cast<const __nv_bfloat16 *>(c->d_grid),
                                              c->d_cmin, c->gd.nx, c->gd.ny, c->gd.nz);
    PM_CUDA(c, cudaGetLastError());
    // cell minima into the texture's array
    cudaMemcpy3DParms cp{};
    cp.srcPtr = make_cudaPitchedPtr(c->d_cmin, c->gd.nx * sizeof(float), c->gd.nx - 1, c->gd.ny);
    cp.dstArray = c->cmin_arr;
    cp.extent = make_cudaExtent(c->gd.nx - 1, c->gd.ny - 1, c->gd.nz - 1);
    cp.kind = cudaMemcpyDeviceToDevice;
    PM_CUDA(c, cudaMemcpy3DAsync(&cp, s));
    c->has_grid = true;
    return PM_OK;
}

pm_status pm::replan_with_scratch(pm_ctx *c, cudaStream_t s, const CallInputs &in, float *U, int K, int H,
                                  int n_iters, float dt, float lambda, uint64_t seed, uint32_t iter0,
                                  float *part, size_t part_floats, float *c0, float *q_out, float *qd_out,
                                  float *u0_out, float *best_out)
{
    std::lock_guard<std::mutex> lk(c->mu);
    TileShape sh;
    pm_status st = pick_shape(c, H, sh);
    if (st != PM_OK) return st;
    KernelPick kp;
    st = pick_kernel(c, K, sh, false, kp);
    if (st != PM_OK) return st;
    const IterKernel fn = kp.fn;
    const size_t smem = kp.smem;
    long long nb = launch_blocks(K, sh, kp.resident);
    const size_t per_block = 2 + static_cast<size_t>(H) * kNJ;
    while (nb > 1 && static_cast<size_t>(nb) * per_block > part_floats) --nb;   // fewer, longer blocks
    if (static_cast<size_t>(nb) * per_block > part_floats)
        return set_err(c, PM_EINVAL, "H=%d needs more than %zu floats of partials", H, part_floats);
    for (int it = 0; it < n_iters; ++it) {
        st = enqueue_iteration(c, s, fn, static_cast<int>(nb), smem, in, U, U, nullptr, part, c0, K, H, dt,
                               lambda, seed, iter0 + static_cast<uint32_t>(it), false, nullptr, nullptr);
        if (st != PM_OK) return st;
    }
    PM_CUDA(c, launch_dependent(replan_advance_kernel, dim3(1), dim3(256), 0, s, in.q0, in.qd0, U, H, dt, in.dyn,
                                q_out, qd_out, u0_out, static_cast<const float *>(c0), best_out));
    PM_CUDA(c, cudaGetLastError());
    return PM_OK;
}

// ===================================================================== ABI
extern "C" {

const char *pm_version(void) { return kVersion; }

const char *pm_last_error(pm_ctx *ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

pm_status pm_create(const pm_robot *rb, const pm_grid_desc *gd, const pm_cost_params *cp,
                    int device, pm_ctx **out)
{
    if (!out) return set_err(nullptr, PM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!rb || !gd || !cp) return set_err(nullptr, PM_EINVAL, "NULL robot, grid or costs");
    if (rb->n_joints != kNJ)
        return set_err(nullptr, PM_EINVAL, "n_joints=%d: the library is compiled for a %d-joint chain", rb->n_joints, kNJ);
    const int n = rb->n_joints;
    if (!rb->a || !rb->d || !rb->alpha || !rb->theta_offset || !rb->q_min || !rb->q_max ||
        !rb->qd_max || !rb->qdd_max)
        return set_err(nullptr, PM_EINVAL, "NULL robot array");
    if (!finite_all(rb->a, n) || !finite_all(rb->d, n) || !finite_all(rb->alpha, n) ||
        !finite_all(rb->theta_offset, n) || !std::isfinite(rb->flange_d) ||
        !finite_all(rb->q_min, n) || !finite_all(rb->q_max, n) || !finite_all(rb->qd_max, n) ||
        !finite_all(rb->qdd_max, n))
        return set_err(nullptr, PM_EINVAL, "non-finite robot parameter");
    for (int j = 0; j < n; ++j) {
        if (!(rb->q_min[j] < rb->q_max[j])) return set_err(nullptr, PM_EINVAL, "q_min >= q_max at joint %d", j);
        if (!(rb->qd_max[j] > 0.f) || !(rb->qdd_max[j] > 0.f))
            return set_err(nullptr, PM_EINVAL, "qd_max/qdd_max must be > 0 at joint %d", j);
    }
    if (rb->n_spheres < 0 || rb->n_spheres > PM_MAX_SPHERES)
        return set_err(nullptr, PM_EINVAL, "n_spheres=%d out of [0, %d]", rb->n_spheres, PM_MAX_SPHERES);
    if (rb->n_spheres > 0 && (!rb->sphere_link || !rb->sphere_offset || !rb->sphere_radius))
        return set_err(nullptr, PM_EINVAL, "NULL sphere array");
    for (int s = 0; s < rb->n_spheres; ++s) {
        if (rb->sphere_link[s] < 1 || rb->sphere_link[s] > n)
            return set_err(nullptr, PM_EINVAL, "sphere_link[%d]=%d out of [1, %d]", s, rb->sphere_link[s], n);
        if (!finite_all(rb->sphere_offset + 3 * s, 3) || !std::isfinite(rb->sphere_radius[s]) ||
            rb->sphere_radius[s] < 0.f)
            return set_err(nullptr, PM_EINVAL, "bad sphere %d", s);
    }
    if (rb->n_self_pairs < 0 || rb->n_self_pairs > kMaxSelfPairs)
        return set_err(nullptr, PM_EINVAL, "n_self_pairs=%d out of [0, %d]", rb->n_self_pairs, kMaxSelfPairs);
    if (rb->n_self_pairs > 0 && !rb->self_pairs) return set_err(nullptr, PM_EINVAL, "self_pairs is NULL");
    for (int i = 0; i < rb->n_self_pairs; ++i)
        for (int k = 0; k < 2; ++k)
            if (rb->self_pairs[2 * i + k] < 0 || rb->self_pairs[2 * i + k] >= rb->n_spheres)
                return set_err(nullptr, PM_EINVAL, "self_pairs[%d][%d]=%d is not a sphere", i, k,
                               rb->self_pairs[2 * i + k]);
    if (gd->nx < 2 || gd->ny < 2 || gd->nz < 2)
        return set_err(nullptr, PM_EINVAL, "grid needs >= 2 voxels per axis");
    const size_t elems = static_cast<size_t>(gd->nx) * gd->ny * gd->nz;
    if (elems >= (1ull << 31) - 2ull * gd->nx * gd->ny)
        return set_err(nullptr, PM_EINVAL, "grid too large for 32-bit voxel indexing");
    if (!std::isfinite(gd->res) || !(gd->res > 0.f) || !finite_all(gd->origin, 3))
        return set_err(nullptr, PM_EINVAL, "grid res/origin invalid");
    if (gd->dtype != PM_F32 && gd->dtype != PM_F16 && gd->dtype != PM_BF16)
        return set_err(nullptr, PM_EINVAL, "grid dtype %d unknown", gd->dtype);
    if (!cp->q_ref || !finite_all(cp->q_ref, n) || !finite_all(cp->Q, 6) || !finite_all(cp->QH, 6))
        return set_err(nullptr, PM_EINVAL, "cost params Q/QH/q_ref invalid");
    const float ws[] = {cp->w_env, cp->d_act, cp->w_self, cp->w_q, cp->w_qd, cp->w_qdd,
                        cp->margin_frac, cp->w_s, cp->w_ns};
    for (float w : ws)
        if (!std::isfinite(w) || w < 0.f) return set_err(nullptr, PM_EINVAL, "cost weights must be finite and >= 0");
    if (!(cp->margin_frac < 0.5f)) return set_err(nullptr, PM_EINVAL, "margin_frac must be < 0.5");

    pm_ctx *c = new pm_ctx();
    c->device = device;
    c->gd = *gd;
    c->grid_elems = elems;
    RobotConst &r = c->rc;
    std::memset(&r, 0, sizeof(r));
    // spheres ordered by link (stable); the cost sums over spheres
    std::vector<int> order(rb->n_spheres);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return rb->sphere_link[x] < rb->sphere_link[y]; });
    r.n_spheres = rb->n_spheres;
    for (int i = 0; i <= n + 1; ++i) r.link_begin[i] = 0;
    for (int i = 0; i < rb->n_spheres; ++i) {
        const int s = order[i];
        for (int k = 0; k < 3; ++k) r.sph_off[i][k] = rb->sphere_offset[3 * s + k];
        r.sph_r[i] = rb->sphere_radius[s];
        const double thr = (static_cast<double>(cp->d_act) + rb->sphere_radius[s]) * (1.0 + 1e-6) + 1e-6;
        r.sph_ls[i].y = std::nextafter(static_cast<float>(thr), INFINITY);
    }
    for (int L = 1; L <= n + 1; ++L) {
        int cnt = 0;
        for (int s = 0; s < rb->n_spheres; ++s) cnt += (rb->sphere_link[s] < L);
        r.link_begin[L] = cnt;
    }
    // frames whose sphere offsets lie on one line through the origin: the
    // direction w is the longest offset, lambda_s = o_s . w / |w|^2, and the
    // line is taken when every offset is within 1e-7 |w| (about one float32
    // ulp) of lambda_s w
    for (int j = 0; j < n; ++j) {
        const int b = r.link_begin[j + 1], e = r.link_begin[j + 2];
        double w[3] = {0.0, 0.0, 0.0}, ww = 0.0;
        for (int i = b; i < e; ++i) {
            double o2 = 0.0;
            for (int k = 0; k < 3; ++k) o2 += static_cast<double>(r.sph_off[i][k]) * r.sph_off[i][k];
            if (o2 > ww) {
                ww = o2;
                for (int k = 0; k < 3; ++k) w[k] = r.sph_off[i][k];
            }
        }
        bool line = e > b;
        for (int i = b; i < e && line; ++i) {
            double lam = 0.0;
            if (ww > 0.0) {
                for (int k = 0; k < 3; ++k) lam += static_cast<double>(r.sph_off[i][k]) * w[k];
                lam /= ww;
            }
            double d2 = 0.0;
            for (int k = 0; k < 3; ++k) {
                const double dk = r.sph_off[i][k] - lam * w[k];
                d2 += dk * dk;
            }
            line = d2 <= 1e-14 * ww + 1e-24;
            r.sph_ls[i].x = static_cast<float>(lam);
        }
        r.link_line[j] = line ? 1 : 0;
        double w2 = 0.0;
        for (int k = 0; k < 3; ++k) {
            r.link_w[j][k] = static_cast<float>(w[k]);
            r.link_wg[j][k] = static_cast<float>(w[k] / static_cast<double>(gd->res));
            w2 += static_cast<double>(r.link_w[j][k]) * r.link_w[j][k];
        }
        r.link_w2[j] = static_cast<float>(w2);
    }
    for (int j = 0; j < n; ++j) {
        r.ca[j] = static_cast<float>(std::cos(static_cast<double>(rb->alpha[j])));
        r.sa[j] = static_cast<float>(std::sin(static_cast<double>(rb->alpha[j])));
        r.a[j] = rb->a[j];
        r.d[j] = rb->d[j];
        r.th0[j] = rb->theta_offset[j];
        const double mf = cp->margin_frac;
        const double lo = rb->q_min[j], hi = rb->q_max[j];
        r.q_lo[j] = static_cast<float>(lo + mf * (hi - lo));
        r.q_hi[j] = static_cast<float>(hi - mf * (hi - lo));
        const double v = rb->qd_max[j], acc = rb->qdd_max[j];
        r.qd_lo[j] = static_cast<float>(-v + mf * 2.0 * v);
        r.qd_hi[j] = static_cast<float>(v - mf * 2.0 * v);
        r.qdd_lo[j] = static_cast<float>(-acc + mf * 2.0 * acc);
        r.qdd_hi[j] = static_cast<float>(acc - mf * 2.0 * acc);
        r.q_ref[j] = cp->q_ref[j];
    }
    r.poly = poly_const();
    r.flange_dg = static_cast<float>(static_cast<double>(rb->flange_d) / static_cast<double>(gd->res));
    for (int i = 0; i < kMaxSpheres + kSpherePad; ++i)
        for (int k = 0; k < 3; ++k) r.sph_off_g[i][k] = static_cast<float>(r.sph_off[i][k] / static_cast<double>(gd->res));
    for (int j = 0; j < kNJ; ++j) {
        r.fk_cs[j] = make_float2(r.ca[j], r.sa[j]);
        r.fk_ad[j] = make_float2(static_cast<float>(r.a[j] / static_cast<double>(gd->res)),
                                 static_cast<float>(r.d[j] / static_cast<double>(gd->res)));
        r.fk_tw[j] = make_float2(r.th0[j], r.link_wg[j][0]);
        r.fk_ww[j] = make_float2(r.link_wg[j][1], r.link_wg[j][2]);
        r.fk_be[j] = make_int2(r.link_begin[j + 1], r.link_begin[j + 2]);
    }
    for (int p = 0; p < kNJ / 2; ++p) {
        r.q_lo_pk[p] = make_float2(r.q_lo[2 * p], r.q_lo[2 * p + 1]);
        r.q_hi_pk[p] = make_float2(r.q_hi[2 * p], r.q_hi[2 * p + 1]);
        r.qd_lo_pk[p] = make_float2(r.qd_lo[2 * p], r.qd_lo[2 * p + 1]);
        r.qd_hi_pk[p] = make_float2(r.qd_hi[2 * p], r.qd_hi[2 * p + 1]);
        r.qdd_lo_pk[p] = make_float2(r.qdd_lo[2 * p], r.qdd_lo[2 * p + 1]);
        r.qdd_hi_pk[p] = make_float2(r.qdd_hi[2 * p], r.qdd_hi[2 * p + 1]);
        r.q_ref_pk[p] = make_float2(r.q_ref[2 * p], r.q_ref[2 * p + 1]);
    }
    r.flange_d = rb->flange_d;
    // self-collision set: pairs in internal sphere order, grouped by their
    // frames (fa <= fb); each frame's bounding sphere around its spheres
    std::vector<float4> self_pairs;
    if (cp->w_self > 0.f && rb->n_self_pairs > 0) {
        std::vector<int> inv(rb->n_spheres);
        for (int i = 0; i < rb->n_spheres; ++i) inv[order[i]] = i;
        double lc[kNJ][3] = {}, lr[kNJ] = {};
        for (int j = 0; j < n; ++j) {
            const int b = r.link_begin[j + 1], e = r.link_begin[j + 2];
            if (e == b) continue;
            for (int i = b; i < e; ++i)
                for (int k = 0; k < 3; ++k) lc[j][k] += r.sph_off[i][k] / static_cast<double>(e - b);
            for (int i = b; i < e; ++i) {
                double d2 = 0.0;
                for (int k = 0; k < 3; ++k) d2 += (r.sph_off[i][k] - lc[j][k]) * (r.sph_off[i][k] - lc[j][k]);
                lr[j] = std::max(lr[j], std::sqrt(d2) + r.sph_r[i]);
            }
            for (int k = 0; k < 3; ++k) r.link_c[j][k] = static_cast<float>(lc[j][k]);
        }
        struct P { int fa, fb, a, b; };
        std::vector<P> ps;
        for (int i = 0; i < rb->n_self_pairs; ++i) {
            int a = inv[rb->self_pairs[2 * i]], b = inv[rb->self_pairs[2 * i + 1]];
            int fa = rb->sphere_link[order[a]] - 1, fb = rb->sphere_link[order[b]] - 1;
            if (fa > fb) { std::swap(a, b); std::swap(fa, fb); }
            ps.push_back(P{fa, fb, a, b});
        }
        std::stable_sort(ps.begin(), ps.end(), [](const P &x, const P &y) {
            if (x.fa != y.fa) return x.fa < y.fa;
            if (x.fb != y.fb) return x.fb < y.fb;
            return x.a != y.a ? x.a < y.a : x.b < y.b;
        });
        int g = -1;
        for (size_t i = 0; i < ps.size(); ++i) {
            if (g < 0 || ps[i].fa != r.grp_fa[g] || ps[i].fb != r.grp_fb[g]) {
                ++g;
                r.grp_fa[g] = static_cast<unsigned char>(ps[i].fa);
                r.grp_fb[g] = static_cast<unsigned char>(ps[i].fb);
                r.grp_begin[g] = static_cast<unsigned short>(i);
                // exact skip with a 0.1 mm + 1e-5 relative margin for FP32 rounding
                const double R = lr[ps[i].fa] + lr[ps[i].fb];
                const double thr = R + 1e-4 + 1e-5 * R;
                r.grp_thr2[g] = std::nextafter(static_cast<float>(thr * thr), INFINITY);
            }
            const unsigned ab = static_cast<unsigned>(ps[i].a) | (static_cast<unsigned>(ps[i].b) << 8);
            const float rs = r.sph_r[ps[i].a] + r.sph_r[ps[i].b];
            // apart beyond (r_a + r_b + 1e-5 m)^2, rounded up: sqrt of any larger
            // FP32 squared distance exceeds r_a + r_b
            const double t = static_cast<double>(rs) + 1e-5;
            float bits;
            std::memcpy(&bits, &ab, sizeof(bits));
            self_pairs.push_back(make_float4(bits, rs, std::nextafter(static_cast<float>(t * t), INFINITY), 0.f));
        }
        r.n_self_groups = g + 1;
        r.grp_begin[g + 1] = static_cast<unsigned short>(ps.size());
        // dense groups: exactly the pairs (a, b) of frame fa's x frame fb's
        // spheres, fa != fb, at most kSelfDense spheres each, in (a, b) order
        for (int k = 0; k <= g; ++k) {
            const int fa = r.grp_fa[k], fb = r.grp_fb[k];
            const int a_lo = r.link_begin[fa + 1], na = r.link_begin[fa + 2] - a_lo;
            const int b_lo = r.link_begin[fb + 1], nb = r.link_begin[fb + 2] - b_lo;
            const int p0 = r.grp_begin[k], np = r.grp_begin[k + 1] - p0;
            bool dense = fa != fb && na >= 1 && nb >= 1 && na <= kSelfDense && nb <= kSelfDense && np == na * nb;
            for (int i = 0; dense && i < np; ++i)
                dense = ps[p0 + i].a == a_lo + i / nb && ps[p0 + i].b == b_lo + i % nb;
            r.grp_dense[k] = dense ? 1 : 0;
        }
        // bounding centres on their frame's line: link_c = link_lc link_w
        bool lc_line[kNJ];
        for (int j = 0; j < n; ++j) {
            double ww = 0.0, lam = 0.0, d2 = 0.0;
            for (int k = 0; k < 3; ++k) ww += static_cast<double>(r.link_w[j][k]) * r.link_w[j][k];
            if (ww > 0.0) {
                for (int k = 0; k < 3; ++k) lam += lc[j][k] * r.link_w[j][k];
                lam /= ww;
            }
            for (int k = 0; k < 3; ++k) {
                const double dk = lc[j][k] - lam * r.link_w[j][k];
                d2 += dk * dk;
            }
            r.link_lc[j] = static_cast<float>(lam);
            lc_line[j] = ww > 0.0 && d2 <= 1e-14 * ww + 1e-24;
        }
        bool frames = true;
        for (int k = 0; k <= g; ++k) {
            const int fa = r.grp_fa[k], fb = r.grp_fb[k];
            frames = frames && r.grp_dense[k] && r.link_line[fa] && r.link_line[fb] && lc_line[fa] && lc_line[fb];
        }
        r.self_frames = frames ? 1 : 0;
    }
    for (int i = 0; i < 6; ++i) { r.Q[i] = cp->Q[i]; r.QH[i] = cp->QH[i]; }
    r.w_env = cp->w_env; r.d_act = cp->d_act; r.w_self = cp->w_self;
    r.w_q = cp->w_q; r.w_qd = cp->w_qd; r.w_qdd = cp->w_qdd;
    r.w_s = cp->w_s; r.w_ns = cp->w_ns;

    auto fail = [&](pm_status st) {
        g_err = c->err;
        pm_destroy(c);
        return st;
    };
    DeviceGuard dg(device);
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        set_err(c, PM_ECUDA, "cudaSetDevice(%d): %s", device, cudaGetErrorString(e));
        return fail(PM_ECUDA);
    }
    auto ck = [&](cudaError_t e2, const char *what) -> bool {
        if (e2 == cudaSuccess) return true;
        set_err(c, e2 == cudaErrorMemoryAllocation ? PM_ENOMEM : PM_ECUDA, "%s: %s", what, cudaGetErrorString(e2));
        return false;
    };
    if (!ck(cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device), "SM count") ||
        !ck(cudaStreamCreateWithFlags(&c->stream, cudaStreamDefault), "stream") ||
        !ck(cudaMalloc(&c->d_grid, elems * dtype_size(gd->dtype)), "grid alloc") ||
        !ck(cudaMalloc(&c->d_rc, sizeof(RobotConst)), "robot constants alloc") ||
        !ck(cudaMalloc(&c->d_cmin, elems * sizeof(float)), "cell-minimum alloc") ||
        !ck(cudaMalloc(&c->d_stage, sizeof(float) * kSlots * kSlotFloats), "staging alloc") ||
        !ck(cudaMallocHost(&c->h_stage, sizeof(float) * kSlots * kSlotFloats), "pinned staging alloc") ||
        !ck(cudaMallocHost(&c->h_U, sizeof(float) * kMaxHorizon * kNJ), "pinned U") ||

        !ck(cudaMalloc(&c->d_gathers, sizeof(unsigned long long)), "counter alloc") ||
        !ck(cudaMemset(c->d_gathers, 0, sizeof(unsigned long long)), "counter zero") ||
        !ck(cudaMalloc(&c->d_c0, 96 * sizeof(float)), "c0") ||
        !ck(cudaMemset(c->d_c0, 0, 96 * sizeof(float)), "c0 zero"))
        return fail(c->err.find("alloc") != std::string::npos ? PM_ENOMEM : PM_ECUDA);
    {
        // cell minima: 3-D array + point-sampled, clamped texture
        const cudaChannelFormatDesc fd = cudaCreateChannelDesc<float>();
        if (!ck(cudaMalloc3DArray(&c->cmin_arr, &fd, make_cudaExtent(gd->nx - 1, gd->ny - 1, gd->nz - 1)),
                "cell-minimum array alloc"))
            return fail(PM_ENOMEM);
        cudaResourceDesc rd{};
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = c->cmin_arr;
        cudaTextureDesc td{};
        td.addressMode[0] = td.addressMode[1] = td.addressMode[2] = cudaAddressModeClamp;
        td.filterMode = cudaFilterModePoint;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        if (!ck(cudaCreateTextureObject(&c->cmin_tex, &rd, &td, nullptr), "cell-minimum texture"))
            return fail(PM_ECUDA);
    }
    for (int k = 0; k < kSlots; ++k)
        if (!ck(cudaEventCreateWithFlags(&c->slot_ev[k], cudaEventDisableTiming), "event"))
            return fail(PM_ECUDA);
    if (!self_pairs.empty()) {
        if (!ck(cudaMalloc(&c->d_self_pairs, self_pairs.size() * sizeof(float4)), "self pairs alloc"))
            return fail(PM_ENOMEM);
        if (!ck(cudaMemcpy(c->d_self_pairs, self_pairs.data(), self_pairs.size() * sizeof(float4),
                           cudaMemcpyHostToDevice), "self pairs copy"))
            return fail(PM_ECUDA);
        c->rc.self_pairs = c->d_self_pairs;
    }
    if (!ck(cudaMemcpy(c->d_rc, &c->rc, sizeof(RobotConst), cudaMemcpyHostToDevice), "robot constants copy"))
        return fail(PM_ECUDA);
#ifdef PM_BOUNDS_CHECK
    if (!ck(cudaMalloc(&c->d_err, sizeof(unsigned)), "bounds word") ||
        !ck(cudaMemset(c->d_err, 0, sizeof(unsigned)), "bounds word"))
        return fail(PM_ECUDA);
#endif
    // Load every iteration kernel this context may launch now (modules load
    // lazily by default), so that the first call of a new tile shape or
    // residency does not stall on it; the occupancy of each is cached.
    {
        const bool self = c->rc.n_self_groups > 0;
        for (const TileShape &sh : kShapes) {
            const size_t smem = iteration_smem_bytes(sh.C) + self_smem_bytes(c->rc);
            const IterKernel fns[2] = {lookup_kernel(c->gd.dtype, sh, false, self),
                                       self ? nullptr : lookup_dense_kernel(c->gd.dtype, sh)};
            for (IterKernel fn : fns)
                if (fn) resident_blocks_per_sm(reinterpret_cast<const void *>(fn), kBlock, smem);
        }
    }
    *out = c;
    return PM_OK;
}

pm_status pm_set_distance_field(pm_ctx *c, const float *grid, int grid_is_device)
{
    if (!c) return set_err(nullptr, PM_EINVAL, "ctx is NULL");
    if (!grid) return set_err(c, PM_EINVAL, "grid is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard dg(c->device);
    if (!grid_is_device) {
        for (size_t i = 0; i < c->grid_elems; ++i)
            if (!std::isfinite(grid[i])) return set_err(c, PM_EINVAL, "grid value %zu is not finite", i);
    }
    const cudaMemcpyKind kind = grid_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (c->gd.dtype == PM_F32) {
        PM_CUDA(c, cudaMemcpyAsync(c->d_grid, grid, c->grid_elems * sizeof(float), kind, c->stream));
    } else {
        float *tmp = nullptr;
        PM_CUDA(c, cudaMalloc(&tmp, c->grid_elems * sizeof(float)));
        cudaError_t e = cudaMemcpyAsync(tmp, grid, c->grid_elems * sizeof(float), kind, c->stream);
        if (e == cudaSuccess) {
            convert_grid_kernel<<<4 * c->n_sm, 256, 0, c->stream>>>(tmp, c->d_grid, c->grid_elems, c->gd.dtype);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        cudaFree(tmp);
        PM_CUDA(c, e);
    }
    pm_status st = finish_distance_field(c, c->stream);
    if (st != PM_OK) return st;
    PM_CUDA(c, cudaStreamSynchronize(c->stream));
    return PM_OK;
}

pm_status pm_smpc_iterate(pm_ctx *c, const float *q0, const float *qd0, const float *T_goal,
                          float *U, int K, int H, float dt, float lambda, const float *sigma,
                          uint64_t seed, uint32_t iter_index, float *costs_out, void *cuda_stream)
{
    if (!c) return set_err(nullptr, PM_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard dg(c->device);
    pm_status st = check_call(c, q0, qd0, T_goal, U, K, H, dt, lambda, sigma, true);
    if (st != PM_OK) return st;
    const bool dU = is_device_ptr(U);
    if (!dU && !finite_all(U, H * kNJ)) return set_err(c, PM_EINVAL, "U has a non-finite entry");
    const bool dC = costs_out && is_device_ptr(costs_out);
    cudaStream_t s = pick_stream(c, cuda_stream);
    cudaGraphExec_t ex = nullptr;
    if (graph_ok(c) && !dU && !dC && !is_device_ptr(q0) && !is_device_ptr(qd0) && !is_device_ptr(T_goal) &&
        graph_get(c, kGraphIterate, K, H, 1, costs_out != nullptr, ex) != PM_OK) {
        c->graphs_on = false;      // capture not possible here: launch directly from now on
        graphs_clear(c);
        cudaGetLastError();
        ex = nullptr;
    }
    if (ex) {
        graph_fill(c, q0, qd0, T_goal, sigma, dt, lambda, seed, iter_index, U, H);
        const size_t nU = static_cast<size_t>(H) * kNJ;
        PM_CUDA(c, cudaMemcpyAsync(c->d_gslot, c->h_gslot, (kGU + nU) * sizeof(float), cudaMemcpyHostToDevice, s));
        PM_CUDA(c, cudaGraphLaunch(ex, s));
        PM_CUDA(c, cudaMemcpyAsync(c->h_gslot + kGU, c->d_gslot + kGU, nU * sizeof(float), cudaMemcpyDeviceToHost, s));
        if (costs_out)
            PM_CUDA(c, cudaMemcpyAsync(c->h_out, c->d_costs, static_cast<size_t>(K) * sizeof(float),
                                       cudaMemcpyDeviceToHost, s));
        PM_CUDA(c, cudaStreamSynchronize(s));
        std::memcpy(U, c->h_gslot + kGU, sizeof(float) * nU);
        if (costs_out) std::memcpy(costs_out, c->h_out, sizeof(float) * K);
        return PM_OK;
    }
    st = ensure_capacity(c, K, H, 1);
    if (st != PM_OK) return st;
    // a host U travels with the inputs through the staging slot
    CallInputs in{};
    SlotIO io;
    st = stage_inputs(c, s, q0, qd0, T_goal, sigma, in, dU ? nullptr : U, H * kNJ, &io);
    if (st != PM_OK) return st;
    float *Ud = dU ? U : io.d + kSlotOut;
    float *Cd = costs_out ? (dC ? costs_out : c->d_costs) : nullptr;
    st = launch_iteration(c, s, in, Ud, Ud, Cd, K, H, dt, lambda, seed, iter_index, false, nullptr);
    if (st != PM_OK) return st;
    if (!dU)
        PM_CUDA(c, cudaMemcpyAsync(io.h + kSlotOut, Ud, sizeof(float) * H * kNJ, cudaMemcpyDeviceToHost, s));
    if (costs_out && !dC)
        PM_CUDA(c, cudaMemcpyAsync(c->h_out, c->d_costs, sizeof(float) * K, cudaMemcpyDeviceToHost, s));
    if (!dU || (costs_out && !dC)) {
        PM_CUDA(c, cudaStreamSynchronize(s));
        if (!dU) std::memcpy(U, io.h + kSlotOut, sizeof(float) * H * kNJ);
        if (costs_out && !dC) std::memcpy(costs_out, c->h_out, sizeof(float) * K);
    }
    return PM_OK;
}

pm_status pm_replan(pm_ctx *c, float *q, float *qd, const float *T_goal, float *U, int K, int H,
                    int n_iters, float dt, float lambda, const float *sigma, uint64_t seed,
                    uint32_t replan_index, float *u0_out, float *best_cost, void *cuda_stream)
{
    if (!c) return set_err(nullptr, PM_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard dg(c->device);
    pm_status st = check_call(c, q, qd, T_goal, U, K, H, dt, lambda, sigma, true);
    if (st != PM_OK) return st;
    if (n_iters < 1 || n_iters > 1024) return set_err(c, PM_EINVAL, "n_iters=%d out of [1, 1024]", n_iters);
    const bool dU = is_device_ptr(U);
    if (!dU && !finite_all(U, H * kNJ)) return set_err(c, PM_EINVAL, "U has a non-finite entry");
    const bool dq = is_device_ptr(q), dqd = is_device_ptr(qd);
    const bool du0 = u0_out && is_device_ptr(u0_out), dbest = best_cost && is_device_ptr(best_cost);
    cudaStream_t s = pick_stream(c, cuda_stream);
    cudaGraphExec_t ex = nullptr;
    if (graph_ok(c) && !dU && !dq && !dqd && !du0 && !dbest && !is_device_ptr(T_goal) &&
        graph_get(c, kGraphReplan, K, H, n_iters, false, ex) != PM_OK) {
        c->graphs_on = false;      // capture not possible here: launch directly from now on
        graphs_clear(c);
        cudaGetLastError();
        ex = nullptr;
    }
    if (ex) {
        graph_fill(c, q, qd, T_goal, sigma, dt, lambda, seed, replan_index * static_cast<uint32_t>(n_iters), U, H);
        const size_t nU = static_cast<size_t>(H) * kNJ;
        PM_CUDA(c, cudaMemcpyAsync(c->d_gslot, c->h_gslot, (kGU + nU) * sizeof(float), cudaMemcpyHostToDevice, s));
        PM_CUDA(c, cudaGraphLaunch(ex, s));
        PM_CUDA(c, cudaMemcpyAsync(c->h_gslot + kGOut, c->d_gslot + kGOut, (kGU - kGOut + nU) * sizeof(float),
                                   cudaMemcpyDeviceToHost, s));
        PM_CUDA(c, cudaStreamSynchronize(s));
        const float *h = c->h_gslot + kGOut;
        std::memcpy(q, h, kNJ * sizeof(float));
        std::memcpy(qd, h + 8, kNJ * sizeof(float));
        if (u0_out) std::memcpy(u0_out, h + 16, kNJ * sizeof(float));
        if (best_cost) *best_cost = h[24];
        std::memcpy(U, c->h_gslot + kGU, sizeof(float) * H * kNJ);
        return PM_OK;
    }
    st = ensure_capacity(c, K, H, 1);
    if (st != PM_OK) return st;
    CallInputs in{};
    SlotIO io;
    st = stage_inputs(c, s, q, qd, T_goal, sigma, in, dU ? nullptr : U, H * kNJ, &io);
    if (st != PM_OK) return st;
    float *Ud = dU ? U : io.d + kSlotOut;
    for (int it = 0; it < n_iters; ++it) {
        st = launch_iteration(c, s, in, Ud, Ud, nullptr, K, H, dt, lambda, seed,
                              replan_index * static_cast<uint32_t>(n_iters) + static_cast<uint32_t>(it),
                              false, nullptr);
        if (st != PM_OK) return st;
    }
    float *small = io.d;  // [q 8][qd 8][u0 8][min S] for host outputs, then U when staged
    PM_CUDA(c, launch_dependent(replan_advance_kernel, dim3(1), dim3(256), 0, s, in.q0, in.qd0, Ud, H, dt,
                                static_cast<const float *>(nullptr), dq ? q : small, dqd ? qd : small + 8,
                                u0_out ? (du0 ? u0_out : small + 16) : static_cast<float *>(nullptr),
                                static_cast<const float *>(c->d_c0),
                                best_cost ? (dbest ? best_cost : small + 24) : static_cast<float *>(nullptr)));
    PM_CUDA(c, cudaGetLastError());
    const bool host_out = !dU || !dq || !dqd || (u0_out && !du0) || (best_cost && !dbest);
    if (host_out) {
        const float *h = io.h;
        const size_t n_back = kSlotOut + (dU ? 0 : static_cast<size_t>(H) * kNJ);
        PM_CUDA(c, cudaMemcpyAsync(io.h, io.d, n_back * sizeof(float), cudaMemcpyDeviceToHost, s));
        PM_CUDA(c, cudaStreamSynchronize(s));
        if (!dq) std::memcpy(q, h, kNJ * sizeof(float));
        if (!dqd) std::memcpy(qd, h + 8, kNJ * sizeof(float));
        if (u0_out && !du0) std::memcpy(u0_out, h + 16, kNJ * sizeof(float));
        if (best_cost && !dbest) *best_cost = h[24];
        if (!dU) std::memcpy(U, h + kSlotOut, sizeof(float) * H * kNJ);
    }
    return PM_OK;
}

pm_status pm_plan_episode(pm_ctx *c, const float *q0, const float *qd0, const float *T_goal, const float *U0,
                          int K, int H, int n_iters, float dt, float lambda, const float *sigma, uint64_t seed,
                          const pm_converge_cfg *cfg, float *q_final, float *qd_final, pm_episode *out,
                          float *log, void *cuda_stream)
{
    if (!c) return set_err(nullptr, PM_EINVAL, "ctx is NULL");
    if (!cfg || !out) return set_err(c, PM_EINVAL, "NULL cfg or out");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard dg(c->device);
    const float Uchk = 0.f;
    pm_status st = check_call(c, q0, qd0, T_goal, U0 ? U0 : &Uchk, K, H, dt, lambda, sigma, true);
    if (st != PM_OK) return st;
    if (n_iters < 1 || n_iters > 1024) return set_err(c, PM_EINVAL, "n_iters=%d out of [1, 1024]", n_iters);
    if (cfg->max_replans < 1 || cfg->n_stable < 1 || !std::isfinite(cfg->pos_tol) || !(cfg->pos_tol > 0.f) ||
        !std::isfinite(cfg->rel_tol) || cfg->rel_tol < 0.f)
        return set_err(c, PM_EINVAL, "bad convergence settings");
    if (U0 && !is_device_ptr(U0) && !finite_all(U0, H * kNJ)) return set_err(c, PM_EINVAL, "U0 has a non-finite entry");
    cudaStream_t s = pick_stream(c, cuda_stream);
    st = ensure_capacity(c, K, H, 1);
    if (st != PM_OK) return st;
    // device state: q [48, 56), qd [56, 64), goal [64, 80), metrics [80, 84) of the small scratch
    float *dq = c->d_c0 + 48, *dqd = c->d_c0 + 56, *dT = c->d_c0 + 64, *dm = c->d_c0 + 80;
    const cudaMemcpyKind k_q = is_device_ptr(q0) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind k_qd = is_device_ptr(qd0) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind k_T = is_device_ptr(T_goal) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (k_q == cudaMemcpyHostToDevice && !finite_all(q0, kNJ)) return set_err(c, PM_EINVAL, "q0 not finite");
    PM_CUDA(c, cudaMemcpyAsync(dq, q0, kNJ * sizeof(float), k_q, s));
    PM_CUDA(c, cudaMemcpyAsync(dqd, qd0, kNJ * sizeof(float), k_qd, s));
    PM_CUDA(c, cudaMemcpyAsync(dT, T_goal, 16 * sizeof(float), k_T, s));
    float *Ud = c->d_U;
    if (U0) PM_CUDA(c, cudaMemcpyAsync(Ud, U0, sizeof(float) * H * kNJ,
                                       is_device_ptr(U0) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    else PM_CUDA(c, cudaMemsetAsync(Ud, 0, sizeof(float) * H * kNJ, s));   // Algorithm 1 initialisation
    CallInputs in{};
    in.q0 = dq;
    in.qd0 = dqd;
    in.Tg = dT;
    for (int j = 0; j < 8; ++j) in.sigma[j] = j < kNJ ? sigma[j] : 0.f;
    pm_episode ep{};
    float *h = c->h_out;
    float prev_best = 0.f;
    int stable = 0;
    for (int t = 0; t < cfg->max_replans; ++t) {
        for (int it = 0; it < n_iters; ++it) {
            st = launch_iteration(c, s, in, Ud, Ud, nullptr, K, H, dt, lambda, seed,
                                  static_cast<uint32_t>(t) * static_cast<uint32_t>(n_iters) + static_cast<uint32_t>(it),
                                  false, nullptr);
            if (st != PM_OK) return st;
        }
        PM_CUDA(c, launch_dependent(episode_step_kernel, dim3(1), dim3(256), 0, s, c->rc,
                                    static_cast<const float *>(dT), dq, dqd, Ud, H, dt,
                                    static_cast<const float *>(c->d_c0), dm));
        PM_CUDA(c, cudaMemcpyAsync(h, dm, 4 * sizeof(float), cudaMemcpyDeviceToHost, s));
        PM_CUDA(c, cudaStreamSynchronize(s));
        ep.replans = t + 1;
        ep.e_pos = h[0];
        ep.e_ori = h[1];
        ep.best_cost = h[2];
        ep.path_length += h[3];
        if (log) {
            log[4 * t] = h[0];
            log[4 * t + 1] = h[1];
            log[4 * t + 2] = h[2];
            log[4 * t + 3] = ep.path_length;
        }
        // convergence (Sec. V-A): relative improvement of the objective below
        // rel_tol and position error below pos_tol, n_stable replans in a row
        const bool small_gain = t > 0 && (prev_best - h[2]) < cfg->rel_tol * std::fabs(prev_best);
        stable = (small_gain && h[0] < cfg->pos_tol) ? stable + 1 : 0;
        prev_best = h[2];
        if (stable >= cfg->n_stable) {
            ep.converged = 1;
            break;
        }
    }
    ep.motion_time = static_cast<float>(ep.replans) * dt;
    PM_CUDA(c, cudaMemcpyAsync(h, dq, 16 * sizeof(float), cudaMemcpyDeviceToHost, s));
    PM_CUDA(c, cudaStreamSynchronize(s));
    if (q_final) {
        if (is_device_ptr(q_final)) PM_CUDA(c, cudaMemcpy(q_final, dq, kNJ * sizeof(float), cudaMemcpyDeviceToDevice));
        else std::memcpy(q_final, h, kNJ * sizeof(float));
    }
    if (qd_final) {
        if (is_device_ptr(qd_final)) PM_CUDA(c, cudaMemcpy(qd_final, dqd, kNJ * sizeof(float), cudaMemcpyDeviceToDevice));
        else std::memcpy(qd_final, h + 8, kNJ * sizeof(float));
    }
    *out = ep;
    return PM_OK;
}

pm_status pm_rollout_trace(pm_ctx *c, const float *q0, const float *qd0, const float *T_goal,
                           const float *U, int K, int H, float dt, const float *sigma,
                           uint64_t seed, uint32_t iter_index, float *trace)
{
    if (!c) return set_err(nullptr, PM_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard dg(c->device);
    pm_status st = check_call(c, q0, qd0, T_goal, U, K, H, dt, 1.0f, sigma, false);
    if (st != PM_OK) return st;
    if (!trace || !is_device_ptr(trace)) return set_err(c, PM_EINVAL, "trace must be device memory");
    cudaStream_t s = c->stream;
    st = ensure_capacity(c, K, H, 1);
    if (st != PM_OK) return st;
    CallInputs in{};
    st = stage_inputs(c, s, q0, qd0, T_goal, sigma, in);
    if (st != PM_OK) return st;
    const float *Ud = U;
    if (!is_device_ptr(U)) {
        std::memcpy(c->h_U, U, sizeof(float) * H * kNJ);
        PM_CUDA(c, cudaMemcpyAsync(c->d_U, c->h_U, sizeof(float) * H * kNJ, cudaMemcpyHostToDevice, s));
        Ud = c->d_U;
    }
    PM_CUDA(c, cudaMemsetAsync(trace, 0, sizeof(float) * static_cast<size_t>(K) * (H + 1) * kTraceCols, s));
    st = launch_iteration(c, s, in, Ud, nullptr, nullptr, K, H, dt, 1.0f, seed, iter_index, true, trace);
    if (st != PM_OK) return st;
    PM_CUDA(c, cudaStreamSynchronize(s));
    return PM_OK;
}

pm_status pm_fp32_fma_peak(int device, double *tflops)
{
    if (!tflops) return PM_EINVAL;
    DeviceGuard dg(device);
    if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return PM_ECUDA; }
    int n_sm = 0;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        return PM_ECUDA;
    }
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t s = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(float));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    const int blocks = 8 * n_sm, threads = 256, iters = 8192;
    double best_ms = 1e30;
    for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, s);
        fma_peak_kernel<<<blocks, threads, 0, s>>>(sink, iters, 0.999999f, 1e-7f);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best_ms = std::min(best_ms, static_cast<double>(ms));   // first launch warms up
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (s) cudaStreamDestroy(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PM_ECUDA;
    }
    const double flops = 2.0 * 8.0 * iters * static_cast<double>(blocks) * threads;
    *tflops = flops / (best_ms * 1e-3) / 1e12;
    return PM_OK;
}

pm_status pm_philox4x32_10(const uint32_t *ctr, uint64_t key, uint32_t *out, size_t n, void *cuda_stream)
{
    if (!ctr || !out) return set_err(nullptr, PM_EINVAL, "NULL argument");
    if (n == 0) return PM_OK;
    if (!is_device_ptr(ctr) || !is_device_ptr(out)) return set_err(nullptr, PM_EINVAL, "ctr/out must be device memory");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const unsigned blocks = static_cast<unsigned>(std::min<size_t>((n + 255) / 256, 65535));
    philox_words_kernel<<<blocks, 256, 0, s>>>(ctr, static_cast<uint32_t>(key & 0xffffffffu),
                                               static_cast<uint32_t>(key >> 32), out, n);
    PM_CUDA(nullptr, cudaGetLastError());
    return PM_OK;
}

pm_status pm_pose_error(const float *T_goal, const float *T, float *xi, size_t n, void *cuda_stream)
{
    if (!T_goal || !T || !xi) return set_err(nullptr, PM_EINVAL, "NULL argument");
    if (n == 0) return PM_OK;
    if (!is_device_ptr(T_goal) || !is_device_ptr(T) || !is_device_ptr(xi))
        return set_err(nullptr, PM_EINVAL, "T_goal/T/xi must be device memory");
    const unsigned blocks = static_cast<unsigned>(std::min<size_t>((n + 127) / 128, 65535));
    pose_error_kernel<<<blocks, 128, 0, static_cast<cudaStream_t>(cuda_stream)>>>(T_goal, T, xi, n);
    PM_CUDA(nullptr, cudaGetLastError());
    return PM_OK;
}

pm_status pm_joint_sincos(const float *x, float *sc, float *sc_ref, size_t n, void *cuda_stream)
{
    if (!x || !sc) return set_err(nullptr, PM_EINVAL, "NULL argument");
    if (n == 0) return PM_OK;
    if (!is_device_ptr(x) || !is_device_ptr(sc) || (sc_ref && !is_device_ptr(sc_ref)))
        return set_err(nullptr, PM_EINVAL, "x/sc/sc_ref must be device memory");
    const PolyConst kp = poly_const();
    const unsigned blocks = static_cast<unsigned>(std::min<size_t>((n + 127) / 128, 65535));
    joint_sincos_kernel<<<blocks, 128, 0, static_cast<cudaStream_t>(cuda_stream)>>>(x, sc, sc_ref, n, kp);
    PM_CUDA(nullptr, cudaGetLastError());
    return PM_OK;
}

pm_status pm_sample_noise(int K, int H, const float *sigma, uint64_t seed, uint32_t iter_index,
                          float *eps, void *cuda_stream)
{
    if (!sigma || !eps) return set_err(nullptr, PM_EINVAL, "NULL argument");
    if (K < 1 || H < 1 || K > PM_MAX_ROLLOUTS || H > PM_MAX_HORIZON) return set_err(nullptr, PM_EINVAL, "K/H out of range");
    if (!is_device_ptr(eps)) return set_err(nullptr, PM_EINVAL, "eps must be device memory");
    if (is_device_ptr(sigma) || !finite_all(sigma, kNJ)) return set_err(nullptr, PM_EINVAL, "sigma must be finite host memory");
    Sigma sg{};
    for (int j = 0; j < kNJ; ++j) sg.s[j] = sigma[j];
    const size_t total = static_cast<size_t>(K) * H;
    const unsigned blocks = static_cast<unsigned>(std::min<size_t>((total + 255) / 256, 65535));
    const PolyConst kp = poly_const();
    sample_noise_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
        K, H, sg, static_cast<uint32_t>(seed & 0xffffffffu), static_cast<uint32_t>(seed >> 32), iter_index, eps, kp);
    PM_CUDA(nullptr, cudaGetLastError());
    return PM_OK;
}

pm_status pm_profile_enable(pm_ctx *c, int flags)
{
    if (!c) return set_err(nullptr, PM_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    c->prof = (flags & PM_PROFILE_TIME) != 0;
    c->count_gathers = (flags & PM_PROFILE_GATHERS) != 0;
    return PM_OK;
}

pm_status pm_profile_gathers(pm_ctx *c, uint64_t *gathers, int reset)
{
    if (!c) return set_err(nullptr, PM_EINVAL, "ctx is NULL");
    if (!gathers) return set_err(c, PM_EINVAL, "NULL output");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard dg(c->device);
    unsigned long long v = 0;
    PM_CUDA(c, cudaMemcpy(&v, c->d_gathers, sizeof(v), cudaMemcpyDeviceToHost));
    *gathers = v;
    if (reset) PM_CUDA(c, cudaMemset(c->d_gathers, 0, sizeof(unsigned long long)));
    return PM_OK;
}

pm_status pm_set_noise_dtype(pm_ctx *c, int dtype)
{
    if (!c) return set_err(nullptr, PM_EINVAL, "ctx is NULL");
    if (dtype != PM_F32 && dtype != PM_F16 && dtype != PM_BF16)
        return set_err(c, PM_EINVAL, "noise dtype %d unknown", dtype);
    std::lock_guard<std::mutex> lk(c->mu);
    c->noise_dtype = dtype;
    ++c->graph_gen;
    return PM_OK;
}

int pm_bounds_checked(void)
{
#ifdef PM_BOUNDS_CHECK
    return 1;
#else
    return 0;
#endif
}

pm_status pm_bounds_status(pm_ctx *c, unsigned *word, int reset)
{
    if (!c || !word) return set_err(c, PM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard dg(c->device);
    *word = 0;
    if (!c->d_err) return PM_OK;
    PM_CUDA(c, cudaDeviceSynchronize());
    PM_CUDA(c, cudaMemcpy(word, c->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (reset) PM_CUDA(c, cudaMemset(c->d_err, 0, sizeof(unsigned)));
    return PM_OK;
}

pm_status pm_set_call_graphs(pm_ctx *c, int enable)
{
    if (!c) return set_err(nullptr, PM_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard dg(c->device);
    c->graphs_on = enable != 0;
    if (!c->graphs_on) graphs_clear(c);
    return PM_OK;
}

pm_status pm_set_tile_shape(pm_ctx *c, int C, int L, int P)
{
    if (!c) return set_err(nullptr, PM_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    const TileShape t{C, L, P};
    if (C == 0 && L == 0 && P == 0) {
        c->forced = t;
        ++c->graph_gen;
        return PM_OK;
    }
    if (!shape_known(t)) return set_err(c, PM_EINVAL, "no kernel for tile shape C=%d L=%d P=%d", C, L, P);
    c->forced = t;
    ++c->graph_gen;
    return PM_OK;
}

pm_status pm_profile_read(pm_ctx *c, double *total_ms, uint64_t *launches, int reset)
{
    if (!c) return set_err(nullptr, PM_EINVAL, "ctx is NULL");
    if (!total_ms || !launches) return set_err(c, PM_EINVAL, "NULL output");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard dg(c->device);
    double tot = 0.0;
    for (size_t i = 0; i + 1 < c->prof_used; i += 2) {
        PM_CUDA(c, cudaEventSynchronize(c->prof_ev[i + 1]));
        float ms = 0.f;
        PM_CUDA(c, cudaEventElapsedTime(&ms, c->prof_ev[i], c->prof_ev[i + 1]));
        tot += ms;
    }
    *total_ms = tot;
    *launches = c->prof_used / 2;
    if (reset) c->prof_used = 0;
    return PM_OK;
}

void pm_destroy(pm_ctx *c)
{
    if (!c) return;
    {
        DeviceGuard dg(c->device);
        if (c->stream) cudaStreamSynchronize(c->stream);
        cudaFree(c->d_grid);
        cudaFree(c->d_rc);
        cudaFree(c->d_map_occ);
        cudaFree(c->d_map_a);
        cudaFree(c->d_map_b);
        cudaFree(c->d_phi_table);
        cudaFree(c->d_mask_spheres);
        cudaFree(c->d_self_pairs);
        cudaFree(c->d_cmin);
        if (c->cmin_tex) cudaDestroyTextureObject(c->cmin_tex);
        if (c->cmin_arr) cudaFreeArray(c->cmin_arr);
        cudaFree(c->d_stage);
        cudaFreeHost(c->h_stage);
        cudaFreeHost(c->h_U);
        cudaFree(c->d_U);
        cudaFree(c->d_costs);
        cudaFreeHost(c->h_out);
        cudaFree(c->d_part);

        cudaFree(c->d_c0);
        cudaFree(c->d_err);
        cudaFree(c->d_gathers);
        graphs_clear(c);
        cudaFree(c->d_gslot);
        cudaFreeHost(c->h_gslot);
        if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
        for (cudaEvent_t e : c->slot_ev)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
        if (c->stream) cudaStreamDestroy(c->stream);
    }
    delete c;
}

} // extern "C"

// ============================================================ no-allocation
// pm_smpc_iterate_noalloc: the same iteration kernel, with its scratch
// (the block partials of the soft-min merge and the k = 0 state term) in one file-scope device array instead of memory the
// context allocates on demand.  It is for callers that must not allocate
// device memory once they are running -- for instance a fixed-rate control
// loop that forbids allocation after start-up, or a process whose device
// memory is fully reserved by another allocator.
namespace {

constexpr size_t kStaticScratchFloats = 512 * 1024;   // 2 MiB, held by every GPU that loads us
constexpr size_t kStaticHeaderFloats = 64;            // c0 [0, 2); partials start 256-B aligned

static __device__ __align__(256) float g_static_scratch[kStaticScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
float *g_static_addr[kMaxDevices] = {};

// Device address of g_static_scratch on `device` (the caller made it current).
// Resolved once per device and cached.
pm_status static_scratch(pm_ctx *c, int device, float **out)
{
    if (device < 0 || device >= kMaxDevices) return set_err(c, PM_EINVAL, "device %d out of range", device);
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return set_err(c, PM_ECUDA, "cudaGetSymbolAddress(static scratch) on device %d: %s", device,
                           cudaGetErrorString(e));
        g_static_addr[device] = static_cast<float *>(p);
    }
    *out = g_static_addr[device];
    return PM_OK;
}

// Blocks of a launch whose partials live in the static array: fewer, longer
// running blocks when nb blocks' partials would not fit; 0 if none fits.
long long static_blocks(long long nb, int H)
{
    const size_t per_block = 2 + static_cast<size_t>(H) * kNJ;
    auto fits = [&](long long n) { return kStaticHeaderFloats + static_cast<size_t>(n) * per_block <= kStaticScratchFloats; };
    while (nb > 1 && !fits(nb)) --nb;
    return fits(nb) ? nb : 0;
}

} // namespace

extern "C" pm_status pm_smpc_iterate_noalloc(pm_ctx *c, const float *q0, const float *qd0,
                                             const float *T_goal, float *U, int K, int H, float dt,
                                             float lambda, const float *sigma, uint64_t seed,
                                             uint32_t iter_index, float *costs_out, void *cuda_stream)
{
    if (!c) return set_err(nullptr, PM_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard dg(c->device);
    pm_status st = check_call(c, q0, qd0, T_goal, U, K, H, dt, lambda, sigma, true);
    if (st != PM_OK) return st;
    if (!is_device_ptr(q0) || !is_device_ptr(qd0) || !is_device_ptr(T_goal) || !is_device_ptr(U) ||
        (costs_out && !is_device_ptr(costs_out)))
        return set_err(c, PM_EINVAL, "pm_smpc_iterate_noalloc needs q0, qd0, T_goal, U and costs_out in device memory");
    float *scratch = nullptr;
    st = static_scratch(c, c->device, &scratch);
    if (st != PM_OK) return st;

    TileShape sh;
    st = pick_shape(c, H, sh);
    if (st != PM_OK) return st;
    KernelPick kp;
    st = pick_kernel(c, K, sh, false, kp);
    if (st != PM_OK) return st;
    const IterKernel fn = kp.fn;
    const size_t smem = kp.smem;
    const long long nb = static_blocks(launch_blocks(K, sh, kp.resident), H);
    if (nb < 1)
        return set_err(c, PM_EINVAL, "H=%d needs more than the %zu-float static scratch", H, kStaticScratchFloats);

    cudaStream_t s = pick_stream(c, cuda_stream);
    CallInputs in{};
    in.q0 = q0;
    in.qd0 = qd0;
    in.Tg = T_goal;
    for (int j = 0; j < 8; ++j) in.sigma[j] = j < kNJ ? sigma[j] : 0.f;
    // every word of the array that the kernels read is written earlier in the
    // same call (partials by the iteration kernel, c0 by its first warp), so
    // nothing has to be cleared between calls
    return enqueue_iteration(c, s, fn, static_cast<int>(nb), smem, in, U, U, costs_out,
                             scratch + kStaticHeaderFloats, scratch, K, H, dt, lambda, seed,
                             iter_index, false, nullptr, nullptr);
}

extern "C" pm_status pm_launch_plan(pm_ctx *c, int K, int H, int noalloc, int out[4])
{
    if (!c || !out) return set_err(c, PM_EINVAL, "NULL argument");
    if (K < 1 || H < 1 || K > PM_MAX_ROLLOUTS || H > PM_MAX_HORIZON)
        return set_err(c, PM_EINVAL, "K=%d / H=%d out of range", K, H);
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard dg(c->device);
    TileShape sh;
    pm_status st = pick_shape(c, H, sh);
    if (st != PM_OK) return st;
    KernelPick kp;
    st = pick_kernel(c, K, sh, false, kp);
    if (st != PM_OK) return st;
    long long nb = launch_blocks(K, sh, kp.resident);
    if (noalloc) nb = static_blocks(nb, H);
    out[0] = sh.C;
    out[1] = sh.L;
    out[2] = sh.P;
    out[3] = static_cast<int>(nb);
    return PM_OK;
}
