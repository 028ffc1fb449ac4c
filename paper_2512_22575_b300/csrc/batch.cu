// Batched SMPC iterations over many arms (contexts) in one persistent launch.
//
// A batch holds instances of different K, H and distance fields.  Each
// instance is cut into nb_i "local blocks" (its share of the work in units
// of one thread block, each running the same per-block roll-out loop as the
// single-instance kernel); the (instance, local block) items form a work
// list, heaviest instances first, that a persistent grid pulls from an
// atomic counter.  Because every item's tiles and block partial belong to
// one instance, the per-instance soft-min merge is the same as for a single
// call.  Tile shape and nb_i per instance make up a plan; plans are chosen
// by an autotuner (timed candidates) or a work-proportional default and
// cached per batch structure; a structure's sequence of launches can be
// captured once as a CUDA graph and replayed.
#include "ctx_internal.h"
#include "softmin_merge.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <sstream>

using namespace pm;

namespace pm {

constexpr int kBatchCMax = 4;                         // C of the widest shape in a batch
constexpr int kBatchMaxSteps = kBatchCMax * 32 * 2;   // C * L * P of that shape

struct BatchInstance {
    const RobotConst *rc;     // the arm's constants (device copy kept by its context)
    GridConst g;
    CallInputs in;            // q0, qd0, T_goal (device), sigma
    TileJob job;              // job.iter: index of the first iteration of the call
    float *Uout;              // [H][7] (= job.Ubar, updated in place)
    float *c0;                // [2]: k = 0 terms, min S
    float *q_out, *qd_out, *u0_out, *best_out;   // replan outputs (device) or null
    int C, L, P;
};

struct BatchArgs {
    const BatchInstance *inst;
    const int2 *work;         // (instance, local block)
    int n_work;
    unsigned *queue;          // next work item, zero at launch
    uint32_t it;              // iteration offset added to every instance's iter
};

template <typename GT, bool SELF>
__global__ void __launch_bounds__(kBlock, 4) smpc_batch_kernel(const __grid_constant__ BatchArgs ba)
{
    extern __shared__ float s_dyn[];
    __shared__ RobotConst s_rc;
    __shared__ BatchInstance s_inst;
    __shared__ __align__(16) float s_tot[kWarps / 2 + 1][2 * kNJ];
    __shared__ float s_S[kWarps / 2 + 1][2][2];
    __shared__ float s_state[kStateFloats];
    __shared__ float s_blk[kBatchMaxSteps * kNJ];
    __shared__ float s_wm[kWarps], s_wz[kWarps];
    __shared__ float4 s_grp[SELF ? kMaxSelfGroups * kSelfGroupRec : 1];
    __shared__ int s_item;
    const int tid = threadIdx.x;
    grid_dependency_prologue();

    int cur = -1;          // the instance whose descriptor, constants and state are in shared memory
    for (;;) {
        __syncthreads();   // the previous item is done with shared memory
        if (tid == 0) s_item = static_cast<int>(atomicAdd(ba.queue, 1u));
        __syncthreads();
        const int item = s_item;
        if (item >= ba.n_work) return;
        const int2 w = ba.work[item];
        // items come instance by instance, so a block's next item is mostly
        // of the same instance: then its shared copies are kept
        if (w.x != cur) {
            {
                const int *src = reinterpret_cast<const int *>(ba.inst + w.x);
                int *dst = reinterpret_cast<int *>(&s_inst);
                for (int i = tid; i < static_cast<int>(sizeof(BatchInstance) / 4); i += kBlock) dst[i] = src[i];
            }
            __syncthreads();
            {
                const int *src = reinterpret_cast<const int *>(s_inst.rc);
                int *dst = reinterpret_cast<int *>(&s_rc);
                for (int i = tid; i < static_cast<int>(sizeof(RobotConst) / 4); i += kBlock) dst[i] = __ldg(src + i);
            }
            load_state(s_inst.in, CallScalars{s_inst.job.seed_lo, s_inst.job.seed_hi, s_inst.job.iter, s_inst.job.dt, s_inst.job.inv_lambda}, s_state);
            __syncthreads();
            if (SELF && s_rc.n_self_groups > 0 && s_rc.self_frames) {
                build_self_groups(s_rc, s_inst.g, s_grp);
                __syncthreads();
            }
            cur = w.x;
        }
        const InstanceState &st = *reinterpret_cast<const InstanceState *>(s_state);
        TileJob job = s_inst.job;
        job.iter += ba.it;
        job.c0 = s_inst.c0;
        const int C = s_inst.C;
        BlockSmem sm{s_dyn, s_dyn + kWarps * C * kNJ * 32, s_tot, s_S, s_blk, s_wm, s_wz,
                     (SELF && s_rc.n_self_groups > 0) ? s_dyn + 2 * kWarps * kBatchCMax * kNJ * 32 : nullptr,
                     nullptr, (SELF && s_rc.n_self_groups > 0 && s_rc.self_frames) ? s_grp : nullptr};
        unsigned ngath = 0;
        run_block<GT, false, SELF, false>(s_rc, s_inst.g, st, job, nullptr, C, s_inst.L, s_inst.P, w.y, sm, ngath);
    }
}

// The same work list when every item has a one-step shape ((1,16,1),
// (1,32,1) or (1,32,2): H <= 64, the default shapes up to there): with one
// step per lane fixed at compile time, each step's state is staged in
// shared memory as in the single-instance kernel, and the kernel is fitted
// to MINB blocks per SM (the run-time-shape kernel above holds 4).  The
// block loop exists twice: with L = 32 folded (P at run time) for the
// (1,32,1) and (1,32,2) items, and with L at run time for (1,16,1).  Three
// compile-time copies, one per shape, missed the instruction cache (3.8
// stalls per issue on an empty instruction buffer); one copy with L and P
// at run time issued 34% more instructions per roll-out step than the
// single-instance kernel (7.0 against 6.4 G roll-out steps/s for two
// copies against one on the uneven batch).
constexpr int kBatchC1Steps = 64;   // C * L * P of the widest one-step shape

template <typename GT, bool SELF, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) smpc_batch_kernel_c1(const __grid_constant__ BatchArgs ba)
{
    extern __shared__ float s_dyn[];
    __shared__ RobotConst s_rc;
    __shared__ BatchInstance s_inst;
    __shared__ __align__(16) float s_tot[kWarps / 2 + 1][2 * kNJ];
    __shared__ float s_S[kWarps / 2 + 1][2][2];
    __shared__ float s_state[kStateFloats];
    __shared__ float s_blk[kBatchC1Steps * kNJ];
    __shared__ float s_wm[kWarps], s_wz[kWarps];
    __shared__ float s_qs[kWarps * kStageFloats * 32];
    __shared__ float4 s_grp[SELF ? kMaxSelfGroups * kSelfGroupRec : 1];
    __shared__ int s_item;
    const int tid = threadIdx.x;
    grid_dependency_prologue();

    int cur = -1;          // the instance whose descriptor, constants and state are in shared memory
    for (;;) {
        __syncthreads();   // the previous item is done with shared memory
        if (tid == 0) s_item = static_cast<int>(atomicAdd(ba.queue, 1u));
        __syncthreads();
        const int item = s_item;
        if (item >= ba.n_work) return;
        const int2 w = ba.work[item];
        // items come instance by instance, so a block's next item is mostly
        // of the same instance: then its shared copies are kept
        if (w.x != cur) {
            {
                const int *src = reinterpret_cast<const int *>(ba.inst + w.x);
                int *dst = reinterpret_cast<int *>(&s_inst);
                for (int i = tid; i < static_cast<int>(sizeof(BatchInstance) / 4); i += kBlock) dst[i] = src[i];
            }
            __syncthreads();
            {
                const int *src = reinterpret_cast<const int *>(s_inst.rc);
                int *dst = reinterpret_cast<int *>(&s_rc);
                for (int i = tid; i < static_cast<int>(sizeof(RobotConst) / 4); i += kBlock) dst[i] = __ldg(src + i);
            }
            load_state(s_inst.in, CallScalars{s_inst.job.seed_lo, s_inst.job.seed_hi, s_inst.job.iter, s_inst.job.dt, s_inst.job.inv_lambda}, s_state);
            __syncthreads();
            if (SELF && s_rc.n_self_groups > 0 && s_rc.self_frames) {
                build_self_groups(s_rc, s_inst.g, s_grp);
                __syncthreads();
            }
            cur = w.x;
        }
        const InstanceState &st = *reinterpret_cast<const InstanceState *>(s_state);
        TileJob job = s_inst.job;
        job.iter += ba.it;
        job.c0 = s_inst.c0;
        BlockSmem sm{s_dyn, s_dyn + kWarps * kNJ * 32, s_tot, s_S, s_blk, s_wm, s_wz,
                     (SELF && s_rc.n_self_groups > 0) ? s_dyn + 2 * kWarps * kNJ * 32 : nullptr, s_qs,
                     (SELF && s_rc.n_self_groups > 0 && s_rc.self_frames) ? s_grp : nullptr};
        unsigned ngath = 0;
        if (s_inst.L == 32)
            run_block<GT, false, SELF, true>(s_rc, s_inst.g, st, job, nullptr, 1, 32, s_inst.P, w.y, sm, ngath);
        else
            run_block<GT, false, SELF, true>(s_rc, s_inst.g, st, job, nullptr, 1, s_inst.L, 1, w.y, sm, ngath);
    }
}

// Merge items: (instance, first output); one block per kMergeRows outputs
// of an instance's U*, as the single-instance merge (merge_rows).  The
// instance's first item also writes min S and adds the k = 0 terms to its
// costs.
__global__ void __launch_bounds__(kMergeThreads)
batch_merge_kernel(const BatchInstance *inst, const int2 *rows)
{
    grid_dependency_prologue();
    const int2 row = rows[blockIdx.x];
    const BatchInstance &I = inst[row.x];
    const float M = merge_rows(I.job.part, I.job.nb, I.job.H * kNJ, row.y, I.job.inv_lambda, I.job.Ubar, I.Uout);
    if (row.y == 0) {
        const float k0 = I.c0[0];
        if (threadIdx.x == 0) I.c0[1] = M + k0;
        if (I.job.costs)
            for (int i = threadIdx.x; i < I.job.K; i += blockDim.x) I.job.costs[i] += k0;
    }
}

// End of a call, one block per instance: min S to best_out and, for a
// replan (Sec. IV-C), execute u0*, advance the state and shift U left by one
// step repeating the last row.
__global__ void batch_finish_kernel(const BatchInstance *inst, int replan)
{
    grid_dependency_prologue();
    const BatchInstance &I = inst[blockIdx.x];
    if (threadIdx.x == 0 && I.best_out) *I.best_out = I.c0[1];
    if (!replan) return;
    __shared__ float sU[kMaxHorizon * kNJ];
    const int n = I.job.H * kNJ;
    for (int i = threadIdx.x; i < n; i += blockDim.x) sU[i] = I.Uout[i];
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) I.Uout[i] = (i < n - kNJ) ? sU[i + kNJ] : sU[i];
    if (threadIdx.x < kNJ) {
        const int j = threadIdx.x;
        const float u0 = sU[j];
        const float qd = fmaf(I.job.dt, u0, I.in.qd0[j]);
        const float q = fmaf(I.job.dt, qd, I.in.q0[j]);
        if (I.q_out) I.q_out[j] = q;
        if (I.qd_out) I.qd_out[j] = qd;
        if (I.u0_out) I.u0_out[j] = u0;
    }
}

} // namespace pm

// ====================================================================== engine
namespace {

struct Plan {
    std::vector<TileShape> shape;
    std::vector<int> nb;
    bool c1 = false;            // every shape one-step: smpc_batch_kernel_c1
    double us = 0.0;            // measured time of the autotuned candidate (0 = default)
    std::string how;
};

constexpr int kBatchC1MinBlocks = 6;   // residency the one-step batch kernel is fitted to

constexpr size_t kMaxPlans = 1024;   // cached plans per engine
constexpr size_t kMaxGraphs = 64;    // cached executable graphs per engine

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    int n_inst = 0;
    size_t gen = 0;             // workspace generation it was captured with
};

} // namespace

struct pm_batch {
    int device = 0;
    int n_sm = 0;
    int blocks_per_sm = 1;      // resident batch blocks per SM without the self-collision region
    int bps_call = 1;           // ... for the current call's shared memory
    size_t smem_call = 0;       // dynamic shared memory of the current call
    int bps_c1 = 1;             // resident one-step batch blocks per SM without the self-collision region
    int bps_c1_call = 1;        // resident one-step batch blocks per SM for the current call
    size_t smem_c1_call = 0;    // dynamic shared memory of the one-step kernel for the current call
    bool self_call = false;     // an item of the current call has the self-collision term
    std::mutex mu;
    std::string err;
    // workspace
    BatchInstance *d_inst = nullptr, *h_inst = nullptr;
    int2 *d_work = nullptr, *h_work = nullptr;
    int2 *d_rows = nullptr, *h_rows = nullptr;
    float *d_part = nullptr;
    float *d_c0 = nullptr;
    unsigned *d_queue = nullptr;
    float *d_tune = nullptr;    // scratch copies of U / state / outputs for the autotuner
    size_t cap_inst = 0, cap_work = 0, cap_rows = 0, cap_part = 0, cap_c0 = 0, cap_queue = 0, cap_tune = 0;
    size_t cap_hinst = 0, cap_hwork = 0, cap_hrows = 0;
    size_t gen = 1;             // bumped whenever a workspace buffer moves
    cudaEvent_t done = nullptr; // the last call's staging reads are complete
    bool pending = false;
    cudaStream_t own = nullptr;         // blocking: ordered with the legacy default stream
    cudaStream_t cap = nullptr;         // non-blocking, for graph capture only
    std::map<std::string, Plan> plans;
    std::map<std::string, GraphEntry> graphs;
};

namespace {

pm_status berr(pm_batch *b, pm_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    b->err = buf;
    return st;
}

#define PM_BCUDA(b, call)                                                                 \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return berr((b), e_ == cudaErrorMemoryAllocation ? PM_ENOMEM : PM_ECUDA,      \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

template <typename T>
pm_status grow_dev(pm_batch *b, T **p, size_t *cap, size_t n)
{
    if (n <= *cap) return PM_OK;
    size_t c = std::max(n, *cap * 2);
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    PM_BCUDA(b, cudaMalloc(p, c * sizeof(T)));
    *cap = c;
    ++b->gen;
    return PM_OK;
}

template <typename T>
pm_status grow_host(pm_batch *b, T **p, size_t *cap, size_t n)
{
    if (n <= *cap) return PM_OK;
    size_t c = std::max(n, *cap * 2);
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    *cap = 0;
    PM_BCUDA(b, cudaMallocHost(p, c * sizeof(T)));
    *cap = c;
    ++b->gen;
    return PM_OK;
}

size_t batch_smem() { return 2u * kWarps * kBatchCMax * kNJ * 32 * sizeof(float); }
size_t batch_c1_smem() { return 2u * kWarps * kNJ * 32 * sizeof(float); }

using BatchKernel = void (*)(BatchArgs);

// with the self term the slots' shared memory allows 5 blocks per SM, so
// that variant is fitted to 5 (96 registers instead of spilling at 80)
BatchKernel c1_kernel(bool self)
{
    return self ? smpc_batch_kernel_c1<float, true, kBatchC1MinBlocks - 1>
                : smpc_batch_kernel_c1<float, false, kBatchC1MinBlocks>;
}

int blocks_needed(int K, int H, TileShape s)
{
    (void)H;
    const int R = 32 / s.L;
    const long long tiles = (static_cast<long long>(K) + R - 1) / R;
    return static_cast<int>(std::max(1LL, (tiles * s.P + kWarps - 1) / kWarps));
}

bool batch_shape_ok(TileShape s, int H) { return s.C <= kBatchCMax && s.C * s.L * s.P >= H; }

// Work-proportional plan: instance i gets blocks in proportion to K_i H_i,
// scaled to `scale` times the resident grid, capped by what it can use.
Plan make_plan(pm_batch *b, const pm_batch_item *it, int n, double scale, bool wide)
{
    Plan p;
    double total = 0.0;
    p.c1 = true;
    for (int i = 0; i < n; ++i) {
        total += static_cast<double>(it[i].K) * it[i].H;
        TileShape s = default_shape(it[i].H);
        if (wide && it[i].H > 32 && it[i].H <= 64) s = TileShape{2, 32, 1};
        if (wide && it[i].H > 16 && it[i].H <= 32) s = TileShape{1, 32, 1};
        p.shape.push_back(s);
        p.c1 = p.c1 && s.C == 1;
    }
    const double B = scale * b->n_sm * (p.c1 ? b->bps_c1_call : b->bps_call);
    for (int i = 0; i < n; ++i) {
        const TileShape s = p.shape[i];
        const int need = blocks_needed(it[i].K, it[i].H, s);
        const int share = static_cast<int>(std::lround(B * it[i].K * it[i].H / total));
        p.nb.push_back(std::max(1, std::min(need, share)));
    }
    std::ostringstream os;
    os << "scale=" << scale << (wide ? " wide" : " default") << (p.c1 ? " one-step" : "");
    p.how = os.str();
    return p;
}

// Dynamic shared memory of a batch: the tile arrays plus, if any item has
// the self-collision term on, the largest item's self slots.
size_t call_smem(const pm_batch_item *it, int n)
{
    size_t extra = 0;
    for (int i = 0; i < n; ++i)
        if (it[i].ctx) extra = std::max(extra, self_smem_bytes(it[i].ctx->rc));
    return batch_smem() + extra;
}

std::string structure_key(const pm_batch_item *it, int n, int n_iters, int flags)
{
    std::ostringstream os;
    os << n_iters << ':' << (flags & PM_BATCH_REPLAN) << ':' << call_smem(it, n) << ':';
    for (int i = 0; i < n; ++i) os << it[i].K << ',' << it[i].H << ';';
    return os.str();
}

// Fill the descriptors and lay out partials, work list and merge rows for a
// plan; `tune` redirects every output to the autotuner's scratch.
pm_status stage_batch(pm_batch *b, const pm_batch_item *it, int n, const Plan &p, int flags,
                      bool tune, int *n_work, int *n_rows)
{
    size_t part = 0, rows = 0, work = 0, tune_f = 0;
    for (int i = 0; i < n; ++i) {
        const size_t na = static_cast<size_t>(it[i].H) * kNJ;
        part += static_cast<size_t>(p.nb[i]) * (2 + na);
        rows += (na + kMergeRows - 1) / kMergeRows;
        work += p.nb[i];
        tune_f += na + static_cast<size_t>(it[i].K) + 32;
    }
    pm_status st;
    if ((st = grow_dev(b, &b->d_inst, &b->cap_inst, n)) != PM_OK) return st;
    if ((st = grow_host(b, &b->h_inst, &b->cap_hinst, n)) != PM_OK) return st;
    if ((st = grow_dev(b, &b->d_work, &b->cap_work, work)) != PM_OK) return st;
    if ((st = grow_host(b, &b->h_work, &b->cap_hwork, work)) != PM_OK) return st;
    if ((st = grow_dev(b, &b->d_rows, &b->cap_rows, rows)) != PM_OK) return st;
    if ((st = grow_host(b, &b->h_rows, &b->cap_hrows, rows)) != PM_OK) return st;
    if ((st = grow_dev(b, &b->d_part, &b->cap_part, part)) != PM_OK) return st;
    if ((st = grow_dev(b, &b->d_c0, &b->cap_c0, 2 * static_cast<size_t>(n))) != PM_OK) return st;
    if (tune && (st = grow_dev(b, &b->d_tune, &b->cap_tune, tune_f)) != PM_OK) return st;

    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return static_cast<long long>(it[x].K) * it[x].H > static_cast<long long>(it[y].K) * it[y].H;
    });
    size_t off = 0, toff = 0;
    int wi = 0, ri = 0;
    for (int i = 0; i < n; ++i) {
        const pm_batch_item &x = it[i];
        pm_ctx *c = x.ctx;
        BatchInstance &I = b->h_inst[i];
        std::memset(&I, 0, sizeof(I));
        I.rc = c->d_rc;
        I.g = grid_const(c);
        I.in.q0 = x.q;
        I.in.qd0 = x.qd;
        I.in.Tg = x.T_goal;
        for (int j = 0; j < 8; ++j) I.in.sigma[j] = j < kNJ ? x.sigma[j] : 0.f;
        I.in.dyn = nullptr;
        const size_t na = static_cast<size_t>(x.H) * kNJ;
        I.job.Ubar = x.U;
        I.Uout = x.U;
        I.job.costs = x.costs_out;
        I.job.part = b->d_part + off;
        I.job.K = x.K;
        I.job.H = x.H;
        I.job.nb = p.nb[i];
        I.job.seed_lo = static_cast<uint32_t>(x.seed & 0xffffffffu);
        I.job.seed_hi = static_cast<uint32_t>(x.seed >> 32);
        I.job.iter = x.iter_index;
        I.job.dt = x.dt;
        I.job.inv_lambda = 1.0f / x.lambda;
        I.job.noise_dtype = c->noise_dtype;
        I.job.dyn = nullptr;
        I.job.rk = nullptr;         // the batch kernels derive the round keys (one key per instance)
        I.c0 = b->d_c0 + 2 * i;
        if (flags & PM_BATCH_REPLAN) {
            I.q_out = x.q;
            I.qd_out = x.qd;
            I.u0_out = x.u0_out;
        }
        I.best_out = x.best_cost;
        I.C = p.shape[i].C;
        I.L = p.shape[i].L;
        I.P = p.shape[i].P;
        if (tune) {
            float *t = b->d_tune + toff;
            I.Uout = t;                                // read Ubar, write scratch
            I.job.costs = x.costs_out ? t + na : nullptr;
            I.q_out = I.qd_out = I.u0_out = I.best_out = nullptr;
            toff += na + x.K + 32;
        }
        off += static_cast<size_t>(p.nb[i]) * (2 + na);
        for (int t = 0; t < static_cast<int>(na); t += kMergeRows) b->h_rows[ri++] = int2{i, t};
    }
    for (int i : order)
        for (int lb = 0; lb < p.nb[i]; ++lb) b->h_work[wi++] = int2{i, lb};
    *n_work = wi;
    *n_rows = ri;
    return PM_OK;
}

// Enqueue (or capture) the whole call: descriptor copies, then per
// iteration the batch kernel and the merge, then the replan step.
pm_status enqueue_batch(pm_batch *b, int n, int n_work, int n_rows, int n_iters, int flags,
                        bool tune, bool c1, cudaStream_t s)
{
    PM_BCUDA(b, cudaMemcpyAsync(b->d_inst, b->h_inst, sizeof(BatchInstance) * n, cudaMemcpyHostToDevice, s));
    PM_BCUDA(b, cudaMemcpyAsync(b->d_work, b->h_work, sizeof(int2) * n_work, cudaMemcpyHostToDevice, s));
    PM_BCUDA(b, cudaMemcpyAsync(b->d_rows, b->h_rows, sizeof(int2) * n_rows, cudaMemcpyHostToDevice, s));
    PM_BCUDA(b, cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned) * n_iters, s));
    const int grid = std::max(1, std::min(n_work, b->n_sm * (c1 ? b->bps_c1_call : b->bps_call)));
    const BatchKernel kern = c1 ? c1_kernel(b->self_call)
                                : (b->self_call ? smpc_batch_kernel<float, true> : smpc_batch_kernel<float, false>);
    const size_t smem = c1 ? b->smem_c1_call : b->smem_call;
    for (int itn = 0; itn < n_iters; ++itn) {
        BatchArgs a{b->d_inst, b->d_work, n_work, b->d_queue + itn, static_cast<uint32_t>(itn)};
        PM_BCUDA(b, launch_dependent(kern, dim3(grid), dim3(kBlock), smem, s, a));
        PM_BCUDA(b, launch_dependent(batch_merge_kernel, dim3(n_rows), dim3(kMergeThreads), 0, s,
                                     static_cast<const BatchInstance *>(b->d_inst),
                                     static_cast<const int2 *>(b->d_rows)));
    }
    if (!tune)
        PM_BCUDA(b, launch_dependent(batch_finish_kernel, dim3(n), dim3(256), 0, s,
                                     static_cast<const BatchInstance *>(b->d_inst),
                                     (flags & PM_BATCH_REPLAN) ? 1 : 0));
    return PM_OK;
}

pm_status validate(pm_batch *b, const pm_batch_item *it, int n, int n_iters)
{
    if (!it || n < 1) return berr(b, PM_EINVAL, "need at least one item");
    if (n_iters < 1 || n_iters > 1024) return berr(b, PM_EINVAL, "n_iters=%d out of [1, 1024]", n_iters);
    for (int i = 0; i < n; ++i) {
        const pm_batch_item &x = it[i];
        if (!x.ctx) return berr(b, PM_EINVAL, "item %d: ctx is NULL", i);
        if (x.ctx->device != b->device) return berr(b, PM_EINVAL, "item %d: context on another device", i);
        if (!x.ctx->has_grid) return berr(b, PM_EINVAL, "item %d: no distance field set", i);
        if (x.ctx->gd.dtype != PM_F32) return berr(b, PM_EINVAL, "item %d: batches take float32 fields", i);
        if (!x.q || !x.qd || !x.T_goal || !x.U) return berr(b, PM_EINVAL, "item %d: NULL buffer", i);
        if (x.K < 1 || x.K > PM_MAX_ROLLOUTS) return berr(b, PM_EINVAL, "item %d: K=%d out of range", i, x.K);
        if (x.H < 1 || x.H > kBatchMaxSteps) return berr(b, PM_EINVAL, "item %d: H=%d out of [1, %d]", i, x.H, kBatchMaxSteps);
        if (!std::isfinite(x.dt) || x.dt < 0.f) return berr(b, PM_EINVAL, "item %d: bad dt", i);
        if (!std::isfinite(x.lambda) || !(x.lambda > 0.f)) return berr(b, PM_EINVAL, "item %d: bad lambda", i);
        for (int j = 0; j < kNJ; ++j)
            if (!std::isfinite(x.sigma[j]) || x.sigma[j] < 0.f) return berr(b, PM_EINVAL, "item %d: bad sigma", i);
    }
    return PM_OK;
}

pm_status time_candidate(pm_batch *b, const pm_batch_item *it, int n, int n_iters, int flags,
                         const Plan &p, cudaStream_t s, double *us)
{
    int nw, nr;
    pm_status st = stage_batch(b, it, n, p, flags, true, &nw, &nr);
    if (st != PM_OK) return st;
    if ((st = grow_dev(b, &b->d_queue, &b->cap_queue, static_cast<size_t>(n_iters))) != PM_OK) return st;
    cudaEvent_t e0, e1;
    PM_BCUDA(b, cudaEventCreate(&e0));
    PM_BCUDA(b, cudaEventCreate(&e1));
    double best = 1e30;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, s);
        st = enqueue_batch(b, n, nw, nr, n_iters, flags, true, p.c1, s);
        cudaEventRecord(e1, s);
        if (st != PM_OK) break;
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = std::min(best, 1e3 * ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *us = best;
    return st;
}

} // namespace

pm_status pm::batch_reserve(pm_batch *b, int max_items, int flags)
{
    if (!b || max_items < 1) return PM_EINVAL;
    std::lock_guard<std::mutex> lk(b->mu);
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    struct Restore { int p, d; ~Restore() { if (p >= 0 && p != d) cudaSetDevice(p); } } restore{prev, b->device};
    if (b->pending) {
        PM_BCUDA(b, cudaEventSynchronize(b->done));
        b->pending = false;
    }
    // make_plan gives each item max(1, min(need, share)) blocks with shares
    // rounding to at most scale * resident + n/2 in all
    const size_t n = static_cast<size_t>(max_items);
    const double scale = (flags & PM_BATCH_AUTOTUNE) ? 4.0 : 1.0;
    const size_t work = static_cast<size_t>(scale * b->n_sm * std::max(b->blocks_per_sm, b->bps_c1)) + 2 * n;
    const size_t rows = n * ((kBatchMaxSteps * kNJ + kMergeRows - 1) / kMergeRows);
    pm_status st;
    if ((st = grow_dev(b, &b->d_inst, &b->cap_inst, n)) != PM_OK) return st;
    if ((st = grow_host(b, &b->h_inst, &b->cap_hinst, n)) != PM_OK) return st;
    if ((st = grow_dev(b, &b->d_work, &b->cap_work, work)) != PM_OK) return st;
    if ((st = grow_host(b, &b->h_work, &b->cap_hwork, work)) != PM_OK) return st;
    if ((st = grow_dev(b, &b->d_rows, &b->cap_rows, rows)) != PM_OK) return st;
    if ((st = grow_host(b, &b->h_rows, &b->cap_hrows, rows)) != PM_OK) return st;
    if ((st = grow_dev(b, &b->d_part, &b->cap_part, work * (2 + static_cast<size_t>(kBatchMaxSteps) * kNJ))) != PM_OK)
        return st;
    if ((st = grow_dev(b, &b->d_c0, &b->cap_c0, 2 * n)) != PM_OK) return st;
    return grow_dev(b, &b->d_queue, &b->cap_queue, static_cast<size_t>(1024));
}

// ========================================================================= ABI
extern "C" {

pm_status pm_batch_create(int device, pm_batch **out)
{
    if (!out) return PM_EINVAL;
    *out = nullptr;
    pm_batch *b = new pm_batch();
    b->device = device;
    int prev = -1;
    cudaGetDevice(&prev);
    auto fail = [&](pm_status st) {
        pm_batch_destroy(b);
        if (prev >= 0) cudaSetDevice(prev);
        return st;
    };
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->own, cudaStreamDefault) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return fail(PM_ECUDA);
    }
    b->blocks_per_sm = resident_blocks_per_sm(reinterpret_cast<const void *>(smpc_batch_kernel<float, false>),
                                              kBlock, batch_smem());
    if (b->blocks_per_sm < 1) return fail(PM_ECUDA);
    b->bps_c1 = resident_blocks_per_sm(reinterpret_cast<const void *>(c1_kernel(false)), kBlock, batch_c1_smem());
    if (b->bps_c1 < 1) return fail(PM_ECUDA);
    b->bps_c1_call = b->bps_c1;
    b->smem_c1_call = batch_c1_smem();
    b->bps_call = b->blocks_per_sm;
    b->smem_call = batch_smem();
    if (prev >= 0) cudaSetDevice(prev);
    *out = b;
    return PM_OK;
}

pm_status pm_batch_run(pm_batch *b, const pm_batch_item *items, int n, int n_iters, int flags,
                       void *cuda_stream)
{
    if (!b) return PM_EINVAL;
    std::lock_guard<std::mutex> lk(b->mu);
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    struct Restore { int p, d; ~Restore() { if (p >= 0 && p != d) cudaSetDevice(p); } } restore{prev, b->device};
    pm_status st = validate(b, items, n, n_iters);
    if (st != PM_OK) return st;
    cudaStream_t s = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : b->own;
    if (b->pending) {
        PM_BCUDA(b, cudaEventSynchronize(b->done));   // pinned staging is about to be rewritten
        b->pending = false;
    }
    b->smem_call = call_smem(items, n);
    b->self_call = b->smem_call > batch_smem();
    b->bps_call = b->self_call
                      ? resident_blocks_per_sm(reinterpret_cast<const void *>(smpc_batch_kernel<float, true>), kBlock,
                                               b->smem_call)
                      : b->blocks_per_sm;
    if (b->bps_call < 1) return berr(b, PM_ECUDA, "cannot give the batch kernel %zu bytes of shared memory", b->smem_call);
    b->smem_c1_call = batch_c1_smem() + (b->smem_call - batch_smem());
    b->bps_c1_call = resident_blocks_per_sm(reinterpret_cast<const void *>(c1_kernel(b->self_call)), kBlock,
                                            b->smem_c1_call);
    if (b->bps_c1_call < 1)
        return berr(b, PM_ECUDA, "cannot give the one-step batch kernel %zu bytes of shared memory", b->smem_c1_call);
    const std::string key = structure_key(items, n, n_iters, flags);
    auto pit = b->plans.find(key);
    if (pit == b->plans.end()) {
        if (b->plans.size() >= kMaxPlans) b->plans.clear();   // bounded cache: start over
        Plan best = make_plan(b, items, n, 1.0, false);
        if (flags & PM_BATCH_AUTOTUNE) {
            double best_us = 1e30;
            for (double scale : {1.0, 2.0, 4.0, 8.0, 16.0})
                for (bool wide : {false, true}) {
                    Plan cand = make_plan(b, items, n, scale, wide);
                    double us = 0.0;
                    if ((st = time_candidate(b, items, n, n_iters, flags, cand, s, &us)) != PM_OK) return st;
                    if (us < best_us) {
                        best_us = us;
                        best = cand;
                        best.us = us;
                    }
                }
        }
        pit = b->plans.emplace(key, best).first;
    }
    const Plan &p = pit->second;
    int nw = 0, nr = 0;
    if ((st = stage_batch(b, items, n, p, flags, false, &nw, &nr)) != PM_OK) return st;
    if ((st = grow_dev(b, &b->d_queue, &b->cap_queue, static_cast<size_t>(n_iters))) != PM_OK) return st;

    if (flags & PM_BATCH_GRAPH) {
        if (b->graphs.size() >= kMaxGraphs && !b->graphs.count(key)) {
            // bounded cache; an executable graph still running is freed when it completes
            for (auto &kv : b->graphs)
                if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
            b->graphs.clear();
        }
        GraphEntry &g = b->graphs[key];
        if (!g.exec || g.gen != b->gen || g.n_inst != n) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
            cudaStream_t cap = b->cap;
            cudaGraph_t graph;
            PM_BCUDA(b, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
            pm_status cst = enqueue_batch(b, n, nw, nr, n_iters, flags, false, p.c1, cap);
            cudaError_t ce = cudaStreamEndCapture(cap, &graph);
            if (cst != PM_OK) return cst;
            PM_BCUDA(b, ce);
            ce = cudaGraphInstantiate(&g.exec, graph, 0);
            cudaGraphDestroy(graph);
            PM_BCUDA(b, ce);
            g.gen = b->gen;
            g.n_inst = n;
        }
        PM_BCUDA(b, cudaGraphLaunch(g.exec, s));
    } else {
        if ((st = enqueue_batch(b, n, nw, nr, n_iters, flags, false, p.c1, s)) != PM_OK) return st;
    }
    PM_BCUDA(b, cudaEventRecord(b->done, s));
    b->pending = true;
    return PM_OK;
}

pm_status pm_batch_plan(pm_batch *b, const pm_batch_item *items, int n, int n_iters, int flags,
                        int *shapes, int *blocks, double *tuned_us)
{
    if (!b || !items) return PM_EINVAL;
    std::lock_guard<std::mutex> lk(b->mu);
    auto pit = b->plans.find(structure_key(items, n, n_iters, flags));
    if (pit == b->plans.end()) return berr(b, PM_EINVAL, "no plan for this batch structure yet");
    for (int i = 0; i < n; ++i) {
        if (shapes) {
            shapes[3 * i] = pit->second.shape[i].C;
            shapes[3 * i + 1] = pit->second.shape[i].L;
            shapes[3 * i + 2] = pit->second.shape[i].P;
        }
        if (blocks) blocks[i] = pit->second.nb[i];
    }
    if (tuned_us) *tuned_us = pit->second.us;
    return PM_OK;
}

const char *pm_batch_last_error(pm_batch *b) { return b ? b->err.c_str() : ""; }

void pm_batch_destroy(pm_batch *b)
{
    if (!b) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    if (b->pending) cudaEventSynchronize(b->done);
    for (auto &kv : b->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    cudaFree(b->d_inst);
    cudaFreeHost(b->h_inst);
    cudaFree(b->d_work);
    cudaFreeHost(b->h_work);
    cudaFree(b->d_rows);
    cudaFreeHost(b->h_rows);
    cudaFree(b->d_part);
    cudaFree(b->d_c0);
    cudaFree(b->d_queue);
    cudaFree(b->d_tune);
    if (b->done) cudaEventDestroy(b->done);
    if (b->own) cudaStreamDestroy(b->own);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (prev >= 0) cudaSetDevice(prev);
    delete b;
}

} // extern "C"
