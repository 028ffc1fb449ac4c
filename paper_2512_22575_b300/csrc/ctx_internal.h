// Internal definition of the context (shared by paramap.cu and batch.cu).
#pragma once

#include "paramap.h"
#include "smpc_dispatch.h"

#include <mutex>
#include <string>
#include <utility>
#include <vector>

struct pm_ctx {
    int device = 0;
    int n_sm = 0;
    pm::RobotConst rc{};
    pm::RobotConst *d_rc = nullptr;     // device copy (read by the batched kernels)
    unsigned char *d_map_occ = nullptr; // mapping scratch: occupancy copy, two int32 EDT buffers
    int *d_map_a = nullptr, *d_map_b = nullptr;
    float *d_phi_table = nullptr;       // res * sqrt(D) for D = 0 .. phi_table_n - 1 (or null)
    float4 *d_mask_spheres = nullptr;   // robot mask: sphere centres and radii [kMaxSpheres]
    size_t phi_table_n = 0;
    float4 *d_self_pairs = nullptr;     // self-collision pairs, grouped (rc.self_pairs)
    pm_grid_desc gd{};
    size_t grid_elems = 0;
    void *d_grid = nullptr;
    float *d_cmin = nullptr;            // per-cell corner minimum of the stored field
    // The same minima in a 3-D array of (nx-1) x (ny-1) x (nz-1) cells read
    // through a point-sampled texture (see GridConst::cmin_tex).
    cudaArray_t cmin_arr = nullptr;
    cudaTextureObject_t cmin_tex = 0;
    bool has_grid = false;
    cudaStream_t stream = nullptr;
    // Ring of staging slots for host inputs: slot i holds q0 [0..7], qd0
    // [8..15] and T_goal [16..31]; its event marks the copy as done so the
    // pinned slot can be reused.
    float *d_stage = nullptr;
    float *h_stage = nullptr;           // pinned
    cudaEvent_t slot_ev[16] = {};
    bool slot_pending[16] = {};
    int slot = 0;
    float *d_U = nullptr;
    size_t cap_U = 0;
    float *h_U = nullptr;               // pinned [PM_MAX_HORIZON * 8]
    float *d_costs = nullptr;
    size_t cap_costs = 0;
    float *h_out = nullptr;             // pinned: costs / small outputs
    size_t cap_h_out = 0;
    float *d_part = nullptr;            // block partials
    size_t cap_part = 0;

    unsigned *d_err = nullptr;          // bounds-checked builds: violation word of the kernels
    float *d_c0 = nullptr;              // small scratch: [0] c0, [1] best, [8, 32) replan q, qd, u0,
                                        // [32, 40) the robot mask's configuration,
                                        // [48, 84) an episode's q, qd, goal and metrics
    pm::TileShape forced{0, 0, 0};          // tile shape set by pm_set_tile_shape (0 = default)
    unsigned long long *d_gathers = nullptr;  // 8-corner lookups, counted while enabled
    bool count_gathers = false;
    int noise_dtype = PM_F32;           // rounding of the sampled perturbations
    bool prof = false;                  // bracket iteration kernels with events
    std::vector<cudaEvent_t> prof_ev;   // pairs (start, end)
    size_t prof_used = 0;               // events recorded since the last reset
    cudaStream_t prof_stream = nullptr;
    // Host-buffer calls replayed as CUDA graphs (one per call shape): the
    // call's inputs and scalars go through one fixed pinned block and its
    // device mirror, so a call is one graph launch instead of 2-17 launches.
    struct Graph {
        int kind, K, H, n_iters;
        bool costs;
        unsigned gen;
        const void *part, *costs_d, *costs_h, *c0;   // scratch captured into the graph
        cudaGraphExec_t exec;
    };
    std::vector<Graph> graphs;          // most recently used last
    unsigned graph_gen = 0;             // bumped when a setting captured in a graph changes
    bool graphs_on = true;
    float *d_gslot = nullptr;           // [kGraphSlotFloats] device
    float *h_gslot = nullptr;           // its pinned mirror
    cudaStream_t cap_stream = nullptr;  // private stream the graphs are captured on
    std::string err;
    std::mutex mu;
};


namespace pm {

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// After d_grid holds a new field: its cell minima, the texture's array, and
// has_grid; enqueued on s (called with the context's lock held).
pm_status finish_distance_field(pm_ctx *c, cudaStream_t s);

// Kernel view of a context's distance field.
inline GridConst grid_const(const pm_ctx *c)
{
    GridConst g;
    g.phi = c->d_grid;
    g.cmin = c->d_cmin;
    g.cmin_tex = c->cmin_tex;
    g.nx = c->gd.nx; g.ny = c->gd.ny; g.nz = c->gd.nz;
    g.inv_res = 1.0f / c->gd.res;
    g.bx = static_cast<float>(-static_cast<double>(c->gd.origin[0]) / c->gd.res - 0.5);
    g.by = static_cast<float>(-static_cast<double>(c->gd.origin[1]) / c->gd.res - 0.5);
    g.bz = static_cast<float>(-static_cast<double>(c->gd.origin[2]) / c->gd.res - 0.5);
    g.mx = static_cast<float>(c->gd.nx - 1);
    g.my = static_cast<float>(c->gd.ny - 1);
    g.mz = static_cast<float>(c->gd.nz - 1);
    g.inv_res_pk = make_float2(g.inv_res, g.inv_res);
    g.bxy = make_float2(g.bx, g.by);
    g.res = c->gd.res;
    g.mbxy = make_float2(static_cast<float>(-static_cast<double>(g.bx) * c->gd.res),
                         static_cast<float>(-static_cast<double>(g.by) * c->gd.res));
    g.mbz = static_cast<float>(-static_cast<double>(g.bz) * c->gd.res);
    g.err = c->d_err;
    return g;
}

// Launch a kernel that may start while its predecessor in the stream is
// still running (programmatic dependent launch): the kernel's
// grid_dependency_prologue() waits for the predecessor's completion and
// memory before anything else, so only the launch latency overlaps.
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                             Args &&...args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Resident blocks per SM of an iteration kernel (raises its dynamic shared
// memory limit on first use); -1 if the limit cannot be set.
int resident_blocks_per_sm(const void *fn, int block, size_t smem);

// One replan (n_iters iterations with the shape-specialised kernels, then u0*
// executed and U shifted) on stream s, with the block partials and the
// [c0, best] pair in caller-owned device scratch instead of the context's,
// so that nothing is allocated.  Inputs, U and outputs are device pointers;
// q_out / qd_out may alias in.q0 / in.qd0.  Uses fewer blocks when the
// partials would not fit part_floats.
pm_status replan_with_scratch(pm_ctx *c, cudaStream_t s, const CallInputs &in, float *U, int K, int H,
                              int n_iters, float dt, float lambda, uint64_t seed, uint32_t iter0,
                              float *part, size_t part_floats, float *c0, float *q_out, float *qd_out,
                              float *u0_out, float *best_out);

// Grow a batch's workspace (device and pinned) to what any call with up to
// max_items items of up to kMaxHorizon steps needs under the given flags, so
// that later calls allocate nothing.
pm_status batch_reserve(pm_batch *b, int max_items, int flags);

} // namespace pm
