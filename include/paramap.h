/*
 * paramap.h -- C ABI of the B300 (sm_103a) sampling-based MPC hot path.
 *
 * One SMPC iteration (ParaMaP, arXiv 2512.22575, Algorithm 1 and Sec. IV-C)
 * over a batch of K candidate roll-outs of a 7-DoF arm: Gaussian
 * perturbations of the nominal joint-acceleration sequence (Eq. 27),
 * Euler roll-out (Eq. 7), forward kinematics (Eq. 6), collision-sphere
 * clearance from a dense distance field (Eqs. 17-20), SE(3) pose error
 * (Eqs. 11-16), joint-limit, smoothness, null-space and terminal costs
 * (Eqs. 21-25), soft-min weights (Eq. 29) and the weighted-mean update of
 * the nominal sequence (Eq. 30).  All of it runs in the library's CUDA
 * kernels on one GPU.
 *
 * Conventions shared by every entry point:
 *  - Every call returns a pm_status; nothing throws across the ABI.  On any
 *    status other than PM_OK the caller's output buffers are left untouched
 *    and pm_last_error() describes the failure.
 *  - Pointers marked "host or device" may point to host memory (pageable or
 *    pinned) or to device memory of the context's GPU; the library detects
 *    which.  If any output pointer is host memory the call waits for its
 *    stream before returning; if all inputs and outputs are device memory
 *    the call only enqueues work on the stream (outputs are valid once the
 *    stream reaches that point).
 *  - Streams: device inputs must be ready when the stream reaches the call.
 *    A NULL cuda_stream selects the context's (or batch's) own stream,
 *    which is a blocking stream: it waits for earlier work on the legacy
 *    default stream and that stream waits for it, so callers that produce
 *    inputs on the default stream need no synchronisation.  Inputs made on
 *    any other stream need that stream passed (or synchronised).
 *  - The caller owns every buffer it passes.  The library copies the robot
 *    description, cost parameters and distance field into memory it owns.
 *  - A context may be used from one host thread at a time (calls on one
 *    context are serialised by an internal lock); different contexts are
 *    independent.
 *  - Layouts: joint vectors are float[n_joints]; control sequences U are
 *    row-major float[H][n_joints]; poses are row-major float[16]
 *    homogeneous matrices; the distance field is float[nz][ny][nx]
 *    (x fastest).
 *  - The library compiles the kinematic chain for n_joints == 7.
 */
#ifndef PARAMAP_H
#define PARAMAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PM_MAX_JOINTS 8
#define PM_MAX_SPHERES 64
#define PM_MAX_HORIZON 256
#define PM_MAX_ROLLOUTS (1 << 22)

typedef struct pm_ctx pm_ctx;

typedef enum {
    PM_OK = 0,
    PM_EINVAL = 1,     /* an argument is out of range, NaN or missing        */
    PM_ENOMEM = 2,     /* a device or pinned-host allocation failed          */
    PM_EBUSY = 3,      /* serving: request not admitted before its deadline  */
    PM_ETIMEOUT = 4,   /* a bounded device wait gave up (status word set)    */
    PM_ECUDA = 5,      /* a CUDA runtime call failed                         */
    PM_ENOTREADY = 6,  /* serving: the ticket's result is not ready yet      */
    PM_EINTERNAL = 7
} pm_status;

typedef enum { PM_F32 = 0, PM_F16 = 1, PM_BF16 = 2 } pm_dtype;

/*
 * Arm description (Sec. IV-A, Eq. 6; sphere model of Sec. IV-B-2, Fig. 2).
 * Modified (Craig) DH per joint i = 1..n, stored at index i-1:
 *   T_i = T_{i-1} RotX(alpha[i-1]) TransX(a[i-1]) RotZ(q_i + theta_offset[i-1])
 *         TransZ(d[i-1]),
 * and the end effector is the flange T_n TransZ(flange_d).
 * Sphere s is centred at R^{L} sphere_offset[s] + t^{L} with L =
 * sphere_link[s] in 1..n (frame index) and has radius sphere_radius[s].
 * self_pairs lists sphere index pairs (i, j) of the self-collision set S of
 * Eq. 18 (may be empty; n_self_pairs = 0).
 */
typedef struct {
    int n_joints;
    const float *a, *d, *alpha, *theta_offset;   /* [n_joints]            */
    float flange_d;
    const float *q_min, *q_max;                  /* [n_joints] rad        */
    const float *qd_max, *qdd_max;               /* [n_joints], symmetric */
    int n_spheres;                               /* 0..PM_MAX_SPHERES     */
    const int *sphere_link;                      /* [n_spheres]           */
    const float *sphere_offset;                  /* [n_spheres][3]        */
    const float *sphere_radius;                  /* [n_spheres]           */
    int n_self_pairs;
    const int *self_pairs;                       /* [n_self_pairs][2]     */
} pm_robot;

/*
 * Dense distance field phi of Eq. 17 (unsigned Euclidean distance in metres
 * to the nearest occupied voxel centre, 0 inside obstacles).  Voxel (i, j, l)
 * has centre origin + (i + 0.5, j + 0.5, l + 0.5) * res; each axis needs at
 * least 2 voxels.  phi(p) is the trilinear interpolation of the centre
 * samples with p clamped to the grid (edge replication outside).
 * dtype selects the device copy's storage: PM_F32, or PM_F16 / PM_BF16 to
 * halve the gather traffic (the lookup arithmetic stays FP32).
 */
typedef struct {
    int nx, ny, nz;
    float res;
    float origin[3];
    int dtype;
} pm_grid_desc;

/*
 * Cost weights (Sec. IV-B).  Q and QH are the diagonals of Q_k (k < H) and
 * Q_H acting on xi = [v; omega] (Eqs. 16, 25).  w_env, d_act: Eqs. 19-20;
 * w_self: Eqs. 19-20 over self_pairs; w_q, w_qd, w_qdd with the box tightened by
 * margin_frac * (max - min) per joint: Eqs. 21-22; w_s: Eq. 23; w_ns with
 * q_ref[n_joints]: Eq. 24.
 */
typedef struct {
    float Q[6], QH[6];
    float w_env, d_act, w_self;
    float w_q, w_qd, w_qdd, margin_frac;
    float w_s, w_ns;
    const float *q_ref;
} pm_cost_params;

/*
 * Create a planning context on CUDA device `device` for one arm and one
 * distance-field geometry.  Copies *robot and *costs; allocates the device
 * field of the size grid describes (filled by pm_set_distance_field).
 * Errors: PM_EINVAL (n_joints != 7, a count out of range, NaN, grid axis
 * < 2), PM_ECUDA, PM_ENOMEM.  On success *out owns all device memory until
 * pm_destroy.
 */
pm_status pm_create(const pm_robot *robot, const pm_grid_desc *grid,
                    const pm_cost_params *costs, int device, pm_ctx **out);

/*
 * Copy the dense float32 distance field [nz][ny][nx] into the context
 * (converting to the context's storage dtype).  `grid` is host memory if
 * grid_is_device == 0, else device memory of the context's GPU.  The copy
 * completes before the call returns.  Errors: PM_EINVAL (NULL), PM_ECUDA.
 */
pm_status pm_set_distance_field(pm_ctx *ctx, const float *grid, int grid_is_device);

/*
 * One SMPC iteration (Algorithm 1; Eqs. 27-30).
 *   q0, qd0   [7]     start state q_0, qdot_0 (host or device)
 *   T_goal    [16]    target pose T_g, row-major (host or device)
 *   U         [H][7]  in: nominal sequence Ubar; out: U* of Eq. 30
 *                     (host or device; device buffers are updated in place)
 *   K                 number of roll-outs M, 1..PM_MAX_ROLLOUTS
 *   H                 horizon, 1..PM_MAX_HORIZON
 *   dt                integration step of Eq. 7 (semi-implicit Euler:
 *                     qd_{k+1} = qd_k + dt u_k, q_{k+1} = q_k + dt qd_{k+1})
 *   lambda            temperature of Eq. 29, > 0
 *   sigma     [7]     per-joint standard deviation of D (host)
 *   seed, iter_index  noise of roll-out m at step k is Philox4x32-10 with
 *                     key (seed lo, seed hi) and counter (m, k, b, iter_index)
 *                     mapped by Box-Muller (b = 0: joints 0-3, b = 1: 4-6)
 *   costs_out [K]     S^(m) of Eq. 28, or NULL (host or device)
 *   cuda_stream       cudaStream_t to run on, or NULL for the context's own
 * When U or costs_out is host memory the call returns once they are
 * written; otherwise it only enqueues (host inputs are staged first).
 * Calls on one context
 * share its scratch (partials, staging): calls on different streams must
 * not overlap on the GPU.
 * Errors: PM_EINVAL (range, NaN in q0/qd0/T_goal/sigma, no field set; U is
 * left untouched), PM_ENOMEM, PM_ECUDA.
 */
pm_status pm_smpc_iterate(pm_ctx *ctx, const float *q0, const float *qd0,
                          const float *T_goal, float *U, int K, int H, float dt,
                          float lambda, const float *sigma, uint64_t seed,
                          uint32_t iter_index, float *costs_out, void *cuda_stream);

/*
 * One receding-horizon replan (Sec. IV-C, last paragraph): n_iters SMPC
 * iterations from the nominal U with iter_index = replan_index * n_iters +
 * it, then the first control u_0* is executed for one step of the same
 * integrator and the sequence is shifted one step left (last row repeated)
 * to warm-start the next replan.
 *   q, qd     [7]    in: current state; out: state after u_0* (host or device)
 *   T_goal    [16]   target pose for this replan (host or device)
 *   U         [H][7] in: nominal; out: shifted U* (host or device)
 *   u0_out    [7]    executed control u_0*, or NULL (host or device)
 *   best_cost [1]    min_m S^(m) of the last iteration, or NULL (host or device)
 * Other arguments as pm_smpc_iterate.  Errors as pm_smpc_iterate.
 */
pm_status pm_replan(pm_ctx *ctx, float *q, float *qd, const float *T_goal, float *U,
                    int K, int H, int n_iters, float dt, float lambda,
                    const float *sigma, uint64_t seed, uint32_t replan_index,
                    float *u0_out, float *best_cost, void *cuda_stream);

/*
 * pm_smpc_iterate without any allocation (the paper has no counterpart; this
 * serves callers that may not allocate device memory while running, such as
 * a fixed-rate control loop that forbids allocation after start-up or a
 * process whose device memory another allocator has fully reserved).
 * Same arguments and result as pm_smpc_iterate, except that q0, qd0, T_goal,
 * U and costs_out (if not NULL) must be device memory; sigma is host memory.
 * Only enqueues work on the stream.
 * Scratch: the soft-min merge partials live in one 2 MiB static device
 * array that every GPU loading the library holds until exit.  The array's
 * device address is resolved with cudaGetSymbolAddress on the first call on
 * each device, with that device current; make that first call before any
 * stream capture.  The address is cached for the life of the process: it
 * does not survive cudaDeviceReset or a re-created primary context, after
 * which this entry point must not be called.  Every call shares the array and keeps what the previous
 * call left there; each call writes every word it reads before reading it,
 * so nothing needs clearing, but calls must not overlap on the GPU (calls on
 * different streams, or from different contexts, that run concurrently race
 * on the array).  The launch uses fewer blocks when the partials of the
 * usual grid do not fit the array (for H above about 128); H up to
 * PM_MAX_HORIZON is accepted.
 * Errors: PM_EINVAL (as pm_smpc_iterate, or a host pointer), PM_ECUDA.
 */
pm_status pm_smpc_iterate_noalloc(pm_ctx *ctx, const float *q0, const float *qd0,
                                  const float *T_goal, float *U, int K, int H, float dt,
                                  float lambda, const float *sigma, uint64_t seed,
                                  uint32_t iter_index, float *costs_out, void *cuda_stream);

/*
 * Memory-safety checks (no counterpart in the paper).  The library built
 * with PM_BOUNDS_CHECK (libparamap_checked.so, from the same sources)
 * checks the index of every distance-field gather, shared-memory slot and
 * cost / partial / trace write of the iteration kernels against the extent
 * of its array; a violation skips the access (a read takes element 0) and
 * sets a bit in the context's violation word: 1 field gather, 2 tile
 * arrays, 4 staged states, 8 block accumulator, 16 nominal sequence read,
 * 32 cost write, 64 block partial, 128 trace, 256 self-collision slots.
 * Nothing traps.  pm_bounds_checked returns 1 in that build and 0 in the
 * normal one.  pm_bounds_status waits for the device, stores the context's
 * word in *word (always 0 in the normal build) and clears it if reset.
 * Errors: PM_EINVAL, PM_ECUDA.
 */
int pm_bounds_checked(void);
pm_status pm_bounds_status(pm_ctx *ctx, unsigned *word, int reset);

/*
 * pm_set_call_graphs: with enable != 0 (the default), a pm_smpc_iterate or
 * pm_replan call whose q0/q, qd0/qd, T_goal, U and outputs are all host
 * memory is replayed from a CUDA graph the context captures on the first
 * call of each shape (K, H, n_iters, costs wanted; at most 32 kept, least
 * recently used dropped): one graph launch per call instead of 2 n_iters + 1
 * kernel launches.  The graph's kernels read the call's inputs and scalars
 * (sigma, dt, lambda, seed, iteration index) from a fixed device block that
 * the call fills with one copy from a pinned host block (one copy brings the
 * outputs back), and compute exactly what the direct launches compute (same
 * results, bit for bit).
 * Applies to contexts with a float field and no self-collision term while
 * profiling and gather counting are off; other calls launch directly.  The
 * first call of a shape pays the capture (about a millisecond).  enable = 0
 * drops the captured graphs and launches every call directly.  No
 * counterpart in the paper.  If a capture fails (a driver without graph
 * support for these launches), the context turns the replay off and the
 * call, like every later one, launches directly.  Errors: PM_EINVAL.
 */
pm_status pm_set_call_graphs(pm_ctx *ctx, int enable);

/*
 * pm_launch_plan: the launch an iteration of K roll-outs over horizon H
 * would use on this context (no counterpart in the paper; for tests and
 * tuning): out[0..2] = the tile shape (C steps per lane, L lanes per
 * roll-out, P warps per roll-out), out[3] = thread blocks of the iteration
 * kernel.  With noalloc != 0 the block count is the one
 * pm_smpc_iterate_noalloc launches (reduced so that the partials fit its
 * static array; 0 if they cannot).  Launches nothing.  Errors: PM_EINVAL.
 */
pm_status pm_launch_plan(pm_ctx *ctx, int K, int H, int noalloc, int out[4]);

/*
 * Batched iterations: many arms, each with its own context (robot, costs,
 * float32 distance field), K, H and inputs, advanced together in one
 * persistent launch per SMPC iteration (Algorithm 1 for every item).  An
 * item's roll-outs are cut into thread-block work items that a persistent
 * grid pulls from a queue; the soft-min merge stays per item.  Every buffer
 * of an item must be device memory of the batch's GPU (not checked).
 *   q, qd        [7]    start state; with PM_BATCH_REPLAN replaced by the
 *                       state after executing u0* (Sec. IV-C)
 *   T_goal       [16]   target pose (row-major)
 *   U            [H][7] nominal in, U* out (shifted one step with PM_BATCH_REPLAN)
 *   costs_out    [K]    S^(m) of the last iteration, or NULL
 *   u0_out       [7]    executed control (PM_BATCH_REPLAN), or NULL
 *   best_cost    [1]    min_m S^(m) of the last iteration, or NULL
 *   iteration it (0..n_iters-1) uses iter_index + it; H <= 256.
 * pm_batch_run enqueues n_iters iterations (plus the replan step) on
 * cuda_stream (NULL: the batch's own stream) and returns.  Flags:
 *   PM_BATCH_REPLAN    execute u0*, advance q/qd and shift U after the iterations
 *   PM_BATCH_GRAPH     capture the call's launches once per batch structure
 *                      (the items' K, H and n_iters) as a CUDA graph and replay it;
 *                      up to 64 graphs and 1024 plans are cached per batch, the
 *                      cache starts over when full
 *   PM_BATCH_AUTOTUNE  the first time a structure is seen, time candidate plans
 *                      (tile shape per item, thread blocks per item) and keep
 *                      the fastest; otherwise a work-proportional default plan
 * pm_batch_plan reports the plan used for a structure: shapes [n][3] as
 * (C, L, P), blocks [n], and the autotuned time in microseconds (0 if the
 * default plan was used).  Calls on one batch are serialised; they must not
 * overlap on the GPU.  Errors: PM_EINVAL (item out of range, context without
 * a float32 field or on another device), PM_ENOMEM, PM_ECUDA.
 * The paper runs one arm; batching many is this library's addition.
 */
typedef struct pm_batch pm_batch;

typedef struct {
    pm_ctx *ctx;
    float *q, *qd;
    const float *T_goal;
    float *U;
    float *costs_out;
    float *u0_out;
    float *best_cost;
    int K, H;
    float dt, lambda;
    float sigma[7];
    uint64_t seed;
    uint32_t iter_index;
} pm_batch_item;

#define PM_BATCH_REPLAN 1
#define PM_BATCH_GRAPH 2
#define PM_BATCH_AUTOTUNE 4

pm_status pm_batch_create(int device, pm_batch **out);
pm_status pm_batch_run(pm_batch *batch, const pm_batch_item *items, int n, int n_iters,
                       int flags, void *cuda_stream);
pm_status pm_batch_plan(pm_batch *batch, const pm_batch_item *items, int n, int n_iters,
                        int flags, int *shapes, int *blocks, double *tuned_us);
const char *pm_batch_last_error(pm_batch *batch);
void pm_batch_destroy(pm_batch *batch);

/*
 * Replanning server (continuous batching; the paper runs one arm at 50 Hz,
 * Sec. V -- serving many arms is this library's addition).
 * pm_server_create starts a scheduler thread on `device`.  Arms are
 * registered with pm_server_add_arm (a context with a float32 field; the
 * server keeps the arm's nominal sequence resident on the device, 2 x 7 KiB).
 * pm_submit copies a request and returns a ticket at once; the scheduler
 * batches pending requests -- at most one per arm and one n_iters per
 * batch, oldest first, admitted while free device memory covers the batch's
 * workspace plus cfg.hbm_headroom -- and runs each batch as one replan of
 * every request (n_iters iterations of Algorithm 1, then u0* executed and the
 * sequence shifted, Sec. IV-C), with up to cfg.max_inflight batches on the
 * GPU at once.  A request with warm_start starts from its arm's resident
 * sequence (truncated or extended with the last row to its H), otherwise
 * from zeros; on success the arm keeps the shifted result.  pm_poll returns
 * PM_ENOTREADY while the ticket is pending and the result (then forgets it);
 * pm_wait blocks up to timeout_us.  A request not admitted within
 * deadline_us (0 = none) completes with status PM_EBUSY; a failed batch
 * completes its requests with the error and leaves their arms' sequences
 * unchanged.  A batch of one request runs on the single-instance kernels.
 * All device and pinned workspace is reserved by pm_server_create (about
 * 8.5 MiB per in-flight slot on 148 SMs plus the batch engine's), so
 * serving allocates nothing.  A registered context may still be used
 * directly, but its distance field must not change while requests of its
 * arm are pending.  Errors of the calls themselves: PM_EINVAL (unknown arm
 * or ticket, argument out of range or not finite), PM_ENOMEM, PM_EBUSY
 * (server stopping).
 */
typedef struct pm_server pm_server;

typedef struct {
    int max_batch;          /* requests per batch (default 64)             */
    int max_inflight;       /* batches on the GPU at once (default 2)      */
    size_t hbm_headroom;    /* bytes kept free on the device (256 MiB)     */
    int batch_flags;        /* PM_BATCH_GRAPH / PM_BATCH_AUTOTUNE (0)      */
    uint32_t spin_us;       /* the scheduler busy-polls (one host core) for
                               this long after its last activity before it
                               sleeps; 0 = always sleep (default 5000)     */
    uint32_t admit_window_us; /* while a batch is on the GPU, a free slot
                               launches only once the oldest waiting request
                               is this old or max_batch are waiting, so that
                               requests arriving during a batch share the
                               next one (an idle GPU launches at once);
                               0 = launch at once; default 100             */
} pm_server_config;

typedef struct {
    uint32_t arm;
    float q[7], qd[7];      /* current state                               */
    float T_goal[16];       /* target pose, row-major                      */
    int K, H, n_iters;
    float dt, lambda;
    float sigma[7];
    uint64_t seed;
    uint32_t iter_index;    /* first iteration index of the replan         */
    uint32_t deadline_us;   /* admission deadline after submit; 0 = none   */
    int warm_start;
} pm_request;

typedef struct {
    pm_status status;
    float u0[7];            /* executed control u0*                        */
    float q_next[7], qd_next[7];
    float best_cost;        /* min S of the last iteration                 */
    double latency_us;      /* submit to completion                        */
    double queue_us;        /* submit to the launch of its batch           */
    int batch_size;
} pm_result;

typedef struct {
    uint64_t submitted, completed, failed, rejected, deferred, batches, batched_requests;
    double launch_host_us;  /* host time spent forming and enqueuing batches */
    double batch_run_us;    /* sum over batches of launch to completion seen */
} pm_server_stats;

pm_status pm_server_create(int device, const pm_server_config *cfg, pm_server **out);
pm_status pm_server_add_arm(pm_server *server, pm_ctx *ctx, uint32_t *arm_id);
pm_status pm_submit(pm_server *server, const pm_request *req, uint64_t *ticket);
/* n requests at once (all validated first: PM_EINVAL submits none), queued
 * together so that the scheduler sees all of them in its next batch. */
pm_status pm_submit_many(pm_server *server, const pm_request *reqs, int n, uint64_t *tickets);
pm_status pm_poll(pm_server *server, uint64_t ticket, pm_result *out);
pm_status pm_wait(pm_server *server, uint64_t ticket, uint32_t timeout_us, pm_result *out);
pm_status pm_server_get_stats(pm_server *server, pm_server_stats *out);
void pm_server_destroy(pm_server *server);

/*
 * Planning episode with the evaluation's convergence test (Sec. V-A): from
 * (q0, qd0) replan against the fixed goal T_goal -- n_iters SMPC iterations,
 * execute u0*, shift the sequence (pm_replan; replan t uses iteration
 * indices t n_iters + it) -- until, for n_stable consecutive replans, the
 * relative improvement of the objective (min S of the replan's last
 * iteration) is below rel_tol and the position error is below pos_tol, or
 * max_replans replans have run.  U0: initial sequence [H][7] (host or
 * device) or NULL for zeros (Algorithm 1).  Metrics of the executed state
 * after each replan: e_pos = |p_g - p| (flange), e_ori = 2 arccos |q_g . q|
 * (computed as the angle of R_g^T R), path length = sum over replans and
 * joints of |q_{t+1} - q_t|, motion time = replans dt.  q_final, qd_final
 * (host or device, may be NULL) receive the final state; log (host, may be
 * NULL) receives [max_replans][4] rows (e_pos, e_ori, objective, path so
 * far) for the replans run.  Synchronous (one small read-back per replan
 * decides termination).  Errors: as pm_replan, plus PM_EINVAL for bad
 * settings.  The paper's loop runs at 50 Hz with pos_tol = 10 mm and
 * n_stable = 5; rel_tol is not given (see the design notes).
 */
typedef struct {
    int max_replans;
    float pos_tol;          /* m                                           */
    float rel_tol;          /* relative objective improvement              */
    int n_stable;
} pm_converge_cfg;

typedef struct {
    int converged;          /* 1 if the test held for n_stable replans     */
    int replans;
    float e_pos, e_ori;     /* final pose error (m, rad)                   */
    float path_length;      /* rad                                          */
    float motion_time;      /* s                                            */
    float best_cost;        /* objective of the last replan                */
} pm_episode;

pm_status pm_plan_episode(pm_ctx *ctx, const float *q0, const float *qd0, const float *T_goal,
                          const float *U0, int K, int H, int n_iters, float dt, float lambda,
                          const float *sigma, uint64_t seed, const pm_converge_cfg *cfg,
                          float *q_final, float *qd_final, pm_episode *out, float *log,
                          void *cuda_stream);

/*
 * Mapping (Sec. III-B; Sec. IV-B-2, Remark 2).
 *
 * pm_edt_squared: exact squared Euclidean distance transform of an
 *   occupancy grid, in voxel units: d2[v] = min over occupied voxels o of
 *   |v - o|^2, or INT32_MAX when no voxel is occupied.  The separable
 *   three-pass transform along y, x, then z on the native layout
 *   (Sec. III-B): lines up to 256 voxels take a nearest-occupied sweep (first
 *   pass) or a direct minimum over the line in FP32 (later passes, while
 *   every value stays below 2^24, which keeps it exact); longer lines take
 *   the 1-D Felzenszwalb-Huttenlocher lower envelope.  occ: device
 *   uint8 [nz][ny][nx] (non-zero = occupied); d2: device int32 [nz][ny][nx].
 *   Each extent 1..16384.  Enqueued on cuda_stream (NULL:
 *   the legacy default stream); allocates its scratch on that stream.
 *   Errors: PM_EINVAL, PM_ENOMEM, PM_ECUDA.
 * pm_robot_mask: clears (sets to 0) every voxel of occ whose centre lies in
 *   a sphere of the context's model at configuration q (radius + inflate,
 *   closed ball), so that the robot's own body is not fused into the map
 *   (Remark 2).  occ: device uint8 on the context's grid; q: host or device
 *   [7]; inflate >= 0 m.  Enqueued on cuda_stream (NULL: the context's);
 *   waits for it when q is host memory.
 * pm_map_update: the context's distance field from an occupancy grid:
 *   occ (host or device as occ_is_device says, uint8 on the context's grid)
 *   is copied, masked at q_mask if it is not NULL (pm_robot_mask with
 *   inflate), transformed on the GPU (pm_edt_squared), converted to metres
 *   phi = res sqrt(d2) (rounded once from FP64 to the field's storage type;
 *   1e10 m if nothing is occupied) and installed with its skip bounds, as
 *   pm_set_distance_field does.  Enqueued on cuda_stream (NULL: the
 *   context's); the scratch (1 + 8 bytes per voxel) is allocated on first
 *   use.  Iterations reading the field on other streams must not overlap it.
 *   The paper has no separate entry for this; it is the mapping step that
 *   precedes planning.
 */
pm_status pm_edt_squared(const uint8_t *occ, int nx, int ny, int nz, int32_t *d2, void *cuda_stream);
pm_status pm_robot_mask(pm_ctx *ctx, uint8_t *occ, const float *q, float inflate, void *cuda_stream);
pm_status pm_map_update(pm_ctx *ctx, const uint8_t *occ, int occ_is_device, const float *q_mask,
                        float inflate, void *cuda_stream);

/*
 * Diagnostics used by the parity tests (same device code as the hot path).
 *
 * pm_philox4x32_10: out[i][0..3] = Philox4x32-10(ctr[i][0..3], key) for
 *   i < n, as the sampler computes it (Salmon et al., SC'11; Eq. 27).
 *   ctr, out: device memory, uint32[n][4].  Enqueued on cuda_stream.
 * pm_sample_noise: eps[m][k][j] = sigma_j z_j(m, k) for m < K, k < H, j < 7
 *   (sampling step of Algorithm 1).  eps: device float[K][H][7].  Enqueued on cuda_stream.
 * pm_rollout_trace: per-step cost terms of roll-outs 0..K-1 of the iteration
 *   pm_smpc_iterate would run with the same arguments; trace: device
 *   float[K][H+1][8] with columns (pose, env, self, lim_q, lim_qd, lim_qdd,
 *   smooth, ns); row H holds the terminal cost in the pose column.  State
 *   terms of row 0 are the same for every roll-out and are left at 0.
 *   U is read, not updated.  Waits for the stream.
 * pm_pose_error: xi[i] = log(T_goal[i]^{-1} T[i]) = [v; w] (Eqs. 11-15), the
 *   pose error of the pose cost (Eqs. 16, 25) as the iteration evaluates it,
 *   in its three regimes of the rotation angle theta (series below 1e-4,
 *   the quotient form, the symmetric-part axis above pi - 0.05).  T_goal,
 *   T: device float[n][16], row-major homogeneous transforms; xi: device
 *   float[n][6].  Enqueued on cuda_stream.  Errors: PM_EINVAL (NULL or host
 *   pointers), PM_ECUDA.
 * pm_joint_sincos: sc[i] = (sin x[i], cos x[i]) as the forward kinematics
 *   evaluates the joint rotations (Eq. 6): a Cody-Waite reduction by pi/2
 *   and polynomials on [-pi/4, pi/4] fitted for this library (within 2
 *   float32 ulps for |x| <= 64, within 2^-23 absolute up to 1e4 and 2^-21
 *   up to 2^22; NaN for non-finite x).  If
 *   sc_ref is not NULL it receives CUDA's sincosf of the same arguments.
 *   x: device float[n]; sc, sc_ref: device float[n][2].  Enqueued on
 *   cuda_stream.  Errors: PM_EINVAL (NULL x/sc or host pointers), PM_ECUDA.
 */
pm_status pm_philox4x32_10(const uint32_t *ctr, uint64_t key, uint32_t *out, size_t n,
                           void *cuda_stream);
/*
 * pm_fp32_fma_peak: measured FP32 rate of `device` (a yardstick for the
 * iteration kernel, which is bound by FP32 and integer arithmetic; the paper
 * has no counterpart).  Every thread of 8 resident blocks per SM runs 8
 * independent chains of dependent FMAs; *tflops = 2 x FMAs / best of 5
 * event-timed launches, in 1e12 FLOP/s.  Synchronous.  Errors: PM_EINVAL
 * (NULL output), PM_ECUDA.
 */
pm_status pm_fp32_fma_peak(int device, double *tflops);
pm_status pm_sample_noise(int K, int H, const float *sigma, uint64_t seed,
                          uint32_t iter_index, float *eps, void *cuda_stream);
pm_status pm_pose_error(const float *T_goal, const float *T, float *xi, size_t n,
                        void *cuda_stream);
pm_status pm_joint_sincos(const float *x, float *sc, float *sc_ref, size_t n, void *cuda_stream);
pm_status pm_rollout_trace(pm_ctx *ctx, const float *q0, const float *qd0,
                           const float *T_goal, const float *U, int K, int H, float dt,
                           const float *sigma, uint64_t seed, uint32_t iter_index,
                           float *trace);

/*
 * Kernel observability (no counterpart in the paper).  pm_profile_enable
 * takes a mask of PM_PROFILE_TIME and PM_PROFILE_GATHERS (0 turns both off).
 * PM_PROFILE_TIME brackets every SMPC iteration kernel the context launches
 * with a pair of CUDA events recorded on the stream it runs on;
 * pm_profile_read waits for them, returns the summed kernel time in
 * milliseconds and the number of timed launches, and clears the record if
 * reset != 0.  PM_PROFILE_GATHERS counts the sphere lookups that needed the
 * 8-corner interpolation (the others are skipped because the cell's corner
 * minimum proves their collision term is 0); pm_profile_gathers waits for
 * the device and returns the count since the last reset.
 * Errors: PM_EINVAL (NULL ctx / outputs), PM_ECUDA.
 */
#define PM_PROFILE_TIME 1
#define PM_PROFILE_GATHERS 2
pm_status pm_profile_enable(pm_ctx *ctx, int flags);
pm_status pm_profile_read(pm_ctx *ctx, double *total_ms, uint64_t *launches, int reset);
pm_status pm_profile_gathers(pm_ctx *ctx, uint64_t *gathers, int reset);

/*
 * Precision of the sampled perturbations (the reduced-precision variant).
 * With PM_F16 or PM_BF16 every eps = sigma_j z of Eq. 27 is rounded to that
 * format (round to nearest even) right after sampling, and the rounded value
 * is used both in the roll-out and in the update of Eq. 30 -- the values a
 * kernel would read back had it stored the noise in that format.  FK, costs
 * and reductions stay FP32.  Default PM_F32 (no rounding).  Applies to later
 * calls on ctx.  Errors: PM_EINVAL (unknown dtype).
 */
pm_status pm_set_noise_dtype(pm_ctx *ctx, int dtype);

/*
 * Work decomposition of the iteration kernel (no counterpart in the paper).
 * A roll-out of H steps is mapped onto P warps (P = 1 or 2) of L lanes
 * (L = 16 or 32, 32/L roll-outs per warp when P = 1), each lane owning C
 * consecutive steps; C*L*P must be >= H.  Instantiated shapes (C, L, P):
 * (1,16,1) (1,32,1) (3,16,1) (2,32,1) (4,32,1) (8,32,1) (1,32,2) (2,32,2)
 * (4,32,2).  pm_set_tile_shape forces one for all later calls on ctx (an
 * autotuner's hook); (0, 0, 0) restores the default per horizon (H <= 16:
 * (1,16,1); <= 32: (1,32,1); <= 64: (1,32,2); <= 128: (2,32,2); else
 * (4,32,2)).  A call whose H exceeds the forced shape's C*L*P fails with
 * PM_EINVAL.  Errors: PM_EINVAL (unknown shape).
 */
pm_status pm_set_tile_shape(pm_ctx *ctx, int C, int L, int P);

/* Release every resource of the context (NULL is a no-op). */
void pm_destroy(pm_ctx *ctx);

/* Human-readable description of the last failure on ctx (or of the last
 * failure of a context-free call when ctx is NULL).  Valid until the next
 * call on the same context. */
const char *pm_last_error(pm_ctx *ctx);

/* Library version string. */
const char *pm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PARAMAP_H */
