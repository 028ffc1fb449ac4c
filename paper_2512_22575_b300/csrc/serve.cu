// Replanning server: requests from many arms, continuously batched.
//
// Clients submit replan requests (arm, state, target, K, H, iterations,
// deadline) and poll for results.  A scheduler thread forms batches from
// what is pending -- at most one request per arm per batch, oldest first,
// admitted while free device memory covers the batch's workspace plus a
// headroom -- and runs each batch through the batch engine (one persistent
// launch per SMPC iteration, then the replan step).  Up to max_inflight
// batches run at once on separate streams, so requests that arrive while a
// batch is on the GPU start as soon as a slot frees and overlap its tail.
// Each arm's nominal sequence stays resident on the device between requests
// (warm start, Sec. IV-C); a batch writes into the arm's spare buffer and
// the arm switches to it only when the batch succeeded, so a failed request
// leaves the arm's sequence unchanged.  Requests whose deadline passes
// before they are admitted complete with PM_EBUSY.
//
// A batch of one request runs through the shape-specialised single-instance
// kernels instead of the persistent batch kernel.  Every workspace (batch
// engine, block partials, pinned staging) is reserved when the server is
// created, so serving allocates nothing: a cudaFree would wait for the whole
// device.  Completion is signalled by a host function enqueued behind each
// batch, which only wakes the scheduler (it takes no lock the scheduler
// holds across CUDA calls); the batch's event stays the authority on whether
// it finished.
#include "ctx_internal.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>
#include <unordered_set>

using namespace pm;

namespace {

using Clock = std::chrono::steady_clock;

double now_us()
{
    return std::chrono::duration<double, std::micro>(Clock::now().time_since_epoch()).count();
}

constexpr double kMemInfoUs = 2000.0;
constexpr int kIoFloats = 64;   // per request: q [0,8) qd [8,16) T [16,32) u0 [32,40) best [40]

struct PrepItem {
    const float *src;           // resident U of the arm
    float *dst;                 // the arm's spare buffer, receives the start sequence
    int H, H_src, warm;
};

// Start sequence of every request of a batch: the arm's resident sequence
// truncated or extended (last row repeated) to the request's horizon, or
// zeros (Algorithm 1 initialisation) without warm start.
__global__ void prepare_u_kernel(const PrepItem *items)
{
    const PrepItem p = items[blockIdx.x];
    const int n = p.H * kNJ;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int k = i / kNJ, j = i % kNJ;
        float v = 0.f;
        if (p.warm && p.H_src > 0) v = p.src[min(k, p.H_src - 1) * kNJ + j];
        p.dst[i] = v;
    }
}

struct Arm {
    pm_ctx *ctx = nullptr;
    float *U[2] = {nullptr, nullptr};   // [kMaxHorizon][7] each
    int cur = 0;
    int H_cur = 0;
    bool busy = false;                  // a request of this arm is in flight
};

struct Req {
    uint64_t ticket;
    pm_request r;
    double t_submit;
};

struct Slot {
    pm_server *server = nullptr;
    bool busy = false;
    cudaStream_t stream = nullptr;
    pm_batch *batch = nullptr;
    cudaEvent_t done = nullptr;
    float *h_io = nullptr, *d_io = nullptr;   // pinned / device [max_batch][kIoFloats]
    PrepItem *h_prep = nullptr, *d_prep = nullptr;
    float *d_part = nullptr;                  // block partials of a one-request batch
    size_t part_floats = 0;
    float *d_c0 = nullptr;                    // [c0, best] of a one-request batch
    std::vector<Req> reqs;
    std::vector<pm_batch_item> items;
    double t_launch = 0.0;
    pm_status launch_status = PM_OK;
};

} // namespace

struct pm_server {
    int device = 0;
    int n_sm = 0;
    pm_server_config cfg{};
    std::vector<Arm> arms;
    std::vector<std::unique_ptr<Slot>> slots;
    std::mutex mu;
    std::condition_variable cv_done;    // clients: a result is ready
    // scheduler wake-up (new request, finished batch, stop); never held
    // across a CUDA call, so the completion host function cannot block on it
    std::mutex wake_mu;
    std::condition_variable wake_cv;
    std::atomic<bool> wake{false};
    std::deque<Req> pending;
    std::unordered_map<uint64_t, pm_result> done;
    std::unordered_set<uint64_t> inflight;
    uint64_t next_ticket = 1;
    bool stop = false;
    size_t free_b = 0;                  // last free-memory figure and its time
    double t_meminfo = -1e30;
    std::thread sched;
    std::string err;
    pm_server_stats stats{};
};

namespace {

void signal(pm_server *s)
{
    {
        std::lock_guard<std::mutex> g(s->wake_mu);
        s->wake.store(true, std::memory_order_release);
    }
    s->wake_cv.notify_one();
}

void CUDART_CB on_batch_done(void *p) { signal(static_cast<Slot *>(p)->server); }

size_t batch_workspace_bytes(const std::vector<Req> &reqs, int n_sm)
{
    // partials of at most the resident grid per request, plus descriptors
    size_t b = 0;
    for (const Req &q : reqs) b += static_cast<size_t>(n_sm) * 8 * (2 + 7 * q.r.H) * sizeof(float);
    return b + reqs.size() * 1024;
}

void publish(pm_server *s, const Req &q, pm_status st, const float *io, double t_end, int batch_size,
             double t_launch)
{
    pm_result res{};
    res.status = st;
    res.queue_us = t_launch > 0.0 ? t_launch - q.t_submit : t_end - q.t_submit;
    if (io && st == PM_OK) {
        for (int j = 0; j < kNJ; ++j) {
            res.q_next[j] = io[j];
            res.qd_next[j] = io[8 + j];
            res.u0[j] = io[32 + j];
        }
        res.best_cost = io[40];
    }
    res.latency_us = t_end - q.t_submit;
    res.batch_size = batch_size;
    s->inflight.erase(q.ticket);
    s->done[q.ticket] = res;
}

// Retire finished batches (called with s->mu held).
void retire(pm_server *s)
{
    for (auto &slp : s->slots) {
        Slot &sl = *slp;
        if (!sl.busy) continue;
        cudaError_t e = cudaEventQuery(sl.done);
        if (e == cudaErrorNotReady) continue;
        const double t = now_us();
        pm_status st = sl.launch_status;
        if (st == PM_OK && e != cudaSuccess) st = PM_ECUDA;
        for (size_t i = 0; i < sl.reqs.size(); ++i) {
            const Req &q = sl.reqs[i];
            Arm &a = s->arms[q.r.arm];
            if (st == PM_OK) {
                a.cur = 1 - a.cur;
                a.H_cur = q.r.H;
            }
            a.busy = false;
            publish(s, q, st, sl.h_io + i * kIoFloats, t, static_cast<int>(sl.reqs.size()), sl.t_launch);
            if (st == PM_OK) ++s->stats.completed; else ++s->stats.failed;
        }
        s->stats.batches += 1;
        s->stats.batched_requests += sl.reqs.size();
        s->stats.batch_run_us += t - sl.t_launch;
        sl.reqs.clear();
        sl.busy = false;
        if (e != cudaSuccess && e != cudaErrorNotReady) cudaGetLastError();
    }
    s->cv_done.notify_all();
}

// Form and launch one batch on a free slot (called with s->mu held).
void launch(pm_server *s, Slot &sl)
{
    const double t = now_us();
    std::vector<Req> take;
    std::unordered_set<uint32_t> arms_in;
    std::deque<Req> keep;
    while (!s->pending.empty()) {
        Req q = s->pending.front();
        s->pending.pop_front();
        if (q.r.deadline_us && t > q.t_submit + q.r.deadline_us) {
            publish(s, q, PM_EBUSY, nullptr, t, 0, 0.0);
            ++s->stats.rejected;
            continue;
        }
        Arm &a = s->arms[q.r.arm];
        // one request per arm (its warm start needs the previous result), one
        // n_iters per batch (iterations are launched batch-wide)
        if (a.busy || arms_in.count(q.r.arm) || static_cast<int>(take.size()) >= s->cfg.max_batch ||
            (!take.empty() && q.r.n_iters != take[0].r.n_iters)) {
            keep.push_back(q);
            continue;
        }
        arms_in.insert(q.r.arm);
        take.push_back(q);
    }
    s->pending.swap(keep);
    if (take.empty()) return;
    // admission by free device memory (the driver query is refreshed at
    // most every kMemInfoUs, and whenever the cached figure would refuse)
    auto refresh = [&] {
        size_t total_b = 0;
        if (cudaMemGetInfo(&s->free_b, &total_b) != cudaSuccess) {
            cudaGetLastError();
            s->free_b = 0;
        }
        s->t_meminfo = now_us();
    };
    if (t - s->t_meminfo > kMemInfoUs) refresh();
    if (batch_workspace_bytes(take, s->n_sm) + s->cfg.hbm_headroom > s->free_b && s->t_meminfo < t) refresh();
    const size_t free_b = s->free_b;
    while (!take.empty() && batch_workspace_bytes(take, s->n_sm) + s->cfg.hbm_headroom > free_b) {
        s->pending.push_front(take.back());   // waits for memory (or its deadline)
        take.pop_back();
        ++s->stats.deferred;
    }
    if (take.empty()) return;

    const int n = static_cast<int>(take.size());
    sl.items.assign(n, pm_batch_item{});
    for (int i = 0; i < n; ++i) {
        const pm_request &r = take[i].r;
        Arm &a = s->arms[r.arm];
        a.busy = true;
        float *io = sl.h_io + i * kIoFloats;
        std::memset(io, 0, sizeof(float) * kIoFloats);
        for (int j = 0; j < kNJ; ++j) {
            io[j] = r.q[j];
            io[8 + j] = r.qd[j];
        }
        std::memcpy(io + 16, r.T_goal, 16 * sizeof(float));
        sl.h_prep[i] = PrepItem{a.U[a.cur], a.U[1 - a.cur], r.H, a.H_cur, r.warm_start ? 1 : 0};
        float *dio = sl.d_io + i * kIoFloats;
        pm_batch_item &it = sl.items[i];
        it.ctx = a.ctx;
        it.q = dio;
        it.qd = dio + 8;
        it.T_goal = dio + 16;
        it.U = a.U[1 - a.cur];
        it.costs_out = nullptr;
        it.u0_out = dio + 32;
        it.best_cost = dio + 40;
        it.K = r.K;
        it.H = r.H;
        it.dt = r.dt;
        it.lambda = r.lambda;
        for (int j = 0; j < kNJ; ++j) it.sigma[j] = r.sigma[j];
        it.seed = r.seed;
        it.iter_index = r.iter_index;
    }
    sl.reqs = take;
    sl.busy = true;
    sl.t_launch = t;
    pm_status st = PM_OK;
    cudaStream_t str = sl.stream;
    const int n_iters = take[0].r.n_iters;
    if (cudaMemcpyAsync(sl.d_io, sl.h_io, sizeof(float) * kIoFloats * n, cudaMemcpyHostToDevice, str) != cudaSuccess ||
        cudaMemcpyAsync(sl.d_prep, sl.h_prep, sizeof(PrepItem) * n, cudaMemcpyHostToDevice, str) != cudaSuccess)
        st = PM_ECUDA;
    if (st == PM_OK) {
        prepare_u_kernel<<<n, 256, 0, str>>>(sl.d_prep);
        if (cudaGetLastError() != cudaSuccess) st = PM_ECUDA;
    }
    if (st == PM_OK && n == 1) {
        // one request: the shape-specialised kernels, partials in the slot's scratch
        const pm_batch_item &it = sl.items[0];
        CallInputs in{};
        in.q0 = it.q;
        in.qd0 = it.qd;
        in.Tg = it.T_goal;
        for (int j = 0; j < 8; ++j) in.sigma[j] = j < kNJ ? it.sigma[j] : 0.f;
        st = replan_with_scratch(it.ctx, str, in, it.U, it.K, it.H, n_iters, it.dt, it.lambda, it.seed,
                                 it.iter_index, sl.d_part, sl.part_floats, sl.d_c0, sl.d_io, sl.d_io + 8,
                                 it.u0_out, it.best_cost);
    } else if (st == PM_OK) {
        st = pm_batch_run(sl.batch, sl.items.data(), n, n_iters, PM_BATCH_REPLAN | s->cfg.batch_flags, str);
    }
    if (st == PM_OK &&
        cudaMemcpyAsync(sl.h_io, sl.d_io, sizeof(float) * kIoFloats * n, cudaMemcpyDeviceToHost, str) != cudaSuccess)
        st = PM_ECUDA;
    sl.launch_status = st;
    cudaEventRecord(sl.done, str);
    if (cudaLaunchHostFunc(str, on_batch_done, &sl) != cudaSuccess) cudaGetLastError();   // polled instead
    if (st != PM_OK) cudaGetLastError();
    s->stats.launch_host_us += now_us() - t;
}

void scheduler(pm_server *s)
{
    cudaSetDevice(s->device);
    double t_active = now_us();
    for (;;) {
        bool any_busy = false, has_pending = false;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->stop) break;
            retire(s);
            // with an admission window, a free slot waits, while another
            // batch is on the GPU, until the oldest waiting request is that
            // old or a full batch is waiting (an idle GPU launches at once)
            bool other_busy = false;
            for (auto &slp : s->slots) other_busy |= slp->busy;
            const bool ripe = !s->pending.empty() &&
                              (s->cfg.admit_window_us == 0 || !other_busy ||
                               static_cast<int>(s->pending.size()) >= s->cfg.max_batch ||
                               now_us() - s->pending.front().t_submit >= s->cfg.admit_window_us);
            for (auto &slp : s->slots) {
                if (!slp->busy && ripe && !s->pending.empty()) launch(s, *slp);
                any_busy |= slp->busy;
            }
            has_pending = !s->pending.empty();
        }
        const double t_now = now_us();
        if (any_busy || has_pending) t_active = t_now;
        if (t_now - t_active < s->cfg.spin_us) {
            // busy-poll (keeps this core awake, so launches and retirement
            // do not pay a sleeping thread's wake-up) and re-examine the
            // slots at least every 20 us
            while (!s->wake.load(std::memory_order_acquire) && now_us() < t_now + 20.0)
                std::this_thread::yield();
            s->wake.store(false, std::memory_order_relaxed);
            continue;
        }
        // in-flight batches wake us through their host function (the timeout
        // covers a batch whose host function never runs); pending requests
        // blocked on memory are re-examined every 100 us
        const auto wait = has_pending ? std::chrono::microseconds(100)
                        : any_busy    ? std::chrono::microseconds(2000)
                                      : std::chrono::microseconds(50000);
        std::unique_lock<std::mutex> wk(s->wake_mu);
        s->wake_cv.wait_for(wk, wait, [&] { return s->wake.load(std::memory_order_acquire); });
        s->wake.store(false, std::memory_order_relaxed);
    }
    // drain
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto &slp : s->slots)
        if (slp->busy) cudaEventSynchronize(slp->done);
    retire(s);
    for (Req &q : s->pending) publish(s, q, PM_EBUSY, nullptr, now_us(), 0, 0.0);
    s->pending.clear();
    s->cv_done.notify_all();
}

// Called with s->mu held.
bool valid_request(const pm_server *s, const pm_request &r)
{
    if (r.arm >= s->arms.size()) return false;
    if (r.K < 1 || r.K > PM_MAX_ROLLOUTS || r.H < 1 || r.H > PM_MAX_HORIZON || r.n_iters < 1 || r.n_iters > 1024)
        return false;
    if (!std::isfinite(r.lambda) || !(r.lambda > 0.f) || !std::isfinite(r.dt) || r.dt < 0.f) return false;
    for (int j = 0; j < kNJ; ++j)
        if (!std::isfinite(r.q[j]) || !std::isfinite(r.qd[j]) || !std::isfinite(r.sigma[j]) || r.sigma[j] < 0.f)
            return false;
    for (int j = 0; j < 16; ++j)
        if (!std::isfinite(r.T_goal[j])) return false;
    return true;
}

} // namespace

extern "C" {

pm_status pm_server_create(int device, const pm_server_config *cfg, pm_server **out)
{
    if (!out) return PM_EINVAL;
    *out = nullptr;
    pm_server_config c{};
    c.max_batch = 64;
    c.max_inflight = 2;
    c.hbm_headroom = static_cast<size_t>(256) << 20;
    c.batch_flags = 0;   // batch mixes rarely repeat, so graphs seldom pay off
    c.spin_us = 5000;
    c.admit_window_us = 100;
    if (cfg) c = *cfg;
    if (c.max_batch < 1 || c.max_batch > 4096 || c.max_inflight < 1 || c.max_inflight > 8) return PM_EINVAL;
    pm_server *s = new pm_server();
    s->device = device;
    s->cfg = c;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        if (prev >= 0) cudaSetDevice(prev);
        delete s;
        return PM_EINVAL;
    }
    for (int i = 0; i < c.max_inflight; ++i) {
        s->slots.emplace_back(new Slot());
        Slot &sl = *s->slots.back();
        sl.server = s;
        // partials for up to 8 resident blocks per SM at the longest horizon
        sl.part_floats = static_cast<size_t>(s->n_sm) * 8 * (2 + static_cast<size_t>(kMaxHorizon) * kNJ);
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&sl.h_io, sizeof(float) * kIoFloats * c.max_batch) != cudaSuccess ||
            cudaMalloc(&sl.d_io, sizeof(float) * kIoFloats * c.max_batch) != cudaSuccess ||
            cudaMallocHost(&sl.h_prep, sizeof(PrepItem) * c.max_batch) != cudaSuccess ||
            cudaMalloc(&sl.d_prep, sizeof(PrepItem) * c.max_batch) != cudaSuccess ||
            cudaMalloc(&sl.d_part, sizeof(float) * sl.part_floats) != cudaSuccess ||
            cudaMalloc(&sl.d_c0, sizeof(float) * 8) != cudaSuccess ||
            pm_batch_create(device, &sl.batch) != PM_OK ||
            batch_reserve(sl.batch, c.max_batch, c.batch_flags) != PM_OK) {
            cudaGetLastError();
            if (prev >= 0) cudaSetDevice(prev);
            pm_server_destroy(s);
            return PM_ENOMEM;
        }
    }
    if (prev >= 0) cudaSetDevice(prev);
    s->sched = std::thread(scheduler, s);
    *out = s;
    return PM_OK;
}

pm_status pm_server_add_arm(pm_server *s, pm_ctx *ctx, uint32_t *arm_id)
{
    if (!s || !ctx || !arm_id) return PM_EINVAL;
    if (ctx->device != s->device || !ctx->has_grid || ctx->gd.dtype != PM_F32) return PM_EINVAL;
    Arm a;
    a.ctx = ctx;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    const size_t bytes = sizeof(float) * kMaxHorizon * kNJ;
    cudaError_t e = cudaMalloc(&a.U[0], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&a.U[1], bytes);
    if (e == cudaSuccess) e = cudaMemset(a.U[0], 0, bytes);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(a.U[0]);
        cudaFree(a.U[1]);
        return e == cudaErrorMemoryAllocation ? PM_ENOMEM : PM_ECUDA;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    *arm_id = static_cast<uint32_t>(s->arms.size());
    s->arms.push_back(a);
    return PM_OK;
}

pm_status pm_submit_many(pm_server *s, const pm_request *reqs, int n, uint64_t *tickets)
{
    if (!s || !reqs || !tickets || n < 1) return PM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return PM_EBUSY;
    for (int i = 0; i < n; ++i)
        if (!valid_request(s, reqs[i])) return PM_EINVAL;
    const double t = now_us();
    for (int i = 0; i < n; ++i) {
        Req q{s->next_ticket++, reqs[i], t};
        tickets[i] = q.ticket;
        s->inflight.insert(q.ticket);
        s->pending.push_back(q);
    }
    s->stats.submitted += static_cast<uint64_t>(n);
    signal(s);
    return PM_OK;
}

pm_status pm_submit(pm_server *s, const pm_request *req, uint64_t *ticket)
{
    return pm_submit_many(s, req, 1, ticket);
}

pm_status pm_poll(pm_server *s, uint64_t ticket, pm_result *out)
{
    if (!s || !out) return PM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->done.find(ticket);
    if (it != s->done.end()) {
        *out = it->second;
        s->done.erase(it);
        return PM_OK;
    }
    return s->inflight.count(ticket) ? PM_ENOTREADY : PM_EINVAL;
}

pm_status pm_wait(pm_server *s, uint64_t ticket, uint32_t timeout_us, pm_result *out)
{
    if (!s || !out) return PM_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] { return s->done.count(ticket) || !s->inflight.count(ticket); };
    if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) return PM_ENOTREADY;
    auto it = s->done.find(ticket);
    if (it == s->done.end()) return PM_EINVAL;
    *out = it->second;
    s->done.erase(it);
    return PM_OK;
}

pm_status pm_server_get_stats(pm_server *s, pm_server_stats *out)
{
    if (!s || !out) return PM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    return PM_OK;
}

void pm_server_destroy(pm_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    signal(s);
    if (s->sched.joinable()) s->sched.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    for (auto &slp : s->slots) {
        Slot &sl = *slp;
        if (sl.stream) cudaStreamSynchronize(sl.stream);   // host functions included
        pm_batch_destroy(sl.batch);
        cudaFreeHost(sl.h_io);
        cudaFree(sl.d_io);
        cudaFreeHost(sl.h_prep);
        cudaFree(sl.d_prep);
        cudaFree(sl.d_part);
        cudaFree(sl.d_c0);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    for (Arm &a : s->arms) {
        cudaFree(a.U[0]);
        cudaFree(a.U[1]);
    }
    if (prev >= 0) cudaSetDevice(prev);
    delete s;
}

} // extern "C"
