"""Python binding of libparamap.so, the B300 SMPC hot path (ParaMaP, arXiv 2512.22575).

Argument marshalling only: every step of the SMPC iteration runs in the
library's CUDA kernels.  The functions carry the C ABI's names without the
``pm_`` prefix (``create``, ``set_distance_field``, ``smpc_iterate``,
``replan``, ``philox4x32_10``, ``sample_noise``, ``rollout_trace``,
``destroy``, ``last_error``).  Array arguments may be numpy arrays (host
memory) or torch tensors (host or CUDA); they must be contiguous float32
(uint32 for Philox).  A failing call raises ``PmError`` with the library's
message.  Importing this package loads the library and raises if it is
missing: there is no fallback implementation.
"""
import ctypes as C
import sys
import os

import numpy as np

from ._abi import (PM_BF16, PM_F16, PM_F32, PmBatchItem, PmConvergeCfg, PmCostParams, PmEpisode, PmError,
                   PmGridDesc,
                   PmRequest, PmResult, PmRobot, PmServerConfig, PmServerStats, STATUS_NAMES, lib,
                   lib_path)

__all__ = [
    "PM_F32", "PM_F16", "PM_BF16", "PmError", "lib_path", "version",
    "create", "set_distance_field", "smpc_iterate", "smpc_iterate_noalloc", "replan",
    "philox4x32_10",
    "sample_noise", "rollout_trace", "pose_error", "joint_sincos", "profile_enable", "profile_read", "profile_gathers", "launch_plan", "set_call_graphs", "bounds_checked", "bounds_status",
    "set_tile_shape", "set_noise_dtype", "PM_PROFILE_TIME", "PM_PROFILE_GATHERS", "destroy",
    "last_error", "Planner", "Batch", "Server", "PM_BATCH_REPLAN", "PM_BATCH_GRAPH", "PM_BATCH_AUTOTUNE",
]

_DTYPES = {"f32": PM_F32, "f16": PM_F16, "bf16": PM_BF16,
           PM_F32: PM_F32, PM_F16: PM_F16, PM_BF16: PM_BF16}


def version():
    return lib().pm_version().decode()


def last_error(ctx=None):
    return lib().pm_last_error(ctx).decode()


def _check(status, ctx=None):
    if status != 0:
        raise PmError(status, STATUS_NAMES.get(status, str(status)), last_error(ctx))


def _ptr(x, dtype=np.float32, n=None, writable=False):
    """Raw address of a numpy array / torch tensor (None -> NULL)."""
    if x is None:
        return None
    if type(x) is np.ndarray:   # the common host case, kept cheap (it runs per call)
        if x.dtype != dtype or not x.flags.c_contiguous:
            raise ValueError(f"expected a C-contiguous numpy {np.dtype(dtype).name} array")
        if n is not None and x.size < n:
            raise ValueError(f"array has {x.size} elements, need {n}")
        if x.flags.writeable and x.nbytes > 0:
            return C.addressof(C.c_char.from_buffer(x))
        if writable:
            raise ValueError("output array is read-only")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):  # torch tensor
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        want = {np.float32: "torch.float32", np.uint32: "torch.uint32", np.uint8: "torch.uint8",
                np.int32: "torch.int32"}[dtype]
        if str(x.dtype) != want:
            raise ValueError(f"tensor dtype {x.dtype} != {want}")
        if n is not None and x.numel() < n:
            raise ValueError(f"tensor has {x.numel()} elements, need {n}")
        return C.c_void_p(x.data_ptr())
    if not isinstance(x, np.ndarray) or x.dtype != dtype or not x.flags.c_contiguous:
        raise ValueError(f"expected a C-contiguous numpy {np.dtype(dtype).name} array")
    if writable and not x.flags.writeable:
        raise ValueError("output array is read-only")
    if n is not None and x.size < n:
        raise ValueError(f"array has {x.size} elements, need {n}")
    return C.c_void_p(x.ctypes.data)


def _f32(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


class _Keep:
    """Holds the numpy buffers a C struct points into."""

    def __init__(self):
        self.bufs = []

    def f32(self, a, n=None):
        a = _f32(a)
        if n is not None and a.size < n:
            raise ValueError(f"expected at least {n} values, got {a.size}")
        self.bufs.append(a)
        return a.ctypes.data_as(C.POINTER(C.c_float))

    def i32(self, a):
        a = np.ascontiguousarray(np.asarray(a, dtype=np.int32))
        self.bufs.append(a)
        return a.ctypes.data_as(C.POINTER(C.c_int))


def create(robot, grid_desc, costs, device=0, dtype="f32"):
    """pm_create: robot / costs as dicts (see workloads.robot), grid_desc with
    nx, ny, nz, res, origin.  Returns an opaque context handle."""
    keep = _Keep()
    n = int(robot["n_joints"])
    r = PmRobot()
    r.n_joints = n
    r.a = keep.f32(robot["a"], n); r.d = keep.f32(robot["d"], n)
    r.alpha = keep.f32(robot["alpha"], n); r.theta_offset = keep.f32(robot["theta_offset"], n)
    r.flange_d = float(robot["flange_d"])
    r.q_min = keep.f32(robot["q_min"], n); r.q_max = keep.f32(robot["q_max"], n)
    r.qd_max = keep.f32(robot["qd_max"], n); r.qdd_max = keep.f32(robot["qdd_max"], n)
    ns = len(robot["sphere_radius"])
    r.n_spheres = ns
    r.sphere_link = keep.i32(robot["sphere_link"])
    r.sphere_offset = keep.f32(robot["sphere_offset"], 3 * ns)
    r.sphere_radius = keep.f32(robot["sphere_radius"], ns)
    pairs = np.asarray(robot.get("self_pairs", np.zeros((0, 2))), dtype=np.int32).reshape(-1, 2)
    r.n_self_pairs = len(pairs)
    r.self_pairs = keep.i32(pairs) if len(pairs) else None
    g = PmGridDesc()
    g.nx, g.ny, g.nz = int(grid_desc.nx), int(grid_desc.ny), int(grid_desc.nz)
    g.res = float(grid_desc.res)
    for i in range(3):
        g.origin[i] = float(grid_desc.origin[i])
    g.dtype = _DTYPES[dtype]
    cp = PmCostParams()
    for i in range(6):
        cp.Q[i] = float(costs["Q"][i]); cp.QH[i] = float(costs["QH"][i])
    for k in ("w_env", "d_act", "w_self", "w_q", "w_qd", "w_qdd", "margin_frac", "w_s", "w_ns"):
        setattr(cp, k, float(costs[k]))
    cp.q_ref = keep.f32(costs["q_ref"], n)
    out = C.c_void_p()
    _check(lib().pm_create(C.byref(r), C.byref(g), C.byref(cp), int(device), C.byref(out)))
    return out


def set_distance_field(ctx, grid):
    """pm_set_distance_field: grid float32 [nz][ny][nx] (numpy or CUDA tensor)."""
    is_dev = hasattr(grid, "is_cuda") and grid.is_cuda
    if not hasattr(grid, "data_ptr"):
        grid = _f32(grid)
    _check(lib().pm_set_distance_field(ctx, _ptr(grid), int(is_dev)), ctx)


def smpc_iterate(ctx, q0, qd0, T_goal, U, K, dt, lam, sigma, seed, iter_index,
                 costs_out=None, stream=None):
    """pm_smpc_iterate: U [H][7] is updated in place to U*."""
    H = int(U.shape[0])
    sigma = _f32(sigma, 7)
    _check(lib().pm_smpc_iterate(ctx, _ptr(q0, n=7), _ptr(qd0, n=7), _ptr(T_goal, n=16),
                                 _ptr(U, n=7 * H, writable=True), int(K), H, float(dt),
                                 float(lam), _ptr(sigma), C.c_uint64(int(seed)),
                                 C.c_uint32(int(iter_index)), _ptr(costs_out, n=int(K), writable=True),
                                 _stream(stream)), ctx)


def smpc_iterate_noalloc(ctx, q0, qd0, T_goal, U, K, dt, lam, sigma, seed, iter_index,
                         costs_out=None, stream=None):
    """pm_smpc_iterate_noalloc: as smpc_iterate with every array in device memory
    and the merge scratch in the library's static device array, for callers
    that may not allocate device memory while running.  Enqueues only."""
    H = int(U.shape[0])
    sigma = _f32(sigma, 7)
    _check(lib().pm_smpc_iterate_noalloc(ctx, _ptr(q0, n=7), _ptr(qd0, n=7), _ptr(T_goal, n=16),
                                         _ptr(U, n=7 * H, writable=True), int(K), H, float(dt),
                                         float(lam), _ptr(sigma), C.c_uint64(int(seed)),
                                         C.c_uint32(int(iter_index)),
                                         _ptr(costs_out, n=int(K), writable=True),
                                         _stream(stream)), ctx)


def replan(ctx, q, qd, T_goal, U, K, n_iters, dt, lam, sigma, seed, replan_index,
           u0_out=None, best_cost=None, stream=None):
    """pm_replan: q, qd advanced and U shifted in place."""
    H = int(U.shape[0])
    sigma = _f32(sigma, 7)
    _check(lib().pm_replan(ctx, _ptr(q, n=7, writable=True), _ptr(qd, n=7, writable=True),
                           _ptr(T_goal, n=16), _ptr(U, n=7 * H, writable=True), int(K), H,
                           int(n_iters), float(dt), float(lam), _ptr(sigma),
                           C.c_uint64(int(seed)), C.c_uint32(int(replan_index)),
                           _ptr(u0_out, n=7, writable=True), _ptr(best_cost, n=1, writable=True),
                           _stream(stream)), ctx)


def rollout_trace(ctx, q0, qd0, T_goal, U, K, dt, sigma, seed, iter_index, trace):
    """pm_rollout_trace: trace is a CUDA float32 tensor [K][H+1][8]."""
    H = int(U.shape[0])
    sigma = _f32(sigma, 7)
    _check(lib().pm_rollout_trace(ctx, _ptr(q0, n=7), _ptr(qd0, n=7), _ptr(T_goal, n=16),
                                  _ptr(U, n=7 * H), int(K), H, float(dt), _ptr(sigma),
                                  C.c_uint64(int(seed)), C.c_uint32(int(iter_index)),
                                  _ptr(trace, n=int(K) * (H + 1) * 8, writable=True)), ctx)


def plan_episode(ctx, q0, qd0, T_goal, K, H, n_iters, dt, lam, sigma, seed, max_replans=500, pos_tol=0.01,
                 rel_tol=0.01, n_stable=5, U0=None, with_log=False, stream=None):
    """pm_plan_episode: replan to a fixed goal until the convergence test
    holds; returns a dict with converged, replans, e_pos, e_ori, path_length,
    motion_time, best_cost, q_final, qd_final and (with_log) log [replans][4]."""
    H = int(H)
    cfg = PmConvergeCfg(int(max_replans), float(pos_tol), float(rel_tol), int(n_stable))
    ep = PmEpisode()
    qf, qdf = np.empty(7, np.float32), np.empty(7, np.float32)
    log = np.zeros((int(max_replans), 4), np.float32) if with_log else None
    sigma = _f32(sigma, 7)
    U0p = None
    if U0 is not None:
        U0 = U0 if hasattr(U0, "data_ptr") else np.ascontiguousarray(np.asarray(U0, np.float32))
        U0p = _ptr(U0, n=7 * H)
    q0 = q0 if hasattr(q0, "data_ptr") else _f32(q0, 7)
    qd0 = qd0 if hasattr(qd0, "data_ptr") else _f32(qd0, 7)
    T = T_goal if hasattr(T_goal, "data_ptr") else _f32(T_goal, 16)
    _check(lib().pm_plan_episode(ctx, _ptr(q0, n=7), _ptr(qd0, n=7), _ptr(T, n=16), U0p, int(K), H, int(n_iters),
                                 float(dt), float(lam), _ptr(sigma), C.c_uint64(int(seed)), C.byref(cfg),
                                 _ptr(qf, writable=True), _ptr(qdf, writable=True), C.byref(ep),
                                 _ptr(log, writable=True) if log is not None else None, _stream(stream)), ctx)
    r = {n: getattr(ep, n) for n, _ in PmEpisode._fields_}
    r["converged"] = bool(r["converged"])
    r["q_final"], r["qd_final"] = qf, qdf
    if log is not None:
        r["log"] = log[:ep.replans].copy()
    return r


def edt_squared(occ, d2, stream=None):
    """pm_edt_squared: occ CUDA uint8 [nz][ny][nx] -> d2 CUDA int32 (squared
    distances in voxels; 2^31 - 1 when nothing is occupied)."""
    nz, ny, nx = (int(x) for x in occ.shape)
    _check(lib().pm_edt_squared(_ptr(occ, np.uint8, nx * ny * nz), nx, ny, nz,
                                _ptr(d2, np.int32, nx * ny * nz, writable=True), _stream(stream)))


def robot_mask(ctx, occ, q, inflate=0.0, stream=None):
    """pm_robot_mask: clear the voxels of occ (CUDA uint8, the context's grid)
    covered by the sphere model at q."""
    q = q if hasattr(q, "data_ptr") else _f32(q, 7)
    _check(lib().pm_robot_mask(ctx, _ptr(occ, np.uint8, writable=True), _ptr(q, n=7), float(inflate),
                               _stream(stream)), ctx)


def map_update(ctx, occ, q_mask=None, inflate=0.0, stream=None):
    """pm_map_update: the context's field from an occupancy grid (numpy or
    CUDA uint8 [nz][ny][nx]), masked at q_mask if given."""
    dev = hasattr(occ, "data_ptr")
    if not dev:
        occ = np.ascontiguousarray(np.asarray(occ, dtype=np.uint8))
    if q_mask is not None and not hasattr(q_mask, "data_ptr"):
        q_mask = _f32(q_mask, 7)
    _check(lib().pm_map_update(ctx, _ptr(occ, np.uint8), int(dev),
                               _ptr(q_mask, n=7) if q_mask is not None else None, float(inflate),
                               _stream(stream)), ctx)


def fp32_fma_peak(device=0):
    """pm_fp32_fma_peak: measured FP32 FMA rate of the device in TFLOP/s."""
    t = C.c_double()
    _check(lib().pm_fp32_fma_peak(int(device), C.byref(t)))
    return t.value


def philox4x32_10(ctr, key, out, stream=None):
    """pm_philox4x32_10 on CUDA uint32 tensors ctr, out of shape [n][4]."""
    n = ctr.numel() // 4
    _check(lib().pm_philox4x32_10(_ptr(ctr, np.uint32, 4 * n), C.c_uint64(int(key)),
                                  _ptr(out, np.uint32, 4 * n), C.c_size_t(n), _stream(stream)))


def sample_noise(K, H, sigma, seed, iter_index, eps, stream=None):
    """pm_sample_noise into a CUDA float32 tensor eps [K][H][7]."""
    sigma = _f32(sigma, 7)
    _check(lib().pm_sample_noise(int(K), int(H), _ptr(sigma), C.c_uint64(int(seed)),
                                 C.c_uint32(int(iter_index)), _ptr(eps, n=int(K) * int(H) * 7),
                                 _stream(stream)))


def pose_error(T_goal, T, xi, stream=None):
    """pm_pose_error on CUDA float32 tensors T_goal, T [n][16] (row-major 4x4)
    into xi [n][6] = log(T_goal^-1 T) as [v; w]."""
    n = T.numel() // 16
    _check(lib().pm_pose_error(_ptr(T_goal, n=16 * n), _ptr(T, n=16 * n), _ptr(xi, n=6 * n, writable=True),
                               C.c_size_t(n), _stream(stream)))


def joint_sincos(x, sc, sc_ref=None, stream=None):
    """pm_joint_sincos on CUDA float32 tensors: x [n] into sc [n][2] = (sin, cos)
    as the forward kinematics computes them; sc_ref, if given, gets CUDA's sincosf."""
    n = x.numel()
    _check(lib().pm_joint_sincos(_ptr(x, n=n), _ptr(sc, n=2 * n, writable=True),
                                 None if sc_ref is None else _ptr(sc_ref, n=2 * n, writable=True),
                                 C.c_size_t(n), _stream(stream)))


PM_PROFILE_TIME, PM_PROFILE_GATHERS = 1, 2


def profile_enable(ctx, flags=PM_PROFILE_TIME):
    """pm_profile_enable: PM_PROFILE_TIME | PM_PROFILE_GATHERS (0 = off)."""
    _check(lib().pm_profile_enable(ctx, int(flags)), ctx)


def profile_gathers(ctx, reset=True):
    """pm_profile_gathers: 8-corner lookups performed since the last reset."""
    n = C.c_uint64()
    _check(lib().pm_profile_gathers(ctx, C.byref(n), int(bool(reset))), ctx)
    return n.value


def set_noise_dtype(ctx, dtype="f32"):
    """pm_set_noise_dtype: round the sampled perturbations to f16 / bf16."""
    _check(lib().pm_set_noise_dtype(ctx, _DTYPES[dtype]), ctx)


def set_tile_shape(ctx, C_steps=0, L=0, P=0):
    """pm_set_tile_shape: force (C, L, P) for later calls; (0, 0, 0) = default."""
    _check(lib().pm_set_tile_shape(ctx, int(C_steps), int(L), int(P)), ctx)


def bounds_checked():
    """pm_bounds_checked: True in the bounds-checked build."""
    return bool(lib().pm_bounds_checked())


def bounds_status(ctx, reset=True):
    """pm_bounds_status: the context's violation word (0 = no violation)."""
    w = C.c_uint()
    _check(lib().pm_bounds_status(ctx, C.byref(w), int(bool(reset))), ctx)
    return w.value


def set_call_graphs(ctx, enable=True):
    """pm_set_call_graphs: replay host-buffer calls from captured CUDA graphs
    (default on) or launch every call directly."""
    _check(lib().pm_set_call_graphs(ctx, int(bool(enable))), ctx)


def launch_plan(ctx, K, H, noalloc=False):
    """pm_launch_plan: ((C, L, P), thread blocks) of an iteration of K
    roll-outs over horizon H (of pm_smpc_iterate_noalloc with noalloc)."""
    out = (C.c_int * 4)()
    _check(lib().pm_launch_plan(ctx, int(K), int(H), int(bool(noalloc)), out), ctx)
    return (out[0], out[1], out[2]), out[3]


def profile_read(ctx, reset=True):
    """pm_profile_read: (summed kernel milliseconds, timed launches)."""
    ms = C.c_double()
    n = C.c_uint64()
    _check(lib().pm_profile_read(ctx, C.byref(ms), C.byref(n), int(bool(reset))), ctx)
    return ms.value, n.value


def destroy(ctx):
    lib().pm_destroy(ctx)


def _stream(stream):
    """cudaStream_t of `stream`: a torch.cuda.Stream, a raw handle, or None
    for PyTorch's current stream when torch has initialised CUDA (so a call
    is ordered after the torch work that produced its inputs), else NULL."""
    if stream is None:
        torch = sys.modules.get("torch")
        if torch is not None and torch.cuda.is_initialized():
            raw = getattr(torch._C, "_cuda_getCurrentRawStream", None)
            if raw is not None:     # the handle without building a Stream object
                return raw(torch.cuda.current_device())
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


PM_BATCH_REPLAN, PM_BATCH_GRAPH, PM_BATCH_AUTOTUNE = 1, 2, 4


class Batch:
    """pm_batch_*: many contexts advanced together in one persistent launch.

    Items are dicts with keys ctx (a Planner or a context handle), q, qd,
    T_goal, U, and optionally costs_out, u0_out, best_cost (CUDA float32
    tensors), K, dt, lam, sigma, seed, iter_index.  H is U's first dimension.
    """

    def __init__(self, device=0):
        out = C.c_void_p()
        _check(lib().pm_batch_create(int(device), C.byref(out)))
        self.b = out

    def _items(self, items):
        arr = (PmBatchItem * len(items))()
        for i, it in enumerate(items):
            x = arr[i]
            ctx = it["ctx"]
            x.ctx = ctx.ctx if hasattr(ctx, "ctx") else ctx
            H = int(it["U"].shape[0])
            x.q = _ptr(it["q"], n=7); x.qd = _ptr(it["qd"], n=7)
            x.T_goal = _ptr(it["T_goal"], n=16); x.U = _ptr(it["U"], n=7 * H)
            x.costs_out = _ptr(it.get("costs_out"), n=int(it["K"]))
            x.u0_out = _ptr(it.get("u0_out"), n=7)
            x.best_cost = _ptr(it.get("best_cost"), n=1)
            x.K = int(it["K"]); x.H = H
            x.dt = float(it.get("dt", 0.02)); x.lambda_ = float(it.get("lam", 0.05))
            sig = _f32(it.get("sigma", np.full(7, 0.5)), 7)
            for j in range(7):
                x.sigma[j] = float(sig[j])
            x.seed = int(it.get("seed", 0)); x.iter_index = int(it.get("iter_index", 0))
        return arr

    def run(self, items, n_iters=1, flags=0, stream=None):
        arr = self._items(items)
        st = lib().pm_batch_run(self.b, arr, len(items), int(n_iters), int(flags), _stream(stream))
        if st != 0:
            raise PmError(st, STATUS_NAMES.get(st, str(st)), lib().pm_batch_last_error(self.b).decode())

    def plan(self, items, n_iters=1, flags=0):
        """(shapes [(C, L, P)], blocks per item, autotuned time in us or 0)."""
        n = len(items)
        arr = self._items(items)
        shapes = (C.c_int * (3 * n))()
        blocks = (C.c_int * n)()
        us = C.c_double()
        st = lib().pm_batch_plan(self.b, arr, n, int(n_iters), int(flags), shapes, blocks, C.byref(us))
        if st != 0:
            raise PmError(st, STATUS_NAMES.get(st, str(st)), lib().pm_batch_last_error(self.b).decode())
        return ([tuple(shapes[3 * i:3 * i + 3]) for i in range(n)], list(blocks), us.value)

    def close(self):
        if self.b is not None:
            lib().pm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """pm_server_*: continuously batched replanning for many arms.

    submit() copies a request and returns a ticket; poll() returns None while
    it is pending, else a dict with status (a STATUS_NAMES string), u0,
    q_next, qd_next, best_cost, latency_us, queue_us and batch_size."""

    def __init__(self, device=0, max_batch=64, max_inflight=2, hbm_headroom=256 << 20,
                 batch_flags=0, spin_us=5000, admit_window_us=100):
        cfg = PmServerConfig(int(max_batch), int(max_inflight), int(hbm_headroom), int(batch_flags),
                             int(spin_us), int(admit_window_us))
        out = C.c_void_p()
        _check(lib().pm_server_create(int(device), C.byref(cfg), C.byref(out)))
        self.s = out

    def add_arm(self, planner):
        aid = C.c_uint32()
        _check(lib().pm_server_add_arm(self.s, planner.ctx if hasattr(planner, "ctx") else planner,
                                       C.byref(aid)))
        return aid.value

    @staticmethod
    def _request(arm, q, qd, T_goal, K, H, n_iters=8, dt=0.02, lam=0.05, sigma=None, seed=0,
                 iter_index=0, deadline_us=0, warm_start=True, r=None):
        r = PmRequest() if r is None else r
        r.arm = int(arm)
        q = _f32(q, 7); qd = _f32(qd, 7); T = _f32(T_goal, 16)
        sig = _f32(np.full(7, 0.5) if sigma is None else sigma, 7)
        for j in range(7):
            r.q[j] = float(q[j]); r.qd[j] = float(qd[j]); r.sigma[j] = float(sig[j])
        for j in range(16):
            r.T_goal[j] = float(T[j])
        r.K, r.H, r.n_iters = int(K), int(H), int(n_iters)
        r.dt, r.lambda_ = float(dt), float(lam)
        r.seed, r.iter_index = int(seed), int(iter_index)
        r.deadline_us, r.warm_start = int(deadline_us), int(bool(warm_start))
        return r

    def submit(self, arm, q, qd, T_goal, K, H, n_iters=8, **kw):
        """pm_submit; further keyword arguments dt, lam, sigma, seed,
        iter_index, deadline_us, warm_start."""
        r = self._request(arm, q, qd, T_goal, K, H, n_iters, **kw)
        t = C.c_uint64()
        _check(lib().pm_submit(self.s, C.byref(r), C.byref(t)))
        return t.value

    def submit_many(self, requests):
        """pm_submit_many: requests is a list of dicts with submit()'s
        arguments; returns the tickets in order."""
        n = len(requests)
        arr = (PmRequest * n)()
        for i, kw in enumerate(requests):
            self._request(r=arr[i], **kw)
        t = (C.c_uint64 * n)()
        _check(lib().pm_submit_many(self.s, arr, n, t))
        return list(t)

    @staticmethod
    def _result(res):
        return {"status": STATUS_NAMES.get(res.status, str(res.status)),
                "u0": np.array(res.u0[:], np.float32), "q_next": np.array(res.q_next[:], np.float32),
                "qd_next": np.array(res.qd_next[:], np.float32), "best_cost": res.best_cost,
                "latency_us": res.latency_us, "queue_us": res.queue_us, "batch_size": res.batch_size}

    def poll(self, ticket):
        res = PmResult()
        st = lib().pm_poll(self.s, C.c_uint64(int(ticket)), C.byref(res))
        if st == 6:  # PM_ENOTREADY
            return None
        _check(st)
        return self._result(res)

    def wait(self, ticket, timeout_us=10_000_000):
        res = PmResult()
        st = lib().pm_wait(self.s, C.c_uint64(int(ticket)), int(timeout_us), C.byref(res))
        _check(st)
        return self._result(res)

    def stats(self):
        st = PmServerStats()
        _check(lib().pm_server_get_stats(self.s, C.byref(st)))
        return {n: getattr(st, n) for n, _ in PmServerStats._fields_}

    def close(self):
        if self.s is not None:
            lib().pm_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Planner:
    """Owns one context; methods forward to the functions above."""

    def __init__(self, robot, grid_desc, costs, device=0, dtype="f32"):
        self.ctx = create(robot, grid_desc, costs, device, dtype)
        self.grid_desc = grid_desc

    def set_distance_field(self, grid):
        set_distance_field(self.ctx, grid)

    def map_update(self, occ, q_mask=None, inflate=0.0, stream=None):
        map_update(self.ctx, occ, q_mask, inflate, stream)

    def robot_mask(self, occ, q, inflate=0.0, stream=None):
        robot_mask(self.ctx, occ, q, inflate, stream)

    def plan_episode(self, *a, **kw):
        return plan_episode(self.ctx, *a, **kw)

    def smpc_iterate(self, *a, **kw):
        smpc_iterate(self.ctx, *a, **kw)

    def smpc_iterate_noalloc(self, *a, **kw):
        smpc_iterate_noalloc(self.ctx, *a, **kw)

    def replan(self, *a, **kw):
        replan(self.ctx, *a, **kw)

    def rollout_trace(self, *a, **kw):
        rollout_trace(self.ctx, *a, **kw)

    def profile_enable(self, flags=PM_PROFILE_TIME):
        profile_enable(self.ctx, flags)

    def profile_gathers(self, reset=True):
        return profile_gathers(self.ctx, reset)

    def set_noise_dtype(self, dtype="f32"):
        set_noise_dtype(self.ctx, dtype)

    def set_tile_shape(self, C_steps=0, L=0, P=0):
        set_tile_shape(self.ctx, C_steps, L, P)

    def profile_read(self, reset=True):
        return profile_read(self.ctx, reset)

    def launch_plan(self, K, H, noalloc=False):
        return launch_plan(self.ctx, K, H, noalloc)

    def set_call_graphs(self, enable=True):
        set_call_graphs(self.ctx, enable)

    def bounds_status(self, reset=True):
        return bounds_status(self.ctx, reset)

    def close(self):
        if self.ctx is not None:
            destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


lib()  # load now: a missing or unbuilt library is an import error, never a fallback
