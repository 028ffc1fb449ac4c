"""ctypes declarations of include/paramap.h (loading only; no compute)."""
import ctypes as C
import os

PM_F32, PM_F16, PM_BF16 = 0, 1, 2
STATUS_NAMES = {0: "PM_OK", 1: "PM_EINVAL", 2: "PM_ENOMEM", 3: "PM_EBUSY", 4: "PM_ETIMEOUT",
                5: "PM_ECUDA", 6: "PM_ENOTREADY", 7: "PM_EINTERNAL"}

_PF = C.POINTER(C.c_float)
_PI = C.POINTER(C.c_int)
_V = C.c_void_p


class PmError(RuntimeError):
    def __init__(self, status, name, message):
        super().__init__(f"{name}: {message}")
        self.status = status
        self.name = name


class PmRobot(C.Structure):
    _fields_ = [("n_joints", C.c_int), ("a", _PF), ("d", _PF), ("alpha", _PF),
                ("theta_offset", _PF), ("flange_d", C.c_float), ("q_min", _PF), ("q_max", _PF),
                ("qd_max", _PF), ("qdd_max", _PF), ("n_spheres", C.c_int), ("sphere_link", _PI),
                ("sphere_offset", _PF), ("sphere_radius", _PF), ("n_self_pairs", C.c_int),
                ("self_pairs", _PI)]


class PmGridDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("res", C.c_float),
                ("origin", C.c_float * 3), ("dtype", C.c_int)]


class PmCostParams(C.Structure):
    _fields_ = [("Q", C.c_float * 6), ("QH", C.c_float * 6), ("w_env", C.c_float),
                ("d_act", C.c_float), ("w_self", C.c_float), ("w_q", C.c_float),
                ("w_qd", C.c_float), ("w_qdd", C.c_float), ("margin_frac", C.c_float),
                ("w_s", C.c_float), ("w_ns", C.c_float), ("q_ref", _PF)]


class PmBatchItem(C.Structure):
    _fields_ = [("ctx", _V), ("q", _V), ("qd", _V), ("T_goal", _V), ("U", _V), ("costs_out", _V),
                ("u0_out", _V), ("best_cost", _V), ("K", C.c_int), ("H", C.c_int),
                ("dt", C.c_float), ("lambda_", C.c_float), ("sigma", C.c_float * 7),
                ("seed", C.c_uint64), ("iter_index", C.c_uint32)]


class PmServerConfig(C.Structure):
    _fields_ = [("max_batch", C.c_int), ("max_inflight", C.c_int), ("hbm_headroom", C.c_size_t),
                ("batch_flags", C.c_int), ("spin_us", C.c_uint32), ("admit_window_us", C.c_uint32)]


class PmRequest(C.Structure):
    _fields_ = [("arm", C.c_uint32), ("q", C.c_float * 7), ("qd", C.c_float * 7),
                ("T_goal", C.c_float * 16), ("K", C.c_int), ("H", C.c_int), ("n_iters", C.c_int),
                ("dt", C.c_float), ("lambda_", C.c_float), ("sigma", C.c_float * 7),
                ("seed", C.c_uint64), ("iter_index", C.c_uint32), ("deadline_us", C.c_uint32),
                ("warm_start", C.c_int)]


class PmResult(C.Structure):
    _fields_ = [("status", C.c_int), ("u0", C.c_float * 7), ("q_next", C.c_float * 7),
                ("qd_next", C.c_float * 7), ("best_cost", C.c_float), ("latency_us", C.c_double),
                ("queue_us", C.c_double), ("batch_size", C.c_int)]


class PmConvergeCfg(C.Structure):
    _fields_ = [("max_replans", C.c_int), ("pos_tol", C.c_float), ("rel_tol", C.c_float), ("n_stable", C.c_int)]


class PmEpisode(C.Structure):
    _fields_ = [("converged", C.c_int), ("replans", C.c_int), ("e_pos", C.c_float), ("e_ori", C.c_float),
                ("path_length", C.c_float), ("motion_time", C.c_float), ("best_cost", C.c_float)]


class PmServerStats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("submitted", "completed", "failed", "rejected", "deferred",
                                          "batches", "batched_requests")] + \
               [("launch_host_us", C.c_double), ("batch_run_us", C.c_double)]


# Every exported entry point of include/paramap.h with its ctypes signature.
SIGNATURES = {
    "pm_create": (C.c_int, [C.POINTER(PmRobot), C.POINTER(PmGridDesc), C.POINTER(PmCostParams),
                            C.c_int, C.POINTER(C.c_void_p)]),
    "pm_set_distance_field": (C.c_int, [_V, _V, C.c_int]),
    "pm_smpc_iterate": (C.c_int, [_V, _V, _V, _V, _V, C.c_int, C.c_int, C.c_float, C.c_float, _V,
                                  C.c_uint64, C.c_uint32, _V, _V]),
    "pm_smpc_iterate_noalloc": (C.c_int, [_V, _V, _V, _V, _V, C.c_int, C.c_int, C.c_float,
                                          C.c_float, _V, C.c_uint64, C.c_uint32, _V, _V]),
    "pm_replan": (C.c_int, [_V, _V, _V, _V, _V, C.c_int, C.c_int, C.c_int, C.c_float, C.c_float,
                            _V, C.c_uint64, C.c_uint32, _V, _V, _V]),
    "pm_philox4x32_10": (C.c_int, [_V, C.c_uint64, _V, C.c_size_t, _V]),
    "pm_sample_noise": (C.c_int, [C.c_int, C.c_int, _V, C.c_uint64, C.c_uint32, _V, _V]),
    "pm_pose_error": (C.c_int, [_V, _V, _V, C.c_size_t, _V]),
    "pm_joint_sincos": (C.c_int, [_V, _V, _V, C.c_size_t, _V]),
    "pm_launch_plan": (C.c_int, [_V, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "pm_set_call_graphs": (C.c_int, [_V, C.c_int]),
    "pm_bounds_checked": (C.c_int, []),
    "pm_bounds_status": (C.c_int, [_V, C.POINTER(C.c_uint), C.c_int]),
    "pm_rollout_trace": (C.c_int, [_V, _V, _V, _V, _V, C.c_int, C.c_int, C.c_float, _V,
                                   C.c_uint64, C.c_uint32, _V]),
    "pm_profile_enable": (C.c_int, [_V, C.c_int]),
    "pm_profile_read": (C.c_int, [_V, C.POINTER(C.c_double), C.POINTER(C.c_uint64), C.c_int]),
    "pm_profile_gathers": (C.c_int, [_V, C.POINTER(C.c_uint64), C.c_int]),
    "pm_set_tile_shape": (C.c_int, [_V, C.c_int, C.c_int, C.c_int]),
    "pm_set_noise_dtype": (C.c_int, [_V, C.c_int]),
    "pm_batch_create": (C.c_int, [C.c_int, C.POINTER(C.c_void_p)]),
    "pm_batch_run": (C.c_int, [_V, C.POINTER(PmBatchItem), C.c_int, C.c_int, C.c_int, _V]),
    "pm_batch_plan": (C.c_int, [_V, C.POINTER(PmBatchItem), C.c_int, C.c_int, C.c_int,
                                C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "pm_batch_last_error": (C.c_char_p, [_V]),
    "pm_batch_destroy": (None, [_V]),
    "pm_server_create": (C.c_int, [C.c_int, C.POINTER(PmServerConfig), C.POINTER(C.c_void_p)]),
    "pm_server_add_arm": (C.c_int, [_V, _V, C.POINTER(C.c_uint32)]),
    "pm_submit": (C.c_int, [_V, C.POINTER(PmRequest), C.POINTER(C.c_uint64)]),
    "pm_submit_many": (C.c_int, [_V, C.POINTER(PmRequest), C.c_int, C.POINTER(C.c_uint64)]),
    "pm_fp32_fma_peak": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
    "pm_plan_episode": (C.c_int, [_V, _V, _V, _V, _V, C.c_int, C.c_int, C.c_int, C.c_float, C.c_float, _V,
                                  C.c_uint64, C.POINTER(PmConvergeCfg), _V, _V, C.POINTER(PmEpisode), _V, _V]),
    "pm_edt_squared": (C.c_int, [_V, C.c_int, C.c_int, C.c_int, _V, _V]),
    "pm_robot_mask": (C.c_int, [_V, _V, _V, C.c_float, _V]),
    "pm_map_update": (C.c_int, [_V, _V, C.c_int, _V, C.c_float, _V]),
    "pm_poll": (C.c_int, [_V, C.c_uint64, C.POINTER(PmResult)]),
    "pm_wait": (C.c_int, [_V, C.c_uint64, C.c_uint32, C.POINTER(PmResult)]),
    "pm_server_get_stats": (C.c_int, [_V, C.POINTER(PmServerStats)]),
    "pm_server_destroy": (None, [_V]),
    "pm_destroy": (None, [_V]),
    "pm_last_error": (C.c_char_p, [_V]),
    "pm_version": (C.c_char_p, []),
}

_lib = None


LIB_NAMES = ("libparamap.so", "libparamap_checked.so")


def lib_path():
    """The library this process loads: libparamap.so, or the bounds-checked
    build when the environment sets PARAMAP_LIB=libparamap_checked.so."""
    name = os.environ.get("PARAMAP_LIB", "libparamap.so")
    if name not in LIB_NAMES:
        raise ImportError(f"PARAMAP_LIB={name!r}: expected one of {LIB_NAMES}")
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), name)


def lib():
    """Load libparamap.so (built in-tree by paper_2512_22575_b300.build)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with "
                              "`python paper_2512_22575_b300/build.py`")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib
