"""Python access to the FP64 CPU oracle (test infrastructure only).

The oracle is plain C (``smpc_oracle.c``) compiled by ``oracle/build.py`` and
loaded here with ctypes.  It is the reference definition of one SMPC
iteration (ParaMaP, Sec. IV, Algorithm 1) that the CUDA path is checked
against.  Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline may import this package; the product never does.  Nothing here is
shared with the CUDA path.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

MAX_J, MAX_S, MAX_P = 8, 64, 2048
T_COLS = 8  # pose, env, self, lim_q, lim_qd, lim_qdd, smooth, ns
T_NAMES = ("pose", "env", "self", "lim_q", "lim_qd", "lim_qdd", "smooth", "ns")

_D = C.c_double
_PD = C.POINTER(C.c_double)


class OrRobot(C.Structure):
    _fields_ = [
        ("n_joints", C.c_int),
        ("a", _D * MAX_J), ("d", _D * MAX_J), ("alpha", _D * MAX_J),
        ("theta_offset", _D * MAX_J), ("flange_d", _D),
        ("q_min", _D * MAX_J), ("q_max", _D * MAX_J),
        ("qd_max", _D * MAX_J), ("qdd_max", _D * MAX_J),
        ("n_spheres", C.c_int), ("sphere_link", C.c_int * MAX_S),
        ("sphere_offset", (_D * 3) * MAX_S), ("sphere_radius", _D * MAX_S),
        ("n_pairs", C.c_int), ("pairs", (C.c_int * 2) * MAX_P),
    ]


class OrGrid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("res", _D),
                ("origin", _D * 3), ("phi", C.POINTER(C.c_float))]


class OrCost(C.Structure):
    _fields_ = [("Q", _D * 6), ("QH", _D * 6), ("w_env", _D), ("d_act", _D), ("w_self", _D),
                ("w_q", _D), ("w_qd", _D), ("w_qdd", _D), ("margin_frac", _D),
                ("w_s", _D), ("w_ns", _D), ("q_ref", _D * MAX_J)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
        L.or_word_to_uniform.argtypes = [C.c_uint32]
        L.or_word_to_uniform.restype = _D
        L.or_normals.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, _PD]
        L.or_fk.argtypes = [C.POINTER(OrRobot), _PD, _PD]
        L.or_sphere_centres.argtypes = [C.POINTER(OrRobot), _PD, _PD]
        L.or_phi.argtypes = [C.POINTER(OrGrid), _PD]
        L.or_phi.restype = _D
        L.or_se3_log.argtypes = [_PD, _PD]
        L.or_pose_error.argtypes = [_PD, _PD, _PD]
        L.or_integrate.argtypes = [C.c_int, C.c_int, _D, _PD, _PD, _PD, _PD, _PD]
        L.or_rollout.argtypes = [C.POINTER(OrRobot), C.POINTER(OrGrid), C.POINTER(OrCost),
                                 _PD, _PD, _PD, _PD, C.c_int, _D, _PD]
        L.or_rollout.restype = _D
        L.or_smpc_iterate.argtypes = [C.POINTER(OrRobot), C.POINTER(OrGrid), C.POINTER(OrCost),
                                      _PD, _PD, _PD, _PD, C.c_int, C.c_int, _D, _D, _PD,
                                      C.c_uint64, C.c_uint32, _PD, _PD, C.c_int]
        L.or_smpc_iterate.restype = C.c_int
        L.or_replan.argtypes = [C.POINTER(OrRobot), C.POINTER(OrGrid), C.POINTER(OrCost),
                                _PD, _PD, _PD, _PD, C.c_int, C.c_int, _D, _D, _PD,
                                C.c_uint64, C.c_uint32, C.c_int, _PD, _PD, C.c_int]
        L.or_replan.restype = C.c_int
        L.or_edt_bruteforce.argtypes = [C.POINTER(C.c_uint8), C.c_int, C.c_int, C.c_int,
                                        C.POINTER(C.c_int64)]
        L.or_eps_range.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, C.c_int, C.c_int, _PD, _PD]
        L.or_pose_metrics.argtypes = [C.POINTER(OrRobot), _PD, _PD, _PD]
        L.or_robot_mask.argtypes = [C.POINTER(OrRobot), _PD, C.c_int, C.c_int, C.c_int, C.c_double,
                                    _PD, C.c_double, C.POINTER(C.c_uint8)]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_PD)


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


# ----------------------------------------------------------- input structs
def make_robot(rb) -> OrRobot:
    r = OrRobot()
    n = int(rb["n_joints"])
    r.n_joints = n
    for j in range(n):
        r.a[j] = float(rb["a"][j]); r.d[j] = float(rb["d"][j])
        r.alpha[j] = float(rb["alpha"][j]); r.theta_offset[j] = float(rb["theta_offset"][j])
        r.q_min[j] = float(rb["q_min"][j]); r.q_max[j] = float(rb["q_max"][j])
        r.qd_max[j] = float(rb["qd_max"][j]); r.qdd_max[j] = float(rb["qdd_max"][j])
    r.flange_d = float(rb["flange_d"])
    ns = len(rb["sphere_radius"])
    assert ns <= MAX_S
    r.n_spheres = ns
    for s in range(ns):
        r.sphere_link[s] = int(rb["sphere_link"][s])
        for c in range(3):
            r.sphere_offset[s][c] = float(rb["sphere_offset"][s][c])
        r.sphere_radius[s] = float(rb["sphere_radius"][s])
    pairs = np.asarray(rb.get("self_pairs", np.zeros((0, 2))), dtype=np.int64).reshape(-1, 2)
    assert len(pairs) <= MAX_P
    r.n_pairs = len(pairs)
    for p, (a, b) in enumerate(pairs):
        r.pairs[p][0] = int(a); r.pairs[p][1] = int(b)
    return r


class Grid:
    """Keeps the float32 field alive while the C struct points into it."""

    def __init__(self, desc, phi):
        self.phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float32))
        assert self.phi.shape == (desc.nz, desc.ny, desc.nx)
        g = OrGrid()
        g.nx, g.ny, g.nz = desc.nx, desc.ny, desc.nz
        g.res = float(desc.res)
        for i in range(3):
            g.origin[i] = float(desc.origin[i])
        g.phi = self.phi.ctypes.data_as(C.POINTER(C.c_float))
        self.c = g


def make_cost(cp, n_joints=7) -> OrCost:
    c = OrCost()
    for i in range(6):
        c.Q[i] = float(cp["Q"][i]); c.QH[i] = float(cp["QH"][i])
    for k in ("w_env", "d_act", "w_self", "w_q", "w_qd", "w_qdd", "margin_frac", "w_s", "w_ns"):
        setattr(c, k, float(cp[k]))
    for j in range(n_joints):
        c.q_ref[j] = float(cp["q_ref"][j])
    return c


# ----------------------------------------------------------- primitives
def philox(ctr, key):
    """Philox4x32-10 of each counter row (N x 4 uint32) under key (2 uint32)."""
    ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    key = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.empty_like(ctr)
    L = lib()
    P = C.POINTER(C.c_uint32)
    for i in range(len(ctr)):
        L.or_philox4x32_10(ctr[i].ctypes.data_as(P), key.ctypes.data_as(P),
                           out[i].ctypes.data_as(P))
    return out


def word_to_uniform(x):
    return lib().or_word_to_uniform(int(x))


def normals(seed, it, m, k):
    z = np.empty(8)
    lib().or_normals(int(seed), int(it), int(m), int(k), _dp(z))
    return z


def eps_range(seed, it, m0, count, H, sigma, n=7):
    """eps of roll-outs m0 .. m0+count-1: array (count, H, n), as eps_tensor."""
    sig = _f64(sigma)
    out = np.empty((int(count), int(H), n))
    lib().or_eps_range(int(seed), int(it), int(m0), int(count), int(H), n, _dp(sig), _dp(out))
    return out


def eps_tensor(seed, it, K, H, sigma, n=7):
    """eps[m, k, j] = sigma_j z_j(m, k) of the sampling step of Algorithm 1 (FP64)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    out = np.empty((K, H, n))
    z = np.empty(8)
    L = lib()
    for m in range(K):
        for k in range(H):
            L.or_normals(int(seed), int(it), m, k, _dp(z))
            out[m, k] = sigma[:n] * z[:n]
    return out


def fk(robot, q):
    """Frames T^0..T^n and the flange T^{n+1}: array (n+2, 4, 4)."""
    n = int(robot.n_joints)
    q = _f64(q)
    T = np.empty((n + 2, 4, 4))
    lib().or_fk(C.byref(robot), _dp(q), _dp(T))
    return T


def sphere_centres(robot, q):
    T = fk(robot, q)
    p = np.empty((robot.n_spheres, 3))
    lib().or_sphere_centres(C.byref(robot), _dp(T), _dp(p))
    return p


def phi(grid: Grid, points):
    pts = _f64(points).reshape(-1, 3)
    L = lib()
    return np.array([L.or_phi(C.byref(grid.c), _dp(np.ascontiguousarray(p))) for p in pts])


def se3_log(T):
    T = _f64(T, (4, 4))
    xi = np.empty(6)
    lib().or_se3_log(_dp(T), _dp(xi))
    return xi


def pose_error(Tg, Tee):
    Tg = _f64(Tg, (4, 4)); Tee = _f64(Tee, (4, 4))
    xi = np.empty(6)
    lib().or_pose_error(_dp(Tg), _dp(Tee), _dp(xi))
    return xi


def integrate(q0, qd0, u, dt):
    u = _f64(u)
    H, n = u.shape
    q = np.empty((H + 1, n)); qd = np.empty((H + 1, n))
    lib().or_integrate(n, H, float(dt), _dp(_f64(q0)), _dp(_f64(qd0)), _dp(u), _dp(q), _dp(qd))
    return q, qd


def rollout_cost(robot, grid, cost, q0, qd0, Tg, u, dt, trace=False):
    """S of Eq. 28 for one control sequence u [H][n]; optionally per-step terms."""
    u = _f64(u)
    H = u.shape[0]
    tr = np.empty((H + 1, T_COLS)) if trace else None
    S = lib().or_rollout(C.byref(robot), C.byref(grid.c), C.byref(cost),
                         _dp(_f64(q0)), _dp(_f64(qd0)), _dp(_f64(Tg, (4, 4))), _dp(u),
                         H, float(dt), _dp(tr) if trace else None)
    return (S, tr) if trace else S


def smpc_iterate(robot, grid, cost, q0, qd0, Tg, U, K, dt, lam, sigma, seed, it, n_threads=1):
    """One iteration of Alg. 1.  Returns (U*, costs S[K], weights w[K])."""
    U = _f64(U).copy()
    H = U.shape[0]
    S = np.empty(K); w = np.empty(K)
    rc = lib().or_smpc_iterate(C.byref(robot), C.byref(grid.c), C.byref(cost),
                               _dp(_f64(q0)), _dp(_f64(qd0)), _dp(_f64(Tg, (4, 4))), _dp(U),
                               int(K), int(H), float(dt), float(lam), _dp(_f64(sigma)),
                               int(seed), int(it), _dp(S), _dp(w), int(n_threads))
    if rc:
        raise ValueError(f"or_smpc_iterate failed: {rc}")
    return U, S, w


def replan(robot, grid, cost, q, qd, Tg, U, K, dt, lam, sigma, seed, replan_index, n_iters,
           n_threads=1):
    """One receding-horizon replan.  Returns (q', qd', U_shifted, u0*, best S)."""
    q = _f64(q).copy(); qd = _f64(qd).copy(); U = _f64(U).copy()
    H = U.shape[0]
    u0 = np.empty(U.shape[1]); best = np.empty(1)
    rc = lib().or_replan(C.byref(robot), C.byref(grid.c), C.byref(cost), _dp(q), _dp(qd),
                         _dp(_f64(Tg, (4, 4))), _dp(U), int(K), int(H), float(dt), float(lam),
                         _dp(_f64(sigma)), int(seed), int(replan_index), int(n_iters),
                         _dp(u0), _dp(best), int(n_threads))
    if rc:
        raise ValueError(f"or_replan failed: {rc}")
    return q, qd, U, u0, float(best[0])


def edt_bruteforce(occ):
    """Exact squared distances (voxel units) for occ of shape (nz, ny, nx)."""
    occ = np.ascontiguousarray(np.asarray(occ, dtype=np.uint8))
    nz, ny, nx = occ.shape
    D = np.empty(occ.shape, dtype=np.int64)
    lib().or_edt_bruteforce(occ.ctypes.data_as(C.POINTER(C.c_uint8)), nx, ny, nz,
                            D.ctypes.data_as(C.POINTER(C.c_int64)))
    return D


def cores_available():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def robot_mask(robot, grid_desc, q, occ, inflate=0.0):
    """Copy of occ (nz, ny, nx) with the voxels covered by the sphere model at
    q cleared (Sec. IV-B-2, Remark 2)."""
    out = np.ascontiguousarray(np.array(occ, dtype=np.uint8, copy=True))
    nz, ny, nx = out.shape
    origin = _f64(grid_desc.origin)
    lib().or_robot_mask(C.byref(robot), _dp(_f64(q)), nx, ny, nz, float(grid_desc.res), _dp(origin),
                        float(inflate), out.ctypes.data_as(C.POINTER(C.c_uint8)))
    return out


def pose_metrics(robot, q, Tg):
    """(e_pos [m], e_ori [rad]) of configuration q against the goal pose Tg
    (Sec. V-A pose error metrics)."""
    out = np.empty(2)
    lib().or_pose_metrics(C.byref(robot), _dp(_f64(q)), _dp(_f64(Tg).reshape(16).copy()), _dp(out))
    return float(out[0]), float(out[1])

