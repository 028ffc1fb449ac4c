"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test checks one function of oracle/smpc_oracle.c against something
independent of it: a hand-derived closed form, a library routine (scipy's
matrix exponential/logarithm and exact distance transform, Triton's Philox
run by its CPU interpreter), an invariant of the mathematics, or brute force.
The mistakes they are meant to catch are the plausible ones: a dropped term,
a wrong sign or index, a transposed operand, an off-by-one in the horizon.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
from scipy import stats

import oracle
import workloads
from workloads import scenes as ws

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def rb():
    return workloads.panda_robot()


@pytest.fixture(scope="module")
def R(rb):
    return oracle.make_robot(rb)


def rand_rot(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def hat(w):
    return np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])


def twist_matrix(xi):
    M = np.zeros((4, 4))
    M[:3, :3] = hat(xi[3:])
    M[:3, 3] = xi[:3]
    return M


# ------------------------------------------------------------------ Philox
def test_philox_matches_triton_interpreter():
    """Bit-exact against Triton's Philox4x32-10 (library), run on the CPU."""
    os.environ["TRITON_INTERPRET"] = "1"
    torch = pytest.importorskip("torch")
    triton = pytest.importorskip("triton")
    import triton.language as tl

    @triton.jit
    def philox_kernel(out_ptr, c_ptr, seed, N: tl.constexpr):
        i = tl.arange(0, N)
        c0 = tl.load(c_ptr + 4 * i)
        c1 = tl.load(c_ptr + 4 * i + 1)
        c2 = tl.load(c_ptr + 4 * i + 2)
        c3 = tl.load(c_ptr + 4 * i + 3)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
        tl.store(out_ptr + 4 * i, a)
        tl.store(out_ptr + 4 * i + 1, b)
        tl.store(out_ptr + 4 * i + 2, c)
        tl.store(out_ptr + 4 * i + 3, d)

    rng = np.random.default_rng(7)
    N = 64
    for seed in (0, 1, 0xDEADBEEF12345678, 2**64 - 1):
        ctr = rng.integers(0, 2**32, size=(N, 4), dtype=np.uint64).astype(np.uint32)
        ctr[0] = 0
        ctr[1] = 0xFFFFFFFF
        out = torch.zeros(4 * N, dtype=torch.uint32)
        cin = torch.from_numpy(ctr.view(np.int32).copy()).view(torch.uint32)
        philox_kernel[(1,)](out, cin, seed, N)
        tri = out.numpy().view(np.uint32).reshape(N, 4)
        orc = oracle.philox(ctr, [seed & 0xFFFFFFFF, seed >> 32])
        assert np.array_equal(tri, orc), f"seed {seed:#x}"


def test_uniform_map_endpoints_and_fp32_exactness():
    assert oracle.word_to_uniform(0) == 2.0**-24
    assert oracle.word_to_uniform(0xFFFFFFFF) == 1.0 - 2.0**-24
    assert oracle.word_to_uniform(0x80000000) == 0.5 + 2.0**-24
    # every value is a float32 number, so an FP32 implementation draws it exactly
    xs = np.random.default_rng(0).integers(0, 2**32, 20000, dtype=np.uint64).tolist()
    xs += [0, 1, 2**31 - 1, 2**31, 2**32 - 512, 2**32 - 1]
    for x in xs:
        u = oracle.word_to_uniform(x)
        assert float(np.float32(u)) == u and 0.0 < u < 1.0


def test_box_muller_invariants():
    """z0^2 + z1^2 = -2 ln u0 and atan2(z1, z0) = 2 pi u1 (mod 2 pi)."""
    seed, it = 0x1234, 5
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for m, k in [(0, 0), (3, 17), (255, 31), (4095, 63)]:
        z = oracle.normals(seed, it, m, k)
        for b in range(2):
            w = oracle.philox([[m, k, b, it]], key)[0]
            for p in range(2):
                u0 = oracle.word_to_uniform(w[2 * p])
                u1 = oracle.word_to_uniform(w[2 * p + 1])
                z0, z1 = z[4 * b + 2 * p], z[4 * b + 2 * p + 1]
                assert math.isclose(z0 * z0 + z1 * z1, -2 * math.log(u0), rel_tol=1e-12)
                ang = math.atan2(z1, z0) % (2 * math.pi)
                assert math.isclose(ang, (2 * math.pi * u1) % (2 * math.pi), abs_tol=1e-9)


def test_normals_moments_and_chi2():
    e = oracle.eps_tensor(99, 0, 512, 32, np.ones(7))  # 114 688 draws
    z = e.ravel()
    assert abs(z.mean()) < 0.015
    assert abs(z.var() - 1.0) < 0.02
    assert abs(stats.skew(z)) < 0.03
    assert abs(stats.kurtosis(z)) < 0.06
    edges = stats.norm.ppf(np.linspace(0, 1, 41))
    counts, _ = np.histogram(z, bins=edges)
    chi2 = ((counts - len(z) / 40) ** 2 / (len(z) / 40)).sum()
    assert chi2 < stats.chi2.ppf(0.999, 39)
    c = np.corrcoef(e.reshape(-1, 7).T)
    # 21 pairs of 16 384 samples: the correlation's standard error is 1/sqrt(N)
    assert np.abs(c - np.eye(7)).max() < 4.5 / math.sqrt(e.shape[0] * e.shape[1])


# --------------------------------------------------------------- kinematics
def test_home_pose_golden(R):
    g = json.load(open(os.path.join(GOLDEN, "home_pose.json")))
    T = oracle.fk(R, np.zeros(7))
    # the DH inputs are float32 values (0.0825f, pi/2 as float32 whose cosine
    # is -4.4e-8), which moves the closed form by ~1e-8 m
    assert np.allclose(T[-1][:3, 3], g["flange_position"], atol=1e-7)
    assert np.allclose(T[-1][:3, :3], g["flange_rotation"], atol=1e-7)
    for i, z in g["frame_origins_z"].items():
        assert math.isclose(T[int(i)][2, 3], z, abs_tol=1e-7)


def test_fk_matches_product_of_exponentials(R, rb):
    """Space-frame PoE from the home frames equals the DH chain at random q."""
    n = 7
    H0 = oracle.fk(R, np.zeros(n))
    M = H0[-1]
    screws = []
    for i in range(1, n + 1):
        w = H0[i][:3, 2]
        p = H0[i][:3, 3]
        screws.append(np.concatenate([-np.cross(w, p), w]))
    rng = np.random.default_rng(3)
    for _ in range(20):
        q = rng.uniform(rb["q_min"], rb["q_max"])
        T = np.eye(4)
        for S, qi in zip(screws, q):
            T = T @ sla.expm(twist_matrix(S) * qi)
        T = T @ M
        Td = oracle.fk(R, q)
        assert np.allclose(Td[-1], T, atol=1e-10)
        Rm = Td[-1][:3, :3]
        assert np.allclose(Rm.T @ Rm, np.eye(3), atol=1e-12)


def test_sphere_centres_on_link_segments(R, rb):
    """Centres sit at fractions (j+0.5)/4 of frame i -> frame i+1 origins."""
    rng = np.random.default_rng(4)
    for _ in range(5):
        q = rng.uniform(rb["q_min"], rb["q_max"])
        T = oracle.fk(R, q)
        p = oracle.sphere_centres(R, q)
        for s in range(len(rb["sphere_radius"])):
            L = int(rb["sphere_link"][s])
            frac = (s % 4 + 0.5) / 4
            a, b = T[L][:3, 3], T[L + 1][:3, 3]
            if np.linalg.norm(b - a) < 1e-9:  # zero-length link: -z of frame L
                exp = a + frac * T[L][:3, :3] @ np.array([0, 0, -0.10])
            else:
                exp = a + frac * (b - a)
            assert np.allclose(p[s], exp, atol=1e-6)


# ------------------------------------------------------------ distance field
def test_trilinear_exact_on_affine_field():
    g = ws.GridDesc(9, 7, 6, 0.05, (-0.2, 0.1, 0.0))
    x, y, z = ws.voxel_centres(g)
    a = np.array([0.3, -0.7, 1.1])
    field = (a[0] * x + a[1] * y + a[2] * z + 0.25).astype(np.float32)
    G = oracle.Grid(g, field)
    rng = np.random.default_rng(5)
    lo = np.array(g.origin) + 0.5 * g.res
    hi = np.array(g.origin) + (np.array([g.nx, g.ny, g.nz]) - 0.5) * g.res
    pts = rng.uniform(lo, hi, size=(200, 3))
    ref = pts @ a + 0.25
    # the float32 grid samples carry ~1e-7 rounding; interpolation is exact
    assert np.abs(oracle.phi(G, pts) - ref).max() < 5e-7
    # voxel centres return the stored value
    for (i, j, l) in [(0, 0, 0), (8, 6, 5), (3, 2, 4)]:
        c = np.array(g.origin) + (np.array([i, j, l]) + 0.5) * g.res
        assert oracle.phi(G, c)[0] == float(field[l, j, i])
    # outside: clamped to the nearest in-grid point (edge replication)
    out = np.array([[-5.0, 0.3, 0.1], [0.0, 9.0, -3.0]])
    clamped = np.clip(out, lo, hi)
    assert np.allclose(oracle.phi(G, out), oracle.phi(G, clamped), atol=0)


def _analytic_distance(obstacles, pts):
    d = np.full(len(pts), np.inf)
    for ob in obstacles:
        c = np.asarray(ob["center"])
        if ob["type"] == "box":
            q = np.maximum(np.abs(pts - c) - np.asarray(ob["half"]), 0.0)
            d = np.minimum(d, np.linalg.norm(q, axis=1))
        else:
            d = np.minimum(d, np.maximum(np.linalg.norm(pts - c, axis=1) - ob["radius"], 0.0))
    return d


@pytest.mark.parametrize("name", ["cfg1_seed0", "cfg1_seed3"])
def test_grid_equals_bruteforce_edt(name):
    """The input grid (scipy EDT) equals the oracle's brute-force transform."""
    sc = workloads.load_scene(name)
    g = sc["grid"]
    occ = ws.occupancy_grid(sc["obstacles"], g)
    D = oracle.edt_bruteforce(occ)
    ref = (np.sqrt(D.astype(np.float64)) * g.res).astype(np.float32)
    assert np.array_equal(ref, workloads.build_scene_grid(sc))


def test_bruteforce_edt_tiny_exhaustive():
    rng = np.random.default_rng(6)
    occ = (rng.random((5, 6, 7)) < 0.08).astype(np.uint8)
    occ[2, 3, 4] = 1
    D = oracle.edt_bruteforce(occ)
    idx = np.argwhere(occ)
    for l in range(5):
        for j in range(6):
            for i in range(7):
                ref = ((idx - [l, j, i]) ** 2).sum(1).min()
                assert D[l, j, i] == ref


@pytest.mark.parametrize("name", ["cfg1_seed1", "cfg1_seed5"])
def test_grid_brackets_analytic_distance(name):
    """d <= phi_vox <= d + sqrt(3) res at voxel centres (convex obstacles).

    phi_vox is a distance to a point inside an obstacle, so it cannot be
    below the distance d to the union; and for obstacles several voxels
    thick an occupied centre lies within res along the normal and res/2
    tangentially of the nearest surface point, i.e. within sqrt(3) res.
    """
    sc = workloads.load_scene(name)
    g = sc["grid"]
    phi = workloads.build_scene_grid(sc)
    x, y, z = ws.voxel_centres(g)
    pts = np.stack(np.broadcast_arrays(x, y, z), -1).reshape(-1, 3)
    d = _analytic_distance(sc["obstacles"], pts)
    f = phi.reshape(-1).astype(np.float64)
    assert np.all(f >= d - 1e-6)
    assert np.all(f <= d + math.sqrt(3) * g.res + 1e-6)


# -------------------------------------------------------------------- SE(3)
def test_se3_log_identity_is_zero():
    assert np.array_equal(oracle.se3_log(np.eye(4)), np.zeros(6))


def test_se3_log_matches_scipy_logm_and_expm():
    rng = np.random.default_rng(8)
    for trial in range(60):
        th = [1e-7, 1e-4, 0.01, 0.5, 1.5, 2.5, 3.0, math.pi - 0.01][trial % 8]
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        T = np.eye(4)
        T[:3, :3] = sla.expm(hat(th * axis))
        T[:3, 3] = rng.normal(size=3) * 0.5
        xi = oracle.se3_log(T)
        assert np.allclose(sla.expm(twist_matrix(xi)), T, atol=1e-10)
        L = np.real(sla.logm(T))
        ref = np.concatenate([L[:3, 3], [L[2, 1], L[0, 2], L[1, 0]]])
        assert np.allclose(xi, ref, atol=1e-8), (th, xi, ref)


def test_se3_log_near_pi_represents_rotation():
    rng = np.random.default_rng(9)
    for th in [math.pi - 1e-7, math.pi]:
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        T = np.eye(4)
        T[:3, :3] = sla.expm(hat(th * axis))
        T[:3, 3] = [0.1, -0.2, 0.3]
        xi = oracle.se3_log(T)
        assert math.isclose(np.linalg.norm(xi[3:]), th, abs_tol=1e-6)
        assert np.allclose(sla.expm(twist_matrix(xi)), T, atol=1e-6)


def test_pose_error_special_cases():
    rng = np.random.default_rng(10)
    Tg = np.eye(4)
    Tg[:3, :3] = rand_rot(rng)
    Tg[:3, 3] = [0.3, -0.1, 0.6]
    assert np.allclose(oracle.pose_error(Tg, Tg), 0, atol=1e-12)
    # pure translation in the goal frame: v = d, omega = 0
    d = np.array([0.05, -0.02, 0.1])
    Te = Tg.copy()
    Te[:3, 3] = Tg[:3, 3] + Tg[:3, :3] @ d
    xi = oracle.pose_error(Tg, Te)
    assert np.allclose(xi[:3], d, atol=1e-12) and np.allclose(xi[3:], 0, atol=1e-12)
    # pure rotation about the goal origin: v = 0, omega = theta a (goal frame)
    a = np.array([1.0, 2.0, -2.0]) / 3.0
    Te = Tg.copy()
    Te[:3, :3] = Tg[:3, :3] @ sla.expm(hat(0.7 * a))
    xi = oracle.pose_error(Tg, Te)
    assert np.allclose(xi[:3], 0, atol=1e-12) and np.allclose(xi[3:], 0.7 * a, atol=1e-12)


# --------------------------------------------------------------- integrator
def test_integrator_constant_acceleration_closed_form():
    H, dt = 40, 0.02
    q0 = np.array([0.1, -0.2, 0.3, -1.0, 0.0, 1.2, 0.5])
    qd0 = np.array([0.5, 0.0, -0.3, 0.2, 0.1, 0.0, -0.4])
    u = np.array([1.0, -2.0, 0.5, 0.0, 3.0, -1.0, 0.25])
    q, qd = oracle.integrate(q0, qd0, np.tile(u, (H, 1)), dt)
    k = np.arange(H + 1)[:, None]
    assert np.allclose(qd, qd0 + k * dt * u, atol=1e-13)
    assert np.allclose(q, q0 + k * dt * qd0 + dt * dt * u * k * (k + 1) / 2, atol=1e-13)


# -------------------------------------------------------------------- costs
@pytest.fixture(scope="module")
def flat_grid():
    g = ws.GridDesc(8, 8, 8, 0.25, (-1.0, -1.0, 0.0))
    return g


def _costs(**over):
    cp = {"Q": np.zeros(6), "QH": np.zeros(6), "w_env": 0.0, "d_act": 0.05, "w_self": 0.0,
          "w_q": 0.0, "w_qd": 0.0, "w_qdd": 0.0, "margin_frac": 0.05, "w_s": 0.0, "w_ns": 0.0,
          "q_ref": np.zeros(7)}
    cp.update(over)
    return cp


def _grid(g, value):
    return oracle.Grid(g, np.full((g.nz, g.ny, g.nx), value, dtype=np.float32))


def _pose_cost(Q, Tg, Tee):
    L = np.real(sla.logm(np.linalg.inv(Tg) @ Tee))
    xi = np.concatenate([L[:3, 3], [L[2, 1], L[0, 2], L[1, 0]]])
    return 0.5 * np.sum(np.asarray(Q) * xi * xi)


def test_static_pose_and_terminal_costs(R, rb, flat_grid):
    """Static arm (qd0 = 0, u = 0): S = H pose_Q + pose_QH, both via logm."""
    H, dt = 12, 0.02
    q0 = workloads.READY_POSE.astype(np.float64)
    Tg = np.eye(4)
    Tg[:3, :3] = sla.expm(hat([0.3, -0.2, 0.5]))
    Tg[:3, 3] = [0.4, 0.2, 0.5]
    Q = [0.2, 0.3, 0.4, 0.05, 0.06, 0.07]
    QH = [2.0, 1.0, 3.0, 0.5, 0.2, 0.1]
    Tee = oracle.fk(R, q0)[-1]
    G = _grid(flat_grid, 1.0)
    S, tr = oracle.rollout_cost(R, G, oracle.make_cost(_costs(Q=Q)), q0, np.zeros(7), Tg,
                                np.zeros((H, 7)), dt, trace=True)
    assert math.isclose(S, H * _pose_cost(Q, Tg, Tee), rel_tol=1e-10)
    assert tr[H].sum() == 0.0  # Q is not applied at k = H
    S = oracle.rollout_cost(R, G, oracle.make_cost(_costs(QH=QH)), q0, np.zeros(7), Tg,
                            np.zeros((H, 7)), dt)
    assert math.isclose(S, _pose_cost(QH, Tg, Tee), rel_tol=1e-10)


def test_terminal_cost_uses_state_H(R, flat_grid):
    """Constant u: the terminal cost is evaluated at q_H (not q_{H-1})."""
    H, dt = 10, 0.05
    q0 = workloads.READY_POSE.astype(np.float64)
    u = np.array([0.5, -0.4, 0.3, 0.2, -0.6, 0.1, 0.7])
    qH = q0 + dt * dt * u * H * (H + 1) / 2
    Tg = oracle.fk(R, q0)[-1]
    QH = [1.0, 1.0, 1.0, 0.3, 0.3, 0.3]
    S = oracle.rollout_cost(R, _grid(flat_grid, 1.0), oracle.make_cost(_costs(QH=QH)), q0,
                            np.zeros(7), Tg, np.tile(u, (H, 1)), dt)
    assert math.isclose(S, _pose_cost(QH, Tg, oracle.fk(R, qH)[-1]), rel_tol=1e-9)


def test_env_cost_uniform_field(R, rb, flat_grid):
    """phi = c everywhere: each sphere adds w (max(0, d_act - (c - r)))^2 per step."""
    H, dt = 6, 0.02
    q0 = workloads.READY_POSE.astype(np.float64)
    r = rb["sphere_radius"].astype(np.float64)
    for c in (0.0, 0.09, 0.12, 1.0):
        S = oracle.rollout_cost(R, _grid(flat_grid, c), oracle.make_cost(_costs(w_env=100.0)),
                                q0, np.zeros(7), np.eye(4), np.zeros((H, 7)), dt)
        ref = H * 100.0 * np.sum(np.maximum(0.0, 0.05 - (np.float32(c) - r)) ** 2)
        assert math.isclose(S, ref, rel_tol=1e-12, abs_tol=1e-15)


def test_env_cost_affine_field(R, rb):
    """Affine field: phi(p) at each sphere centre is a.p + b (FK-independent check)."""
    g = ws.GridDesc(40, 40, 40, 0.05, (-1.0, -1.0, 0.0))
    x, y, z = ws.voxel_centres(g)
    a = np.array([0.01, 0.02, 0.05])
    G = oracle.Grid(g, (a[0] * x + a[1] * y + a[2] * z + 0.02).astype(np.float32))
    q0 = workloads.READY_POSE.astype(np.float64)
    p = oracle.sphere_centres(R, q0)
    r = rb["sphere_radius"].astype(np.float64)
    S = oracle.rollout_cost(R, G, oracle.make_cost(_costs(w_env=7.0, d_act=0.2)), q0,
                            np.zeros(7), np.eye(4), np.zeros((1, 7)), 0.02)
    ref = 7.0 * np.sum(np.maximum(0.0, 0.2 - (p @ a + 0.02 - r)) ** 2)
    assert math.isclose(S, ref, rel_tol=1e-6)


def test_self_collision_cost(R, rb, flat_grid):
    """Pairs on one link: |p_i - p_j| = |i - j| L/4 on a straight segment."""
    rbp = dict(rb)
    rbp["self_pairs"] = np.array([[4, 5], [4, 6], [8, 10]], dtype=np.int32)
    Rp = oracle.make_robot(rbp)
    q0 = workloads.READY_POSE.astype(np.float64)
    T = oracle.fk(Rp, q0)
    r = rb["sphere_radius"].astype(np.float64)
    ref = 0.0
    for i, j in rbp["self_pairs"]:
        L = np.linalg.norm(T[rb["sphere_link"][i] + 1][:3, 3] - T[rb["sphere_link"][i]][:3, 3])
        d = abs(int(i) - int(j)) * L / 4 - (r[i] + r[j])
        ref += 3.0 * max(0.0, -d) ** 2
    S = oracle.rollout_cost(Rp, _grid(flat_grid, 5.0), oracle.make_cost(_costs(w_self=3.0)),
                            q0, np.zeros(7), np.eye(4), np.zeros((1, 7)), 0.02)
    assert ref > 0
    # sphere offsets are float32-rounded fractions of the segment (~1e-8 m)
    assert math.isclose(S, ref, rel_tol=1e-6)


def test_joint_limit_costs(R, rb, flat_grid):
    """Known violations of the tightened box for q, qd and qdd."""
    H, dt = 5, 0.01
    lo, hi = rb["q_min"].astype(np.float64), rb["q_max"].astype(np.float64)
    e = 0.05 * (hi - lo)
    q0 = 0.5 * (lo + hi)
    q0[1] = hi[1] - e[1] + 0.03           # q above the tightened maximum
    q0[3] = lo[3] + e[3] - 0.02           # q below the tightened minimum
    qdm = rb["qd_max"].astype(np.float64)
    qddm = rb["qdd_max"].astype(np.float64)
    u = np.zeros(7)
    u[5] = -(qddm[5] - 0.1 * qddm[5]) - 0.5  # 0.5 below -qdd_max + eps
    cp = _costs(w_q=2.0, w_qd=3.0, w_qdd=5.0)
    q, qd = oracle.integrate(q0, np.zeros(7), np.tile(u, (H, 1)), dt)
    ref = 0.0
    for k in range(H):
        for j in range(7):
            for x, l, h, w in ((q[k, j], lo[j], hi[j], 2.0), (qd[k, j], -qdm[j], qdm[j], 3.0),
                               (u[j], -qddm[j], qddm[j], 5.0)):
                eps = 0.05 * (h - l)
                dv = max(0.0, x - (h - eps)) + min(0.0, x - (l + eps))
                ref += w * dv * dv
    S = oracle.rollout_cost(R, _grid(flat_grid, 5.0), oracle.make_cost(cp), q0, np.zeros(7),
                            np.eye(4), np.tile(u, (H, 1)), dt)
    assert math.isclose(S, ref, rel_tol=1e-12)
    # first step alone: w_q (0.03^2 + 0.02^2) + w_qdd 0.5^2 (qd_0 = 0)
    S1 = oracle.rollout_cost(R, _grid(flat_grid, 5.0), oracle.make_cost(cp), q0, np.zeros(7),
                             np.eye(4), np.tile(u, (1, 1)), dt)
    assert math.isclose(S1, 2.0 * (0.03**2 + 0.02**2) + 5.0 * 0.5**2, rel_tol=1e-9)


def test_smooth_and_nullspace_costs(R, flat_grid):
    H, dt = 7, 0.02
    q0 = workloads.READY_POSE.astype(np.float64)
    qref = q0 + np.array([0.1, -0.1, 0.2, 0.0, 0.05, -0.3, 0.0])
    u = np.array([0.3, -0.2, 0.1, 0.4, -0.5, 0.6, -0.7])
    cp = _costs(w_s=0.7, w_ns=0.9, q_ref=qref)
    q, _ = oracle.integrate(q0, np.zeros(7), np.tile(u, (H, 1)), dt)
    ref = H * 0.7 * np.sum(u * u) + 0.9 * np.sum((q[:H] - qref) ** 2)
    S = oracle.rollout_cost(R, _grid(flat_grid, 5.0), oracle.make_cost(cp), q0, np.zeros(7),
                            np.eye(4), np.tile(u, (H, 1)), dt)
    assert math.isclose(S, ref, rel_tol=1e-12)


# -------------------------------------------------------------- Algorithm 1
@pytest.fixture(scope="module")
def cfg1():
    sc = workloads.load_scene("cfg1_seed2")
    G = oracle.Grid(sc["grid"], workloads.build_scene_grid(sc))
    C = oracle.make_cost(workloads.default_cost_params(sc["q0"]))
    return sc, G, C


def test_zero_noise_reproduces_nominal(R, cfg1):
    sc, G, C = cfg1
    H, K = 16, 32
    rng = np.random.default_rng(11)
    Ubar = rng.normal(size=(H, 7)) * 0.3
    Us, S, w = oracle.smpc_iterate(R, G, C, sc["q0"], sc["qd0"], sc["T_goal"], Ubar, K, 0.02,
                                   0.05, np.zeros(7), 5, 0)
    assert np.array_equal(Us, Ubar)
    nominal = oracle.rollout_cost(R, G, C, sc["q0"], sc["qd0"], sc["T_goal"], Ubar, 0.02)
    assert np.all(S == nominal)
    assert np.allclose(w, 1.0 / K)


def test_lambda_to_zero_selects_argmin(R, cfg1):
    sc, G, C = cfg1
    H, K, sig = 16, 64, np.full(7, 0.5)
    Ubar = np.zeros((H, 7))
    Us, S, w = oracle.smpc_iterate(R, G, C, sc["q0"], sc["qd0"], sc["T_goal"], Ubar, K, 0.02,
                                   1e-12, sig, 6, 2)
    eps = oracle.eps_tensor(6, 2, K, H, sig)
    m = int(np.argmin(S))
    assert np.allclose(Us, Ubar + eps[m], atol=1e-15)


def test_lambda_to_infinity_averages(R, cfg1):
    sc, G, C = cfg1
    H, K, sig = 16, 64, np.full(7, 0.5)
    Us, S, w = oracle.smpc_iterate(R, G, C, sc["q0"], sc["qd0"], sc["T_goal"], np.zeros((H, 7)),
                                   K, 0.02, 1e12, sig, 6, 2)
    eps = oracle.eps_tensor(6, 2, K, H, sig)
    assert np.allclose(Us, eps.mean(0), atol=1e-12)


def test_iterate_costs_weights_update_consistent(R, cfg1):
    """S_m equals the single roll-out of U + eps_m; U* = sum_m w_m U^(m); sum w = 1."""
    sc, G, C = cfg1
    H, K, sig, lam = 16, 48, np.array([0.5, 0.4, 0.3, 0.5, 0.6, 0.7, 0.2]), 0.05
    rng = np.random.default_rng(12)
    Ubar = rng.normal(size=(H, 7)) * 0.2
    Us, S, w = oracle.smpc_iterate(R, G, C, sc["q0"], sc["qd0"], sc["T_goal"], Ubar, K, 0.02,
                                   lam, sig, 77, 3)
    eps = oracle.eps_tensor(77, 3, K, H, sig)
    for m in (0, 17, K - 1):
        ref = oracle.rollout_cost(R, G, C, sc["q0"], sc["qd0"], sc["T_goal"], Ubar + eps[m], 0.02)
        assert S[m] == ref
    assert math.isclose(w.sum(), 1.0, rel_tol=1e-14)
    assert w[np.argmin(S)] == w.max()
    assert np.allclose(Us, np.einsum("m,mkj->kj", w, Ubar[None] + eps), atol=1e-13)
    # weights depend only on cost differences: exp(-(S_a - S_b)/lam) = w_a / w_b
    a, b = 3, 9
    assert math.isclose(w[a] / w[b], math.exp(-(S[a] - S[b]) / lam), rel_tol=1e-10)


def test_costs_independent_of_K(R, cfg1):
    sc, G, C = cfg1
    H, sig = 16, np.full(7, 0.5)
    _, S1, _ = oracle.smpc_iterate(R, G, C, sc["q0"], sc["qd0"], sc["T_goal"], np.zeros((H, 7)),
                                   32, 0.02, 0.05, sig, 8, 0)
    _, S2, _ = oracle.smpc_iterate(R, G, C, sc["q0"], sc["qd0"], sc["T_goal"], np.zeros((H, 7)),
                                   96, 0.02, 0.05, sig, 8, 0)
    assert np.array_equal(S1, S2[:32])


def test_replan_shift_and_state_advance(R, cfg1):
    sc, G, C = cfg1
    H, K, sig, dt = 8, 16, np.full(7, 0.5), 0.02
    U0 = np.zeros((H, 7))
    q, qd, Un, u0, best = oracle.replan(R, G, C, sc["q0"], sc["qd0"], sc["T_goal"], U0, K, dt,
                                        0.05, sig, 21, 4, 3)
    U = U0.copy()
    for it in range(3):
        U, S, _ = oracle.smpc_iterate(R, G, C, sc["q0"], sc["qd0"], sc["T_goal"], U, K, dt, 0.05,
                                      sig, 21, 4 * 3 + it)
    assert np.array_equal(u0, U[0])
    assert best == S.min()
    qd_ref = sc["qd0"].astype(np.float64) + dt * U[0]
    assert np.allclose(qd, qd_ref, atol=0) and np.allclose(q, sc["q0"] + dt * qd_ref, atol=0)
    assert np.array_equal(Un[:-1], U[1:]) and np.array_equal(Un[-1], U[-1])


def test_robot_mask_single_sphere():
    """One sphere at the origin of frame 1, which sits at (0, 0, d_1) for every
    q: the mask clears exactly the voxels whose centres lie in that closed
    ball (radius + inflate) and nothing else."""
    rb = workloads.panda_robot()
    one = dict(rb)
    one["sphere_link"] = np.array([1], np.int32)
    one["sphere_offset"] = np.zeros((1, 3), np.float32)
    one["sphere_radius"] = np.array([0.05], np.float32)
    one["self_pairs"] = np.zeros((0, 2), np.int32)
    R1 = oracle.make_robot(one)
    g = workloads.GridDesc(nx=24, ny=20, nz=30, res=0.01, origin=(-0.12, -0.1, 0.2))
    rng = np.random.default_rng(4)
    occ = (rng.random(g.shape) < 0.5).astype(np.uint8)
    centre = np.array([0.0, 0.0, float(rb["d"][0])])
    l, j, i = np.meshgrid(np.arange(g.nz), np.arange(g.ny), np.arange(g.nx), indexing="ij")
    cx = g.origin[0] + (i + 0.5) * g.res
    cy = g.origin[1] + (j + 0.5) * g.res
    cz = g.origin[2] + (l + 0.5) * g.res
    d2 = (cx - centre[0]) ** 2 + (cy - centre[1]) ** 2 + (cz - centre[2]) ** 2
    for inflate in (0.0, 0.013):
        q = rng.uniform(-1.0, 1.0, 7)
        got = oracle.robot_mask(R1, g, q, occ, inflate)
        inside = d2 <= (float(np.float32(0.05)) + inflate) ** 2
        assert inside.sum() > 100
        assert np.array_equal(got, np.where(inside, 0, occ))


def test_pose_metrics_against_scipy_rotations(R):
    """e_pos is the flange distance; e_ori = 2 arccos|q_g . q| equals the
    magnitude of the relative rotation R_g^T R (scipy), including near pi."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(8)
    for t in range(20):
        q = rng.uniform(-2.0, 2.0, 7)
        T = oracle.fk(R, q)[-1]
        if t < 10:
            rot = Rotation.from_rotvec(rng.normal(size=3) * (0.3 + 0.3 * t))
        else:   # near pi
            ax = rng.normal(size=3)
            rot = Rotation.from_rotvec(ax / np.linalg.norm(ax) * (np.pi - 10.0 ** -(t - 8)))
        Tg = np.eye(4)
        Tg[:3, :3] = T[:3, :3] @ rot.as_matrix()
        Tg[:3, 3] = T[:3, 3] + rng.normal(size=3) * 0.05
        e_pos, e_ori = oracle.pose_metrics(R, q, Tg)
        assert math.isclose(e_pos, np.linalg.norm(Tg[:3, 3] - T[:3, 3]), rel_tol=1e-12)
        ref = Rotation.from_matrix(Tg[:3, :3].T @ T[:3, :3]).magnitude()
        assert abs(e_ori - ref) <= 2e-7, (t, e_ori, ref)


def test_eps_range_equals_eps_tensor():
    sig = np.array([0.5, 0.1, 1.0, 2.0, 0.25, 0.75, 1.5])
    full = oracle.eps_tensor(99, 4, 12, 9, sig)
    assert np.array_equal(oracle.eps_range(99, 4, 5, 6, 9, sig), full[5:11])
