"""The SE(3) pose error of the CUDA path in every regime of its rotation angle.

The kernel's log map (Eqs. 12-15) has three branches in theta: a series below
1e-4 (and for the V(theta)^-1 coefficient below 1e-2), the quotient form in
between, and above pi - 0.05 an axis taken from the symmetric part of the
rotation with the sign from its skew part.  The cost of Eqs. 16 and 25 is
discontinuous at theta = pi, where both signs of the axis are valid logs.

Checks, all against the FP64 oracle:
  * pm_pose_error (the kernel's device function) on float32 pose pairs whose
    relative rotation is set to theta in {0, 1e-6, ..., pi - 1e-5} about
    several axes, with translations up to 1 m: xi = [v; w] component by
    component, against the oracle's log of the relative pose (and, where the
    oracle's quotient branch is well conditioned, of the same float32 pair);
  * at theta = pi (ambiguous sign): |w| = pi and exp(xi) reproduces the
    relative pose;
  * pm_rollout_trace with sigma = 0, U = 0 and zero start velocity (every
    step holds the start pose) against goals at those angles: the pose terms
    of every step and the terminal term;
  * full iterations whose roll-outs sweep the near-pi and the small-angle
    branches: costs of every roll-out (those passing within 1e-3 of pi are
    skipped and counted, as the cost is discontinuous there), U* and the
    FP64 update from the GPU's own costs.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm

import oracle
from parity_common import S_REL, U_ABS, U_ISO, Scene, fp64_update_from_costs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2512_22575_b300 as pm  # noqa: E402

DEV = torch.device("cuda:0")
PI = math.pi
THETAS = [0.0, 1e-6, 5e-5, 1e-4, 2e-4, 5e-3, 9e-3, 1.1e-2, 1.0, 2.5, PI - 0.1, PI - 0.06,
          PI - 0.04, PI - 1e-2, PI - 1e-3, PI - 1e-5]
# Tolerances of xi = [v; w] from float32 poses.  The inputs are rounded to
# float32, so the relative rotation they represent is orthogonal only to a
# few units of 2^-24, and the log's axis from the skew part of R (the
# quotient branch) amplifies that by kappa = theta / (2 sin theta): up to 31
# at pi - 0.05, where the kernel switches to the symmetric part (kappa ~ 1).
# Bar: |xi - xi_ref| <= XI_ATOL + XI_RTOL |xi_ref| + 8 2^-24 kappa (1 + |t|).
XI_ATOL = 2e-6
XI_RTOL = 1e-5
POSE_RTOL = 1e-4       # pose terms of the trace, as the other per-step terms
POSE_ATOL = 1e-9


def kernel_kappa(th):
    """Condition number of the kernel's branch for theta (1 in the series and
    symmetric-part branches)."""
    return th / (2 * math.sin(th)) if 1e-4 <= th < PI - 0.05 else 1.0


def rot(axis, th):
    """Rotation by th about a unit axis (Rodrigues; an input generator)."""
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * K @ K


def pose(R, t):
    T = np.eye(4)
    T[:3, :3], T[:3, 3] = R, t
    return T


AXES = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1), (0.3, -0.8, 0.52), (-0.6, 0.1, -0.79)]


def pose_pairs(rng):
    """(T_g, T, theta, T_delta) with T_g^-1 T = T_delta = (Rot(theta, axis),
    t_delta) before T_g and T are rounded to float32."""
    out = []
    for th in THETAS:
        for ax in AXES:
            for tn in (0.0, 0.05, 1.0):
                Rg = rot(rng.normal(size=3), rng.uniform(0, PI))
                Tg = pose(Rg, rng.uniform(-0.8, 0.8, 3))
                td = rng.normal(size=3)
                td = tn * td / np.linalg.norm(td)
                D = pose(rot(ax, th), td)
                out.append((Tg.astype(np.float32), (Tg @ D).astype(np.float32), th, D))
    return out


def gpu_pose_error(Tg, T):
    n = len(Tg)
    a = torch.from_numpy(np.ascontiguousarray(Tg).reshape(n, 16)).to(DEV)
    b = torch.from_numpy(np.ascontiguousarray(T).reshape(n, 16)).to(DEV)
    xi = torch.empty((n, 6), dtype=torch.float32, device=DEV)
    pm.pose_error(a, b, xi)
    torch.cuda.synchronize()
    return xi.cpu().numpy().astype(np.float64)


def test_pose_error_in_every_regime_matches_oracle():
    """Every theta: the kernel's xi from the float32 poses against the
    oracle's log of the relative pose those poses represent (FP64, exactly
    orthogonal); where the oracle's own branch is well conditioned
    (theta <= 2.5), also against the oracle on the same float32 poses."""
    rng = np.random.default_rng(2024)
    pairs = pose_pairs(rng)
    xi = gpu_pose_error(np.stack([p[0] for p in pairs]), np.stack([p[1] for p in pairs]))
    worst = {}
    for i, (g, e, th, D) in enumerate(pairs):
        tn = float(np.linalg.norm(D[:3, 3]))
        slack = 8 * 2.0 ** -24 * kernel_kappa(th) * (1 + tn)
        ref = oracle.se3_log(D)
        err = np.abs(xi[i] - ref)
        assert np.all(err <= XI_ATOL + XI_RTOL * np.abs(ref) + slack), (th, tn, xi[i], ref)
        if th <= 2.5:
            ref32 = oracle.pose_error(g.astype(np.float64), e.astype(np.float64))
            err32 = np.abs(xi[i] - ref32)
            assert np.all(err32 <= XI_ATOL + XI_RTOL * np.abs(ref32) + slack), (th, tn, xi[i], ref32)
        worst[th] = max(worst.get(th, 0.0), float(err.max()))
    ths = np.array([p[2] for p in pairs])
    # every branch of the kernel was reached
    assert (ths < 1e-4).any() and ((ths >= 1e-4) & (ths < 1e-2)).any()
    assert ((ths >= 1e-2) & (ths < PI - 0.05)).any() and (ths >= PI - 0.05).any()
    print("max |xi - xi_ref| by theta:", {f"{k:.6g}": f"{v:.1e}" for k, v in worst.items()})


def test_pose_error_at_pi_is_a_valid_log():
    """theta = pi: either sign of the axis is a logarithm.  What is unique is
    checked: |w| = pi and exp([v; w]) = the relative pose."""
    rng = np.random.default_rng(7)
    Tgs, Ts, rels = [], [], []
    for ax in AXES:
        for tn in (0.0, 0.3):
            Tg = pose(rot(rng.normal(size=3), rng.uniform(0, PI)), rng.uniform(-0.5, 0.5, 3))
            td = rng.normal(size=3)
            td = tn * td / np.linalg.norm(td)
            T = Tg @ pose(rot(ax, PI), td)
            Tg32, T32 = Tg.astype(np.float32), T.astype(np.float32)
            Tgs.append(Tg32)
            Ts.append(T32)
            rels.append(np.linalg.inv(Tg32.astype(np.float64)) @ T32.astype(np.float64))
    xi = gpu_pose_error(np.stack(Tgs), np.stack(Ts))
    for x, D in zip(xi, rels):
        assert abs(np.linalg.norm(x[3:]) - PI) <= 1e-5
        tw = np.zeros((4, 4))
        w = x[3:]
        tw[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
        tw[:3, 3] = x[:3]
        assert np.abs(expm(tw) - D).max() <= 1e-5


# ------------------------------------------------ through the iteration kernel
@pytest.fixture(scope="module")
def scene():
    return Scene("cfg1_seed0")


def start_flange(sc, q):
    return oracle.fk(sc.R, q.astype(np.float64))[-1]


@pytest.mark.parametrize("th", [0.0, 1e-6, 1e-4, 5e-3, 1.0, PI - 0.1, PI - 0.04, PI - 1e-3, PI - 1e-5])
def test_pose_terms_at_fixed_angles_through_the_trace(scene, th):
    """sigma = 0, U = 0, zero start velocity: every step's pose is the start
    pose, so every pose term sees relative rotation theta (set per goal, about
    several axes, with a small translation).  Running terms (Q) of steps
    1..H-1 and the terminal term (Q_H) against or_rollout's trace."""
    sc = scene
    K, H = 2, 8
    q0 = sc.q0
    qd0 = np.zeros(7, np.float32)
    Tee = start_flange(sc, q0)
    rng = np.random.default_rng(int(th * 1e6) + 3)
    p = sc.planner()
    U = np.zeros((H, 7), np.float32)
    for ax in AXES:
        td = rng.normal(size=3)
        td = 0.04 * td / np.linalg.norm(td)
        Tg = (Tee @ np.linalg.inv(pose(rot(ax, th), td))).astype(np.float32)
        tr = torch.zeros((K, H + 1, 8), dtype=torch.float32, device=DEV)
        p.rollout_trace(q0, qd0, Tg, U, K, 0.02, np.zeros(7, np.float32), 3, 0, tr)
        torch.cuda.synchronize()
        tr = tr.cpu().numpy()
        _, ref = oracle.rollout_cost(sc.R, sc.G, sc.C, q0, qd0, Tg, U, 0.02, trace=True)
        xi = oracle.pose_error(Tg.astype(np.float64), Tee)
        assert abs(np.linalg.norm(xi[3:]) - th) <= 1e-5     # the goal sets theta
        for m in range(K):
            got, want = tr[m, 1:, 0], ref[1:, 0]
            assert np.all(np.abs(got - want) <= POSE_ATOL + POSE_RTOL * np.abs(want)), (ax, got, want)
    p.close()


def rollout_angles(sc, q0, qd0, Tg, U, dt):
    """Relative rotation angle of every step k = 1..H of one roll-out (oracle FK)."""
    q, _ = oracle.integrate(q0, qd0, U, dt)
    Tg64 = Tg.astype(np.float64)
    return np.array([np.linalg.norm(oracle.pose_error(Tg64, oracle.fk(sc.R, q[k])[-1])[3:])
                     for k in range(1, len(q))])


def iterate_and_compare(sc, Tg, sigma, K, H, seed, min_branch):
    q0, qd0 = sc.q0, np.zeros(7, np.float32)
    p = sc.planner()
    Ug = np.zeros((H, 7), np.float32)
    Sg = np.empty(K, np.float32)
    p.smpc_iterate(q0, qd0, Tg, Ug, K, 0.02, 0.05, sigma, seed, 0, costs_out=Sg)
    p.close()
    Uo, So, _ = oracle.smpc_iterate(sc.R, sc.G, sc.C, q0, qd0, Tg, np.zeros((H, 7)), K, 0.02, 0.05,
                                    sigma, seed, 0, n_threads=0)
    eps = oracle.eps_tensor(seed, 0, K, H, sigma)
    ths = np.stack([rollout_angles(sc, q0, qd0, Tg, eps[m], 0.02) for m in range(K)])
    near_pi = np.any(np.abs(PI - ths) < 1e-3, axis=1)
    ok = ~near_pi
    assert ok.sum() >= K // 2
    rel = np.abs(Sg - So) / np.abs(So)
    assert rel[ok].max() <= S_REL, f"max rel cost error {rel[ok].max():.2e}"
    Uiso, w = fp64_update_from_costs(Sg, eps, np.zeros((H, 7)), 0.05)
    assert np.abs(Ug - Uiso).max() <= U_ISO
    if not near_pi.any():
        assert np.abs(Ug - Uo).max() <= U_ABS
    assert min_branch(ths)
    return int(near_pi.sum())


def test_iteration_sweeping_the_near_pi_branch(scene):
    """Goal rotated pi - 0.03 from the start flange: the roll-outs' angles
    spread over the symmetric-part branch (theta > pi - 0.05) and some cross
    pi; their costs match except where a step passes within 1e-3 of pi
    (skipped and counted)."""
    sc = scene
    Tee = start_flange(sc, sc.q0)
    Tg = (Tee @ np.linalg.inv(pose(rot((0.2, 0.9, -0.4), PI - 0.03), np.array([0.02, -0.03, 0.01])))
          ).astype(np.float32)
    sigma = np.full(7, 0.5, np.float32)
    skipped = iterate_and_compare(sc, Tg, sigma, 256, 32, 61,
                                  lambda ths: (ths > PI - 0.05).mean() > 0.5)
    print(f"near-pi iteration: {skipped} of 256 roll-outs pass within 1e-3 of pi (skipped)")


def test_iteration_sweeping_the_small_angle_branches(scene):
    """Goal = the start flange moved 2 cm, no rotation, small sigma: the early
    steps of every roll-out sit in the series branches (theta < 1e-4 for the
    log, < 1e-2 for V^-1)."""
    sc = scene
    Tee = start_flange(sc, sc.q0)
    Tg = (Tee @ np.linalg.inv(pose(np.eye(3), np.array([0.02, 0.0, -0.01])))).astype(np.float32)
    sigma = np.full(7, 0.05, np.float32)
    iterate_and_compare(sc, Tg, sigma, 256, 32, 62,
                        lambda ths: (ths < 1e-4).any() and ((ths > 1e-4) & (ths < 1e-2)).mean() > 0.3)

