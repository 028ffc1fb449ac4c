"""The 7-DoF arm used by every workload: modified-DH chain, limits, sphere model.

The kinematic chain is the one the workloads are specified on (a Panda-class
arm): per joint i = 1..7 the modified-DH tuple (a_{i-1}, d_i, alpha_{i-1}) and
a fixed flange translation of 0.107 m along the last z axis.  The paper gives
the chain only in words (forward kinematics, Sec. IV-A, Eq. 6); the numbers
below are the workload's.

The sphere model (Sec. IV-B-2, Fig. 2: n_s spheres with centres fixed in link
frames) is not given numerically by the paper.  Chosen here: 4 spheres per
moving link, radii uniform in [0.04, 0.08] m from a seeded draw, centres at
fractions (j + 0.5)/4 of the segment from frame i's origin to frame i+1's
origin, expressed in frame i.  That segment is the constant vector
(a_i, -sin(alpha_i) d_{i+1}, cos(alpha_i) d_{i+1}) of the next joint's DH
tuple (frame 8 is the flange).  A zero-length segment is replaced by 0.10 m
along the link's -z axis.  The offsets are data handed to both sides, so this
choice never affects parity.

Joint position, velocity and acceleration limits follow the public datasheet
of that arm class; the penalty box of Sec. IV-B-3 is tightened from them by a
margin proportional to the range (margin_frac).
"""
import math

import numpy as np

F32 = np.float32

# Modified-DH tuple per joint i = 1..7: a_{i-1} [m], d_i [m], alpha_{i-1} [rad].
DH_A = [0.0, 0.0, 0.0, 0.0825, -0.0825, 0.0, 0.088]
DH_D = [0.333, 0.0, 0.316, 0.0, 0.384, 0.0, 0.0]
DH_ALPHA = [0.0, -math.pi / 2, math.pi / 2, math.pi / 2, -math.pi / 2, math.pi / 2, math.pi / 2]
FLANGE_D = 0.107

Q_MIN = [-2.8973, -1.7628, -2.8973, -3.0718, -2.8973, -0.0175, -2.8973]
Q_MAX = [2.8973, 1.7628, 2.8973, -0.0698, 2.8973, 3.7525, 2.8973]
QD_MAX = [2.1750, 2.1750, 2.1750, 2.1750, 2.6100, 2.6100, 2.6100]
QDD_MAX = [15.0, 7.5, 10.0, 12.5, 15.0, 20.0, 20.0]

# Ready configuration the start states are perturbed around.
READY_POSE = np.array(
    [0.0, -math.pi / 4, 0.0, -3 * math.pi / 4, 0.0, math.pi / 2, math.pi / 4], dtype=F32
)

SPHERES_PER_LINK = 4
ZERO_SEGMENT = (0.0, 0.0, -0.10)


def _segment(i_next_a, i_next_alpha, i_next_d):
    """Constant offset of frame i+1's origin in frame i (from the DH tuple)."""
    return (
        i_next_a,
        -math.sin(i_next_alpha) * i_next_d,
        math.cos(i_next_alpha) * i_next_d,
    )


def panda_robot(seed: int = 0, spheres_per_link: int = SPHERES_PER_LINK):
    """Return the arm description as a dict of float32/int32 numpy arrays.

    Keys: n_joints, a, d, alpha, theta_offset, flange_d, q_min, q_max, qd_max,
    qdd_max, sphere_link (1-based frame index), sphere_offset (n_s x 3, link
    frame), sphere_radius (n_s,), self_pairs (P x 2, empty by default).
    """
    n = 7
    rng = np.random.default_rng(np.random.SeedSequence([0x5EED, seed]))
    # next-joint tuples, with the flange as the 8th "joint" (a=0, alpha=0).
    nxt_a = DH_A[1:] + [0.0]
    nxt_alpha = DH_ALPHA[1:] + [0.0]
    nxt_d = DH_D[1:] + [FLANGE_D]
    links, offsets, radii = [], [], []
    for i in range(n):  # link frame i+1 (1-based)
        seg = _segment(nxt_a[i], nxt_alpha[i], nxt_d[i])
        if math.sqrt(sum(s * s for s in seg)) < 1e-9:
            seg = ZERO_SEGMENT
        for j in range(spheres_per_link):
            frac = (j + 0.5) / spheres_per_link
            links.append(i + 1)
            offsets.append([frac * s for s in seg])
            radii.append(rng.uniform(0.04, 0.08))
    return {
        "n_joints": n,
        "a": np.array(DH_A, dtype=F32),
        "d": np.array(DH_D, dtype=F32),
        "alpha": np.array(DH_ALPHA, dtype=F32),
        "theta_offset": np.zeros(n, dtype=F32),
        "flange_d": F32(FLANGE_D),
        "q_min": np.array(Q_MIN, dtype=F32),
        "q_max": np.array(Q_MAX, dtype=F32),
        "qd_max": np.array(QD_MAX, dtype=F32),
        "qdd_max": np.array(QDD_MAX, dtype=F32),
        "sphere_link": np.array(links, dtype=np.int32),
        "sphere_offset": np.array(offsets, dtype=F32).reshape(-1, 3),
        "sphere_radius": np.array(radii, dtype=F32),
        "self_pairs": np.zeros((0, 2), dtype=np.int32),
    }


def self_collision_pairs(robot, min_link_gap: int = 2):
    """Sphere pairs (i, j), i < j, whose links are at least `min_link_gap` apart.

    The paper leaves the set S of Sec. IV-B-2 unspecified; this is the chosen
    rule for workloads that switch the self-collision term on.
    """
    link = robot["sphere_link"]
    pairs = [
        (i, j)
        for i in range(len(link))
        for j in range(i + 1, len(link))
        if abs(int(link[j]) - int(link[i])) >= min_link_gap
    ]
    return np.array(pairs, dtype=np.int32).reshape(-1, 2)


def default_cost_params(q_ref):
    """Cost weights of Sec. IV-B (values chosen; the paper gives none).

    Q_k = diag(w_pos I3, w_rot I3) with w_pos = 0.2, w_rot = 0.02 acting on
    xi = [v; omega] for k < H and Q_H = diag(2 I3, 0.2 I3) at the terminal
    step; w_env with activation distance d_act; self-collision off; joint-limit
    weights with a 5 % range margin; small smoothness and null-space weights
    with q_ref = start pose.

    The pose weights set the cost scale against the temperature lambda = 0.05
    of Eq. 29: at this scale the weights keep an effective sample size of
    roughly 20-75 % of K, and the FP32 rounding of S moves U* by well under
    1e-5 (ten times larger pose weights make the update an argmin and push
    FP32 rounding of S above that).
    """
    return {
        "Q": np.array([0.2, 0.2, 0.2, 0.02, 0.02, 0.02], dtype=F32),
        "QH": np.array([2.0, 2.0, 2.0, 0.2, 0.2, 0.2], dtype=F32),
        "w_env": F32(100.0),
        "d_act": F32(0.05),
        "w_self": F32(0.0),
        "w_q": F32(10.0),
        "w_qd": F32(10.0),
        "w_qdd": F32(10.0),
        "margin_frac": F32(0.05),
        "w_s": F32(1e-3),
        "w_ns": F32(1e-3),
        "q_ref": np.asarray(q_ref, dtype=F32).copy(),
    }
