"""Write the stored scene files under workloads/scenes/ (run once; committed).

Test infrastructure.  The scene definitions (obstacles, start and target
configurations, target poses) need forward kinematics for their rejection
tests: obstacles may not touch the start configuration's spheres (+2 cm) or
the base column, and the target configuration must be collision-free, keep
its flange inside the grid, and differ from the start by a rotation well
below pi (the SE(3) log is discontinuous at pi, Eq. 12).  This script calls
only the oracle and the seeded generators in ``workloads``; every stored
number is float32-exact, so both sides read identical inputs.

    python -m oracle.make_scenes
"""
import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
import workloads  # noqa: E402
from workloads import scenes as ws  # noqa: E402

F32 = np.float32
OUT = ws.SCENE_DIR


def f32list(a):
    return [float(F32(x)) for x in np.asarray(a).ravel()]


def tightened(rb, frac=0.05):
    lo = rb["q_min"].astype(np.float64)
    hi = rb["q_max"].astype(np.float64)
    e = frac * (hi - lo)
    return lo + e, hi - e


def sphere_hits(ob, centres, radii, pad):
    c = np.asarray(ob["center"], dtype=np.float64)
    if ob["type"] == "box":
        h = np.asarray(ob["half"], dtype=np.float64)
        d = np.maximum(np.abs(centres - c) - h, 0.0)
        dist = np.linalg.norm(d, axis=1)
        return bool(np.any(dist < radii + pad))
    dist = np.linalg.norm(centres - c, axis=1)
    return bool(np.any(dist < radii + ob["radius"] + pad))


def rotation_angle(Ra, Rb):
    c = 0.5 * (np.trace(Ra.T @ Rb) - 1.0)
    return math.acos(max(-1.0, min(1.0, c)))


def make_scene(name, seed, g, n_obstacles, kinds, rb, R, extra=None):
    """One scene: start state, obstacles, target; deterministic in `seed`."""
    rng = np.random.default_rng(np.random.SeedSequence([0x5CE7E, seed]))
    lo, hi = tightened(rb)
    q0 = np.clip(workloads.READY_POSE.astype(np.float64) + rng.normal(0.0, 0.1, 7), lo, hi)
    q0 = q0.astype(F32)
    start_p = oracle.sphere_centres(R, q0.astype(np.float64))
    radii = rb["sphere_radius"].astype(np.float64)
    ext_lo = np.array(g.origin) + 0.05
    ext_hi = np.array(g.origin) + np.array([g.nx, g.ny, g.nz]) * g.res - 0.05
    reg_lo = np.maximum(ext_lo, [-0.75, -0.75, 0.05])
    reg_hi = np.minimum(ext_hi, [0.75, 0.75, 1.15])
    obstacles = []
    while len(obstacles) < n_obstacles:
        kind = kinds[len(obstacles) % len(kinds)]
        if kind == "box":
            ob = ws.sample_box(rng, (0.1, 0.3), reg_lo, reg_hi)
        else:
            ob = ws.sample_sphere(rng, (0.05, 0.15), reg_lo, reg_hi)
        if ws.touches_base_column(ob) or sphere_hits(ob, start_p, radii, 0.02):
            continue
        obstacles.append(ob)
    occ = ws.occupancy_grid(obstacles, g)
    if not occ.any():  # every obstacle fell between voxel centres: force one
        return make_scene(name, seed + 1000003, g, n_obstacles, kinds, rb, R, extra)
    phi = ws.distance_grid(occ, g.res)
    grid = oracle.Grid(g, phi)
    T0 = oracle.fk(R, q0.astype(np.float64))[-1]
    for _ in range(100000):
        qt = rng.uniform(lo, hi).astype(F32)
        T = oracle.fk(R, qt.astype(np.float64))
        ee = T[-1]
        if not (np.all(ee[:3, 3] > ext_lo) and np.all(ee[:3, 3] < ext_hi)):
            continue
        if ee[2, 3] < 0.10:
            continue
        dist = np.linalg.norm(ee[:3, 3] - T0[:3, 3])
        if not (0.15 <= dist <= 0.6):
            continue
        if rotation_angle(T0[:3, :3], ee[:3, :3]) > 2.6:
            continue
        p = oracle.sphere_centres(R, qt.astype(np.float64))
        clear = oracle.phi(grid, p) - radii
        if clear.min() <= 0.01:
            continue
        break
    else:
        raise RuntimeError(f"{name}: no target configuration found")
    scene = {
        "name": name,
        "seed": int(seed),
        "grid": g.to_json(),
        "obstacles": obstacles,
        "q0": f32list(q0),
        "qd0": [0.0] * 7,
        "q_target": f32list(qt),
        "T_goal": f32list(T[-1]),
    }
    if extra:
        scene.update(extra)
    return scene


def write(name, data):
    os.makedirs(OUT, exist_ok=True)
    with open(os.path.join(OUT, name + ".json"), "w") as fh:
        json.dump(data, fh, indent=1)
        fh.write("\n")


def main():
    rb = workloads.panda_robot()
    R = oracle.make_robot(rb)
    # Plain single iteration: K=256, H=32, 64^3 grid at 2 cm, 5 boxes; seeds 0-9.
    for s in range(10):
        g = ws.GridDesc(64, 64, 64, float(F32(0.02)), (float(F32(-0.64)), float(F32(-0.64)), 0.0))
        write(f"cfg1_seed{s}", make_scene(f"cfg1_seed{s}", s, g, 5, ("box",), rb, R,
                                          {"K": 256, "H": 32, "dt": 0.02, "lambda": 0.05,
                                           "sigma": 0.5}))
    # Replanning loop: K=4096, H=64, 160x160x120 grid at 1 cm, 20 boxes and balls.
    g = ws.GridDesc(160, 160, 120, float(F32(0.01)), (float(F32(-0.8)), float(F32(-0.8)), 0.0))
    write("cfg2", make_scene("cfg2", 100, g, 20, ("box", "sphere"), rb, R,
                             {"K": 4096, "H": 64, "dt": 0.02, "lambda": 0.05, "sigma": 0.5,
                              "iters": 8, "replans": 200, "path_seed": 100,
                              "target_speed": 0.2}))
    # Batched uneven instances: 64 instances.
    rng = np.random.default_rng(np.random.SeedSequence([0xB47C4, 3]))
    inst = []
    for i in range(64):
        n = int(rng.integers(64, 129))
        res = float(F32(rng.uniform(0.01, 0.02)))
        g = ws.centred_grid(n, n, res)
        nob = int(rng.integers(5, 31))
        extra = {"K": int(rng.choice([256, 512, 1024, 2048, 4096])),
                 "H": int(rng.choice([16, 32, 48, 64])),
                 "dt": 0.02, "lambda": 0.05, "sigma": 0.5}
        inst.append(make_scene(f"cfg3_{i}", 300 + i, g, nob, ("box", "sphere"), rb, R, extra))
    write("cfg3", {"name": "cfg3", "instances": inst})
    # Serving: 256 arms, grids 96^3-128^3 at 1 cm with 10-25 obstacles.
    rng = np.random.default_rng(np.random.SeedSequence([0x5E7E, 5]))
    arms = []
    for i in range(256):
        n = int(rng.integers(96, 129))
        g = ws.centred_grid(n, n, 0.01)
        nob = int(rng.integers(10, 26))
        arms.append(make_scene(f"cfg5_{i}", 500 + i, g, nob, ("box", "sphere"), rb, R,
                               {"dt": 0.02, "lambda": 0.05, "sigma": 0.5}))
    write("cfg5", {"name": "cfg5", "instances": arms})


if __name__ == "__main__":
    main()
