"""Obstacle scenes, occupancy grids and dense distance fields (seeded inputs).

Grid convention (the paper's EDF of Sec. III-B; conventions chosen where it is
silent): voxel (i, j, l) has centre origin + (i + 0.5, j + 0.5, l + 0.5) * res
and is stored x-fastest, i.e. the array has shape (nz, ny, nx).  A voxel is
occupied iff its centre lies in a closed box or ball.  The distance field
stores the unsigned Euclidean distance in metres from each voxel centre to the
nearest occupied voxel centre (0 inside obstacles), i.e. res * sqrt(D) with D
the exact squared distance in voxel units that the paper's separable transform
computes (Sec. III-B).  The transform here is scipy's exact Euclidean distance
transform, used purely to synthesise the input grid; the oracle pins it
against its own brute-force transform.
"""
import json
import math
import os
from dataclasses import dataclass

import numpy as np
from scipy import ndimage

F32 = np.float32
SCENE_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "scenes")

# Keep-out column around the arm's base (obstacles touching it are redrawn).
BASE_COLUMN_RADIUS = 0.12
BASE_COLUMN_TOP = 0.40


@dataclass(frozen=True)
class GridDesc:
    nx: int
    ny: int
    nz: int
    res: float
    origin: tuple

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def to_json(self):
        return {"nx": self.nx, "ny": self.ny, "nz": self.nz, "res": self.res,
                "origin": list(self.origin)}

    @staticmethod
    def from_json(d):
        return GridDesc(int(d["nx"]), int(d["ny"]), int(d["nz"]),
                        float(F32(d["res"])), tuple(float(F32(o)) for o in d["origin"]))


def centred_grid(n_xy: int, n_z: int, res: float) -> GridDesc:
    """Grid centred on the base in x/y, starting at the floor (z = 0)."""
    res = float(F32(res))
    o = float(F32(-0.5 * n_xy * res))
    return GridDesc(n_xy, n_xy, n_z, res, (o, o, 0.0))


# ---------------------------------------------------------------- obstacles
def sample_box(rng, side_range, region_lo, region_hi):
    side = rng.uniform(side_range[0], side_range[1], size=3)
    centre = rng.uniform(region_lo, region_hi, size=3)
    return {"type": "box", "center": [float(F32(c)) for c in centre],
            "half": [float(F32(0.5 * s)) for s in side]}


def sample_sphere(rng, radius_range, region_lo, region_hi):
    r = rng.uniform(radius_range[0], radius_range[1])
    centre = rng.uniform(region_lo, region_hi, size=3)
    return {"type": "sphere", "center": [float(F32(c)) for c in centre],
            "radius": float(F32(r))}


def touches_base_column(ob) -> bool:
    """Pure geometry: does the obstacle reach into the base keep-out column?"""
    c = np.asarray(ob["center"], dtype=np.float64)
    if ob["type"] == "box":
        h = np.asarray(ob["half"], dtype=np.float64)
        if c[2] - h[2] > BASE_COLUMN_TOP:
            return False
        dx = max(abs(c[0]) - h[0], 0.0)
        dy = max(abs(c[1]) - h[1], 0.0)
        return math.hypot(dx, dy) <= BASE_COLUMN_RADIUS
    r = float(ob["radius"])
    if c[2] - r > BASE_COLUMN_TOP:
        return False
    return math.hypot(c[0], c[1]) <= BASE_COLUMN_RADIUS + r


# ---------------------------------------------------------------- grids
def voxel_centres(g: GridDesc):
    """float64 arrays (x, y, z) of voxel centres, broadcastable to g.shape."""
    x = g.origin[0] + (np.arange(g.nx) + 0.5) * g.res
    y = g.origin[1] + (np.arange(g.ny) + 0.5) * g.res
    z = g.origin[2] + (np.arange(g.nz) + 0.5) * g.res
    return x[None, None, :], y[None, :, None], z[:, None, None]


def occupancy_grid(obstacles, g: GridDesc) -> np.ndarray:
    """uint8 (nz, ny, nx): 1 where the voxel centre lies in a closed obstacle."""
    x, y, z = voxel_centres(g)
    occ = np.zeros(g.shape, dtype=bool)
    for ob in obstacles:
        c = ob["center"]
        if ob["type"] == "box":
            h = ob["half"]
            occ |= ((np.abs(x - c[0]) <= h[0]) & (np.abs(y - c[1]) <= h[1])
                    & (np.abs(z - c[2]) <= h[2]))
        elif ob["type"] == "sphere":
            r = ob["radius"]
            occ |= (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2 <= r * r
        else:
            raise ValueError(f"unknown obstacle type {ob['type']!r}")
    return occ.astype(np.uint8)


def distance_grid(occ: np.ndarray, res: float) -> np.ndarray:
    """float32 (nz, ny, nx) unsigned distance [m] to the nearest occupied centre.

    Requires at least one occupied voxel (the field is undefined otherwise).
    """
    if not occ.any():
        raise ValueError("distance field needs at least one occupied voxel")
    d_vox = ndimage.distance_transform_edt(occ == 0)
    return (d_vox * float(res)).astype(F32)


# ---------------------------------------------------------------- scene files
def scene_path(name: str) -> str:
    return os.path.join(SCENE_DIR, name + ".json")


def scene_names(prefix: str = ""):
    if not os.path.isdir(SCENE_DIR):
        return []
    return sorted(f[:-5] for f in os.listdir(SCENE_DIR)
                  if f.endswith(".json") and f.startswith(prefix))


def load_scene(name: str) -> dict:
    """Read a stored scene (or a scene set) and return it with float32 arrays."""
    with open(scene_path(name)) as fh:
        data = json.load(fh)
    if "instances" in data:
        data["instances"] = [_typed(s) for s in data["instances"]]
        return data
    return _typed(data)


def _typed(s: dict) -> dict:
    out = dict(s)
    out["grid"] = GridDesc.from_json(s["grid"])
    for key in ("q0", "qd0", "q_target"):
        if key in s:
            out[key] = np.asarray(s[key], dtype=F32)
    if "T_goal" in s:
        out["T_goal"] = np.asarray(s["T_goal"], dtype=F32).reshape(4, 4)
    return out


def build_scene_grid(scene: dict) -> np.ndarray:
    """Dense float32 distance field of a stored scene."""
    g = scene["grid"]
    return distance_grid(occupancy_grid(scene["obstacles"], g), g.res)


# ---------------------------------------------------------------- targets
def moving_target(T_goal0: np.ndarray, path_seed: int, t: float,
                  speed: float = 0.2, radius: float = 0.1) -> np.ndarray:
    """Target pose at time t [s] on a seeded circle traversed at `speed` m/s.

    The orientation stays that of T_goal0; the position starts at T_goal0's
    and moves along a circle of the given radius in a seeded random plane.
    Returns a float32 4x4 homogeneous matrix.
    """
    rng = np.random.default_rng(np.random.SeedSequence([0x7A26, path_seed]))
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    e1 = np.cross(n, [0.0, 0.0, 1.0] if abs(n[2]) < 0.9 else [1.0, 0.0, 0.0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    w = speed / radius
    p = radius * ((math.cos(w * t) - 1.0) * e1 + math.sin(w * t) * e2)
    T = np.asarray(T_goal0, dtype=np.float64).copy()
    T[:3, 3] = T[:3, 3] + p
    return T.astype(F32)
