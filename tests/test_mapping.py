"""GPU mapping (Sec. III-B; Sec. IV-B-2, Remark 2) against exact references.

The squared EDT is integer work: it must equal the oracle's brute-force
transform bit for bit, and scipy's exact transform on the full-size grid.
The robot mask must clear exactly the oracle's voxels, except voxels whose
centre lies within 1e-5 m of a sphere's surface, where FP32 and FP64 may
decide differently; those are only checked to be either cleared or kept.
"""
import numpy as np
import pytest
from scipy import ndimage

import oracle
import workloads
from parity_common import SIGMA, Scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2512_22575_b300 as pm  # noqa: E402

DEV = torch.device("cuda:0")
NONE = 2**31 - 1


def gpu_edt(occ):
    o = torch.from_numpy(np.ascontiguousarray(occ, dtype=np.uint8)).to(DEV)
    d2 = torch.empty(occ.shape, dtype=torch.int32, device=DEV)
    pm.edt_squared(o, d2)
    torch.cuda.synchronize()
    return d2.cpu().numpy()


def random_occ(shape, p, seed):
    return (np.random.default_rng(seed).random(shape) < p).astype(np.uint8)


@pytest.mark.parametrize("shape,p,seed", [((7, 5, 3), 0.2, 0), ((19, 23, 37), 0.01, 1), ((19, 23, 37), 0.3, 2),
                                          ((33, 1, 64), 0.05, 3), ((1, 1, 50), 0.04, 4), ((2, 2, 2), 0.3, 5),
                                          ((40, 30, 20), 0.0005, 6)])
def test_edt_matches_bruteforce(shape, p, seed):
    occ = random_occ(shape, p, seed)
    if not occ.any():
        occ.flat[seed % occ.size] = 1
    ref = oracle.edt_bruteforce(occ)
    assert np.array_equal(gpu_edt(occ).astype(np.int64), ref)


def test_edt_edge_cases():
    shape = (9, 11, 13)
    single = np.zeros(shape, np.uint8)
    single[4, 0, 12] = 1
    assert np.array_equal(gpu_edt(single).astype(np.int64), oracle.edt_bruteforce(single))
    assert not gpu_edt(np.ones(shape, np.uint8)).any()
    assert (gpu_edt(np.zeros(shape, np.uint8)) == NONE).all()


def test_edt_scene_grids_match_scipy():
    """cfg1 scene (64^3) against the brute force, the full-size replanning
    grid (160 x 160 x 120) against scipy's exact transform."""
    sc = workloads.load_scene("cfg1_seed3")
    occ = workloads.occupancy_grid(sc["obstacles"], sc["grid"])
    assert np.array_equal(gpu_edt(occ).astype(np.int64), oracle.edt_bruteforce(occ))
    sc2 = workloads.load_scene("cfg2")
    occ2 = workloads.occupancy_grid(sc2["obstacles"], sc2["grid"])
    d = ndimage.distance_transform_edt(occ2 == 0)
    ref = np.rint(d * d).astype(np.int64)
    assert np.array_equal(gpu_edt(occ2).astype(np.int64), ref)


def scipy_edt(occ):
    d = ndimage.distance_transform_edt(occ == 0)
    return np.rint(d * d).astype(np.int64)


@pytest.mark.parametrize("shape,seed", [((6, 10, 300), 7), ((300, 8, 5), 8), ((5, 300, 7), 9)])
def test_edt_long_lines_take_the_envelope(shape, seed):
    """Lines over 256 voxels (x, z, then the first pass along y) go through
    the lower-envelope kernel, the others through the direct passes."""
    occ = random_occ(shape, 0.002, seed)
    occ.flat[seed % occ.size] = 1
    assert np.array_equal(gpu_edt(occ).astype(np.int64), scipy_edt(occ))


def test_edt_passes_whose_values_could_reach_2_24_take_the_envelope():
    """4000 x 900 x 2 voxels: the last (z) pass has short lines, but its
    inputs can reach 899^2 + 3999^2 > 2^24, so it must not use the FP32
    direct pass.  One occupied corner voxel makes the far corner's squared
    distance 3999^2 + 899^2 + 1 > 2^24, where FP32 cannot hold every
    integer."""
    occ = np.zeros((2, 900, 4000), np.uint8)
    occ[0, 0, 0] = 1
    got = gpu_edt(occ).astype(np.int64)
    assert got.max() == 3999**2 + 899**2 + 1 > 2**24
    assert np.array_equal(got, scipy_edt(occ))


def test_map_update_gives_the_same_field_as_the_host_transform():
    """Iterations on a field built by pm_map_update equal, bit for bit, those
    on the field built on the host (scipy EDT x res, rounded to float32)."""
    sc = Scene("cfg1_seed1")
    occ = workloads.occupancy_grid(sc.sc["obstacles"], sc.grid_desc)
    a = sc.planner()                      # host-built field
    b = pm.Planner(sc.robot, sc.grid_desc, sc.cp)
    b.map_update(occ)                     # host occupancy
    c = pm.Planner(sc.robot, sc.grid_desc, sc.cp)
    c.map_update(torch.from_numpy(occ).to(DEV))   # device occupancy
    outs = []
    for p in (a, b, c):
        U = np.zeros((32, 7), np.float32)
        S = np.empty(512, np.float32)
        p.smpc_iterate(sc.q0, sc.qd0, sc.T, U, 512, 0.02, 0.05, SIGMA, 3, 1, costs_out=S)
        outs.append((U, S))
        p.close()
    for U, S in outs[1:]:
        assert np.array_equal(U, outs[0][0]) and np.array_equal(S, outs[0][1])


def robot_covered(sc, q, inflate):
    """Oracle sphere centres and, per voxel, the smallest |c - p| - r."""
    p = oracle.sphere_centres(sc.R, q)
    r = sc.robot["sphere_radius"].astype(np.float64) + inflate
    g = sc.grid_desc
    l, j, i = np.meshgrid(np.arange(g.nz), np.arange(g.ny), np.arange(g.nx), indexing="ij")
    c = np.stack([g.origin[0] + (i + 0.5) * g.res, g.origin[1] + (j + 0.5) * g.res,
                  g.origin[2] + (l + 0.5) * g.res], -1)
    margin = np.full(g.shape, np.inf)
    for s in range(len(r)):
        margin = np.minimum(margin, np.linalg.norm(c - p[s], axis=-1) - r[s])
    return margin


@pytest.mark.parametrize("inflate", [0.0, 0.02])
def test_robot_mask_matches_oracle(inflate):
    sc = Scene("cfg1_seed0")
    g = sc.grid_desc
    occ = workloads.occupancy_grid(sc.sc["obstacles"], g)
    margin = robot_covered(sc, sc.q0, 0.03)
    occ = np.where(margin <= 0, 1, occ).astype(np.uint8)   # the sensor saw the arm (3 cm shell)
    ref = oracle.robot_mask(sc.R, g, sc.q0, occ, inflate)
    p = sc.planner()
    o = torch.from_numpy(occ).to(DEV)
    p.robot_mask(o, sc.q0, inflate)
    got = o.cpu().numpy()
    p.close()
    m = robot_covered(sc, sc.q0, inflate)
    firm = np.abs(m) > 1e-5
    assert (ref != occ).sum() > 500
    assert np.array_equal(got[firm], ref[firm])
    assert np.all((got[~firm] == occ[~firm]) | (got[~firm] == 0))


def test_map_update_with_mask_equals_mask_then_update():
    sc = Scene("cfg1_seed2")
    g = sc.grid_desc
    occ = workloads.occupancy_grid(sc.sc["obstacles"], g)
    occ = np.where(robot_covered(sc, sc.q0, 0.02) <= 0, 1, occ).astype(np.uint8)
    a = pm.Planner(sc.robot, g, sc.cp)
    a.map_update(occ, q_mask=sc.q0, inflate=0.01)
    o = torch.from_numpy(occ).to(DEV)
    b = pm.Planner(sc.robot, g, sc.cp)
    b.robot_mask(o, sc.q0, 0.01)
    b.map_update(o)
    outs = []
    for p in (a, b):
        U = np.zeros((32, 7), np.float32)
        p.smpc_iterate(sc.q0, sc.qd0, sc.T, U, 256, 0.02, 0.05, SIGMA, 5, 0)
        outs.append(U)
        p.close()
    assert np.array_equal(outs[0], outs[1])


def test_bad_arguments():
    with pytest.raises(pm.PmError):
        pm.edt_squared(torch.zeros((1, 1, 20000), dtype=torch.uint8, device=DEV),
                       torch.zeros((1, 1, 20000), dtype=torch.int32, device=DEV))
    sc = Scene("cfg1_seed0")
    p = sc.planner()
    o = torch.zeros(sc.phi.shape, dtype=torch.uint8, device=DEV)
    with pytest.raises(pm.PmError):
        p.robot_mask(o, sc.q0, -1.0)
    q = sc.q0.copy()
    q[3] = np.nan
    with pytest.raises(pm.PmError):
        p.robot_mask(o, q, 0.0)
    p.close()
