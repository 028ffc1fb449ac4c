"""Self-collision term (Eqs. 18-20) on the GPU against the FP64 oracle.

The set S is data.  The tests use sets that always touch (pairs on the same
or adjacent frames, whose spheres overlap at the joints) to exercise the
arithmetic, and a set that touches only when large noise folds the arm
(frames at least three apart) to exercise the exact skip of far groups.  A pair group
is skipped only when its frames' bounding spheres are provably apart, so
every self term must match the oracle, and be exactly 0 where the oracle's
is 0.
"""
import numpy as np
import pytest

import oracle
import workloads
from parity_common import S_REL, SIGMA, U_ABS, Scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2512_22575_b300 as pm  # noqa: E402

DEV = torch.device("cuda:0")


def scene_with_pairs(name, min_gap, w_self):
    sc = Scene(name, cost_overrides={"w_self": np.float32(w_self)})
    sc.robot = dict(sc.robot)
    sc.robot["self_pairs"] = workloads.self_collision_pairs(sc.robot, min_link_gap=min_gap)
    sc.R = oracle.make_robot(sc.robot)
    sc.C = oracle.make_cost(sc.cp)
    return sc


def trace_both(sc, K, H, sigma, seed):
    p = sc.planner()
    tr = torch.zeros((K, H + 1, 8), dtype=torch.float32, device=DEV)
    U = np.zeros((H, 7), np.float32)
    p.rollout_trace(sc.q0, sc.qd0, sc.T, U, K, 0.02, sigma, seed, 0, tr)
    p.close()
    tr = tr.cpu().numpy()
    eps = oracle.eps_tensor(seed, 0, K, H, sigma)
    refs = []
    for m in range(K):
        _, ref = oracle.rollout_cost(sc.R, sc.G, sc.C, sc.q0, sc.qd0, sc.T, U + eps[m], 0.02, trace=True)
        ref = ref.copy()
        ref[0, [0, 1, 2, 3, 4, 7]] = 0.0   # k = 0 state terms are not per roll-out
        refs.append(ref)
    return tr, np.array(refs)


@pytest.mark.parametrize("min_gap", [0, 1])
def test_self_terms_match_oracle_trace(min_gap):
    """Same-frame and adjacent-frame pairs overlap: every step has a self term."""
    sc = scene_with_pairs("cfg1_seed2", min_gap, 0.5)
    tr, ref = trace_both(sc, 8, 32, SIGMA, 5)
    assert (ref[:, 1:32, 2] > 0).all()
    assert np.allclose(tr, ref, rtol=1e-4, atol=1e-7)


def test_partial_pair_sets_match_oracle_trace():
    """A seeded half of the adjacent-frame set, some pairs listed as (b, a):
    no group holds every pair of its two frames, so each is evaluated from
    its pair list rather than as a dense block."""
    sc = Scene("cfg1_seed7", cost_overrides={"w_self": np.float32(0.5)})
    sc.robot = dict(sc.robot)
    full = workloads.self_collision_pairs(sc.robot, min_link_gap=1)
    rng = np.random.default_rng(17)
    pick = full[rng.permutation(len(full))[: len(full) // 2]].copy()
    flip = rng.random(len(pick)) < 0.5
    pick[flip] = pick[flip][:, ::-1]
    sc.robot["self_pairs"] = np.ascontiguousarray(pick, dtype=np.int32)
    sc.R = oracle.make_robot(sc.robot)
    sc.C = oracle.make_cost(sc.cp)
    tr, ref = trace_both(sc, 8, 32, SIGMA, 9)
    assert (ref[:, 1:32, 2] > 0).any()
    assert np.array_equal(tr[:, 1:32, 2] == 0, ref[:, 1:32, 2] == 0)
    assert np.allclose(tr, ref, rtol=1e-4, atol=1e-7)


def test_far_groups_are_skipped_exactly():
    """Pairs on frames >= 3 apart under large noise: the arm folds in some
    steps (about one in eight here); where the oracle's self term is 0 the
    GPU's is exactly 0.  (With this sphere model the wrist's spheres on
    frames 2 apart always overlap, so that set has contact at every step.)"""
    sc = scene_with_pairs("cfg1_seed4", 3, 1.0)
    sigma = np.full(7, 6.0, np.float32)
    tr, ref = trace_both(sc, 32, 64, sigma, 11)
    self_gpu, self_ref = tr[:, 1:64, 2], ref[:, 1:64, 2]
    assert (self_ref > 0).any(), "no self contact: the test would not exercise the pairs"
    assert np.array_equal(self_gpu == 0, self_ref == 0)
    assert np.allclose(self_gpu, self_ref, rtol=1e-4, atol=1e-7)


def test_iteration_with_self_term_matches_oracle():
    sc = scene_with_pairs("cfg1_seed3", 1, 0.1)
    K, H = 256, 32
    p = sc.planner()
    Ug = np.zeros((H, 7), np.float32)
    Sg = np.empty(K, np.float32)
    p.smpc_iterate(sc.q0, sc.qd0, sc.T, Ug, K, 0.02, 0.05, SIGMA, 77, 2, costs_out=Sg)
    p.close()
    Uo, So, _ = sc.oracle_iterate(np.zeros((H, 7), np.float32), K, 0.02, 0.05, SIGMA, 77, 2)
    assert (np.abs(Sg - So) / np.abs(So)).max() <= S_REL
    assert np.abs(Ug - Uo).max() <= U_ABS


def test_batch_mixes_arms_with_and_without_the_term():
    on = scene_with_pairs("cfg1_seed5", 1, 0.1)
    off = Scene("cfg1_seed6")
    K, H = 512, 32
    refs, items, planners = [], [], []
    for sc in (on, off, on):
        p = sc.planner()
        planners.append(p)
        U = np.zeros((H, 7), np.float32)
        S = np.empty(K, np.float32)
        p.smpc_iterate(sc.q0, sc.qd0, sc.T, U, K, 0.02, 0.05, SIGMA, 9, 0, costs_out=S)
        refs.append((U, S))
        items.append(dict(ctx=p, q=torch.from_numpy(sc.q0).to(DEV), qd=torch.from_numpy(sc.qd0).to(DEV),
                          T_goal=torch.from_numpy(sc.T.ravel().copy()).to(DEV),
                          U=torch.zeros((H, 7), device=DEV), costs_out=torch.zeros(K, device=DEV),
                          K=K, dt=0.02, lam=0.05, sigma=SIGMA, seed=9, iter_index=0))
    b = pm.Batch()
    b.run(items, n_iters=1)
    torch.cuda.synchronize()
    for it, (Ur, Sr) in zip(items, refs):
        assert np.abs(it["U"].cpu().numpy() - Ur).max() <= U_ABS
        assert (np.abs(it["costs_out"].cpu().numpy() - Sr) / np.abs(Sr)).max() <= S_REL
    b.close()
    for p in planners:
        p.close()


def test_bad_pairs_are_rejected():
    sc = Scene("cfg1_seed0", cost_overrides={"w_self": np.float32(1.0)})
    rb = dict(sc.robot)
    rb["self_pairs"] = np.array([[0, 5], [3, 28]], dtype=np.int32)   # 28 spheres: 28 is out of range
    with pytest.raises(pm.PmError) as e:
        pm.Planner(rb, sc.grid_desc, sc.cp)
    assert e.value.name == "PM_EINVAL"
