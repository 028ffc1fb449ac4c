"""Batched iterations (pm_batch_*) against single calls and the oracle.

Instances of the uneven batch workload (own K, H and distance field each)
run together in one persistent launch per iteration.  Each instance's result
must match the same instance run alone through pm_smpc_iterate / pm_replan
(within the parity tolerances: the batch may cut the roll-outs into a
different number of thread blocks, which changes the merge's rounding
order), and small instances must match the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
import workloads
from parity_common import S_REL, SIGMA, U_ABS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2512_22575_b300 as pm  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


class Inst:
    """One batch instance: its scene, context and device buffers."""

    def __init__(self, sc, K=None, H=None, seed=0):
        self.sc = sc
        self.K = int(K or sc["K"])
        self.H = int(H or sc["H"])
        self.robot = workloads.panda_robot()
        self.cp = workloads.default_cost_params(sc["q0"])
        self.phi = workloads.build_scene_grid(sc)
        self.planner = pm.Planner(self.robot, sc["grid"], self.cp)
        self.planner.set_distance_field(self.phi)
        rng = np.random.default_rng(seed)
        self.U0 = (rng.normal(size=(self.H, 7)) * 0.2).astype(np.float32)
        self.seed = 1000 + seed
        self.reset()

    def reset(self):
        self.q = dev(self.sc["q0"])
        self.qd = dev(self.sc["qd0"])
        self.T = dev(self.sc["T_goal"].ravel())
        self.U = dev(self.U0)
        self.S = torch.zeros(self.K, dtype=torch.float32, device=DEV)
        self.u0 = torch.zeros(7, dtype=torch.float32, device=DEV)
        self.best = torch.zeros(1, dtype=torch.float32, device=DEV)

    def item(self, it0=0):
        return dict(ctx=self.planner, q=self.q, qd=self.qd, T_goal=self.T, U=self.U,
                    costs_out=self.S, u0_out=self.u0, best_cost=self.best, K=self.K,
                    dt=0.02, lam=0.05, sigma=SIGMA, seed=self.seed, iter_index=it0)


@pytest.fixture(scope="module")
def insts():
    cfg3 = workloads.load_scene("cfg3")["instances"]
    # twelve instances spanning every K and H of the workload; K capped to keep
    # the single-call reference quick
    picks = list(range(12))
    return [Inst(cfg3[i], K=min(int(cfg3[i]["K"]), 2048), seed=i) for i in picks]


def single_iterate(inst, n_iters):
    inst.reset()
    for it in range(n_iters):
        inst.planner.smpc_iterate(inst.q, inst.qd, inst.T, inst.U, inst.K, 0.02, 0.05, SIGMA,
                                  inst.seed, it, costs_out=inst.S)
    torch.cuda.synchronize()
    return inst.U.cpu().numpy().copy(), inst.S.cpu().numpy().copy()


@pytest.mark.parametrize("flags", [0, pm.PM_BATCH_GRAPH, pm.PM_BATCH_AUTOTUNE | pm.PM_BATCH_GRAPH])
def test_batch_matches_single_calls(insts, flags):
    n_iters = 3
    ref = [single_iterate(x, n_iters) for x in insts]
    b = pm.Batch()
    for rep in range(2):  # second run replays the cached plan / graph
        for x in insts:
            x.reset()
        b.run([x.item() for x in insts], n_iters=n_iters, flags=flags)
        torch.cuda.synchronize()
        for x, (Ur, Sr) in zip(insts, ref):
            U = x.U.cpu().numpy()
            S = x.S.cpu().numpy()
            assert np.abs(U - Ur).max() <= U_ABS, (x.K, x.H, rep)
            assert (np.abs(S - Sr) / np.abs(Sr)).max() <= S_REL, (x.K, x.H, rep)
            assert abs(float(x.best.cpu()[0]) - Sr.min()) <= S_REL * abs(Sr.min())
    shapes, blocks, us = b.plan([x.item() for x in insts], n_iters=n_iters, flags=flags)
    assert len(shapes) == len(insts) and all(nb >= 1 for nb in blocks)
    for (C, L, P), x in zip(shapes, insts):
        assert C * L * P >= x.H
    if flags & pm.PM_BATCH_AUTOTUNE:
        assert us > 0
    b.close()


def test_batch_replan_matches_single_replan(insts):
    n_iters = 4
    sub = insts[:6]
    refs = []
    for x in sub:
        x.reset()
        x.planner.replan(x.q, x.qd, x.T, x.U, x.K, n_iters, 0.02, 0.05, SIGMA, x.seed, 0,
                         u0_out=x.u0, best_cost=x.best)
        torch.cuda.synchronize()
        refs.append([t.cpu().numpy().copy() for t in (x.q, x.qd, x.U, x.u0)])
    b = pm.Batch()
    for x in sub:
        x.reset()
    b.run([x.item() for x in sub], n_iters=n_iters, flags=pm.PM_BATCH_REPLAN)
    torch.cuda.synchronize()
    for x, (q, qd, U, u0) in zip(sub, refs):
        assert np.abs(x.U.cpu().numpy() - U).max() <= n_iters * U_ABS
        assert np.abs(x.u0.cpu().numpy() - u0).max() <= n_iters * U_ABS
        assert np.abs(x.qd.cpu().numpy() - qd).max() <= 1e-6
        assert np.abs(x.q.cpu().numpy() - q).max() <= 1e-6
    b.close()


def test_same_alone_and_in_the_mix(insts):
    """An instance's result does not depend on what else is in the batch."""
    b = pm.Batch()
    x = insts[3]
    x.reset()
    b.run([x.item()], n_iters=2)
    torch.cuda.synchronize()
    alone = (x.U.cpu().numpy().copy(), x.S.cpu().numpy().copy())
    for y in insts:
        y.reset()
    b.run([y.item() for y in insts], n_iters=2)
    torch.cuda.synchronize()
    assert np.abs(x.U.cpu().numpy() - alone[0]).max() <= U_ABS
    assert (np.abs(x.S.cpu().numpy() - alone[1]) / np.abs(alone[1])).max() <= S_REL
    b.close()


def test_results_do_not_depend_on_the_order_of_the_batch(insts):
    """Permuting the instances (and with them the work queue) leaves every
    result unchanged bit for bit: an instance's blocks, their roll-outs and
    its merge are fixed by the plan, which depends on the instances and not
    on their order."""
    sub = insts[:8]
    b = pm.Batch()
    for x in sub:
        x.reset()
    b.run([x.item() for x in sub], n_iters=2)
    torch.cuda.synchronize()
    first = [(x.U.cpu().numpy().copy(), x.S.cpu().numpy().copy()) for x in sub]
    perm = [7, 2, 5, 0, 3, 6, 1, 4]
    for x in sub:
        x.reset()
    b.run([sub[i].item() for i in perm], n_iters=2)
    torch.cuda.synchronize()
    for x, (U, S) in zip(sub, first):
        assert np.array_equal(x.U.cpu().numpy(), U), (x.K, x.H)
        assert np.array_equal(x.S.cpu().numpy(), S), (x.K, x.H)
    b.close()


def test_batch_small_instances_match_oracle(insts):
    small = [x for x in insts if x.K <= 512][:3]
    assert small
    b = pm.Batch()
    for x in small:
        x.reset()
    b.run([x.item() for x in small], n_iters=1)
    torch.cuda.synchronize()
    for x in small:
        R = oracle.make_robot(x.robot)
        G = oracle.Grid(x.sc["grid"], x.phi)
        Cc = oracle.make_cost(x.cp)
        Uo, So, _ = oracle.smpc_iterate(R, G, Cc, x.sc["q0"], x.sc["qd0"], x.sc["T_goal"], x.U0,
                                        x.K, 0.02, 0.05, SIGMA, x.seed, 0, n_threads=0)
        assert np.abs(x.U.cpu().numpy() - Uo).max() <= U_ABS
        assert (np.abs(x.S.cpu().numpy() - So) / np.abs(So)).max() <= S_REL
    b.close()


def test_batch_rejects_bad_items(insts):
    b = pm.Batch()
    it = insts[0].item()
    it["K"] = 0
    with pytest.raises(pm.PmError) as e:
        b.run([it])
    assert e.value.name == "PM_EINVAL"
    with pytest.raises(pm.PmError):
        b.run([])
    b.close()
