"""Replanning server (pm_submit / pm_poll): results, warm starts, deadlines.

Every served result must equal the same replan run alone through pm_replan
(within the parity tolerances: a batch may cut the roll-outs into a different
number of thread blocks), whatever else is in the batch.  Failures are made
on the host: a deadline that cannot be met, a memory headroom that cannot be
satisfied, bad requests and tickets.
"""
import numpy as np
import pytest

import workloads
from parity_common import SIGMA, U_ABS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2512_22575_b300 as pm  # noqa: E402

DEV = torch.device("cuda:0")
N_ITERS = 4


class Arm:
    def __init__(self, sc):
        self.sc = sc
        self.robot = workloads.panda_robot()
        self.planner = pm.Planner(self.robot, sc["grid"], workloads.default_cost_params(sc["q0"]))
        self.planner.set_distance_field(workloads.build_scene_grid(sc))
        self.q = sc["q0"].astype(np.float32)
        self.qd = sc["qd0"].astype(np.float32)
        self.T = sc["T_goal"].astype(np.float32).ravel()


@pytest.fixture(scope="module")
def arms():
    cfg5 = workloads.load_scene("cfg5")["instances"]
    return [Arm(sc) for sc in cfg5[:32]]


def reference_replans(arm, requests):
    """Sequential pm_replan calls carrying the shifted sequence, like the server."""
    out = []
    U = None
    q, qd = arm.q.copy(), arm.qd.copy()
    for (K, H, seed, it0, warm) in requests:
        U0 = np.zeros((H, 7), np.float32)
        if warm and U is not None:
            rows = np.minimum(np.arange(H), U.shape[0] - 1)
            U0 = U[rows].copy()
        u0 = np.empty(7, np.float32)
        best = np.empty(1, np.float32)
        qq, qqd = q.copy(), qd.copy()
        arm.planner.replan(qq, qqd, arm.T, U0, K, N_ITERS, 0.02, 0.05, SIGMA, seed, it0 // N_ITERS,
                           u0_out=u0, best_cost=best)
        out.append((qq, qqd, u0, float(best[0])))
        U = U0
    return out


def check(res, ref):
    """A served result against the same replan alone: u0* within the U* bar
    (1e-5; the two differ only in how the roll-outs are cut into blocks, so
    in the merge order of the soft-min sums)."""
    qq, qqd, u0, best = ref
    assert res["status"] == "PM_OK"
    err = np.abs(res["u0"] - u0).max()
    print(f"served vs alone: |u0 - u0_alone| = {err:.1e}")
    assert err <= U_ABS
    assert np.abs(res["qd_next"] - qqd).max() <= 1e-6
    assert np.abs(res["q_next"] - qq).max() <= 1e-6
    assert abs(res["best_cost"] - best) <= 1e-4 * abs(best)


def test_served_equals_alone_in_a_mix_of_arms(arms):
    srv = pm.Server()
    ids = [srv.add_arm(a.planner) for a in arms]
    rng = np.random.default_rng(0)
    reqs = []
    for i, a in enumerate(arms):
        K = int(rng.choice([512, 1024, 2048, 4096]))
        H = int(rng.choice([16, 32, 48, 64]))
        reqs.append((K, H, 40 + i, 0, True))
    # queued together: the scheduler's first batch takes all of them
    tickets = srv.submit_many([dict(arm=ids[i], q=a.q, qd=a.qd, T_goal=a.T, K=K, H=H, n_iters=N_ITERS,
                                    seed=seed, iter_index=it0)
                               for i, (a, (K, H, seed, it0, _)) in enumerate(zip(arms, reqs))])
    results = [srv.wait(t) for t in tickets]
    stats = srv.stats()
    srv.close()
    assert stats["completed"] == len(arms) and stats["failed"] == 0
    assert all(r["batch_size"] == len(arms) for r in results)
    assert stats["batches"] == 1
    for a, r, req in zip(arms, results, reqs):
        check(r, reference_replans(a, [req])[0])


@pytest.mark.parametrize("spin_us", [0, 5000])
def test_warm_start_chain(arms, spin_us):
    """Consecutive requests of one arm start from its resident, shifted sequence
    (with a sleeping and with a busy-polling scheduler)."""
    a = arms[5]
    srv = pm.Server(spin_us=spin_us)
    aid = srv.add_arm(a.planner)
    chain = [(1024, 32, 7, 0, True), (1024, 32, 7, N_ITERS, True), (2048, 48, 8, 2 * N_ITERS, True),
             (512, 16, 9, 3 * N_ITERS, False)]
    results = []
    for (K, H, seed, it0, warm) in chain:
        t = srv.submit(aid, a.q, a.qd, a.T, K, H, N_ITERS, seed=seed, iter_index=it0, warm_start=warm)
        results.append(srv.wait(t))
    srv.close()
    for r, ref in zip(results, reference_replans(a, chain)):
        check(r, ref)


def test_deadline_expires_behind_a_busy_arm(arms):
    a = arms[0]
    srv = pm.Server()
    aid = srv.add_arm(a.planner)
    t1 = srv.submit(aid, a.q, a.qd, a.T, 4096, 64, 8)
    t2 = srv.submit(aid, a.q, a.qd, a.T, 256, 16, 8, deadline_us=1)   # arm busy with t1
    r1, r2 = srv.wait(t1), srv.wait(t2)
    stats = srv.stats()
    srv.close()
    assert r1["status"] == "PM_OK"
    assert r2["status"] == "PM_EBUSY"
    assert stats["rejected"] == 1


def test_admission_refused_when_memory_headroom_cannot_be_met(arms):
    a = arms[1]
    srv = pm.Server(hbm_headroom=1 << 60)   # more than any device has
    aid = srv.add_arm(a.planner)
    t = srv.submit(aid, a.q, a.qd, a.T, 512, 16, 2, deadline_us=20000)
    r = srv.wait(t)
    stats = srv.stats()
    srv.close()
    assert r["status"] == "PM_EBUSY"
    assert stats["deferred"] >= 1 and stats["completed"] == 0


def test_bad_requests_and_tickets(arms):
    a = arms[2]
    srv = pm.Server()
    aid = srv.add_arm(a.planner)
    with pytest.raises(pm.PmError) as e:
        srv.submit(aid + 7, a.q, a.qd, a.T, 512, 16)
    assert e.value.name == "PM_EINVAL"
    bad_q = a.q.copy()
    bad_q[0] = np.nan
    with pytest.raises(pm.PmError):
        srv.submit(aid, bad_q, a.qd, a.T, 512, 16)
    with pytest.raises(pm.PmError):
        srv.submit(aid, a.q, a.qd, a.T, 0, 16)
    with pytest.raises(pm.PmError):
        srv.poll(123456789)
    good = dict(arm=aid, q=a.q, qd=a.qd, T_goal=a.T, K=256, H=16, n_iters=2)
    with pytest.raises(pm.PmError):     # one bad request: none is queued
        srv.submit_many([good, dict(good, lam=float("inf"))])
    assert srv.stats()["submitted"] == 0
    t = srv.submit(aid, a.q, a.qd, a.T, 256, 16, 2)
    r = srv.wait(t)
    assert r["status"] == "PM_OK"
    with pytest.raises(pm.PmError):
        srv.poll(t)            # a result is handed out once
    srv.close()


def test_abandoned_tickets_are_cleaned_up(arms):
    """A client that submits and never polls (e.g. it died) does not block the
    server or its shutdown."""
    a = arms[3]
    srv = pm.Server()
    aid = srv.add_arm(a.planner)
    for i in range(5):
        srv.submit(aid, a.q, a.qd, a.T, 512, 16, 2, seed=i)
    t = srv.submit(aid, a.q, a.qd, a.T, 512, 16, 2, seed=99)
    assert srv.wait(t)["status"] == "PM_OK"
    srv.close()


def test_admission_window_groups_close_arrivals(arms):
    """With an admission window, requests submitted one by one while a batch
    is on the GPU share the next batch (instead of each running alone), and
    each result is still the replan alone."""
    srv = pm.Server(admit_window_us=20000)
    sel = arms[10:14]
    ids = [srv.add_arm(a.planner) for a in sel]
    busy = srv.add_arm(arms[15].planner)
    a15 = arms[15]
    srv.submit(busy, a15.q, a15.qd, a15.T, 4096, 256, 64)    # about 10 ms on the GPU meanwhile
    reqs = [(1024, 32, 60 + i, 0, True) for i in range(len(sel))]
    tickets = [srv.submit(aid, a.q, a.qd, a.T, K, H, N_ITERS, seed=seed, iter_index=it0)
               for aid, a, (K, H, seed, it0, _) in zip(ids, sel, reqs)]
    results = [srv.wait(t) for t in tickets]
    srv.close()
    assert max(r["batch_size"] for r in results) >= 2
    for a, r, req in zip(sel, results, reqs):
        check(r, reference_replans(a, [req])[0])
