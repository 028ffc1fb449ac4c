"""The bounds-checked build (libparamap_checked.so, PM_BOUNDS_CHECK).

compute-sanitizer is not available here, so memory safety is checked by the
library itself: in the checked library every distance-field gather, shared-memory
slot and cost / partial / trace write of the iteration kernels is checked
against its extent, and a violation sets a bit in the context's word and
skips the access (no trap).  A child process loads that build (the
library is chosen when the package is imported) and runs the plain
iteration, ragged and maximal shapes, every tile shape, the trace, the
host-buffer graph path, a replan, a batch through both batch kernels, the
self-collision variant in both slot layouts (alone, traced and batched)
and the no-allocation entry point; every word must
stay 0 and the results must still match the oracle: costs within S_REL, U*
within U_ISO of the FP64 update from the GPU's own costs, and within U_ABS of
the oracle's U* where the soft-min is well conditioned (the conditioning
reading of the cost weights: with few roll-outs and lambda = 0.05 the FP32
rounding of S alone can move U* by more than U_ABS).
"""
import json
import os
import subprocess
import sys
import textwrap

import pytest

from parity_common import S_REL, U_ABS, U_ISO

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import json, sys
    import numpy as np
    import torch
    sys.path.insert(0, {root!r})
    sys.path.insert(0, {tests!r})
    import paper_2512_22575_b300 as pm
    import oracle, workloads
    from parity_common import Scene, SIGMA, S_REL, U_ABS, first_order_bound, fp64_update_from_costs
    out = {{"checked": pm.bounds_checked(), "lib": pm.lib_path(), "words": {{}}, "parity": {{}}}}
    dev = torch.device("cuda:0")
    sc = Scene("cfg1_seed3")
    p = sc.planner()

    def word(tag):
        out["words"][tag] = p.bounds_status(reset=True)

    def both(K, H, seed, it, shape=None, graphs=True):
        p.set_call_graphs(graphs)
        if shape:
            p.set_tile_shape(*shape)
        U = (np.random.default_rng(K + H).normal(size=(H, 7)) * 0.3).astype(np.float32)
        Ug, Sg = U.copy(), np.empty(K, np.float32)
        p.smpc_iterate(sc.q0, sc.qd0, sc.T, Ug, K, 0.02, 0.05, SIGMA, seed, it, costs_out=Sg)
        p.set_tile_shape(0, 0, 0)
        Uo, So, _ = sc.oracle_iterate(U, K, 0.02, 0.05, SIGMA, seed, it)
        eps = oracle.eps_tensor(seed, it, K, H, SIGMA)
        Uiso, _ = fp64_update_from_costs(Sg, eps, U, 0.05)
        return (float((np.abs(Sg - So) / np.abs(So)).max()), float(np.abs(Ug - Uo).max()),
                float(np.abs(Ug - Uiso).max()), first_order_bound(Sg, So, SIGMA, 0.05))

    out["parity"]["cfg1_graph"] = both(256, 32, 7, 0)
    word("cfg1_graph")
    out["parity"]["cfg1_direct"] = both(256, 32, 7, 1, graphs=False)
    word("cfg1_direct")
    for K, H in [(1, 16), (37, 16), (5, 5), (9, 200), (513, 33), (2, 256), (70, 48), (129, 64)]:
        out["parity"][f"ragged_{{K}}_{{H}}"] = both(K, H, 11, 2, graphs=False)
        word(f"ragged_{{K}}_{{H}}")
    for shape in [(1, 16, 1), (1, 32, 1), (3, 16, 1), (2, 32, 1), (4, 32, 1), (8, 32, 1),
                  (1, 32, 2), (2, 32, 2), (4, 32, 2)]:
        C, L, P = shape
        H = max(1, C * L * P - 3)
        out["parity"]["shape_%d_%d_%d" % shape] = both(37, H, 13, 2, shape=shape, graphs=False)
        word("shape_%d_%d_%d" % shape)
    tr = torch.zeros((8, 33, 8), dtype=torch.float32, device=dev)
    p.rollout_trace(sc.q0, sc.qd0, sc.T, np.zeros((32, 7), np.float32), 8, 0.02, SIGMA, 21, 0, tr)
    word("trace")
    q, qd, U = sc.q0.copy(), sc.qd0.copy(), np.zeros((64, 7), np.float32)
    p.replan(q, qd, sc.T, U, 4096, 8, 0.02, 0.05, SIGMA, 100, 0)
    word("replan_graph")
    Ud = torch.zeros((200, 7), dtype=torch.float32, device=dev)
    p.smpc_iterate_noalloc(torch.from_numpy(sc.q0).to(dev), torch.from_numpy(sc.qd0).to(dev),
                           torch.from_numpy(sc.T.ravel().copy()).to(dev), Ud, 300, 0.02, 0.05, SIGMA, 5, 0)
    torch.cuda.synchronize()
    word("noalloc")

    # a batch: one-step shapes only (one-step kernel), then one with H = 100 (run-time shapes)
    insts = workloads.load_scene("cfg3")["instances"][:6]
    planners = []
    for Hs, tag in (([16, 32, 48, 64, 64, 32], "batch_one_step"), ([16, 32, 100, 64, 64, 32], "batch_run_time")):
        items = []
        for i, (s, H) in enumerate(zip(insts, Hs)):
            pl = pm.Planner(workloads.panda_robot(), s["grid"], workloads.default_cost_params(s["q0"]))
            pl.set_distance_field(workloads.build_scene_grid(s))
            planners.append(pl)
            items.append(dict(ctx=pl, q=torch.from_numpy(s["q0"]).to(dev), qd=torch.from_numpy(s["qd0"]).to(dev),
                              T_goal=torch.from_numpy(s["T_goal"].ravel().copy()).to(dev),
                              U=torch.zeros((H, 7), dtype=torch.float32, device=dev), K=int(s["K"]) // 4,
                              seed=30 + i))
        b = pm.Batch(0)
        b.run(items, n_iters=2, flags=pm.PM_BATCH_REPLAN)
        torch.cuda.synchronize()
        b.close()
        out["words"][tag] = max(it["ctx"].bounds_status(reset=True) for it in items)

    # the self-collision variant
    rb = workloads.panda_robot()
    rb["self_pairs"] = workloads.self_collision_pairs(rb, min_link_gap=2)
    cp = dict(sc.cp); cp["w_self"] = np.float32(1.0)
    ps = pm.Planner(rb, sc.grid_desc, cp)
    ps.set_distance_field(sc.phi)
    Us = np.zeros((32, 7), np.float32)
    ps.smpc_iterate(sc.q0, sc.qd0, sc.T, Us, 512, 0.02, 0.05, SIGMA, 3, 0)
    out["words"]["self"] = ps.bounds_status(reset=True)
    # its trace, and the sphere layout (same-frame pairs: groups that are
    # not dense blocks)
    tr = torch.zeros((64, 33, 8), dtype=torch.float32, device=dev)
    ps.rollout_trace(sc.q0, sc.qd0, sc.T, np.zeros((32, 7), np.float32), 64, 0.02, SIGMA, 3, 0, tr)
    out["words"]["self_trace"] = ps.bounds_status(reset=True)
    rb0 = workloads.panda_robot()
    rb0["self_pairs"] = workloads.self_collision_pairs(rb0, min_link_gap=0)
    ps0 = pm.Planner(rb0, sc.grid_desc, cp)
    ps0.set_distance_field(sc.phi)
    Us0 = np.zeros((32, 7), np.float32)
    ps0.smpc_iterate(sc.q0, sc.qd0, sc.T, Us0, 512, 0.02, 0.05, SIGMA, 3, 0)
    out["words"]["self_spheres"] = ps0.bounds_status(reset=True)
    # both layouts through the batch kernels (their group records are built
    # per instance), one-step and run-time shapes
    for H, tag in ((32, "batch_self_one_step"), (100, "batch_self_run_time")):
        items = [dict(ctx=pl, q=torch.from_numpy(sc.q0.astype(np.float32)).to(dev),
                      qd=torch.from_numpy(sc.qd0.astype(np.float32)).to(dev),
                      T_goal=torch.from_numpy(np.asarray(sc.T, np.float32).ravel().copy()).to(dev),
                      U=torch.zeros((H, 7), dtype=torch.float32, device=dev), K=256, seed=50 + i)
                 for i, pl in enumerate((ps, ps0))]
        b = pm.Batch(0)
        b.run(items, n_iters=2, flags=pm.PM_BATCH_REPLAN)
        torch.cuda.synchronize()
        b.close()
        out["words"][tag] = max(it["ctx"].bounds_status(reset=True) for it in items)
    ps0.close()
    ps.close()
    for pl in planners:
        pl.close()
    p.close()
    print("RESULT " + json.dumps(out))
""")


def test_checked_build_finds_no_violation_and_keeps_parity():
    lib = os.path.join(ROOT, "paper_2512_22575_b300", "libparamap_checked.so")
    assert os.path.exists(lib), "build the checked library: python paper_2512_22575_b300/build.py --checked"
    env = dict(os.environ, PARAMAP_LIB="libparamap_checked.so")
    code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1][7:])
    assert res["checked"] is True and res["lib"].endswith("libparamap_checked.so")
    bad = {k: v for k, v in res["words"].items() if v != 0}
    assert not bad, f"bounds violations (bit mask per workload): {bad}"
    assert len(res["words"]) >= 28
    for tag, (s_rel, u_abs, u_iso, bound) in res["parity"].items():
        # costs within S_REL and the update exact given the GPU's costs
        # (U_ISO) everywhere; U* against the oracle's within U_ABS wherever the
        # soft-min is well conditioned (first-order bound of the FP32 cost
        # rounding sigma max|dS|/lambda below U_ABS / 2; on the few-roll-out
        # shapes it is not, and that bound, not the kernel, sets the error)
        assert s_rel <= S_REL and u_iso <= U_ISO, (tag, s_rel, u_iso)
        assert u_abs <= U_ABS or bound > U_ABS / 2, (tag, u_abs, bound)
        print(f"{tag}: S rel {s_rel:.1e}, |U-U_iso| {u_iso:.1e}, |U-U_ref| {u_abs:.1e}, bound {bound:.1e}")
