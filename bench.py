"""Benchmark of the SMPC replanning loop (one 'step' = one replan).

Workload (config 2 of the workloads): 7-DoF arm, K = 4096 roll-outs,
H = 64, 8 SMPC iterations per replan, a 160 x 160 x 120 distance field at
1 cm built from 20 seeded boxes and balls, and a target pose moving on a
seeded circle at 0.2 m/s.  The 200-replan episode repeats until --steps
replans have run (the state restarts every 200).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  'value' is device-timed (inputs resident in
HBM, CUDA events per replan on the launching stream, a 256 MiB buffer
written between replans to flush L2); 'e2e' is the same metric through the
C ABI with host buffers (copies in and out inside the timed region).
With torchrun (N > 1) every rank plans its own arm (independent replicas).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rollout-steps/s; replan p50/p99 ms served vs per-request plain, same GPU"
UNIT = "rollout-steps/s"
EPISODE = 200
# Algorithmic FP32 operations (FMA = 2; transcendental calls, integer Philox
# work and loads not counted), from the kernel's source-level arithmetic.
# A roll-out step: sampling 46, roll-out scans 128, control costs 66,
# kinematics 349, pose error 135, state limits and null space 127,
# accumulation 5 (856 in all) plus, per sphere, its centre 18, cell location
# 18 and the skip test 1 (28 x 37).  A sphere whose cell is not skipped adds
# its trilinear interpolation and cost, 26.  The terminal step (no spheres or
# state limits) is 729.
FLOPS_STEP = 856 + 28 * 37
FLOPS_STEP_ESTIMATE = 2300   # planning estimate: full trilinear evaluation of all 28 spheres
FLOPS_GATHER = 26
FLOPS_TERMINAL = 729
FP32_LANES_PER_SM = 128
SM_MAX_MHZ_NOMINAL = 2032.0


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, world, device=None):
    """Largest value of x over the ranks (all_reduce MAX; NCCL wants a CUDA
    device, gloo the CPU); x itself for one rank."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank, world, max_seconds):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: every rank runs the same workload)."""
    return units_per_rank * world / max_seconds


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- workload
def load_workload():
    import workloads
    sc = workloads.load_scene("cfg2")
    return {
        "scene": sc,
        "phi": workloads.build_scene_grid(sc),
        "robot": workloads.panda_robot(),
        "cp": workloads.default_cost_params(sc["q0"]),
        "K": int(sc["K"]), "H": int(sc["H"]), "iters": int(sc["iters"]),
        "dt": float(sc["dt"]), "lam": float(sc["lambda"]),
        "sigma": np.full(7, sc["sigma"], dtype=np.float32),
    }


def targets(w, n):
    import workloads
    sc = w["scene"]
    T0 = sc["T_goal"].reshape(4, 4)
    return np.stack([workloads.moving_target(T0, sc["path_seed"], (r % EPISODE) * w["dt"],
                                             speed=sc["target_speed"]).ravel()
                     for r in range(n)]).astype(np.float32)


def config_dict(w, world, flush):
    g = w["scene"]["grid"]
    return {"workload": "SMPC replanning loop (config 2): 7-DoF arm, K=4096 roll-outs, H=64, "
                        "8 iterations per replan, 200-replan episodes, moving target",
            "K": w["K"], "H": w["H"], "iters_per_replan": w["iters"],
            "grid": [g.nx, g.ny, g.nz], "voxel_m": g.res, "grid_dtype": "f32",
            "replicas": world, "parallelism": f"replicas{world}",
            "l2": f"flushed between replans ({flush} MiB write)"}


# ------------------------------------------------------------ CPU oracle
def cpu_oracle_time(w, K_sample, iters, budget_s, n_threads, seed=100):
    """Time the FP64 oracle's SMPC iterations on a roll-out sample."""
    import oracle
    sc = w["scene"]
    R = oracle.make_robot(w["robot"])
    G = oracle.Grid(sc["grid"], w["phi"])
    Cc = oracle.make_cost(w["cp"])
    T = sc["T_goal"].reshape(4, 4)
    U = np.zeros((w["H"], 7))
    done, steps = 0, 0
    t0 = time.perf_counter()
    while done < iters:
        U, _, _ = oracle.smpc_iterate(R, G, Cc, sc["q0"], sc["qd0"], T, U, K_sample, w["dt"],
                                      w["lam"], w["sigma"], seed, done, n_threads=n_threads)
        done += 1
        steps += K_sample * w["H"]
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return steps / dt, done, dt


def run_reference(args, rank, world):
    """The oracle as the reference arm (host cores), one bounded sample per step."""
    if rank != 0:
        return
    import oracle
    w = load_workload()
    cores = oracle.cores_available()
    K_sample = 64
    R = oracle.make_robot(w["robot"])
    sc = w["scene"]
    G = oracle.Grid(sc["grid"], w["phi"])
    Cc = oracle.make_cost(w["cp"])
    Ts = targets(w, args.warmup + args.steps)
    q, qd, U = sc["q0"].astype(np.float64), sc["qd0"].astype(np.float64), np.zeros((w["H"], 7))
    t_timed = 0.0
    for r in range(args.warmup + args.steps):
        if r % EPISODE == 0:
            q, qd, U = sc["q0"].astype(np.float64), sc["qd0"].astype(np.float64), np.zeros((w["H"], 7))
        t0 = time.perf_counter()
        q, qd, U, _, _ = oracle.replan(R, G, Cc, q, qd, Ts[r].reshape(4, 4), U, K_sample, w["dt"],
                                       w["lam"], w["sigma"], 100, r % EPISODE, w["iters"],
                                       n_threads=cores)
        if r >= args.warmup:
            t_timed += time.perf_counter() - t0
    units = K_sample * w["H"] * w["iters"] * args.steps
    value = units / t_timed
    sample = (f"{K_sample} of the 4096 roll-outs per replan (same H, iterations, grid and "
              f"target path), {args.steps} replans")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_timed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(w, 1, 0) | {"l2": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- ours
def bench_batched(pm, torch, dev, stream, reps=20):
    """Uneven-instance workload (64 arms, own K, H and field each): one
    replan (8 iterations) of all instances as one batch (persistent kernel,
    CUDA graph, autotuned plan) against the same replans issued one instance
    at a time on one stream."""
    import workloads
    insts = workloads.load_scene("cfg3")["instances"]
    sigma = np.full(7, 0.5, np.float32)
    rb = workloads.panda_robot()
    items, planners = [], []
    units = 0
    for i, sc in enumerate(insts):
        p = pm.Planner(rb, sc["grid"], workloads.default_cost_params(sc["q0"]))
        p.set_distance_field(workloads.build_scene_grid(sc))
        planners.append(p)
        K, H = int(sc["K"]), int(sc["H"])
        units += K * H * 8
        items.append(dict(ctx=p, q=torch.from_numpy(sc["q0"]).to(dev),
                          qd=torch.from_numpy(sc["qd0"]).to(dev),
                          T_goal=torch.from_numpy(sc["T_goal"].ravel().copy()).to(dev),
                          U=torch.zeros((H, 7), dtype=torch.float32, device=dev),
                          u0_out=torch.zeros(7, dtype=torch.float32, device=dev),
                          best_cost=torch.zeros(1, dtype=torch.float32, device=dev),
                          K=K, dt=0.02, lam=0.05, sigma=sigma, seed=300 + i, iter_index=0))
    flags = pm.PM_BATCH_REPLAN | pm.PM_BATCH_GRAPH | pm.PM_BATCH_AUTOTUNE
    b = pm.Batch(dev.index or 0)

    def timed(fn):
        # reps back-to-back rounds between two events on the stream: the
        # host's preparation of a round (marshalling 64 items, descriptors)
        # overlaps the GPU work of the previous one, as in a serving loop
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    with torch.cuda.stream(stream):
        for _ in range(3):
            b.run(items, n_iters=8, flags=flags, stream=stream)
        torch.cuda.synchronize()
        t_batch = timed(lambda: b.run(items, n_iters=8, flags=flags, stream=stream))

        def sequential():
            for it in items:
                it["ctx"].replan(it["q"], it["qd"], it["T_goal"], it["U"], it["K"], 8, 0.02, 0.05,
                                 sigma, it["seed"], 0, u0_out=it["u0_out"], best_cost=it["best_cost"],
                                 stream=stream)
        sequential()
        torch.cuda.synchronize()
        t_seq = timed(sequential)
    shapes, blocks, tuned_us = b.plan(items, n_iters=8, flags=flags)
    b.close()
    for p in planners:
        p.close()
    return {"workload": "64 uneven instances (K 256-4096, H 16-64, fields 64^3-128^3), one replan "
                        "(8 iterations) each",
            "timing": f"{reps} back-to-back rounds between CUDA events on the stream, per round",
            "value": units / (t_batch / 1e3), "unit": UNIT, "ms_per_batch_replan": t_batch,
            "sequential_ms": t_seq, "sequential_value": units / (t_seq / 1e3),
            "speedup_vs_sequential": t_seq / t_batch,
            "plan": {"autotuned_us": tuned_us, "total_blocks": int(sum(blocks)),
                     "shapes": sorted({f"{c}x{l}x{p_}" for c, l, p_ in shapes})}}


SERVE_RATES = (500, 1000, 2000, 3000, 4000, 6000)


def bench_self_collision(pm, torch, dev, stream, w, Ts, n_replans=100, min_link_gap=2):
    """The replanning workload with the self-collision term on (Eqs. 18-20):
    sphere pairs on frames at least min_link_gap apart (2: 240 pairs, the
    wrist's always in contact; 3: 160 pairs), w_self = 1.
    Replans timed with events per replan, then the iteration kernel alone."""
    import workloads
    sc = w["scene"]
    rb = dict(w["robot"])
    rb["self_pairs"] = workloads.self_collision_pairs(rb, min_link_gap=min_link_gap)
    cp = dict(w["cp"])
    cp["w_self"] = np.float32(1.0)
    K, H, iters, dt, lam, sigma = w["K"], w["H"], w["iters"], w["dt"], w["lam"], w["sigma"]
    p = pm.Planner(rb, sc["grid"], cp, device=dev.index or 0)
    p.set_distance_field(w["phi"])
    q0 = torch.from_numpy(sc["q0"].astype(np.float32)).to(dev)
    qd0 = torch.from_numpy(sc["qd0"].astype(np.float32)).to(dev)
    q, qd = q0.clone(), qd0.clone()
    U = torch.zeros((H, 7), dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_replans)]
    with torch.cuda.stream(stream):
        for r in range(3):
            p.replan(q, qd, Ts[r % len(Ts)], U, K, iters, dt, lam, sigma, 100, r, stream=stream)
        q.copy_(q0); qd.copy_(qd0); U.zero_()
        torch.cuda.synchronize()
        for r in range(n_replans):
            ev[r][0].record(stream)
            p.replan(q, qd, Ts[r % len(Ts)], U, K, iters, dt, lam, sigma, 100, r % EPISODE, stream=stream)
            ev[r][1].record(stream)
        torch.cuda.synchronize()
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        p.profile_enable(pm.PM_PROFILE_TIME)
        p.profile_read(reset=True)
        q.copy_(q0); qd.copy_(qd0); U.zero_()
        for r in range(min(n_replans, 50)):
            p.replan(q, qd, Ts[r % len(Ts)], U, K, iters, dt, lam, sigma, 100, r, stream=stream)
        torch.cuda.synchronize()
        kms, kn = p.profile_read(reset=True)
    p.close()
    return {"workload": f"replanning workload (K={K}, H={H}) with the self-collision term: "
                        f"{len(rb['self_pairs'])} sphere pairs on frames >= {min_link_gap} apart, w_self = 1",
            "value": K * H * iters / (ms * 1e-3), "unit": UNIT, "ms_per_replan": ms,
            "kernel_ms_per_launch": kms / max(kn, 1), "replans": n_replans}


def bench_episodes(pm, torch, dev, stream, K=4096, H=32, n_iters=8, max_replans=1000):
    """The evaluation protocol (Sec. V-A) on the synthetic scenes: from each
    cfg1 start state (10 scenes) and the replanning scene, replan at 50 Hz
    (dt = 0.02 s) to the fixed goal until the objective's relative
    improvement is below 1% and the flange is within 10 mm for 5 replans in
    a row.  Pose weights 10x the parity workload's.  Reports the averages the
    paper's Table I reports (planning time per replan, motion time, path
    length, position and orientation error) and how many converged."""
    import workloads
    base = workloads.default_cost_params(np.zeros(7))
    over = {"Q": base["Q"] * 10, "QH": base["QH"] * 10}
    rows = []
    for name in [f"cfg1_seed{i}" for i in range(10)] + ["cfg2"]:
        sc = workloads.load_scene(name)
        cp = workloads.default_cost_params(sc["q0"])
        cp.update(over)
        p = pm.Planner(workloads.panda_robot(), sc["grid"], cp, device=dev.index or 0)
        p.set_distance_field(workloads.build_scene_grid(sc))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = p.plan_episode(sc["q0"], sc["qd0"], sc["T_goal"].ravel(), K, H, n_iters, 0.02, 0.05,
                           np.full(7, 0.5, np.float32), 7, max_replans=max_replans, pos_tol=0.01,
                           rel_tol=0.01, n_stable=5, stream=stream)
        wall = time.perf_counter() - t0
        p.close()
        rows.append((r, wall))
    conv = [r for r, _ in rows if r["converged"]]
    mean = (lambda xs: float(np.mean(xs)) if xs else None)
    return {"workload": f"11 scenes (10 plain + the replanning scene), K={K}, H={H}, {n_iters} iterations per "
                        f"replan, dt = 0.02 s, convergence: <1% objective improvement and <10 mm, 5 replans",
            "converged": len(conv), "episodes": len(rows),
            "planning_ms_per_replan": mean([1e3 * w / r["replans"] for r, w in rows]),
            "motion_time_s": mean([r["motion_time"] for r in conv]),
            "path_length_rad": mean([r["path_length"] for r in conv]),
            "e_pos_mm": mean([1e3 * r["e_pos"] for r in conv]),
            "e_ori_rad": mean([r["e_ori"] for r in conv]),
            "replans": [int(r["replans"]) for r, _ in rows]}


def bench_mapping(pm, torch, dev, stream, w, reps=50):
    """Mapping on the replanning grid (160 x 160 x 120 voxels at 1 cm):
    pm_edt_squared alone, and pm_map_update (occupancy copy, robot mask at
    the start configuration, transform, metres, cell minima), CUDA events on
    the stream.  The transform's traffic model is 21 B per voxel (occupancy
    byte in; three passes of an int32 read and write, the first without the
    read)."""
    import workloads
    sc = w["scene"]
    g = sc["grid"]
    occ = torch.from_numpy(workloads.occupancy_grid(sc["obstacles"], g)).to(dev)
    d2 = torch.empty(occ.shape, dtype=torch.int32, device=dev)
    p = pm.Planner(w["robot"], g, w["cp"], device=dev.index or 0)
    q0 = torch.from_numpy(sc["q0"].astype(np.float32)).to(dev)
    n_vox = occ.numel()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_edt = timed(lambda: pm.edt_squared(occ, d2, stream=stream))
    ms_upd = timed(lambda: p.map_update(occ, q_mask=q0, inflate=0.02, stream=stream))
    p.close()
    return {"workload": f"{g.nx}x{g.ny}x{g.nz} voxels at {g.res:g} m, {len(sc['obstacles'])} obstacles",
            "edt_ms": ms_edt, "edt_voxels_per_s": n_vox / (ms_edt * 1e-3),
            "edt_gbs_model": 21.0 * n_vox / (ms_edt * 1e-3) / 1e9,
            "map_update_ms": ms_upd, "map_update_voxels_per_s": n_vox / (ms_upd * 1e-3)}


def kernel_counters():
    """The committed ncu counters of the iteration kernel, or None when the
    kernel sources changed since they were captured."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "smpc_iteration_kernel_cfg2_counters.json")
    try:
        rec = json.load(open(path))
        h = hashlib.sha256()
        for f in rec["sources"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        return rec if h.hexdigest() == rec["sources_sha256"] else None
    except (OSError, KeyError, ValueError):
        return None


def kernel_traffic_bytes():
    """DRAM bytes (read + write) per launch of the iteration kernel from the
    committed ncu counters, or None when they are stale."""
    rec = kernel_counters()
    if rec is None:
        return None
    return rec["dram_bytes_read_per_launch"] + rec["dram_bytes_write_per_launch"]


def bench_latency_cfg1(pm, torch, dev, stream, reps=200):
    """Single SMPC iteration of the plain workload (K=256, H=32, 64^3 field
    at 2 cm): device time of the iteration (CUDA events around each call on
    the launching stream, the GPU kept busy so the host does not starve it),
    and the host-observed latency of a call with host buffers."""
    import workloads
    sc = workloads.load_scene("cfg1_seed0")
    p = pm.Planner(workloads.panda_robot(), sc["grid"], workloads.default_cost_params(sc["q0"]),
                   device=dev.index or 0)
    p.set_distance_field(workloads.build_scene_grid(sc))
    K, H = int(sc["K"]), int(sc["H"])
    sigma = np.full(7, 0.5, np.float32)
    q0 = torch.from_numpy(sc["q0"].astype(np.float32)).to(dev)
    qd0 = torch.from_numpy(sc["qd0"].astype(np.float32)).to(dev)
    T = torch.from_numpy(sc["T_goal"].astype(np.float32).ravel().copy()).to(dev)
    U = torch.zeros((H, 7), dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    with torch.cuda.stream(stream):
        for i in range(5):
            p.smpc_iterate(q0, qd0, T, U, K, 0.02, 0.05, sigma, 1, i, stream=stream)
        torch.cuda.synchronize()
        torch.cuda._sleep(50_000_000)            # queue the calls behind a busy GPU
        for i in range(reps):
            ev[i][0].record(stream)
            p.smpc_iterate(q0, qd0, T, U, K, 0.02, 0.05, sigma, 1, i, stream=stream)
            ev[i][1].record(stream)
    torch.cuda.synchronize()
    dev_us = np.array([a.elapsed_time(b) * 1e3 for a, b in ev])
    qh, qdh = sc["q0"].astype(np.float32), sc["qd0"].astype(np.float32)
    Th = sc["T_goal"].astype(np.float32).ravel().copy()
    Uh = np.zeros((H, 7), np.float32)
    host_us = []
    for i in range(reps):
        t0 = time.perf_counter()
        p.smpc_iterate(qh, qdh, Th, Uh, K, 0.02, 0.05, sigma, 1, i)
        host_us.append((time.perf_counter() - t0) * 1e6)
    p.close()
    return {"workload": "one SMPC iteration, K=256, H=32, 64^3 field at 2 cm (plain single iteration)",
            "device_us_p50": float(np.percentile(dev_us, 50)), "device_us_p99": float(np.percentile(dev_us, 99)),
            "host_call_us_p50": float(np.percentile(host_us, 50)),
            "host_call_us_p99": float(np.percentile(host_us, 99)),
            "host_call": "pm_smpc_iterate with host buffers (copies in and out, synchronous)",
            "rollout_steps_per_s_device": K * H / (np.percentile(dev_us, 50) * 1e-6)}


def bench_serving(pm, torch, dev, rates=SERVE_RATES, duration_s=0.5, n_iters=8, deadline_ms=10.0,
                  seed=7, spin_us=5000, max_inflight=2, admit_window_us=100):
    """Serving workload: Poisson replan requests from 256 arms (own field of
    96^3-128^3 at 1 cm each; per request K in {512, 1024, 2048, 4096}, H in
    {16, 32, 48, 64}, 8 iterations, warm start from the arm's resident
    sequence, 10 ms admission deadline) at each offered rate, once through
    the server (continuous batching) and once as per-request plain
    pm_replan calls in arrival order on one stream.  Latency runs from the
    request's scheduled arrival to its result on the host."""
    import workloads
    from concurrent.futures import ThreadPoolExecutor
    scenes = workloads.load_scene("cfg5")["instances"]
    rb = workloads.panda_robot()
    with ThreadPoolExecutor(max(1, min(32, os.cpu_count() or 1))) as ex:
        fields = list(ex.map(workloads.build_scene_grid, scenes))
    dev_i = dev.index or 0
    planners = []
    for sc, phi in zip(scenes, fields):
        p = pm.Planner(rb, sc["grid"], workloads.default_cost_params(sc["q0"]), device=dev_i)
        p.set_distance_field(phi)
        planners.append(p)
    del fields
    n_arms = len(planners)
    q0 = [sc["q0"].astype(np.float32) for sc in scenes]
    qd0 = [sc["qd0"].astype(np.float32) for sc in scenes]
    Tg = [sc["T_goal"].astype(np.float32).ravel().copy() for sc in scenes]
    sigma = np.full(7, 0.5, np.float32)
    rng = np.random.default_rng(seed)
    deadline_s = deadline_ms / 1e3

    def arrivals(rate):
        n = max(1, int(rate * duration_s))
        return (np.cumsum(rng.exponential(1.0 / rate, n)), rng.integers(0, n_arms, n),
                rng.choice([512, 1024, 2048, 4096], n), rng.choice([16, 32, 48, 64], n))

    def spin_until(t):
        while time.perf_counter() < t:
            pass

    def summary(lat_s, n, span_s):
        lat = np.asarray(lat_s) * 1e3
        ok = len(lat)
        return {"p50_ms": float(np.percentile(lat, 50)) if ok else None,
                "p99_ms": float(np.percentile(lat, 99)) if ok else None,
                "plans_s": ok / span_s if span_s > 0 else 0.0,
                "completed": ok, "missed_deadline": n - ok}

    srv = pm.Server(dev_i, max_batch=64, max_inflight=max_inflight, spin_us=spin_us,
                    admit_window_us=admit_window_us)
    arm_ids = [srv.add_arm(p) for p in planners]
    stream = torch.cuda.Stream(device=dev)
    U_plain = [torch.zeros((256, 7), dtype=torch.float32, device=dev) for _ in range(n_arms)]
    H_plain = [0] * n_arms
    rounds = [0] * n_arms

    def served(t_arr, arm, K, H):
        tickets, late = [], []
        st0 = srv.stats()
        t0 = time.perf_counter() + 0.01
        for i in range(len(t_arr)):
            spin_until(t0 + t_arr[i])
            a = int(arm[i])
            late.append(time.perf_counter() - (t0 + t_arr[i]))
            tickets.append(srv.submit(arm_ids[a], q0[a], qd0[a], Tg[a], int(K[i]), int(H[i]), n_iters,
                                      seed=1000 + a, iter_index=rounds[a] * n_iters,
                                      deadline_us=int(deadline_ms * 1e3)))
            rounds[a] += 1
        lat, sizes, queue, t_end = [], [], [], t0
        for i, tk in enumerate(tickets):
            r = srv.wait(tk, timeout_us=60_000_000)
            if r["status"] == "PM_OK":
                lat.append(late[i] + r["latency_us"] * 1e-6)
                sizes.append(r["batch_size"])
                queue.append(r["queue_us"])
                t_end = max(t_end, t0 + t_arr[i] + lat[-1])
        st1 = srv.stats()
        out = summary(lat, len(t_arr), t_end - t0)
        out["mean_batch"] = float(np.mean(sizes)) if sizes else 0.0
        out["queue_ms_p50"] = float(np.percentile(queue, 50)) * 1e-3 if queue else None
        nb = st1["batches"] - st0["batches"]
        out["launch_host_ms_mean"] = (st1["launch_host_us"] - st0["launch_host_us"]) * 1e-3 / max(nb, 1)
        out["batch_run_ms_mean"] = (st1["batch_run_us"] - st0["batch_run_us"]) * 1e-3 / max(nb, 1)
        return out

    def plain(t_arr, arm, K, H):
        lat = []
        u0h, besth = np.empty(7, np.float32), np.empty(1, np.float32)
        t0 = time.perf_counter() + 0.01
        t_end = t0
        with torch.cuda.stream(stream):
            for i in range(len(t_arr)):
                arrive = t0 + t_arr[i]
                spin_until(arrive)
                if time.perf_counter() - arrive > deadline_s:
                    continue                      # not started within the deadline
                a, h = int(arm[i]), int(H[i])
                U = U_plain[a]
                if 0 < H_plain[a] < h:            # warm start: extend with the last row
                    U[H_plain[a]:h] = U[H_plain[a] - 1]
                elif H_plain[a] == 0:
                    U[:h].zero_()
                planners[a].replan(q0[a].copy(), qd0[a].copy(), Tg[a], U[:h], int(K[i]), n_iters, 0.02,
                                   0.05, sigma, 1000 + a, rounds[a], u0_out=u0h, best_cost=besth,
                                   stream=stream)
                rounds[a] += 1
                H_plain[a] = h
                t_end = time.perf_counter()
                lat.append(t_end - arrive)
        return summary(lat, len(t_arr), t_end - t0)

    # the request loops run with Python's garbage collector paused, so that a
    # collection in the submitting thread does not delay submissions
    import gc
    gc.collect()
    gc.disable()
    # warm up both paths (kernel loading, plan caches, pinned staging)
    w = arrivals(2000)
    served(*[x[:200] for x in w])
    plain(*[x[:50] for x in w])
    torch.cuda.synchronize()
    results = []
    for rate in rates:
        a = arrivals(rate)
        results.append({"offered_per_s": rate, "requests": len(a[0]),
                        "served": served(*a), "plain": plain(*a)})
    gc.enable()
    stats = srv.stats()
    srv.close()
    for p in planners:
        p.close()
    return {"workload": f"{n_arms} arms, fields 96^3-128^3 at 1 cm, Poisson requests with K in "
                        "{512,1024,2048,4096}, H in {16,32,48,64}, 8 iterations, warm start, "
                        f"{deadline_ms:g} ms admission deadline, {duration_s:g} s per rate",
            "latency": "scheduled arrival to result on the host", "rates": results,
            "server": {"max_batch": 64, "max_inflight": max_inflight, "admit_window_us": admit_window_us,
                       "spin_us": spin_us},
            "server_stats": stats}


def warm_machine(call, seconds, min_calls=1, stream=None, torch=None):
    """Untimed calls for at least `seconds` (and min_calls): the host CPU of
    a freshly started job runs slowly at first (a fixed pure-Python loop
    measured 3.6 ms cold and 0.6 ms after a few hundred calls), and a host
    that enqueues slowly leaves the GPU waiting, so the timed region starts
    only after this warm-up.  The calls use scratch state: the timed
    replans remain the episode's from its start."""
    t0 = time.perf_counter()
    n = 0
    while n < min_calls or time.perf_counter() - t0 < seconds:
        if stream is not None:
            with torch.cuda.stream(stream):
                call(n)
            if n % 8 == 7:
                torch.cuda.synchronize()
        else:
            call(n)
        n += 1
    if torch is not None:
        torch.cuda.synchronize()
    return n


def run_ours(args, rank, world, local):
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    import paper_2512_22575_b300 as pm

    w = load_workload()
    K, H, iters, dt, lam, sigma = w["K"], w["H"], w["iters"], w["dt"], w["lam"], w["sigma"]
    sc = w["scene"]
    seed = 100 + rank
    n_total = args.warmup + args.steps
    Ts_host = targets(w, n_total)

    planner = pm.Planner(w["robot"], sc["grid"], w["cp"], device=local)
    planner.set_distance_field(w["phi"])
    stream = torch.cuda.Stream(device=dev)
    flush_mb = args.flush_mb
    flush = torch.empty(flush_mb << 20, dtype=torch.uint8, device=dev)

    Ts = torch.from_numpy(Ts_host).to(dev)
    q0 = torch.from_numpy(sc["q0"].astype(np.float32)).to(dev)
    qd0 = torch.from_numpy(sc["qd0"].astype(np.float32)).to(dev)
    q, qd = q0.clone(), qd0.clone()
    U = torch.zeros((H, 7), dtype=torch.float32, device=dev)
    u0 = torch.empty(7, dtype=torch.float32, device=dev)
    best = torch.empty(1, dtype=torch.float32, device=dev)
    qw, qdw, Uw = q0.clone(), qd0.clone(), U.clone()     # scratch state of the machine warm-up

    def episode_reset(r):
        if r % EPISODE == 0:
            q.copy_(q0); qd.copy_(qd0); U.zero_()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    # the clock sampler starts before the warm-up, so that no idle gap lies
    # between the warm-up and the timed replans (after an idle gap the host
    # enqueues the first launches slowly and the GPU waits for them)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    warm_machine(lambda r: planner.replan(qw, qdw, Ts[r % len(Ts)], Uw, K, iters, dt, lam, sigma, seed, r,
                                          u0_out=u0, best_cost=best, stream=stream),
                 args.warm_s, stream=stream, torch=torch)
    with torch.cuda.stream(stream):
        for r in range(args.warmup):
            episode_reset(r)
            planner.replan(q, qd, Ts[r], U, K, iters, dt, lam, sigma, seed, r % EPISODE,
                           u0_out=u0, best_cost=best, stream=stream)
            flush.zero_()
    torch.cuda.synchronize()
    # the state the timed replans start from, which the kernel-timing passes
    # below start from too
    q_t, qd_t, U_t = q.clone(), qd.clone(), U.clone()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            r = args.warmup + i
            episode_reset(r)
            ev[i][0].record(stream)
            planner.replan(q, qd, Ts[r], U, K, iters, dt, lam, sigma, seed, r % EPISODE,
                           u0_out=u0, best_cost=best, stream=stream)
            ev[i][1].record(stream)
            flush.zero_()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    # iteration-kernel time (CUDA events around each launch, on its stream)
    # and gathers per launch, over a second timed pass of the same replans:
    # events between the kernels would break the programmatic launch overlap
    # that the first pass measures
    # (three passes, the fastest kept: a pass that the host falls behind in
    # would count its launch gaps into the kernels' event intervals).  Each
    # pass replays the timed replans from their starting state, with the L2
    # flush between replans, so every pass does the timed region's work.
    n_count = min(args.steps, 200)
    per_launch = []
    gathers_per_launch = None
    for rep in range(3):
        q.copy_(q_t); qd.copy_(qd_t); U.copy_(U_t)
        torch.cuda.synchronize()
        planner.profile_enable(pm.PM_PROFILE_TIME | pm.PM_PROFILE_GATHERS)
        planner.profile_read(reset=True)
        planner.profile_gathers(reset=True)
        with torch.cuda.stream(stream):
            for i in range(n_count):
                r = args.warmup + i
                episode_reset(r)
                planner.replan(q, qd, Ts[r], U, K, iters, dt, lam, sigma, seed, r % EPISODE,
                               u0_out=u0, best_cost=best, stream=stream)
                flush.zero_()
        torch.cuda.synchronize()
        kms, kn = planner.profile_read(reset=True)
        per_launch.append(kms / max(kn, 1))
        g = planner.profile_gathers(reset=True) / (n_count * iters)
        gathers_per_launch = g if gathers_per_launch is None else gathers_per_launch
        planner.profile_enable(0)
    launches = n_count * iters
    kernel_ms = min(per_launch) * launches
    step_ms = np.array([s.elapsed_time(e) for s, e in ev])
    total_ms = max_over_ranks(float(step_ms.sum()), world, dev)
    value = whole_job_value(K * H * iters * args.steps, world, total_ms / 1e3)

    # end to end through the C ABI with host buffers (copies inside the region)
    n_e2e = min(args.steps, args.e2e_steps)
    qh, qdh = sc["q0"].astype(np.float32).copy(), sc["qd0"].astype(np.float32).copy()
    Uh = np.zeros((H, 7), np.float32)
    u0h, besth = np.empty(7, np.float32), np.empty(1, np.float32)
    # warm-up calls (the first captures the call's graph), on scratch state
    # for at least --warm-s, then the episode from its start as timed
    warm_machine(lambda r: planner.replan(qh, qdh, Ts_host[r % len(Ts_host)], Uh, K, iters, dt, lam, sigma,
                                          seed, r, u0_out=u0h, best_cost=besth),
                 args.warm_s, min_calls=max(3, args.warmup))
    qh, qdh = sc["q0"].astype(np.float32).copy(), sc["qd0"].astype(np.float32).copy()
    Uh[:] = 0
    if world > 1:
        torch.distributed.barrier()
    t_call = np.empty(n_e2e + 1)
    t0 = time.perf_counter()
    t_call[0] = t0
    for i in range(n_e2e):
        r = i % EPISODE
        if r == 0:
            qh[:] = sc["q0"]; qdh[:] = sc["qd0"]; Uh[:] = 0
        planner.replan(qh, qdh, Ts_host[r], Uh, K, iters, dt, lam, sigma, seed, r,
                       u0_out=u0h, best_cost=besth)
        t_call[i + 1] = time.perf_counter()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e_call_ms = np.diff(t_call) * 1e3
    e2e_value = whole_job_value(K * H * iters * n_e2e, world, e2e_s)
    # the host-buffer replan runs from its graph: one copy in of the call's
    # block (q0, qd0, T_goal, sigma, dt, lambda, seed, iteration: 96 floats
    # with padding) and U, one copy out of the outputs (q, qd, u0, best: 32
    # floats with padding) and U
    h2d = (96 + H * 7) * 4
    d2h = (32 + H * 7) * 4

    # roofline of the iteration kernel (algorithmic FP32 flops / event-timed duration)
    flops_launch = K * ((H - 1) * FLOPS_STEP + FLOPS_TERMINAL) + FLOPS_GATHER * gathers_per_launch
    avg_kernel_s = kernel_ms / 1e3 / max(launches, 1)
    achieved = flops_launch / avg_kernel_s / 1e12
    props = torch.cuda.get_device_properties(dev)
    peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
    fma_peak = pm.fp32_fma_peak(local)
    traffic = kernel_traffic_bytes()
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_measured_fma": fma_peak, "frac_of_measured_fma": achieved / fma_peak,
                "kernel": "smpc_iteration_kernel<C=1,L=32,P=2,float> at K=4096, H=64 "
                          "(72 registers, 7 blocks per SM)",
                "gathered_fraction": gathers_per_launch / (K * (H - 1) * 28),
                "kernel_ms_per_launch": avg_kernel_s * 1e3, "launches_timed": launches,
                "kernel_timing": f"CUDA events around each iteration kernel on its stream, the fastest of "
                                 f"three further passes of {n_count} replans (per-pass means "
                                 f"{', '.join(f'{x * 1e3:.2f}' for x in per_launch)} us)",
                "flops_per_launch": flops_launch,
                # the binding unit is instruction issue: share of issue slots busy
                # in the committed ncu capture (None when stale)
                "issue_slots_busy_ncu": (kernel_counters() or {}).get("issue_active_frac"),
                # FP32 work the kernel executes per roll-out step (2 FFMA + FADD +
                # FMUL, ncu), against the fixed algorithmic count `achieved` uses
                "executed_fp32_flops_per_step_ncu": (kernel_counters() or {}).get("fp32_flop_equiv_per_step"),
                "algorithmic_flops_per_step": flops_launch / (K * H),
                # the same rate with the planning estimate of 2300 FP32 flops per
                # roll-out step (every sphere interpolated, no skip)
                "frac_at_2300_flops_per_step": K * H * FLOPS_STEP_ESTIMATE / avg_kernel_s / 1e12 / peak,
                "peak_basis": f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 lanes "
                              f"x 2 x {SM_MAX_MHZ_NOMINAL:.0f} MHz (unit counts and max clock)"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": config_dict(w, world, flush_mb),
        "replan_ms": {"p50": float(np.percentile(step_ms, 50)),
                      "p99": float(np.percentile(step_ms, 99)), "mean": float(step_ms.mean())},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": n_e2e,
                "ms_per_step": 1e3 * e2e_s / n_e2e,
                "call_ms": {"p50": float(np.percentile(e2e_call_ms, 50)),
                            "p99": float(np.percentile(e2e_call_ms, 99)),
                            "max": float(e2e_call_ms.max())}},
        # per replan: n_iters x (iteration kernel + merge) + the replan step
        "gpu_launches": args.steps * (2 * iters + 1),
        "roofline": roofline,
        "clocks": clk,
    }
    planner.close()

    # reduced-precision variants (field and noise in FP16 / BF16) on the same
    # workload: device time of the replan and of the iteration kernel
    variants = {}
    legs = set(args.legs.split(",")) if args.legs else None
    want = (lambda name: legs is None or name in legs)
    for dt_name in (("f16", "bf16") if want("precision") else ()):
        pv = pm.Planner(w["robot"], sc["grid"], w["cp"], device=local, dtype=dt_name)
        pv.set_distance_field(w["phi"])
        pv.set_noise_dtype(dt_name)
        n_v = min(args.steps, 200)
        qv, qdv, Uv = q0.clone(), qd0.clone(), torch.zeros((H, 7), dtype=torch.float32, device=dev)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(n_v)]
        with torch.cuda.stream(stream):
            for r in range(3):
                pv.replan(qv, qdv, Ts[r], Uv, K, iters, dt, lam, sigma, seed, r, stream=stream)
            qv.copy_(q0); qdv.copy_(qd0); Uv.zero_()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for i in range(n_v):
                evs[i][0].record(stream)
                pv.replan(qv, qdv, Ts[i], Uv, K, iters, dt, lam, sigma, seed, i, stream=stream)
                evs[i][1].record(stream)
                flush.zero_()
        torch.cuda.synchronize()
        # the iteration kernel alone, in a second pass (its timing events sit
        # between the kernels, so they stay out of the replan timing above)
        pv.profile_enable(pm.PM_PROFILE_TIME)
        pv.profile_read(reset=True)
        with torch.cuda.stream(stream):
            for i in range(min(n_v, 50)):
                pv.replan(qv, qdv, Ts[i], Uv, K, iters, dt, lam, sigma, seed, i, stream=stream)
                flush.zero_()
        torch.cuda.synchronize()
        kms, kn = pv.profile_read(reset=True)
        pv.close()
        vms = sum(s_.elapsed_time(e_) for s_, e_ in evs)
        variants[dt_name] = {"value": K * H * iters * n_v / (vms / 1e3), "unit": UNIT,
                             "ms_per_step": vms / n_v, "kernel_ms_per_launch": kms / max(kn, 1),
                             "replans": n_v}
    if variants:
        line["precision_variants"] = variants
    if want("latency"):
        line["latency_cfg1"] = bench_latency_cfg1(pm, torch, dev, stream)
    if want("self"):
        line["self_collision"] = bench_self_collision(pm, torch, dev, stream, w, Ts)
        line["self_collision_gap3"] = bench_self_collision(pm, torch, dev, stream, w, Ts, min_link_gap=3)
    if want("episodes"):
        line["episodes"] = bench_episodes(pm, torch, dev, stream)
    if want("mapping"):
        line["mapping"] = bench_mapping(pm, torch, dev, stream, w)
    if not args.no_batched and want("batched"):
        line["batched"] = bench_batched(pm, torch, dev, stream)
    if not args.no_serving and want("serving"):
        line["serving"] = bench_serving(pm, torch, dev)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        cores = oracle.cores_available()
        v, n_it, secs = cpu_oracle_time(w, K, 1000, args.cpu_budget, cores)
        line["cpu_baseline"] = {
            "value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_it} full SMPC iterations of the config-2 workload (K=4096, H=64) "
                      f"in {secs:.1f} s, OpenMP over roll-outs"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--flush-mb", type=int, default=256)
    ap.add_argument("--e2e-steps", type=int, default=1000)
    ap.add_argument("--legs", default="",
                    help="comma list of the extra legs to run (precision, latency, self, episodes, mapping, "
                         "batched, serving); empty = all")
    ap.add_argument("--warm-s", type=float, default=0.5,
                    help="seconds of untimed calls (scratch state) before each timed region")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
