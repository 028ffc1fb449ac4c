"""Shared set-up of the GPU parity tests: the same seeded inputs for both sides.

Tolerances (written once, used by every parity test):
  S_REL   per-roll-out costs S^(m), relative            1e-4
  U_ABS   updated controls U* (Eq. 30), absolute          1e-5
  NOISE   normals / eps, |gpu - oracle| <= NOISE_ABS + NOISE_REL |oracle|
  U_ISO   U* recomputed in FP64 from the GPU's own FP32 costs vs the GPU U*;
          this isolates the soft-min reduction from the cost arithmetic  1e-6
"""
import numpy as np

import oracle
import workloads

S_REL = 1e-4
U_ABS = 1e-5
NOISE_REL = 2e-6
NOISE_ABS = 2e-6
U_ISO = 1e-6
SIGMA = np.full(7, 0.5, dtype=np.float32)


class Scene:
    """One stored scene with its grid, ready for both sides."""

    def __init__(self, name, cost_overrides=None):
        self.sc = workloads.load_scene(name)
        self.grid_desc = self.sc["grid"]
        self.phi = workloads.build_scene_grid(self.sc)
        self.robot = workloads.panda_robot()
        self.cp = workloads.default_cost_params(self.sc["q0"])
        if cost_overrides:
            self.cp.update(cost_overrides)
        self.q0 = self.sc["q0"].astype(np.float32)
        self.qd0 = self.sc["qd0"].astype(np.float32)
        self.T = self.sc["T_goal"].astype(np.float32).reshape(4, 4)
        # oracle side
        self.R = oracle.make_robot(self.robot)
        self.G = oracle.Grid(self.grid_desc, self.phi)
        self.C = oracle.make_cost(self.cp)

    def planner(self, dtype="f32"):
        import paper_2512_22575_b300 as pm
        p = pm.Planner(self.robot, self.grid_desc, self.cp, device=0, dtype=dtype)
        p.set_distance_field(self.phi)
        return p

    def oracle_iterate(self, U, K, dt, lam, sigma, seed, it, n_threads=0):
        return oracle.smpc_iterate(self.R, self.G, self.C, self.q0, self.qd0, self.T, U, K, dt,
                                   lam, sigma, seed, it, n_threads=n_threads)


def fp64_update_from_costs(S, eps, Ubar, lam):
    """Eqs. 29-30 in FP64 from given costs (used to isolate the reduction)."""
    S = np.asarray(S, dtype=np.float64)
    w = np.exp(-(S - S.min()) / lam)
    w /= w.sum()
    return np.asarray(Ubar, np.float64) + np.einsum("m,mkj->kj", w, eps), w


def first_order_bound(S_gpu, S_ref, sigma, lam):
    """sigma_max * max |dS - mean dS| / lambda: how far U* may move."""
    d = np.asarray(S_gpu, np.float64) - S_ref
    return float(np.max(sigma) * np.max(np.abs(d - d.mean())) / lam)
