"""Host-buffer calls replayed from captured CUDA graphs (pm_set_call_graphs).

A call whose inputs and outputs are all host memory runs as one graph launch;
its kernels read the call's inputs and scalars from a fixed device block.
The results must be bit-identical to the same call launched directly, on the
capturing call and on replays with new inputs, for every tile shape family,
and a changed setting (tile shape, noise rounding) must not replay a graph
captured under the old one.
"""
import numpy as np
import pytest

from parity_common import SIGMA, S_REL, U_ABS, Scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def scene():
    return Scene("cfg1_seed6")


def iterate(p, sc, U, K, seed, it, dt=0.02, lam=0.05, sigma=SIGMA):
    U = U.copy()
    S = np.empty(K, np.float32)
    p.smpc_iterate(sc.q0, sc.qd0, sc.T, U, K, dt, lam, sigma, seed, it, costs_out=S)
    return U, S


def replan(p, sc, U, K, n_iters, seed, r, dt=0.02, lam=0.05):
    q, qd, U = sc.q0.copy(), sc.qd0.copy(), U.copy()
    u0 = np.empty(7, np.float32)
    best = np.empty(1, np.float32)
    p.replan(q, qd, sc.T, U, K, n_iters, dt, lam, SIGMA, seed, r, u0_out=u0, best_cost=best)
    return q, qd, U, u0, best


@pytest.mark.parametrize("K,H", [(256, 32), (4096, 64), (300, 200), (37, 5), (1000, 100)])
def test_graph_iterate_is_bit_identical(scene, K, H):
    pg, pd = scene.planner(), scene.planner()
    pd.set_call_graphs(False)
    rng = np.random.default_rng(K + H)
    U = (rng.normal(size=(H, 7)) * 0.2).astype(np.float32)
    for call in range(3):          # capture, then two replays with new inputs
        seed, it = 50 + call, 7 * call
        lam = 0.05 * (1 + call)
        Ug, Sg = iterate(pg, scene, U, K, seed, it, lam=lam)
        Ud, Sd = iterate(pd, scene, U, K, seed, it, lam=lam)
        assert np.array_equal(Ug, Ud), call
        assert np.array_equal(Sg, Sd), call
        U = Ug
    # without costs (a graph of its own)
    Ug = U.copy()
    pg.smpc_iterate(scene.q0, scene.qd0, scene.T, Ug, K, 0.02, 0.05, SIGMA, 9, 1)
    Ud = U.copy()
    pd.smpc_iterate(scene.q0, scene.qd0, scene.T, Ud, K, 0.02, 0.05, SIGMA, 9, 1)
    assert np.array_equal(Ug, Ud)
    pg.close()
    pd.close()


@pytest.mark.parametrize("K,H,n_iters", [(4096, 64, 8), (512, 16, 3), (2048, 48, 1)])
def test_graph_replan_is_bit_identical(scene, K, H, n_iters):
    pg, pd = scene.planner(), scene.planner()
    pd.set_call_graphs(False)
    U = np.zeros((H, 7), np.float32)
    for r in range(3):
        outs_g = replan(pg, scene, U, K, n_iters, 100, r, dt=0.02 + 0.005 * r)
        outs_d = replan(pd, scene, U, K, n_iters, 100, r, dt=0.02 + 0.005 * r)
        for a, b in zip(outs_g, outs_d):
            assert np.array_equal(a, b), r
        U = outs_g[2]
    pg.close()
    pd.close()


def test_settings_changes_are_not_replayed_from_old_graphs(scene):
    """A graph captured under one tile shape / noise rounding is not replayed
    after the setting changes: results follow the new setting exactly."""
    K, H = 96, 32
    pg, pd = scene.planner(), scene.planner()
    pd.set_call_graphs(False)
    U = np.zeros((H, 7), np.float32)
    iterate(pg, scene, U, K, 3, 0)               # captures under the default shape
    for p in (pg, pd):
        p.set_tile_shape(2, 32, 1)
    b_g, b_d = iterate(pg, scene, U, K, 3, 0), iterate(pd, scene, U, K, 3, 0)
    assert np.array_equal(b_g[0], b_d[0]) and np.array_equal(b_g[1], b_d[1])
    for p in (pg, pd):
        p.set_tile_shape(0, 0, 0)
        p.set_noise_dtype("f16")
    c_g, c_d = iterate(pg, scene, U, K, 3, 0), iterate(pd, scene, U, K, 3, 0)
    assert np.array_equal(c_g[0], c_d[0]) and np.array_equal(c_g[1], c_d[1])
    pg.close()
    pd.close()


def test_graph_calls_match_the_oracle(scene):
    """The replayed path against the FP64 oracle at the parity bars."""
    K, H = 512, 32
    p = scene.planner()
    U = (np.random.default_rng(4).normal(size=(H, 7)) * 0.2).astype(np.float32)
    for it in range(2):
        Ug, Sg = iterate(p, scene, U, K, 77, it)
        Uo, So, _ = scene.oracle_iterate(U, K, 0.02, 0.05, SIGMA, 77, it)
        assert (np.abs(Sg - So) / np.abs(So)).max() <= S_REL
        assert np.abs(Ug - Uo).max() <= U_ABS
        U = Ug
    p.close()
