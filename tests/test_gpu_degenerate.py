"""Degenerate cases of the method on the GPU, checked against closed forms
(no oracle involved) through every solver path: the single-block solver
(grids one block covers), the barrier-free persistent solver (FP32, rows a
multiple of 4 states), the grid-barrier solver (fused=2) and the batched
solvers.

* gamma = 0: Eq. 1 gives V'(s) = R(s) on free states and terminals (0 on
  obstacles) from any start, so value iteration from zero stops after its
  second sweep with V = R exactly.
* A deterministic 1-D chain (p = 1) with one terminal goal: V(s) =
  gamma^dist(s) R_goal in exact arithmetic; FP64 value iteration to 1e-13
  reproduces it to a few units in the last place, and the greedy policy
  moves toward the goal.
* gamma = 1 (undiscounted) on a grid with a free state walled in by
  obstacles and a negative step reward: its value decreases by the step
  reward every sweep, so the solve stops at max_iter with ENOCONV.
"""
import numpy as np
import pytest

import cpmdp_inputs as ci

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2103_00331_gb300 as cp
    return cp


def _expected_gamma0(gw):
    R = np.asarray(gw.reward, dtype=np.float64).reshape(-1)
    cell = np.asarray(gw.cell).reshape(-1)
    return np.where(cell == ci.OBSTACLE, 0.0, R)


@pytest.mark.parametrize("shape", [(10, 10), (16, 16, 16), (7, 9, 13), (37,)])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("fused", [1, 2])
def test_gamma_zero_gives_rewards(cp, shape, prec, fused):
    import torch
    gw = ci.gridworld(shape, p=0.8, gamma=0.0, step_reward=-0.04, goal_rewards=[1.0, -1.0], obstacle_rate=0.1,
                      seed=3)
    f = cp.build_factors(gw, device=0)
    dt = torch.float64 if prec == 1 else torch.float32
    V = torch.zeros(gw.nstates, dtype=dt, device="cuda")
    r = cp.value_iteration(f, cp.F64 if prec == 1 else cp.F32, V, None,
                           opts=cp.default_opts(max_iter=100, fused=fused))
    want = _expected_gamma0(gw).astype(np.float64 if prec == 1 else np.float32)
    assert r["iterations"] == 2 and r["residual"] == 0.0
    assert np.array_equal(V.cpu().numpy(), want)
    f.close()


def test_gamma_zero_batch(cp):
    import torch
    inst = [ci.gridworld(s, p=0.7, gamma=0.0, step_reward=-0.04, goal_rewards=[1.0, -1.0], obstacle_rate=0.1,
                         seed=10 + i) for i, s in enumerate([(10, 10), (48, 48, 48), (130, 150), (9,), (8, 8, 8)])]
    B = cp.batch_build(inst, device=0)
    for fused in (1, 4):
        V = torch.zeros(int(B.total_states), dtype=torch.float32, device="cuda")
        r, it, res = cp.batch_value_iteration(B, V, opts=cp.default_opts(max_iter=100, fused=fused))
        assert np.all(it == 2) and np.all(res == 0.0)
        Vh = V.cpu().numpy()
        for i, gw in enumerate(inst):
            lo = int(B.offsets[i])
            assert np.array_equal(Vh[lo:lo + gw.nstates], _expected_gamma0(gw).astype(np.float32)), (fused, i)
    B.close()


@pytest.mark.parametrize("n,goal,gamma", [(40, 0, 0.9), (57, 31, 0.95), (200, 199, 0.99)])
def test_deterministic_chain_closed_form(cp, n, goal, gamma):
    import torch
    cell = np.zeros(n, np.uint8)
    cell[goal] = ci.TERMINAL
    R = np.zeros(n)
    R[goal] = 1.0
    gw = ci.GridWorld(shape=(n,), p=1.0, gamma=gamma, cell=cell, reward=R)
    f = cp.build_factors(gw, device=0)
    dist = np.abs(np.arange(n) - goal)
    want = gamma ** dist
    for fused in (1, 2):
        V = torch.zeros(n, dtype=torch.float64, device="cuda")
        pi = torch.zeros(n, dtype=torch.uint8, device="cuda")
        r = cp.value_iteration(f, cp.F64, V, pi, opts=cp.default_opts(tol=1e-13, max_iter=5000, fused=fused))
        assert r["status"] == cp.OK
        assert np.abs(V.cpu().numpy() - want).max() <= 1e-13
        p = pi.cpu().numpy()
        assert p[goal] == 255
        assert np.all(p[:goal] == 1) and np.all(p[goal + 1:] == 0)   # action 1 = +1, action 0 = -1
    f.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_undiscounted_walled_state_reaches_max_iter(cp, prec):
    import torch
    shape = (12, 12)
    cell = np.zeros(shape, np.uint8)
    cell[0, 0] = ci.TERMINAL
    cell[5, 4] = cell[5, 6] = cell[4, 5] = cell[6, 5] = ci.OBSTACLE   # state (5, 5) is walled in
    R = np.full(shape, -0.04)
    R[0, 0] = 1.0
    R[cell == ci.OBSTACLE] = 0.0
    gw = ci.GridWorld(shape=shape, p=0.8, gamma=1.0, cell=cell, reward=R)
    f = cp.build_factors(gw, device=0)
    V = torch.zeros(gw.nstates, dtype=torch.float64 if prec == 1 else torch.float32, device="cuda")
    with pytest.raises(cp.CpmdpError) as ei:
        cp.value_iteration(f, cp.F64 if prec == 1 else cp.F32, V, None, opts=cp.default_opts(max_iter=300))
    assert ei.value.status == cp.ENOCONV
    assert abs(float(V[5 * 12 + 5]) - 300 * -0.04) <= 1e-3
    f.close()
