"""The allocation-free value iteration entry point.

Some callers cannot call cudaMalloc (an arena that owns all device memory,
a loop that forbids allocation after start-up); cpmdp_value_iteration_static
keeps its scratch in a fixed static device array instead. These tests call
it through the C ABI, two calls in a row on different grids, and check each
result against the regular cpmdp_value_iteration on the same inputs (values
within the FP32 tolerance the other GPU tests use, sweep counts within one),
against closed forms (a deterministic 1-D chain: V = gamma^dist R_goal; a
grid with no cell array and a constant reward: V = R / (1 - gamma)), that a
second call leaves the device's free memory unchanged, that a cell code
other than 0, 1, 2 is refused, and the size limit. The file name makes
pytest collect it last.
"""
import numpy as np
import pytest

import cpmdp_inputs as ci

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def cp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2103_00331_gb300 as cp
    return cp


def _regular(cp, gw):
    import torch
    f = cp.build_factors(gw, device=0)
    V = torch.zeros(gw.nstates, dtype=torch.float32, device="cuda")
    r = cp.value_iteration(f, cp.F32, V, None, opts=cp.default_opts(max_iter=5000, certify=0))
    f.close()
    return V.double().cpu().numpy(), r["iterations"]


def _static(cp, gw, cell=True, max_iter=5000):
    import torch
    c = torch.as_tensor(gw.cell.reshape(-1)).cuda() if cell else None
    R = torch.as_tensor(gw.reward.reshape(-1), dtype=torch.float32).cuda()
    V = torch.zeros(gw.nstates, dtype=torch.float32, device="cuda")
    k, res = cp.value_iteration_static(gw.shape, gw.p, gw.gamma, c, R, V, tol=1e-6, max_iter=max_iter)
    return V.double().cpu().numpy(), k, res


def test_static_matches_regular_twice(cp):
    for gw in (ci.config_3d(side=64, seed=0),
               ci.gridworld((40, 50, 30), p=0.7, gamma=0.97, step_reward=-0.02,
                            goal_rewards=[1.0, 0.5, -1.0], obstacle_rate=0.1, seed=5)):
        want, k_want = _regular(cp, gw)
        got, k, res = _static(cp, gw)
        assert res < 1e-6
        # same Jacobi iteration in FP32 (operation order may differ by the
        # rounding of a sum): the stopping sweep agrees to within one
        assert abs(k - k_want) <= 1, (k, k_want)
        # both stop below tol: within (2 gamma tol + FP32 rounding) / (1 - gamma)
        eps = 14 * U32 * (np.abs(gw.reward).max() + np.abs(want).max())
        assert np.abs(got - want).max() <= (2 * gw.gamma * 1e-6 + eps) / (1 - gw.gamma)


def test_static_deterministic_chain_closed_form(cp):
    """1-D chain, p = 1 (the move always happens), reward 0 except one
    terminal goal: V(s) = gamma^|s - g| R_goal (1-D branch of the kernel)."""
    n, gamma, rg = 200, 0.95, 2.0
    gw = ci.gridworld((n,), p=1.0, gamma=gamma, step_reward=0.0, goal_rewards=[rg], seed=3)
    g = int(np.flatnonzero(gw.cell.reshape(-1) == ci.TERMINAL)[0])
    got, k, res = _static(cp, gw)
    dist = np.abs(np.arange(n) - g)
    want = rg * gamma ** dist.astype(np.float64)
    # each sweep rounds once per state in FP32; the error after convergence
    # is below tol / (1 - gamma) plus a few ulps per step of distance
    assert np.abs(got - want).max() <= 1e-6 / (1 - gamma) + 4 * U32 * rg * (dist.max() + 1)


def test_static_no_cell_array_2d(cp):
    """10 x 10, 4 actions, p = 0.8, reward -0.04 everywhere, no cell array
    (every state free, no terminal): V = R / (1 - gamma) = -0.4; the regular
    solver on the same all-free grid agrees (2-D weights of the kernel)."""
    gw = ci.gridworld((10, 10), p=0.8, gamma=0.9, step_reward=-0.04, goal_rewards=[], seed=0)
    got, k, res = _static(cp, gw, cell=False, max_iter=1000)
    assert res < 1e-6
    assert np.abs(got + 0.4).max() <= 1e-6 / (1 - 0.9) + 1e-6
    want, k_want = _regular(cp, gw)
    assert abs(k - k_want) <= 1
    assert np.abs(got - want).max() <= (2 * 0.9 * 1e-6 + 1e-6) / (1 - 0.9)


def test_static_allocates_nothing(cp):
    """After a first call (which loads the module), a second call leaves
    the device's free memory exactly as it was."""
    import torch
    gw = ci.config_3d(side=32, seed=4)
    _static(cp, gw)
    torch.cuda.synchronize()
    c = torch.as_tensor(gw.cell.reshape(-1)).cuda()
    R = torch.as_tensor(gw.reward.reshape(-1), dtype=torch.float32).cuda()
    V = torch.zeros(gw.nstates, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    cp.value_iteration_static(gw.shape, gw.p, gw.gamma, c, R, V, tol=1e-6, max_iter=5000)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_rejects_bad_cell_code(cp):
    import torch
    gw = ci.config_3d(side=16, seed=1)
    cell = gw.cell.reshape(-1).copy()
    cell[123] = 7
    c = torch.as_tensor(cell).cuda()
    R = torch.as_tensor(gw.reward.reshape(-1), dtype=torch.float32).cuda()
    V = torch.full((gw.nstates,), 3.0, dtype=torch.float32, device="cuda")
    with pytest.raises(cp.CpmdpError) as ei:
        cp.value_iteration_static(gw.shape, gw.p, gw.gamma, c, R, V)
    assert ei.value.status == cp.EINVAL and "cell codes" in cp.last_error()
    assert bool((V == 3.0).all())   # refused before the first sweep
    # the array is usable again at once
    got, k, res = _static(cp, gw)
    assert res < 1e-6


def test_static_rejects_too_many_states(cp):
    import torch
    R = torch.zeros(1, dtype=torch.float32, device="cuda")
    with pytest.raises(cp.CpmdpError) as ei:
        cp.value_iteration_static((160, 160, 160), 0.8, 0.9, None, R, R)
    assert ei.value.status == cp.EINVAL and "at most" in cp.last_error()
