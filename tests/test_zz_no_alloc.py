"""The allocation-free value iteration entry point.

Some callers cannot call cudaMalloc (an arena that owns all device memory,
a loop that forbids allocation after start-up); cpmdp_value_iteration_static
keeps its scratch in a fixed static device array instead. This test calls
it through the C ABI twice in a row, on two different grids, and checks each
result against the regular cpmdp_value_iteration on the same inputs, within
the FP32 tolerance the other GPU tests use. It also checks the size limit.
The file name makes pytest collect it last.
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


def test_static_matches_regular_twice(cp):
    import torch
    for gw in (ci.config_3d(side=64, seed=0),
               ci.gridworld((40, 50, 30), p=0.7, gamma=0.97, step_reward=-0.02,
                            goal_rewards=[1.0, 0.5, -1.0], obstacle_rate=0.1, seed=5)):
        want, k_want = _regular(cp, gw)
        cell = torch.as_tensor(gw.cell.reshape(-1)).cuda()
        R = torch.as_tensor(gw.reward.reshape(-1), dtype=torch.float32).cuda()
        V = torch.zeros(gw.nstates, dtype=torch.float32, device="cuda")
        k, res = cp.value_iteration_static(gw.shape, gw.p, gw.gamma, cell, R, V, tol=1e-6,
                                           max_iter=5000)
        got = V.double().cpu().numpy()
        assert res < 1e-6
        # both stop below tol: within (2 gamma tol + FP32 rounding) / (1 - gamma)
        eps = 14 * U32 * (np.abs(gw.reward).max() + np.abs(want).max())
        assert np.abs(got - want).max() <= (2 * gw.gamma * 1e-6 + eps) / (1 - gw.gamma)


def test_static_rejects_too_many_states(cp):
    import torch
    R = torch.zeros(1, dtype=torch.float32, device="cuda")
    with pytest.raises(cp.CpmdpError) as ei:
        cp.value_iteration_static((160, 160, 160), 0.8, 0.9, None, R, R)
    assert ei.value.status == cp.EINVAL and "at most" in cp.last_error()
