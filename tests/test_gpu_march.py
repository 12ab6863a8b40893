"""The plane-marching backup sweep of large 3-D grids (the path of
cpmdp_bellman_backup and of the FP64 certifying sweep from 2^23 states on).

Ragged shapes (a z-chunk, a y-tile and an x-tile cut short, rows of 320
states) check the tile and chunk edges. The reference for the FP32 sweep is
the grid-barrier solver's first sweep (value iteration with max_iter = 1,
fused = 2): the same per-state arithmetic, so equal bit for bit. The FP64
certifying sweep and the policies are checked against the C oracle's full
FP64 backup of the same values.
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


@pytest.fixture(scope="module")
def oc():
    from oracle import cpfactor
    cpfactor.build()
    return cpfactor


SHAPES = [(130, 203, 320), (33, 512, 516)]


@pytest.mark.parametrize("shape", SHAPES)
def test_march_sweep_equals_solver_sweep(cp, oc, shape):
    import torch
    gw = ci.gridworld(shape, p=0.8, gamma=0.99, step_reward=-0.01,
                      goal_rewards=list(ci.uniform(1, 12, 8, 0.5, 1.0)), obstacle_rate=0.05, seed=7)
    assert gw.nstates >= 1 << 23
    f = cp.build_factors(gw, device=0)
    V0 = torch.as_tensor(ci.random_values(gw.shape, seed=5).reshape(-1).astype(np.float32)).cuda()
    out = torch.empty_like(V0)
    pi = torch.empty(gw.nstates, dtype=torch.uint8, device="cuda")
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    cp.bellman_backup(f, cp.F32, V0, out, pi, res)
    # the grid-barrier solver's first sweep from the same values
    V1 = V0.clone()
    r = cp.value_iteration(f, cp.F32, V1, None, opts=cp.default_opts(max_iter=1, tol=1e-30, fused=2, certify=0),
                           raise_on_noconv=False)
    assert r["iterations"] == 1 and r["solver"] == cp.SOLVER_GRID_BARRIER
    assert torch.equal(out.view(torch.int32), V1.view(torch.int32))
    assert res.item() == r["residual"]
    # FP32 policy against the oracle's FP64 argmax where rounding cannot flip it
    Vh = V0.double().cpu().numpy()
    Vn, pin, resn, Qn = oc.backup(gw, Vh, want_q=True)
    free = gw.cell.reshape(-1) == ci.FREE
    Qs = np.sort(Qn, axis=0)
    tol = 14 * U32 * 2.0
    sure = free & ((Qs[-1] - Qs[-2]) > 2 * tol)
    assert np.array_equal(pi.cpu().numpy()[sure], pin[sure])
    assert np.all(pi.cpu().numpy()[~free] == 255)
    assert np.abs(out.double().cpu().numpy() - Vn).max() <= tol
    # FP64 certifying sweep of the float values: residual and policy equal
    # the oracle's FP64 backup of the same values
    V2 = V0.clone()
    pi2 = torch.zeros_like(pi)
    r2 = cp.value_iteration(f, cp.F32, V2, pi2, opts=cp.default_opts(max_iter=1, tol=1e-30, fused=2, certify=1),
                            raise_on_noconv=False)
    Vc = V2.double().cpu().numpy()
    Vn2, pin2, resn2, Qn2 = oc.backup(gw, Vc, want_q=True)
    assert abs(r2["certified_residual"] - resn2) <= 1e-12
    Qs2 = np.sort(Qn2, axis=0)
    sure2 = free & ((Qs2[-1] - Qs2[-2]) > 1e-9)
    assert np.array_equal(pi2.cpu().numpy()[sure2], pin2[sure2])
    del V0, out, pi, V1, V2, pi2
    f.close()
    torch.cuda.empty_cache()


def test_march_value_iteration_equals_grid_barrier(cp):
    """Value iteration of a 3-D grid past 2^23 states runs the marching
    sweep from a replayed CUDA graph with the stopping rule on the device:
    the same sweeps, residual trace and values, bit for bit, as the
    grid-barrier solver (fused = 2), its FP64 certificate and policy
    included; a max_iter inside a graph chunk (odd: the result sits in the
    scratch buffer) stops with ENOCONV at exactly max_iter sweeps with the
    grid-barrier solver's values."""
    import torch
    gw = ci.gridworld((130, 256, 256), p=0.8, gamma=0.95, step_reward=-0.01,
                      goal_rewards=list(ci.uniform(3, 12, 8, 0.5, 1.0)), obstacle_rate=0.05, seed=3)
    assert gw.nstates >= 1 << 23
    f = cp.build_factors(gw, device=0)
    out = {}
    for fused in (1, 2, 1):
        V = torch.zeros(gw.nstates, dtype=torch.float32, device="cuda")
        pi = torch.zeros(gw.nstates, dtype=torch.uint8, device="cuda")
        tr = torch.zeros(5000, dtype=torch.float64, device="cuda")
        o = cp.default_opts(max_iter=5000, fused=fused)
        o.trace = tr.data_ptr()
        r = cp.value_iteration(f, cp.F32, V, pi, opts=o)
        assert r["solver"] == (cp.SOLVER_MARCH_GRAPH if fused == 1 else cp.SOLVER_GRID_BARRIER)
        res = (V.cpu().numpy(), pi.cpu().numpy(), r, tr[:r["iterations"]].cpu().numpy())
        if fused in out:   # the second march solve replays the recorded graph
            assert np.array_equal(res[0].view(np.uint32), out[fused][0].view(np.uint32))
        out[fused] = res
    (Va, pa, ra, ta), (Vb, pb, rb, tb) = out[1], out[2]
    assert ra["iterations"] == rb["iterations"] and ra["residual"] == rb["residual"]
    assert np.array_equal(Va.view(np.uint32), Vb.view(np.uint32))
    assert np.array_equal(ta, tb) and np.array_equal(pa, pb)
    assert ra["certified_residual"] == rb["certified_residual"] and ra["backups"] == rb["backups"]
    got = {}
    for fused in (1, 2):
        V = torch.zeros(gw.nstates, dtype=torch.float32, device="cuda")
        r = cp.value_iteration(f, cp.F32, V, None, opts=cp.default_opts(max_iter=21, fused=fused, certify=0),
                               raise_on_noconv=False)
        assert r["status"] == cp.ENOCONV and r["iterations"] == 21
        got[fused] = V.cpu().numpy()
    assert np.array_equal(got[1].view(np.uint32), got[2].view(np.uint32))
    f.close()
