"""The barrier-free FP32 GridWorld solver (sweep-tagged values, stopping
rule checked two sweeps late) against the grid-barrier solver and the
oracle.

Both solvers run the same Jacobi iterates with the same per-state
arithmetic and stop at the same sweep, so their results must be equal bit
for bit: values, policies, sweep counts, rounds, residuals and the
per-sweep residual trace. fused=1 picks the barrier-free solver where it is
eligible (1 to 3 dimensions, rows a multiple of 4 states, one thread per
column of 1, 2 or 4 segments of 4 states in one co-resident grid); fused=2
always takes the grid-barrier solver. The oracle checks the k-sweep
iterates directly.
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


# shapes: 1-D chain; 2-D with rows of 3, 16 and 40 segments (row neighbours
# inside and outside a warp); 3-D with a ragged last warp; the 64^3 bench size
SHAPES = [(400,), (12, 20), (37, 64), (24, 160), (5, 9, 12), (20, 36, 8), (64, 64, 64)]


def _world(shape, seed):
    if len(shape) == 1:
        return ci.gridworld(shape, p=0.8, gamma=0.95, step_reward=-0.04, goal_rewards=[1.0, -1.0],
                            obstacle_rate=0.05, seed=seed)
    if len(shape) == 2:
        return ci.gridworld(shape, p=0.8, gamma=0.97, step_reward=-0.04, goal_rewards=[1.0, -1.0],
                            obstacle_rate=0.05, seed=seed)
    return ci.gridworld(shape, p=0.8, gamma=0.99, step_reward=-0.01,
                        goal_rewards=list(ci.uniform(seed, 99, 8, 0.5, 1.0)), obstacle_rate=0.05, seed=seed)


def _vi(cp, f, gw, fused, **kw):
    import torch
    V = torch.zeros(gw.nstates, dtype=torch.float32, device="cuda")
    pi = torch.zeros(gw.nstates, dtype=torch.uint8, device="cuda")
    mi = kw.pop("max_iter", 5000)
    trace = torch.full((mi,), -1.0, dtype=torch.float64, device="cuda")
    r = cp.value_iteration(f, cp.F32, V, pi, opts=cp.default_opts(fused=fused, max_iter=mi,
                                                                     trace=trace.data_ptr(), **kw),
                           raise_on_noconv=False)
    return V.cpu().numpy(), pi.cpu().numpy(), trace.cpu().numpy(), r


@pytest.mark.parametrize("shape", SHAPES)
def test_vi_equals_grid_barrier_solver(cp, shape):
    gw = _world(shape, seed=len(shape) * 7 + shape[-1])
    f = cp.build_factors(gw, device=0)
    Va, pa, ta, ra = _vi(cp, f, gw, 1)
    Vb, pb, tb, rb = _vi(cp, f, gw, 2)
    assert ra["solver"] == cp.SOLVER_BARRIER_FREE and rb["solver"] == cp.SOLVER_GRID_BARRIER
    assert ra["status"] == cp.OK and rb["status"] == cp.OK
    assert ra["iterations"] == rb["iterations"]
    assert ra["residual"] == rb["residual"]
    assert ra["backups"] == rb["backups"]
    assert np.array_equal(Va.view(np.uint32), Vb.view(np.uint32))
    assert np.array_equal(pa, pb)
    k = ra["iterations"]
    assert np.array_equal(ta[:k], tb[:k])
    assert ra["certified_residual"] == rb["certified_residual"]
    f.close()


@pytest.mark.parametrize("k", [1, 2, 3, 4, 7, 30])
def test_k_sweeps_match_oracle(cp, oc, k):
    """max_iter = k with an unreachable tol: exactly k Jacobi sweeps from
    zero, equal to the grid-barrier solver bit for bit and to k oracle
    sweeps within the FP32 k-sweep bound."""
    gw = _world((20, 36, 8), seed=3)
    f = cp.build_factors(gw, device=0)
    Va, _, ta, ra = _vi(cp, f, gw, 1, max_iter=k, tol=1e-30, certify=0)
    Vb, _, tb, rb = _vi(cp, f, gw, 2, max_iter=k, tol=1e-30, certify=0)
    assert ra["status"] == cp.ENOCONV and ra["iterations"] == k
    assert ra["solver"] == cp.SOLVER_BARRIER_FREE and rb["solver"] == cp.SOLVER_GRID_BARRIER
    assert np.array_equal(Va.view(np.uint32), Vb.view(np.uint32))
    assert np.array_equal(ta, tb)
    Vo = np.zeros(gw.nstates)
    for _ in range(k):
        Vo, _, _, _ = oc.backup(gw, Vo)
    eps = 14 * U32 * (np.abs(gw.reward).max() + np.abs(Vo).max() + 1.0)
    bound = eps * (1 - gw.gamma ** k) / (1 - gw.gamma)
    assert np.abs(Va.astype(np.float64) - Vo).max() <= bound
    f.close()


@pytest.mark.parametrize("shape", [(400,), (3000,), (12, 20), (37, 64), (24, 160), (5, 9, 12), (20, 36, 8),
                                   (64, 64, 64)])
def test_pi_equals_grid_barrier_solver(cp, shape):
    import torch
    gw = _world(shape, seed=11 + shape[0])
    f = cp.build_factors(gw, device=0)
    out = {}
    for fused in (1, 2):
        V = torch.zeros(gw.nstates, dtype=torch.float32, device="cuda")
        pi = torch.zeros(gw.nstates, dtype=torch.uint8, device="cuda")
        r = cp.policy_iteration(f, cp.F32, V, pi, opts=cp.default_opts(fused=fused))
        out[fused] = (V.cpu().numpy(), pi.cpu().numpy(), r)
    (Va, pa, ra), (Vb, pb, rb) = out[1], out[2]
    assert ra["solver"] == cp.SOLVER_BARRIER_FREE and rb["solver"] == cp.SOLVER_GRID_BARRIER
    for key in ("status", "iterations", "rounds", "eval_sweeps", "residual", "backups", "certified_residual"):
        assert ra[key] == rb[key], (key, ra[key], rb[key])
    assert np.array_equal(Va.view(np.uint32), Vb.view(np.uint32))
    assert np.array_equal(pa, pb)
    f.close()


@pytest.mark.parametrize("partial", [0, 1, 2, 3, 4, 8])
def test_pi_partial_evaluation_same_in_both_solvers(cp, partial):
    """Modified policy iteration (evaluations capped at partial_eval sweeps
    until an improvement changes no action; 0 = every evaluation to
    eval_tol): both solvers take the same rounds and sweeps, bit for bit;
    the final policy is the same as with full evaluations wherever the
    values leave no near-tie, and the values agree within the evaluation
    bound 2 eval_tol / (1 - gamma) plus FP32 rounding."""
    import torch
    gw = _world((40, 36, 16), seed=21)
    f = cp.build_factors(gw, device=0)
    out = {}
    for fused in (1, 2):
        V = torch.zeros(gw.nstates, dtype=torch.float32, device="cuda")
        pi = torch.zeros(gw.nstates, dtype=torch.uint8, device="cuda")
        r = cp.policy_iteration(f, cp.F32, V, pi, opts=cp.default_opts(fused=fused, partial_eval=partial))
        out[fused] = (V.cpu().numpy(), pi.cpu().numpy(), r)
    (Va, pa, ra), (Vb, pb, rb) = out[1], out[2]
    for key in ("status", "iterations", "rounds", "eval_sweeps", "residual", "backups"):
        assert ra[key] == rb[key], (key, ra[key], rb[key])
    assert np.array_equal(Va.view(np.uint32), Vb.view(np.uint32)) and np.array_equal(pa, pb)
    V = torch.zeros(gw.nstates, dtype=torch.float32, device="cuda")
    pi = torch.zeros(gw.nstates, dtype=torch.uint8, device="cuda")
    rf = cp.policy_iteration(f, cp.F32, V, pi, opts=cp.default_opts(partial_eval=0))
    Vf, pf = V.cpu().numpy().astype(np.float64), pi.cpu().numpy()
    eps = 14 * U32 * (np.abs(gw.reward).max() + np.abs(Vf).max())
    bound = (2 * 1e-6 + eps) / (1 - gw.gamma)
    assert np.abs(Va - Vf).max() <= bound
    # the policies agree wherever the oracle's Q at the full-evaluation values
    # leaves a gap above twice gamma times that bound plus the keep margin
    from oracle import cpfactor as oc
    _, _, _, Q = oc.backup(gw, Vf, want_q=True)
    free = gw.cell.reshape(-1) == ci.FREE
    Qs = np.sort(Q[:, free], axis=0)
    sure = (Qs[-1] - Qs[-2]) > 2 * gw.gamma * bound + 2e-6 * (1 + np.abs(Qs[-1]))
    assert sure.sum() > 5000
    assert np.array_equal(pa[free][sure], pf[free][sure])
    if partial:
        assert ra["eval_sweeps"] < rf["eval_sweeps"]
    f.close()


def test_pi_round_and_eval_limits(cp):
    """Evaluation and round limits end the solve the same way in both
    solvers (ENOCONV, same partial results)."""
    import torch
    gw = _world((20, 36, 8), seed=5)
    f = cp.build_factors(gw, device=0)
    for kw in (dict(max_eval_iter=1), dict(max_eval_iter=2), dict(max_eval_iter=3),
               dict(max_rounds=1), dict(max_rounds=2, max_eval_iter=5), dict(max_eval_iter=40, partial_eval=6)):
        out = {}
        for fused in (1, 2):
            V = torch.zeros(gw.nstates, dtype=torch.float32, device="cuda")
            pi = torch.zeros(gw.nstates, dtype=torch.uint8, device="cuda")
            r = cp.policy_iteration(f, cp.F32, V, pi, opts=cp.default_opts(fused=fused, **kw),
                                    raise_on_noconv=False)
            out[fused] = (V.cpu().numpy(), pi.cpu().numpy(), r)
        (Va, pa, ra), (Vb, pb, rb) = out[1], out[2]
        assert ra["solver"] == cp.SOLVER_BARRIER_FREE and rb["solver"] == cp.SOLVER_GRID_BARRIER
        for key in ("status", "iterations", "rounds", "eval_sweeps", "residual", "backups"):
            assert ra[key] == rb[key], (kw, key, ra[key], rb[key])
        assert np.array_equal(Va.view(np.uint32), Vb.view(np.uint32)), kw
        assert np.array_equal(pa, pb), kw
    f.close()


def test_warm_start_and_repeated_calls(cp):
    """Many solves on one factors object (the tag base moves on each time)
    and warm starts give the same results as the grid-barrier solver."""
    import torch
    gw = _world((37, 64), seed=8)
    f = cp.build_factors(gw, device=0)
    V0 = torch.as_tensor(ci.random_values(gw.shape, seed=4, lo=-1, hi=1).reshape(-1)).float().cuda()
    ref = None
    for rep in range(6):
        outs = []
        for fused in (1, 2):
            V = V0.clone()
            pi = torch.zeros(gw.nstates, dtype=torch.uint8, device="cuda")
            if rep % 2:
                r = cp.policy_iteration(f, cp.F32, V, pi, opts=cp.default_opts(fused=fused))
            else:
                r = cp.value_iteration(f, cp.F32, V, pi, opts=cp.default_opts(fused=fused))
            outs.append((V.cpu().numpy().view(np.uint32), pi.cpu().numpy(), r["iterations"]))
        assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
        assert outs[0][2] == outs[1][2]
    f.close()


def test_timeout_then_recovery(cp):
    """A stalled block makes the barrier-free solver's bounded waits run out
    (CPMDP_ETIMEOUT, no hang); the rings are cleared and the next solve on
    the same factors object is exact again."""
    import torch
    gw = _world((20, 36, 8), seed=9)
    f = cp.build_factors(gw, device=0)
    for pim in (False, True):
        V = torch.zeros(gw.nstates, dtype=torch.float32, device="cuda")
        pi = torch.zeros(gw.nstates, dtype=torch.uint8, device="cuda")
        with pytest.raises(cp.CpmdpError) as ei:
            if pim:
                cp.policy_iteration(f, cp.F32, V, pi, opts=cp.default_opts(timeout_s=0.2, inject_stall=1))
            else:
                cp.value_iteration(f, cp.F32, V, pi, opts=cp.default_opts(timeout_s=0.2, inject_stall=1))
        assert ei.value.status == cp.ETIMEOUT
    Va, pa, _, ra = _vi(cp, f, gw, 1)
    Vb, pb, _, rb = _vi(cp, f, gw, 2)
    assert ra["iterations"] == rb["iterations"]
    assert np.array_equal(Va.view(np.uint32), Vb.view(np.uint32))
    f.close()


def test_ineligible_shapes_use_grid_barrier(cp):
    """Rows that are not a multiple of 4 states, and 4-D grids, take the
    grid-barrier solver; F64 never runs barrier-free."""
    import torch
    for shape, prec in (((10, 10), cp.F32), ((6, 5, 4, 4), cp.F32), ((16, 16), cp.F64)):
        gw = ci.gridworld(shape, p=0.8, gamma=0.9, step_reward=-0.04, goal_rewards=[1.0, -1.0], seed=1)
        f = cp.build_factors(gw, device=0)
        dt = torch.float64 if prec == cp.F64 else torch.float32
        V = torch.zeros(gw.nstates, dtype=dt, device="cuda")
        r = cp.value_iteration(f, prec, V, None)
        assert r["solver"] == cp.SOLVER_GRID_BARRIER, shape
        f.close()


# Grids past what one 4-state segment per thread covers (152 SMs x 14 warps
# x 32 lanes x 4 = 272,384 states) run with columns of 2 or 4 segments
# stacked along dimension 0 in one thread:
#   (71, 64, 64)  290,816 states: columns of 2, the last group one slice short
#   (73, 72, 72)  378,432 states: columns of 4, the last group three slices short
#   (600, 600)    360,000 states: 2-D, columns of 4 rows
COLUMN_SHAPES = [(71, 64, 64), (73, 72, 72), (600, 600)]


@pytest.mark.parametrize("shape", COLUMN_SHAPES)
def test_columns_equal_grid_barrier_solver(cp, shape):
    import torch
    gw = _world(shape, seed=21 + shape[0])
    f = cp.build_factors(gw, device=0)
    Va, pa, ta, ra = _vi(cp, f, gw, 1)
    Vb, pb, tb, rb = _vi(cp, f, gw, 2)
    assert ra["solver"] == cp.SOLVER_BARRIER_FREE and rb["solver"] == cp.SOLVER_GRID_BARRIER
    assert ra["iterations"] == rb["iterations"] and ra["residual"] == rb["residual"]
    assert np.array_equal(Va.view(np.uint32), Vb.view(np.uint32))
    assert np.array_equal(pa, pb)
    k = ra["iterations"]
    assert np.array_equal(ta[:k], tb[:k])
    # (the large 2-D grid needs hundreds of improvement rounds: stop both after 5)
    kw = dict(max_rounds=5) if len(shape) == 2 else {}
    out = {}
    for fused in (1, 2):
        V = torch.zeros(gw.nstates, dtype=torch.float32, device="cuda")
        pi = torch.zeros(gw.nstates, dtype=torch.uint8, device="cuda")
        r = cp.policy_iteration(f, cp.F32, V, pi, opts=cp.default_opts(fused=fused, **kw), raise_on_noconv=False)
        out[fused] = (V.cpu().numpy(), pi.cpu().numpy(), r)
    (Va, pa, ra), (Vb, pb, rb) = out[1], out[2]
    assert ra["solver"] == cp.SOLVER_BARRIER_FREE
    for key in ("status", "iterations", "rounds", "eval_sweeps", "residual", "backups"):
        assert ra[key] == rb[key], (key, ra[key], rb[key])
    assert np.array_equal(Va.view(np.uint32), Vb.view(np.uint32))
    assert np.array_equal(pa, pb)
    f.close()


def test_columns_k_sweeps_and_limits(cp, oc):
    """Columns of 4 (73 x 72 x 72): k Jacobi sweeps equal the grid-barrier
    solver's and the oracle's; a PI evaluation limit ends both the same way."""
    import torch
    gw = _world((73, 72, 72), seed=4)
    f = cp.build_factors(gw, device=0)
    for k in (1, 2, 3, 5):
        Va, _, ta, ra = _vi(cp, f, gw, 1, max_iter=k, tol=1e-30, certify=0)
        Vb, _, tb, rb = _vi(cp, f, gw, 2, max_iter=k, tol=1e-30, certify=0)
        assert ra["solver"] == cp.SOLVER_BARRIER_FREE and ra["iterations"] == k
        assert np.array_equal(Va.view(np.uint32), Vb.view(np.uint32)) and np.array_equal(ta, tb)
    Vo = np.zeros(gw.nstates)
    for _ in range(5):
        Vo, _, _, _ = oc.backup(gw, Vo)
    eps = 14 * U32 * (np.abs(gw.reward).max() + np.abs(Vo).max() + 1.0)
    assert np.abs(Va.astype(np.float64) - Vo).max() <= eps * 5
    out = {}
    for fused in (1, 2):
        V = torch.zeros(gw.nstates, dtype=torch.float32, device="cuda")
        pi = torch.zeros(gw.nstates, dtype=torch.uint8, device="cuda")
        r = cp.policy_iteration(f, cp.F32, V, pi, opts=cp.default_opts(fused=fused, max_eval_iter=4),
                                raise_on_noconv=False)
        out[fused] = (V.cpu().numpy(), pi.cpu().numpy(), r)
    (Va, pa, ra), (Vb, pb, rb) = out[1], out[2]
    for key in ("status", "iterations", "rounds", "eval_sweeps", "residual"):
        assert ra[key] == rb[key], (key, ra[key], rb[key])
    assert np.array_equal(Va.view(np.uint32), Vb.view(np.uint32)) and np.array_equal(pa, pb)
    f.close()
