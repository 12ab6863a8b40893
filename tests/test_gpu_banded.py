"""GPU parity of the banded (GridWorld) path against the CPU FP64 oracle.

Every GPU call goes through the C ABI (libcpmdp.so via the ctypes binding);
the oracle never sees GPU output as an input except where a test checks a
property of that output (certified residual, policy extraction from it).

Tolerances (derived from the arithmetic; u = 2^-24 for FP32):
* one FP32 sweep: each Q is R + gamma (w_move N + w_perp (sum of 2(D-1)
  pair sums) + w_stay V) with at most 2D + 4 rounded operations, each off
  by at most u times the magnitudes involved, plus the final rounding:
  |V32' - V64'| <= (2D + 8) u (max|R| + max|V|).
* one FP64 sweep: same with u = 2^-53 (we use 1e-13 (max|R| + max|V|)).
* k FP32 sweeps from the same start: errors add up, contracted by gamma
  each sweep: <= eps (1 - gamma^k) / (1 - gamma) with eps the one-sweep bound.
* FP32 and FP64 value iteration to the same tol: each result is within
  gamma tol / (1 - gamma) of V*, so they differ by at most
  (2 gamma tol + eps) / (1 - gamma); the sweep at which an FP32 residual
  crosses tol is not compared (its rounding noise is of the size of tol).
* policies are compared where the oracle's best/second-best Q gap exceeds
  twice the value tolerance (FP32) or 1e-6 (FP64), i.e. where rounding
  cannot flip the argmax.
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


def _dev(x, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def _gap_mask(Q, free):
    Qs = np.sort(Q, axis=0)
    return free, (Qs[-1] - Qs[-2]) if Q.shape[0] > 1 else np.full(Q.shape[1], np.inf)


def _one_sweep(cp, oc, gw, prec, vseed=0, scale=1.0):
    import torch
    dt = torch.float64 if prec == cp.F64 else torch.float32
    V = ci.random_values(gw.shape, seed=vseed, lo=-scale, hi=scale).reshape(-1)
    Vd = _dev(V, dt)
    V = Vd.double().cpu().numpy()                  # the exact values the GPU sees
    f = cp.build_factors(gw, device=0)
    out = torch.empty_like(Vd)
    pi = torch.empty(gw.nstates, dtype=torch.uint8, device="cuda")
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    cp.bellman_backup(f, prec, Vd, out, pi, res)
    torch.cuda.synchronize()
    Vo, pio, reso, Qo = oc.backup(gw, V, want_q=True)
    D = len(gw.shape)
    mag = np.abs(gw.reward).max() + np.abs(V).max()
    tol = (2 * D + 8) * U32 * mag if prec == cp.F32 else 1e-13 * mag
    g = out.double().cpu().numpy()
    err = np.abs(g - Vo).max()
    assert err <= tol, (err, tol)
    free = gw.cell.reshape(-1) == ci.FREE
    _, gap = _gap_mask(Qo, free)
    sure = free & (gap > (2 * tol if prec == cp.F32 else 1e-6))
    gp = pi.cpu().numpy()
    assert np.array_equal(gp[sure], pio[sure])
    assert np.all(gp[~free] == 255)
    live = gw.cell.reshape(-1) != ci.OBSTACLE
    want_res = np.abs(Vo - V)[live].max() if live.any() else 0.0
    assert abs(res.item() - want_res) <= 2 * tol + 1e-300
    f.close()
    return err, tol


SHAPES = [
    ((10, 10), 0.8, 0.0, 2), ((64, 64, 64), 0.8, 0.05, 8), ((13, 7, 5), 0.7, 0.1, 3),
    ((9,), 0.9, 0.2, 1), ((1,), 0.8, 0.0, 0), ((5, 1), 0.6, 0.0, 1), ((3, 4, 2, 6), 0.75, 0.1, 2),
    ((2, 3, 2, 2, 2, 3, 2), 0.8, 0.1, 2), ((2, 2, 2, 2, 2, 2, 2, 2, 4), 0.8, 0.05, 3),
    ((33, 65), 0.8, 0.15, 4), ((40, 30, 64), 0.85, 0.2, 6), ((4, 6), 1.0, 0.0, 1),
]


@pytest.mark.parametrize("shape,p,orate,ngoals", SHAPES)
@pytest.mark.parametrize("prec", [0, 1])
def test_one_backup_matches_oracle(cp, oc, shape, p, orate, ngoals, prec):
    gw = ci.gridworld(shape, p=p, gamma=0.95, step_reward=-0.04,
                      goal_rewards=list(np.linspace(-1, 1, ngoals)), obstacle_rate=orate, seed=11)
    for vseed in range(2):
        _one_sweep(cp, oc, gw, prec, vseed=vseed, scale=3.0)


def test_all_obstacles_and_single_state(cp, oc):
    import torch
    gw = ci.GridWorld(shape=(4, 4), p=0.8, gamma=0.9, cell=np.ones((4, 4), np.uint8),
                      reward=np.zeros((4, 4)))
    f = cp.build_factors(gw, device=0)
    V = torch.full((16,), 3.0, dtype=torch.float64, device="cuda")
    pi = torch.zeros(16, dtype=torch.uint8, device="cuda")
    r = cp.value_iteration(f, cp.F64, V, pi)
    assert r["iterations"] == 1 and np.all(V.cpu().numpy() == 0) and np.all(pi.cpu().numpy() == 255)
    # one free state, no move possible: V = R / (1 - gamma)
    gw = ci.GridWorld(shape=(1,), p=0.8, gamma=0.9, cell=np.zeros(1, np.uint8),
                      reward=np.array([0.5]))
    f = cp.build_factors(gw, device=0)
    V = torch.zeros(1, dtype=torch.float64, device="cuda")
    pi = torch.zeros(1, dtype=torch.uint8, device="cuda")
    cp.value_iteration(f, cp.F64, V, pi, opts=cp.default_opts(tol=1e-13, max_iter=100000))
    assert abs(V.item() - 5.0) < 1e-11


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_vi_pi_small_2d_fp64(cp, oc, seed):
    """10x10, A=4, p=0.8, gamma=0.9: FP64 VI and PI to 1e-6 against the
    tabular oracle (same stopping rule): |dV| <= 1e-6 relative, same sweep
    count, policies equal wherever the oracle's gap exceeds 1e-6."""
    import torch
    from oracle import tabular as T
    gw = ci.config_small_2d(seed)
    P = T.transition_tabular(gw.shape, gw.cell, gw.p)
    Vo, pio, ko, reso = T.value_iteration(P, gw.reward, gw.gamma, gw.cell, tol=1e-6)
    _, _, Qo = T.backup(P, gw.reward, gw.gamma, gw.cell, Vo)
    f = cp.build_factors(gw, device=0)
    V = torch.zeros(gw.nstates, dtype=torch.float64, device="cuda")
    pi = torch.zeros(gw.nstates, dtype=torch.uint8, device="cuda")
    r = cp.value_iteration(f, cp.F64, V, pi)
    assert r["iterations"] == ko
    g = V.cpu().numpy()
    assert np.abs(g - Vo).max() <= 1e-6 * max(1.0, np.abs(Vo).max())
    assert np.abs(g - Vo).max() <= 1e-12
    free = gw.cell.reshape(-1) == ci.FREE
    _, gap = _gap_mask(Qo, free)
    sure = free & (gap > 1e-6)
    assert np.array_equal(pi.cpu().numpy()[sure], pio[sure])
    # certified residual: the oracle's own FP64 backup of the returned V
    Vn, _, _ = T.backup(P, gw.reward, gw.gamma, gw.cell, g)
    assert abs(r["certified_residual"] - np.abs(Vn - g).max()) <= 1e-14
    # policy iteration
    Vp, pip, _ = T.policy_iteration(P, gw.reward, gw.gamma, gw.cell)
    _, _, Qp = T.backup(P, gw.reward, gw.gamma, gw.cell, Vp)
    V2 = torch.zeros(gw.nstates, dtype=torch.float64, device="cuda")
    pi2 = torch.zeros(gw.nstates, dtype=torch.uint8, device="cuda")
    r2 = cp.policy_iteration(f, cp.F64, V2, pi2)
    assert r2["rounds"] >= 1
    _, gap = _gap_mask(Qp, free)
    sure = free & (gap > 1e-6)
    assert np.array_equal(pi2.cpu().numpy()[sure], pip[sure])
    # evaluation stops at 1e-10, so |V - V_pi| <= 1e-10 gamma / (1 - gamma)
    assert np.abs(V2.cpu().numpy() - Vp).max() <= 1e-8


def test_k_sweeps_persistent_matches_oracle(cp, oc):
    """The device-resident loop (grid barrier, residual slots, buffer swaps)
    equals k separate oracle sweeps, for odd and even k."""
    import torch
    gw = ci.config_3d(side=40, seed=3)
    f = cp.build_factors(gw, device=0)
    for k in (1, 2, 7, 30):
        V = torch.zeros(gw.nstates, dtype=torch.float64, device="cuda")
        trace = torch.zeros(k, dtype=torch.float64, device="cuda")
        r = cp.value_iteration(f, cp.F64, V, None, opts=cp.default_opts(tol=1e-30, max_iter=k,
                                                                          trace=trace.data_ptr()),
                               raise_on_noconv=False)
        assert r["status"] == cp.ENOCONV and r["iterations"] == k
        Vo = np.zeros(gw.nstates)
        ress = []
        for _ in range(k):
            Vn, _, res, _ = oc.backup(gw, Vo)
            ress.append(res)
            Vo = Vn
        assert np.abs(V.cpu().numpy() - Vo).max() <= 1e-12
        np.testing.assert_allclose(trace.cpu().numpy(), ress, rtol=1e-9, atol=1e-14)


@pytest.mark.parametrize("prec", [0, 1])
def test_vi_3d_64_matches_oracle(cp, oc, prec):
    """64^3, A=6, p=0.8, 5% obstacles, 8 goals, gamma=0.99: VI to 1e-6.
    FP64: same sweeps, |dV| <= 1e-12. FP32: within the k-sweep rounding
    bound; the FP64 certified residual equals the oracle's recomputation;
    the FP64 policy equals the oracle's argmax of the same V."""
    import torch
    gw = ci.config_3d(side=64, seed=0)
    Vo, pio, ko, reso = oc.value_iteration(gw, tol=1e-6, max_iter=5000)
    f = cp.build_factors(gw, device=0)
    dt = torch.float64 if prec == cp.F64 else torch.float32
    V = torch.zeros(gw.nstates, dtype=dt, device="cuda")
    pi = torch.zeros(gw.nstates, dtype=torch.uint8, device="cuda")
    r = cp.value_iteration(f, prec, V, pi, opts=cp.default_opts(max_iter=5000))
    g = V.double().cpu().numpy()
    free = gw.cell.reshape(-1) == ci.FREE
    if prec == cp.F64:
        assert r["iterations"] == ko
        assert np.abs(g - Vo).max() <= 1e-12
    else:
        # both runs stop with a residual below tol: each is within
        # gamma tol / (1 - gamma) of V*; FP32 rounding adds eps / (1 - gamma)
        eps = 14 * U32 * (np.abs(gw.reward).max() + np.abs(Vo).max())
        bound = (2 * gw.gamma * 1e-6 + eps) / (1 - gw.gamma)
        err = np.abs(g - Vo).max()
        assert err <= bound, (err, bound)
    # certified residual and policy from the FP64 sweep of the returned V
    Vn, pin, resn, Qn = oc.backup(gw, g, want_q=True)
    assert abs(r["certified_residual"] - resn) <= 1e-12
    _, gap = _gap_mask(Qn, free)
    sure = free & (gap > 1e-9)
    assert np.array_equal(pi.cpu().numpy()[sure], pin[sure])
    assert np.all(pi.cpu().numpy()[~free] == 255)
    # true error bound of the returned values against V* (oracle to 1e-12)
    Vs, _, _, _ = oc.value_iteration(gw, tol=1e-12, max_iter=20000, V0=Vo)
    assert np.abs(g - Vs).max() <= r["error_bound"] * (1 + 1e-6) + 1e-12


@pytest.mark.parametrize("prec", [0, 1])
def test_pi_3d_matches_optimal_policy(cp, oc, prec):
    """Policy iteration on 64^3 returns the optimal policy wherever the
    optimal Q gap exceeds what its value error could flip."""
    import torch
    gw = ci.config_3d(side=64, seed=1)
    Vs, pis, _, _ = oc.value_iteration(gw, tol=1e-12, max_iter=20000)
    _, _, _, Qs = oc.backup(gw, Vs, want_q=True)
    f = cp.build_factors(gw, device=0)
    dt = torch.float64 if prec == cp.F64 else torch.float32
    V = torch.zeros(gw.nstates, dtype=dt, device="cuda")
    pi = torch.zeros(gw.nstates, dtype=torch.uint8, device="cuda")
    r = cp.policy_iteration(f, prec, V, pi, opts=cp.default_opts(max_iter=5000))
    g = V.double().cpu().numpy()
    err = np.abs(g - Vs).max()
    bound = 1e-8 if prec == cp.F64 else (1e-6 + 14 * U32 * 2) / (1 - gw.gamma)
    assert err <= bound, (err, bound)
    free = gw.cell.reshape(-1) == ci.FREE
    _, gap = _gap_mask(Qs, free)
    sure = free & (gap > 2 * gw.gamma * bound + 1e-9)
    assert sure.sum() > 0.5 * free.sum()
    assert np.array_equal(pi.cpu().numpy()[sure], pis[sure])
    assert r["rounds"] >= 2


def test_plain_baseline_matches_fused(cp):
    import torch
    gw = ci.config_3d(side=32, seed=5)
    f = cp.build_factors(gw, device=0)
    out = {}
    for fused in (1, 0):
        V = torch.zeros(gw.nstates, dtype=torch.float64, device="cuda")
        pi = torch.zeros(gw.nstates, dtype=torch.uint8, device="cuda")
        r = cp.value_iteration(f, cp.F64, V, pi, opts=cp.default_opts(fused=fused, max_iter=5000))
        out[fused] = (V.cpu().numpy(), pi.cpu().numpy(), r)
    assert out[0][2]["iterations"] == out[1][2]["iterations"]
    assert np.abs(out[0][0] - out[1][0]).max() <= 1e-12
    assert np.mean(out[0][1] == out[1][1]) > 0.999


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_plain_device_stop_equals_host_stop(cp, prec):
    """fused = 3 runs the plain kernels of fused = 0 with the stopping rule
    taken on the device and a recorded 32-sweep graph: same sweep count,
    same values bit for bit, same residual and policy, called twice (graph
    replay); and max_iter inside a chunk (45: odd, the result sits in the
    scratch buffer; 44: even) stops with ENOCONV at exactly max_iter sweeps
    with the values of the host-checked run."""
    import torch
    dt = torch.float32 if prec == "f32" else torch.float64
    P = cp.F32 if prec == "f32" else cp.F64
    for side, seed in ((32, 5), (24, 6)):
        gw = ci.config_3d(side=side, seed=seed)
        f = cp.build_factors(gw, device=0)
        out = {}
        for fused in (0, 3, 3):
            V = torch.zeros(gw.nstates, dtype=dt, device="cuda")
            pi = torch.zeros(gw.nstates, dtype=torch.uint8, device="cuda")
            r = cp.value_iteration(f, P, V, pi, opts=cp.default_opts(fused=fused, max_iter=5000, certify=0))
            assert r["solver"] == cp.SOLVER_PLAIN
            if fused in out:
                assert r["iterations"] == out[fused][2]["iterations"]
            out[fused] = (V.cpu().numpy(), pi.cpu().numpy(), r)
        (V0, p0, r0), (V3, p3, r3) = out[0], out[3]
        assert r0["iterations"] == r3["iterations"] and r0["residual"] == r3["residual"]
        assert np.array_equal(V0, V3) and np.array_equal(p0, p3)
        for mi in (45, 44):
            got = {}
            for fused in (0, 3):
                V = torch.zeros(gw.nstates, dtype=dt, device="cuda")
                r = cp.value_iteration(f, P, V, None, opts=cp.default_opts(fused=fused, max_iter=mi, certify=0),
                                       raise_on_noconv=False)
                assert r["status"] == cp.ENOCONV and r["iterations"] == mi
                got[fused] = V.cpu().numpy()
            assert np.array_equal(got[0], got[3])
        f.close()


def test_wait_timeout_returns_status(cp):
    """A block that never arrives at the grid barrier (inject_stall) makes the
    other blocks' bounded waits run out: the call returns CPMDP_ETIMEOUT
    after about timeout_s (no hang, no fault) and the context stays usable."""
    import time
    import torch
    gw = ci.config_3d(side=64, seed=0)
    f = cp.build_factors(gw, device=0)
    V = torch.zeros(gw.nstates, dtype=torch.float32, device="cuda")
    for prec, dt in ((cp.F32, torch.float32), (cp.F64, torch.float64)):
        V = torch.zeros(gw.nstates, dtype=dt, device="cuda")
        t0 = time.perf_counter()
        with pytest.raises(cp.CpmdpError) as ei:
            cp.value_iteration(f, prec, V, None, opts=cp.default_opts(timeout_s=0.2, inject_stall=1))
        el = time.perf_counter() - t0
        assert ei.value.status == cp.ETIMEOUT
        assert 0.15 < el < 10.0
    V = torch.zeros(gw.nstates, dtype=torch.float32, device="cuda")
    V.zero_()
    r = cp.value_iteration(f, cp.F32, V, None)
    assert r["status"] == cp.OK
    torch.cuda.synchronize()


def test_large_512_sampled(cp, oc):
    """512^3 (134M states, FP32): one backup through the C ABI, checked on
    4096 sampled states against the oracle's per-state FP64 Q."""
    import torch
    gw = ci.gridworld((512, 512, 512), p=0.8, gamma=0.99, step_reward=-0.01,
                      goal_rewards=list(ci.uniform(0, 12, 8, 0.5, 1.0)), obstacle_rate=0.05, seed=2)
    f = cp.build_factors(gw, device=0)
    V = _dev(ci.random_values(gw.shape, seed=4).reshape(-1).astype(np.float32), torch.float32)
    out = torch.empty_like(V)
    pi = torch.empty(gw.nstates, dtype=torch.uint8, device="cuda")
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    cp.bellman_backup(f, cp.F32, V, out, pi, res)
    torch.cuda.synchronize()
    states = ci.integers(0, 77, 4096, 0, gw.nstates - 1)
    states = np.concatenate([states, [0, gw.nstates - 1, 511, 512 * 512 - 1]])
    Vh = V.double().cpu().numpy()
    Q = oc.q_states(gw, Vh, states)
    cell = gw.cell.reshape(-1)[states]
    R = gw.reward.reshape(-1)[states]
    want = np.where(cell == ci.FREE, Q.max(axis=1), np.where(cell == ci.TERMINAL, R, 0.0))
    got = out[torch.as_tensor(states, device="cuda")].double().cpu().numpy()
    tol = 14 * U32 * (1.0 + 1.0)
    assert np.abs(got - want).max() <= tol
    free = cell == ci.FREE
    Qs = np.sort(Q, axis=1)
    sure = free & ((Qs[:, -1] - Qs[:, -2]) > 2 * tol)
    gp = pi[torch.as_tensor(states, device="cuda")].cpu().numpy()
    assert np.array_equal(gp[sure], Q.argmax(axis=1)[sure])
    del V, out, pi
    f.close()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("shape", [(7,), (5, 6), (4, 5, 3), (3, 2, 3, 2)])
def test_device_factors_components_match_host(cp, shape):
    """Factors on a device keep no host codes (the codes are built on the GPU);
    their Definition-3 components, derived per state on the host, equal those
    of host-only factors built by the other routine, for every state and
    action (walls, obstacles and terminals included)."""
    gw = ci.gridworld(shape, p=0.7, gamma=0.9, step_reward=-0.04, goal_rewards=[1.0, -1.0],
                      obstacle_rate=0.2, seed=5)
    fd = cp.build_factors(gw, device=0)
    fh = cp.build_factors(gw, device=-1)
    for s in range(gw.nstates):
        for a in range(2 * len(shape)):
            assert cp.components(fd, s, a) == cp.components(fh, s, a)
    fd.close()
    fh.close()


def test_device_build_checks_inputs_on_the_device(cp):
    """A device GridWorld build checks every reward (finite) and cell code
    (0, 1 or 2) in its conversion and code kernels instead of on the host:
    the same EINVAL and message as a host-only build, and the device stays
    usable (the next build and solve succeed)."""
    import torch
    base = ci.gridworld((6, 7, 9), p=0.8, gamma=0.95, step_reward=-0.04, goal_rewards=[1.0], obstacle_rate=0.1,
                        seed=5)
    r = np.asarray(base.reward, dtype=np.float64).reshape(-1).copy()
    r[123] = np.nan
    pr = cp.make_problem(shape=base.shape, nactions=6, kind=cp.GRIDWORLD, reward=r, gamma=0.95, p_success=0.8,
                         cell=np.asarray(base.cell, dtype=np.uint8).reshape(-1))
    with pytest.raises(cp.CpmdpError) as ei:
        cp.build_factors(pr, device=0)
    assert ei.value.status == cp.EINVAL and "reward[123] is not finite" in cp.last_error()
    c = np.asarray(base.cell, dtype=np.uint8).reshape(-1).copy()
    c[200] = 7
    pr = cp.make_problem(shape=base.shape, nactions=6, kind=cp.GRIDWORLD,
                         reward=np.asarray(base.reward, dtype=np.float64).reshape(-1), gamma=0.95, p_success=0.8, cell=c)
    with pytest.raises(cp.CpmdpError) as ei:
        cp.build_factors(pr, device=0)
    assert ei.value.status == cp.EINVAL and "cell[200] = 7" in cp.last_error()
    # the device is fine: a valid build solves, and its host query reads the cells back from the device
    f = cp.build_factors(base, device=0)
    V = torch.zeros(base.nstates, dtype=torch.float32, device="cuda")
    res = cp.value_iteration(f, cp.F32, V, None, opts=cp.default_opts(max_iter=5000))
    assert res["status"] == cp.OK
    free = int(np.flatnonzero(np.asarray(base.cell).reshape(-1) == 0)[0])
    comps = cp.components(f, free, 0)
    assert comps and abs(sum(pr_ for _, pr_ in comps) - 1.0) < 1e-12
    f.close()


@pytest.mark.parametrize("shape,prec", [((10, 10), 1), ((10, 10), 0), ((37,), 1), ((5, 6, 7), 1), ((3, 9, 5), 0),
                                         ((21, 23), 1), ((2, 2), 1)])
def test_single_block_solver_equals_grid_barrier(cp, shape, prec):
    """Grids one block covers (at most 256 segments) run value and policy
    iteration in a single block with the values in shared memory (fused=1);
    the grid-barrier kernels (fused=2) run the same per-state arithmetic and
    stopping rules through global memory: values, policies, sweep, round and
    evaluation counts and the last residual equal, bit for bit (FP64 and
    FP32, rows of odd and even length, 1-D to 3-D)."""
    import torch
    gw = ci.gridworld(shape, p=0.8, gamma=0.93, step_reward=-0.04,
                      goal_rewards=[1.0, -1.0][:min(2, int(np.prod(shape)) - 1)], obstacle_rate=0.1, seed=41)
    f = cp.build_factors(gw, device=0)
    dt = torch.float64 if prec == 1 else torch.float32
    pr = cp.F64 if prec == 1 else cp.F32
    out = {}
    for fused in (1, 2):
        V = torch.zeros(gw.nstates, dtype=dt, device="cuda")
        pi = torch.zeros(gw.nstates, dtype=torch.uint8, device="cuda")
        r = cp.value_iteration(f, pr, V, pi, opts=cp.default_opts(max_iter=5000, fused=fused))
        V2 = torch.zeros(gw.nstates, dtype=dt, device="cuda")
        pi2 = torch.zeros(gw.nstates, dtype=torch.uint8, device="cuda")
        r2 = cp.policy_iteration(f, pr, V2, pi2, opts=cp.default_opts(max_iter=5000, fused=fused))
        out[fused] = (V.cpu().numpy(), pi.cpu().numpy(), r, V2.cpu().numpy(), pi2.cpu().numpy(), r2)
    a, b = out[1], out[2]
    assert np.array_equal(a[0].view(np.uint8), b[0].view(np.uint8)) and np.array_equal(a[1], b[1])
    assert a[2]["iterations"] == b[2]["iterations"] and a[2]["residual"] == b[2]["residual"]
    assert a[2]["certified_residual"] == b[2]["certified_residual"]
    assert np.array_equal(a[3].view(np.uint8), b[3].view(np.uint8)) and np.array_equal(a[4], b[4])
    for k in ("iterations", "rounds", "eval_sweeps", "residual"):
        assert a[5][k] == b[5][k], (k, a[5][k], b[5][k])
    f.close()
