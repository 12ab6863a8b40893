"""Batched value iteration: one persistent launch over many uneven GridWorlds.

Each instance is checked against the FP64 C oracle run to the same stopping
rule and against the single-instance fused solver (same arithmetic: same
sweep count, values within 1e-6). Against the oracle only values are
compared: both runs stop with a residual below tol, so each is within
gamma tol / (1 - gamma) of V*, and FP32 rounding adds at most
eps / (1 - gamma) with eps = 14 u (max|R| + max|V|), u = 2^-24. Near tol
the FP32 residual carries rounding noise of the same size, so the sweep at
which it crosses tol is not compared.
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


def _instances():
    inst = ci.batch_gridworlds(count=192, seed=7)
    # edge cases: a 1-D chain, a single state, a ragged thin grid, an all-obstacle grid
    inst.append(ci.gridworld((37,), p=0.9, gamma=0.95, step_reward=-0.04, goal_rewards=[1.0], seed=1))
    inst.append(ci.GridWorld(shape=(1,), p=0.8, gamma=0.9, cell=np.zeros(1, np.uint8), reward=np.array([0.3])))
    inst.append(ci.gridworld((3, 129), p=0.7, gamma=0.97, step_reward=-0.04, goal_rewards=[1.0, -1.0],
                             obstacle_rate=0.1, seed=2))
    inst.append(ci.GridWorld(shape=(4, 4), p=0.8, gamma=0.9, cell=np.ones((4, 4), np.uint8),
                             reward=np.zeros((4, 4))))
    return inst


def test_batch_matches_oracle_and_single(cp, oc_lib=None):
    import torch
    from oracle import cpfactor as oc
    inst = _instances()
    B = cp.batch_build(inst, device=0)
    assert B.count == len(inst)
    V = torch.zeros(int(B.total_states), dtype=torch.float32, device="cuda")
    r, iters, res = cp.batch_value_iteration(B, V, opts=cp.default_opts(max_iter=5000))
    assert r["status"] == cp.OK and np.all(res < 1e-6)
    Vh = V.double().cpu().numpy()
    picks = list(range(0, 192, 8)) + list(range(192, len(inst)))
    for i in picks:
        gw = inst[i]
        lo, n = int(B.offsets[i]), gw.nstates
        got = Vh[lo:lo + n]
        Vo, _, ko, _ = oc.value_iteration(gw, tol=1e-6, max_iter=5000)
        eps = 14 * U32 * (np.abs(gw.reward).max() + np.abs(Vo).max())
        bound = (2 * gw.gamma * 1e-6 + eps) / (1 - gw.gamma)
        assert np.abs(got - Vo).max() <= bound, (i, np.abs(got - Vo).max(), bound, iters[i], ko)
    # the single-instance fused solver on a few instances
    for i in picks[:6] + [len(inst) - 2]:
        gw = inst[i]
        f = cp.build_factors(gw, device=0)
        Vs = torch.zeros(gw.nstates, dtype=torch.float32, device="cuda")
        rs = cp.value_iteration(f, cp.F32, Vs, None, opts=cp.default_opts(max_iter=5000, certify=0))
        lo = int(B.offsets[i])
        assert rs["iterations"] == int(iters[i])
        assert np.abs(Vs.double().cpu().numpy() - Vh[lo:lo + gw.nstates]).max() <= 1e-6
        f.close()
    # a second solve replays the recorded graph and reproduces the result
    V2 = V.clone().zero_()
    V.zero_()
    r2, it2, _ = cp.batch_value_iteration(B, V, opts=cp.default_opts(max_iter=5000))
    assert np.array_equal(it2, iters) and np.array_equal(V.double().cpu().numpy(), Vh)
    assert r2["rounds"] in (0, 1)
    B.close()


def test_batch_max_iter_and_warm_start(cp):
    import torch
    inst = ci.batch_gridworlds(count=40, seed=3)
    B = cp.batch_build(inst, device=0)
    V = torch.zeros(int(B.total_states), dtype=torch.float32, device="cuda")
    r, iters, _ = cp.batch_value_iteration(B, V, opts=cp.default_opts(max_iter=7), raise_on_noconv=False)
    assert r["status"] == cp.ENOCONV and np.all(iters <= 7)
    # continuing from the partial result converges and uses fewer sweeps than from zero
    r, it_warm, res = cp.batch_value_iteration(B, V, opts=cp.default_opts(max_iter=5000))
    V0 = torch.zeros_like(V)
    r0, it_zero, _ = cp.batch_value_iteration(B, V0, opts=cp.default_opts(max_iter=5000))
    assert np.all(res < 1e-6)
    assert it_warm.sum() < it_zero.sum()
    B.close()


def test_batch_rejects_invalid_instance(cp):
    bad = ci.config_small_2d(0)
    bad.reward = bad.reward.copy()
    bad.reward[0, 0] = np.nan
    with pytest.raises(cp.CpmdpError) as ei:
        cp.batch_build([ci.config_small_2d(1), bad], device=0)
    assert ei.value.status == cp.EINVAL and "instance 1" in cp.last_error()


@pytest.mark.parametrize("k", [1, 4, 9])
def test_batch_k_sweeps_match_oracle(cp, k):
    """k sweeps with tol too small to stop, on instances of every shape class:
    row lengths not a multiple of 4 (4-state segments that span rows, single
    neighbour loads), multiples of 4 (16-byte row loads), 1-D, 2-D and 3-D,
    odd and even state counts (padding). Each instance equals k oracle sweeps
    from zero within the FP32 bound eps (1 - gamma^k) / (1 - gamma)."""
    import torch
    from oracle import cpfactor as oc
    shapes = [(5,), (8,), (3, 7), (6, 6), (4, 12), (5, 9, 3), (4, 4, 8), (7, 5, 11), (2, 3, 4), (9, 1, 6)]
    inst = [ci.gridworld(s, p=0.75, gamma=0.93, step_reward=-0.04, goal_rewards=[1.0, -1.0][:min(2, int(np.prod(s)) - 1)],
                         obstacle_rate=0.15, seed=50 + i) for i, s in enumerate(shapes)]
    B = cp.batch_build(inst, device=0)
    V = torch.zeros(int(B.total_states), dtype=torch.float32, device="cuda")
    r, iters, _ = cp.batch_value_iteration(B, V, opts=cp.default_opts(tol=1e-30, max_iter=k), raise_on_noconv=False)
    assert np.all(iters == k)
    Vh = V.double().cpu().numpy()
    for i, gw in enumerate(inst):
        Vo = np.zeros(gw.nstates)
        for _ in range(k):
            Vo = oc.backup(gw, Vo)[0]
        lo = int(B.offsets[i])
        eps = 14 * U32 * (np.abs(gw.reward).max() + np.abs(Vo).max())
        err = np.abs(Vh[lo:lo + gw.nstates] - Vo).max()
        assert err <= eps * (1 - gw.gamma ** k) / (1 - gw.gamma) + 1e-30, (i, gw.shape, err)
    B.close()


def test_batch_tail_equals_batched_kernel(cp):
    """fused=4: once the running instances fit one co-resident grid, the
    batched kernel hands them to the barrier-free tail, each instance at its
    own pace. Same sweeps, values and residuals, bit for bit, as the batched
    kernel run to the end (fused=2)."""
    import torch
    inst = ci.batch_gridworlds(count=300, seed=11)
    inst.append(ci.gridworld((37,), p=0.9, gamma=0.95, step_reward=-0.04, goal_rewards=[1.0], seed=1))
    inst.append(ci.gridworld((3, 129), p=0.7, gamma=0.99, step_reward=-0.04, goal_rewards=[1.0, -1.0],
                             obstacle_rate=0.1, seed=2))
    B = cp.batch_build(inst, device=0)
    out = {}
    for fused in (4, 2):
        V = torch.zeros(int(B.total_states), dtype=torch.float32, device="cuda")
        r, it, res = cp.batch_value_iteration(B, V, opts=cp.default_opts(max_iter=5000, fused=fused))
        out[fused] = (V.cpu().numpy(), it, res, r)
    (Va, ia, ra, xa), (Vb, ib, rb, xb) = out[4], out[2]
    assert xa["tail_from"] > 0 and xb["tail_from"] == 0
    assert np.array_equal(ia, ib)
    assert np.array_equal(ra, rb)
    assert np.array_equal(Va.view(np.uint32), Vb.view(np.uint32))
    assert xa["iterations"] == xb["iterations"]
    # max_iter inside the tail: the same partial result
    for fused in (4, 2):
        V = torch.zeros(int(B.total_states), dtype=torch.float32, device="cuda")
        r, it, res = cp.batch_value_iteration(B, V, opts=cp.default_opts(max_iter=xa["tail_from"] + 5, fused=fused),
                                              raise_on_noconv=False)
        out[fused] = (V.cpu().numpy(), it, res, r)
    (Va, ia, ra, xa), (Vb, ib, rb, xb) = out[4], out[2]
    assert xa["status"] == cp.ENOCONV and np.array_equal(ia, ib) and np.array_equal(ra, rb)
    assert np.array_equal(Va.view(np.uint32), Vb.view(np.uint32))
    B.close()


def test_batch_resident_equals_batched_kernel(cp):
    """fused=1 (default): every instance held in shared memory for its whole
    solve, in one CTA (several small instances per CTA in lockstep) or cut
    into slices over the CTAs of a cluster (the slices next to a part read
    through distributed shared memory). Same per-state arithmetic as the
    batched kernel: sweeps, values and residuals equal those of fused=2 bit
    for bit, on the first solve (bundles from a gamma-based guess), on the
    second (bundles re-made from the first solve's sweep counts) and with
    max_iter stopping part of the instances."""
    import torch
    inst = ci.batch_gridworlds(count=160, seed=13)
    extra = [(48, 48, 48), (40, 47, 45), (33, 37, 28), (128, 128), (127, 101), (3, 129), (37,), (1,), (8, 8),
             (2, 3, 4), (9, 1, 6), (45, 30, 21)]
    for j, s in enumerate(extra):
        inst.append(ci.gridworld(s, p=0.6 + 0.03 * j, gamma=0.9 + 0.008 * j, step_reward=-0.04,
                                 goal_rewards=[1.0, -1.0][:min(2, int(np.prod(s)) - 1)] or [1.0],
                                 obstacle_rate=0.05 if int(np.prod(s)) > 2 else 0.0, seed=300 + j))
    inst.append(ci.GridWorld(shape=(4, 4), p=0.8, gamma=0.9, cell=np.ones((4, 4), np.uint8),
                             reward=np.zeros((4, 4))))
    B = cp.batch_build(inst, device=0)
    nS = int(B.total_states)

    def solve(fused, max_iter=5000):
        V = torch.zeros(nS, dtype=torch.float32, device="cuda")
        r, it, res = cp.batch_value_iteration(B, V, opts=cp.default_opts(max_iter=max_iter, fused=fused),
                                              raise_on_noconv=False)
        return V.cpu().numpy(), it, res, r

    Vb, ib, rb, xb = solve(2)
    for rep in range(2):
        Va, ia, ra, xa = solve(1)
        assert xa["solver"] == cp.SOLVER_BATCH_RESIDENT and xb["solver"] == cp.SOLVER_BATCH
        assert xa["status"] == cp.OK
        assert np.array_equal(ia, ib), (rep, np.nonzero(ia != ib)[0][:5])
        assert np.array_equal(ra, rb)
        assert np.array_equal(Va.view(np.uint32), Vb.view(np.uint32))
        assert xa["iterations"] == xb["iterations"] and xa["backups"] == xb["backups"]
    k = int(np.median(ib))
    Vb, ib, rb, xb = solve(2, k)
    Va, ia, ra, xa = solve(1, k)
    assert xa["status"] == cp.ENOCONV and xb["status"] == cp.ENOCONV
    assert np.array_equal(ia, ib) and np.array_equal(ra, rb)
    assert np.array_equal(Va.view(np.uint32), Vb.view(np.uint32))
    B.close()


@pytest.mark.parametrize("shapes", [
    # 2-D grids larger than one CTA (cut into row ranges over a cluster of 2), small ones beside them
    [(150, 200), (201, 140), (9, 7), (64, 64), (3, 5, 7)],
    # a 3-D grid that needs 6 CTAs (clusters of 8), 1-D and 2-D instances beside it
    [(100, 40, 40), (40, 47, 45), (37,), (120, 9), (8, 8, 8)],
])
def test_batch_resident_cluster_sizes(cp, shapes):
    """The resident solver's cluster size is the smallest power of two that
    fits every instance (2 and 8 here); parts of one instance on
    neighbouring ranks exchange their edge slices (rows in 2-D, planes in
    3-D). Sweeps, values and residuals equal the batched kernel's (fused=2)
    bit for bit, and every instance matches the FP64 oracle within the value
    bound of the first test."""
    import torch
    from oracle import cpfactor as oc
    inst = [ci.gridworld(s, p=0.7 + 0.04 * j, gamma=0.93 + 0.01 * j, step_reward=-0.04,
                         goal_rewards=[1.0, -1.0], obstacle_rate=0.05, seed=700 + j) for j, s in enumerate(shapes)]
    B = cp.batch_build(inst, device=0)
    out = {}
    for fused in (1, 2):
        V = torch.zeros(int(B.total_states), dtype=torch.float32, device="cuda")
        r, it, res = cp.batch_value_iteration(B, V, opts=cp.default_opts(max_iter=5000, fused=fused))
        out[fused] = (V.cpu().numpy(), it, res, r)
    (Va, ia, ra, xa), (Vb, ib, rb, xb) = out[1], out[2]
    assert xa["solver"] == cp.SOLVER_BATCH_RESIDENT
    assert np.array_equal(ia, ib) and np.array_equal(ra, rb)
    assert np.array_equal(Va.view(np.uint32), Vb.view(np.uint32))
    Vh = Va.astype(np.float64)
    for i, gw in enumerate(inst):
        lo, n = int(B.offsets[i]), gw.nstates
        Vo, _, ko, _ = oc.value_iteration(gw, tol=1e-6, max_iter=5000)
        eps = 14 * U32 * (np.abs(gw.reward).max() + np.abs(Vo).max())
        bound = (2 * gw.gamma * 1e-6 + eps) / (1 - gw.gamma)
        assert np.abs(Vh[lo:lo + n] - Vo).max() <= bound, (i, gw.shape)
    B.close()


def test_batch_certify_policy_matches_oracle(cp):
    """cpmdp_batch_certify after a batched solve: per instance the certified
    residual equals the oracle's own FP64 backup of the returned values
    (max |T(V) - V| over non-obstacle states), the policy equals the oracle's
    argmax of that backup wherever its best and second-best Q differ by
    more than FP64 rounding, and it equals the policy of the oracle's own
    value iteration wherever that gap exceeds twice gamma times the distance
    bound between the two results (both within residual / (1 - gamma) of
    V*). Obstacles and terminals get 255; the padding between instances is
    not written."""
    import torch
    from oracle import cpfactor as oc
    inst = _instances()
    B = cp.batch_build(inst, device=0)
    V = torch.zeros(int(B.total_states), dtype=torch.float32, device="cuda")
    r, iters, res = cp.batch_value_iteration(B, V, opts=cp.default_opts(max_iter=5000))
    pi = torch.full((int(B.total_states),), 77, dtype=torch.uint8, device="cuda")
    cert = cp.batch_certify(B, V, pi)
    Vh = V.double().cpu().numpy()
    ph = pi.cpu().numpy()
    for i in range(len(inst) - 1):   # padding after instance i, before instance i + 1
        lo, hi = int(B.offsets[i]) + inst[i].nstates, int(B.offsets[i + 1])
        assert np.all(ph[lo:hi] == 77)
    picks = list(range(0, 192, 6)) + list(range(192, len(inst)))
    compared = 0
    for i in picks:
        gw = inst[i]
        lo, n = int(B.offsets[i]), gw.nstates
        got, gp = Vh[lo:lo + n], ph[lo:lo + n]
        TV, opi, ores, Q = oc.backup(gw, got, want_q=True)
        free = gw.cell.reshape(-1) != ci.OBSTACLE
        want = float(np.abs(TV - got)[free].max()) if free.any() else 0.0
        assert abs(cert[i] - want) <= 1e-13 * (1 + np.abs(got).max()), (i, cert[i], want)
        inner = gw.cell.reshape(-1) == ci.FREE
        assert np.all(gp[~inner] == 255)
        if not inner.any():
            continue
        Qs = np.sort(Q[:, inner], axis=0)
        gap = Qs[-1] - Qs[-2] if Q.shape[0] > 1 else np.full(inner.sum(), np.inf)
        sure = gap > 1e-12 * (1 + np.abs(Qs[-1]))
        assert np.array_equal(gp[inner][sure], opi[inner][sure]), i
        # against the oracle's own value iteration
        Vo, po, ko, ro = oc.value_iteration(gw, tol=1e-6, max_iter=5000)
        bound = (cert[i] + gw.gamma * ro) / (1 - gw.gamma)
        _, _, _, Qo = oc.backup(gw, Vo, want_q=True)
        Qos = np.sort(Qo[:, inner], axis=0)
        gapo = Qos[-1] - Qos[-2] if Qo.shape[0] > 1 else np.full(inner.sum(), np.inf)
        sure_o = gapo > max(1e-6, 2 * gw.gamma * bound)
        assert np.array_equal(gp[inner][sure_o], po[inner][sure_o]), i
        compared += int(sure_o.sum())
    assert compared > 1000
    B.close()


def test_batch_full_4096_certified_and_sampled(cp):
    """The full 4096-instance batch (2-D sides 8..128, 3-D sides 8..48) in the
    configuration the benchmark times (shared-memory-resident solver,
    default options, second solve scheduled from the first's sweep counts):
    every instance converges, its FP64 certified residual (the FP64 backup
    of the returned values) is at most tol plus one FP32 backup's rounding
    bound eps = 14 u (max|R| + max|V|), and every 128th instance plus the
    slowest one equal the FP64 oracle's value iteration within the value
    bound of the first test."""
    import torch
    from oracle import cpfactor as oc
    inst = ci.batch_gridworlds(count=4096, seed=0)
    B = cp.batch_build(inst, device=0)
    V = torch.zeros(int(B.total_states), dtype=torch.float32, device="cuda")
    cp.batch_value_iteration(B, V, opts=cp.default_opts(max_iter=5000))
    V.zero_()
    r, iters, res = cp.batch_value_iteration(B, V, opts=cp.default_opts(max_iter=5000))
    assert r["status"] == cp.OK and r["solver"] == cp.SOLVER_BATCH_RESIDENT and np.all(res < 1e-6)
    cert = cp.batch_certify(B, V)
    Vh = V.double().cpu().numpy()
    for i, gw in enumerate(inst):
        lo, n = int(B.offsets[i]), gw.nstates
        eps = 14 * U32 * (np.abs(gw.reward).max() + np.abs(Vh[lo:lo + n]).max())
        assert cert[i] <= 1e-6 + eps, (i, cert[i], eps)
    picks = sorted(set(range(0, 4096, 128)) | {int(np.argmax(iters))})
    for i in picks:
        gw = inst[i]
        lo, n = int(B.offsets[i]), gw.nstates
        Vo, _, ko, _ = oc.value_iteration(gw, tol=1e-6, max_iter=5000)
        eps = 14 * U32 * (np.abs(gw.reward).max() + np.abs(Vo).max())
        bound = (2 * gw.gamma * 1e-6 + eps) / (1 - gw.gamma)
        assert np.abs(Vh[lo:lo + n] - Vo).max() <= bound, (i, gw.shape)
    B.close()
