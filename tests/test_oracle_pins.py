"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: exact
rational arithmetic, closed forms, brute force over every policy, a printed
textbook example, the contraction property, or a second, independently
written oracle. Chosen so that a dropped slip term, a wrong move sign, a
transposed dimension, a wrong wall or obstacle rule or wrong terminal
handling each fails at least one test.
"""
from collections import deque
from fractions import Fraction
import os

import numpy as np
import pytest

import cpmdp_inputs as ci
from oracle import dense as OD
from oracle import tabular as T

FREE, OBST, TERM = ci.FREE, ci.OBSTACLE, ci.TERMINAL
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid(shape, cells=(), p=0.8, gamma=0.9, step=0.0, seed=0):
    shape = tuple(shape)
    cell = np.zeros(shape, dtype=np.uint8)
    reward = np.full(shape, float(step))
    for (idx, kind, r) in cells:
        cell[idx] = kind
        reward[idx] = r if kind == TERM else (0.0 if kind == OBST else step)
    return ci.GridWorld(shape=shape, p=p, gamma=gamma, cell=cell, reward=reward, seed=seed)


# --- exact (rational) structure: Definition 3, row sums, CP reconstruction ---

EXACT_CASES = [
    ((2, 3), [((1, 1), OBST, 0)], Fraction(4, 5)),
    ((3, 4), [((0, 3), TERM, 1), ((1, 1), OBST, 0), ((1, 2), TERM, -1)], Fraction(4, 5)),
    ((2, 2, 3), [((0, 1, 1), OBST, 0), ((1, 0, 2), TERM, 1)], Fraction(4, 5)),
    ((5,), [((2,), OBST, 0)], Fraction(3, 4)),
    ((3, 2, 2, 2), [((1, 1, 0, 1), OBST, 0)], Fraction(7, 10)),
]


@pytest.mark.parametrize("shape,cells,p", EXACT_CASES)
def test_cp_reconstruction_equals_tabular_exactly(shape, cells, p):
    """CP factors (Kronecker sum of shift/identity factors) plus the obstacle
    correction reproduce the rule-based tabular P exactly, entry by entry,
    in rational arithmetic."""
    gw = _grid(shape, cells)
    P_rules = T.transition_tabular(shape, gw.cell, p, dtype=object)
    P_cp = T.expand_cp(T.gridworld_cp_factors(shape, p, Fraction(1)), shape, gw.cell)
    assert P_rules.shape == P_cp.shape
    assert all(x == y for x, y in zip(P_rules.ravel(), P_cp.ravel()))


@pytest.mark.parametrize("shape,cells,p", EXACT_CASES)
def test_rows_stochastic_exactly(shape, cells, p):
    gw = _grid(shape, cells)
    P = T.transition_tabular(shape, gw.cell, p, dtype=object)
    cellf = gw.cell.reshape(-1)
    for a in range(P.shape[0]):
        for s in range(P.shape[1]):
            total = sum(P[a, s, :], Fraction(0))
            assert total == (1 if cellf[s] == FREE else 0)
            # nothing ever lands on an obstacle
            assert all(P[a, s, t] == 0 for t in np.flatnonzero(cellf == OBST))


def test_definition3_counts_interior_and_corner():
    """Definition 3: C(s) counts transitions with P > 0. In an open grid an
    interior state has 2D-1 distinct successors per action; a corner merges
    the wall-blocked moves into s."""
    shape = (4, 5)
    gw = _grid(shape)
    P = T.transition_tabular(shape, gw.cell, 0.8)
    _, counts = T.definition3_components(P)
    D, A = 2, 4
    interior = np.ravel_multi_index((1, 2), shape)
    assert counts[interior] == A * (2 * D - 1)
    corner = np.ravel_multi_index((0, 0), shape)
    # per action at (0,0): moving into a wall merges with the bounce of the
    # blocked perpendicular move; count by hand: N:{s,(0,1)}=2, S:{(1,0),s,(0,1)}=3,
    # W:{s,(1,0)}=2, E:{(0,1),s,(1,0)}=3
    assert counts[corner] == 10


def test_action_directions():
    """a = 2d + (sigma > 0): action 1 moves +1 along dimension 0, action 2
    moves -1 along dimension 1 (deterministic moves)."""
    shape = (3, 4)
    gw = _grid(shape)
    P = T.transition_tabular(shape, gw.cell, 1.0)
    s = np.ravel_multi_index((1, 1), shape)
    assert P[1, s, np.ravel_multi_index((2, 1), shape)] == 1.0
    assert P[0, s, np.ravel_multi_index((0, 1), shape)] == 1.0
    assert P[2, s, np.ravel_multi_index((1, 0), shape)] == 1.0
    assert P[3, s, np.ravel_multi_index((1, 2), shape)] == 1.0


# --- closed forms -------------------------------------------------------------

def _bfs_dist(cell, goal):
    shape = cell.shape
    dist = np.full(shape, -1, dtype=np.int64)
    dist[goal] = 0
    q = deque([goal])
    while q:
        c = q.popleft()
        for d in range(len(shape)):
            for st in (-1, 1):
                t = list(c)
                t[d] += st
                t = tuple(t)
                if 0 <= t[d] < shape[d] and cell[t] != OBST and dist[t] < 0:
                    dist[t] = dist[c] + 1
                    if cell[t] == FREE:
                        q.append(t)
    return dist


def test_deterministic_chain_closed_form(oracle_c):
    """1-D chain, p = 1, zero step reward, terminal goal: V = gamma^dist R_goal,
    and the policy points toward the goal."""
    N, g, gamma = 9, 6, 0.9
    gw = _grid((N,), [((g,), TERM, 2.0)], p=1.0, gamma=gamma)
    want = 2.0 * gamma ** np.abs(np.arange(N) - g)
    P = T.transition_tabular(gw.shape, gw.cell, 1.0)
    V, pi, _, _ = T.value_iteration(P, gw.reward, gamma, gw.cell, tol=1e-14, max_iter=5000)
    np.testing.assert_allclose(V, want, rtol=0, atol=1e-12)
    assert list(pi[:g]) == [1] * g and list(pi[g + 1:]) == [0] * (N - g - 1) and pi[g] == 255
    Vc, pic, _, _ = oracle_c.value_iteration(gw, tol=1e-14, max_iter=5000)
    np.testing.assert_allclose(Vc, want, rtol=0, atol=1e-12)
    assert np.array_equal(pic, pi)


def test_deterministic_grid_with_obstacles_closed_form(oracle_c):
    """Non-square 2-D and 3-D grids, p = 1, zero step reward, one goal:
    V = gamma^(shortest path length around obstacles) * R_goal, 0 where the
    goal is unreachable."""
    for shape, goal, obst in [((5, 7), (3, 1), []),
                              ((6, 5), (0, 4), [(1, 3), (1, 4), (2, 1), (3, 2), (4, 4)]),
                              ((3, 4, 5), (2, 0, 3), [(1, 0, 3), (2, 1, 3), (0, 2, 2)])]:
        gamma = 0.8
        gw = _grid(shape, [(goal, TERM, 1.0)] + [(o, OBST, 0) for o in obst], p=1.0, gamma=gamma)
        dist = _bfs_dist(gw.cell, goal)
        want = np.where(dist >= 0, gamma ** np.maximum(dist, 0), 0.0)
        want[gw.cell == OBST] = 0.0
        Vc, pic, _, _ = oracle_c.value_iteration(gw, tol=1e-15, max_iter=10000)
        np.testing.assert_allclose(Vc.reshape(shape), want, rtol=0, atol=1e-12)
        P = T.transition_tabular(shape, gw.cell, 1.0)
        V, pi, _, _ = T.value_iteration(P, gw.reward, gamma, gw.cell, tol=1e-15, max_iter=10000)
        np.testing.assert_allclose(V.reshape(shape), want, rtol=0, atol=1e-12)
        # each chosen move of a reachable state goes one step closer to the goal
        for s in np.flatnonzero((gw.cell.reshape(-1) == FREE) & (dist.reshape(-1) > 0)):
            a = int(pi[s])
            c = list(np.unravel_index(s, shape))
            c[a // 2] += 1 if a % 2 else -1
            assert 0 <= c[a // 2] < shape[a // 2]
            assert dist[tuple(c)] == dist.reshape(-1)[s] - 1


def test_constant_reward_closed_form(oracle_c):
    """No terminals or obstacles, constant reward r: every policy earns
    V = r / (1 - gamma)."""
    gw = _grid((4, 3, 5), p=0.65, gamma=0.93, step=0.7)
    want = 0.7 / (1 - 0.93)
    Vc, _, _, _ = oracle_c.value_iteration(gw, tol=1e-13, max_iter=20000)
    np.testing.assert_allclose(Vc, want, rtol=1e-11)
    P = T.transition_tabular(gw.shape, gw.cell, gw.p)
    V, _, _, _ = T.value_iteration(P, gw.reward, gw.gamma, gw.cell, tol=1e-13, max_iter=20000)
    np.testing.assert_allclose(V, want, rtol=1e-11)


def test_textbook_4x3_world():
    """The 4x3 world of Russell and Norvig (golden file, cited there): the
    same slip model, walls, obstacle and terminal rules as this oracle."""
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "aima_4x3_utilities.txt"))
            if ln.strip() and not ln.startswith("#")]
    shape = (3, 4)
    cell = np.zeros(shape, dtype=np.uint8)
    reward = np.full(shape, -0.04)
    want = np.zeros(shape)
    for i, row in enumerate(rows):
        for j, tok in enumerate(row):
            if tok == "X":
                cell[i, j] = OBST
                reward[i, j] = 0.0
            elif tok.startswith("+") or tok == "-1":
                cell[i, j] = TERM
                reward[i, j] = float(tok)
                want[i, j] = float(tok)
            else:
                want[i, j] = float(tok)
    P = T.transition_tabular(shape, cell, 0.8)
    V, pi, _, _ = T.value_iteration(P, reward, 1.0, cell, tol=1e-13, max_iter=100000)
    np.testing.assert_allclose(V.reshape(shape), want, rtol=0, atol=6e-4)
    Vpi, pipi, _ = T.policy_iteration(P, reward, 0.999999, cell)
    np.testing.assert_allclose(Vpi.reshape(shape), want, rtol=0, atol=2e-3)


# --- brute force over every policy ---------------------------------------------

@pytest.mark.parametrize("shape,cells,p,gamma", [
    ((2, 3), [((0, 2), TERM, 1.0), ((1, 1), OBST, 0)], 0.8, 0.9),
    ((2, 3), [((1, 0), TERM, -1.0), ((0, 2), TERM, 1.0)], 0.6, 0.95),
    ((2, 2, 2), [((1, 1, 1), TERM, 1.0), ((0, 1, 0), OBST, 0)], 0.8, 0.9),
])
def test_brute_force_optimum(shape, cells, p, gamma, oracle_c):
    gw = _grid(shape, cells, p=p, gamma=gamma, step=-0.04)
    P = T.transition_tabular(shape, gw.cell, p)
    Vstar, optimal = T.brute_force_optimum(P, gw.reward, gamma, gw.cell)
    V, pi, _, _ = T.value_iteration(P, gw.reward, gamma, gw.cell, tol=1e-13, max_iter=10000)
    np.testing.assert_allclose(V, Vstar, rtol=0, atol=1e-10)
    assert any(np.array_equal(pi, o) for o in optimal)
    Vp, pip, _ = T.policy_iteration(P, gw.reward, gamma, gw.cell)
    np.testing.assert_allclose(Vp, Vstar, rtol=0, atol=1e-10)
    assert any(np.array_equal(pip, o) for o in optimal)
    Vc, pic, _, _ = oracle_c.value_iteration(gw, tol=1e-13, max_iter=10000)
    np.testing.assert_allclose(Vc, Vstar, rtol=0, atol=1e-10)
    assert any(np.array_equal(pic, o) for o in optimal)


# --- invariants ----------------------------------------------------------------

def test_contraction_and_monotonicity(oracle_c):
    gw = ci.gridworld((6, 5, 4), p=0.7, gamma=0.9, step_reward=0.1, goal_rewards=[1.0, 0.5],
                      obstacle_rate=0.1, seed=3)
    live = gw.cell.reshape(-1) != OBST
    for seed in range(5):
        V = ci.random_values(gw.shape, seed=seed, lo=-3, hi=3).reshape(-1)
        W = ci.random_values(gw.shape, seed=seed + 100, lo=-3, hi=3).reshape(-1)
        TV = oracle_c.backup(gw, V)[0]
        TW = oracle_c.backup(gw, W)[0]
        assert np.max(np.abs(TV - TW)[live]) <= gw.gamma * np.max(np.abs(V - W)[live]) + 1e-12
    # R >= 0: value iteration from 0 is monotone non-decreasing
    V = np.zeros(gw.nstates)
    for _ in range(30):
        Vn = oracle_c.backup(gw, V)[0]
        assert np.all(Vn >= V - 1e-15)
        V = Vn


def test_vi_pi_agree_and_fixed_point(oracle_c):
    """Config-1 shape: VI and PI (tabular exact and C iterative) give the
    same policy wherever the best/second-best Q gap exceeds 1e-6, and the
    Bellman residual of the returned V is below the tolerance."""
    gw = ci.config_small_2d(seed=1)
    P = T.transition_tabular(gw.shape, gw.cell, gw.p)
    V, pi, k, res = T.value_iteration(P, gw.reward, gw.gamma, gw.cell, tol=1e-6)
    assert res < 1e-6 and k < 1000
    Vn, _, Q = T.backup(P, gw.reward, gw.gamma, gw.cell, V)
    assert np.max(np.abs(Vn - V)) < 1e-6
    Vp, pip, _ = T.policy_iteration(P, gw.reward, gw.gamma, gw.cell)
    Vc, pic, _ = oracle_c.policy_iteration(gw)
    free = gw.cell.reshape(-1) == FREE
    Qs = np.sort(Q, axis=0)
    gap = Qs[-1] - Qs[-2]
    sure = free & (gap > 1e-6)
    assert np.array_equal(pi[sure], pip[sure]) and np.array_equal(pic[sure], pip[sure])
    np.testing.assert_allclose(Vc, Vp, rtol=0, atol=1e-10)
    # V from VI at residual 1e-6 is within gamma/(1-gamma) * res of V*
    assert np.max(np.abs(V - Vp)) <= gw.gamma / (1 - gw.gamma) * res + 1e-12


# --- the two oracles agree -----------------------------------------------------

@pytest.mark.parametrize("shape,p,orate,seed", [
    ((3, 4), 0.8, 0.2, 0), ((2, 3, 4), 0.7, 0.15, 1), ((7,), 0.9, 0.2, 2),
    ((3, 2, 2, 3), 0.6, 0.1, 3), ((1, 5), 0.8, 0.0, 4),
])
def test_c_oracle_matches_tabular(shape, p, orate, seed, oracle_c):
    gw = ci.gridworld(shape, p=p, gamma=0.9, step_reward=-0.04, goal_rewards=[1.0, -1.0],
                      obstacle_rate=orate, seed=seed)
    P = T.transition_tabular(shape, gw.cell, p)
    for vs in range(3):
        V = ci.random_values(shape, seed=vs).reshape(-1)
        Vt, pit, Qt = T.backup(P, gw.reward, gw.gamma, gw.cell, V)
        Vc, pic, _, Qc = oracle_c.backup(gw, V, want_q=True)
        np.testing.assert_allclose(Vc, Vt, rtol=0, atol=1e-14)
        free = gw.cell.reshape(-1) == FREE
        np.testing.assert_allclose(Qc[:, free], Qt[:, free], rtol=0, atol=1e-14)
        Qs = np.sort(Qt, axis=0)
        sure = free & ((Qs[-1] - Qs[-2]) > 1e-12)
        assert np.array_equal(pic[sure], pit[sure])
        pin = np.where(free, pit, 255).astype(np.uint8)
        Ve, _, _, _ = oracle_c.backup(gw, V, fixed_pi=pin)
        want = np.where(free, Qt[np.where(free, pit, 0), np.arange(V.size)],
                        np.where(gw.cell.reshape(-1) == TERM, gw.reward.reshape(-1), 0))
        np.testing.assert_allclose(Ve, want, rtol=0, atol=1e-14)


# --- dense CP ------------------------------------------------------------------

def test_dense_mode_products_match_kronecker():
    dc = ci.dense_cp((3, 4, 2), nactions=3, rank=4, gamma=0.9, seed=5)
    P = T.dense_tabular(dc.factors, dc.lam, dc.shape)
    np.testing.assert_allclose(P.sum(axis=2), 1.0, rtol=0, atol=1e-13)
    V = ci.random_values(dc.shape, seed=1).reshape(-1)
    Qt = T.bellman_q(P, dc.reward, dc.gamma, V)
    Qm = OD.q_values(dc, V)
    np.testing.assert_allclose(Qm, Qt, rtol=0, atol=1e-13)
    for coords in [(0, 0, 0), (2, 3, 1), (1, 2, 0)]:
        s = np.ravel_multi_index(coords, dc.shape)
        np.testing.assert_allclose(OD.q_at(dc, V, coords), Qt[:, s], rtol=0, atol=1e-13)
    Vt, pit, _, _ = T.dense_value_iteration(P, dc.reward, dc.gamma, tol=1e-12)
    Vm, pim, _, _ = OD.value_iteration(dc, tol=1e-12)
    np.testing.assert_allclose(Vm, Vt, rtol=0, atol=1e-10)


def test_dense_uniform_and_identity_closed_forms():
    shape, gamma = (3, 4, 5), 0.9
    R = ci.random_values(shape, seed=7)
    uni = [[[np.full((n, n), 1.0 / n) for n in shape] for _ in range(2)] for _ in range(2)]
    dc = ci.DenseCP(shape=shape, factors=uni, lam=np.full((2, 2), 0.5), reward=R, gamma=gamma)
    V, _, _, _ = OD.value_iteration(dc, tol=1e-13, max_iter=5000)
    np.testing.assert_allclose(V, (R + gamma * R.mean() / (1 - gamma)).reshape(-1), atol=1e-11)
    ident = [[[np.eye(n) for n in shape]] for _ in range(3)]
    dc = ci.DenseCP(shape=shape, factors=ident, lam=np.ones((3, 1)), reward=R, gamma=gamma)
    V, _, _, _ = OD.value_iteration(dc, tol=1e-13, max_iter=5000)
    np.testing.assert_allclose(V, (R / (1 - gamma)).reshape(-1), atol=1e-11)


def test_c_oracle_sampled_q_matches_full(oracle_c):
    gw = ci.gridworld((5, 6, 7), p=0.7, gamma=0.9, step_reward=-0.04, goal_rewards=[1.0, -1.0],
                      obstacle_rate=0.1, seed=9)
    V = ci.random_values(gw.shape, seed=2).reshape(-1)
    _, _, _, Q = oracle_c.backup(gw, V, want_q=True)
    states = np.array([0, 17, 101, gw.nstates - 1, 55])
    Qs = oracle_c.q_states(gw, V, states)
    free = gw.cell.reshape(-1)[states] == FREE
    np.testing.assert_array_equal(Qs[free], Q[:, states].T[free])
    assert np.all(Qs[~free] == 0)
