"""Tabular FP64 oracle: the plain definitions on expanded transition matrices.

Test infrastructure only (see the package header). Everything here works on
the dense |S| x |S| matrix P_a of each action, so it is meant for small
grids (a few thousand states at most), like the tabular baseline the paper
compares against.

Parity pins (tests/test_oracle_pins.py): integer-exact row sums and
Definition 3 counts; closed forms (deterministic chains and grids give
gamma^dist * R_goal, constant reward gives R/(1-gamma), uniform and
identity dense factors); brute-force enumeration of every policy on tiny
grids; the contraction property; agreement with the independent C
CP-factor oracle.

Conventions
-----------
* States are flat C-order indices over (N_1, ..., N_D) (Definition 2: the
  last dimension varies fastest).
* Action ``a = 2*d + (sigma > 0)`` moves along dimension ``d`` by ``sigma``
  (two actions per axis, |A| = 2D; GridWorld scenario section).
* Slip model: the intended move happens with probability ``p``; the rest is
  spread evenly over the 2(D-1) perpendicular unit moves. For D = 1 there is
  no perpendicular move and the agent stays put with probability 1 - p.
* A move that would leave the grid or enter an obstacle leaves the agent
  where it is. Obstacle cells are not states (value 0, no action).
* Terminal cells end the interaction: V(t) = R(t), with no continuation.
"""
from __future__ import annotations

import itertools
from fractions import Fraction

import numpy as np

FREE, OBSTACLE, TERMINAL = 0, 1, 2


def slip_moves(D: int, a: int, p):
    """The rank-1 terms of action ``a``: a list of (dim, step, weight).

    ``step`` is -1, +1 or 0 (stay). Weights are taken in the arithmetic of
    ``p`` (float or Fraction), so integer-unit tests stay exact.
    """
    d, sigma = a // 2, (1 if a % 2 else -1)
    moves = [(d, sigma, p)]
    if D == 1:
        moves.append((d, 0, 1 - p))
    else:
        q = (1 - p) / (2 * (D - 1))
        for d2 in range(D):
            if d2 != d:
                moves.append((d2, -1, q))
                moves.append((d2, +1, q))
    return moves


def transition_tabular(shape, cell, p, dtype=np.float64):
    """P[a, s, s'] expanded directly from the GridWorld rules.

    Follows the scenario section (|A| = 2|D|, obstacles not accessible,
    terminals end the interaction) with Definition 2's state order. Rows of
    obstacle and terminal states are zero. ``p`` may be a ``Fraction``: with
    ``dtype=object`` the entries are then exact rationals.
    """
    shape = tuple(int(n) for n in shape)
    D = len(shape)
    S = int(np.prod(shape))
    A = 2 * D
    cellf = np.asarray(cell).reshape(-1)
    P = np.zeros((A, S, S), dtype=dtype)
    if dtype is object:
        P[...] = Fraction(0)
    for s in range(S):
        if cellf[s] != FREE:
            continue
        c = np.unravel_index(s, shape)
        for a in range(A):
            for (dd, step, w) in slip_moves(D, a, p):
                t = list(c)
                t[dd] += step
                if not (0 <= t[dd] < shape[dd]):
                    t = list(c)
                tf = int(np.ravel_multi_index(t, shape))
                if cellf[tf] == OBSTACLE:
                    tf = s
                P[a, s, tf] += w
    return P


def shift_matrix(n, step, one=1):
    """N x N per-dimension factor of a unit move: row i holds ``one`` at column
    i + step, or at column i when i + step leaves [0, n) (the wall sends the
    agent back). ``step = 0`` gives the identity."""
    U = np.zeros((n, n), dtype=object if not isinstance(one, (int, float)) else type(one))
    if U.dtype == object:
        U[...] = 0 * one
    for i in range(n):
        j = i + step
        U[i, j if 0 <= j < n else i] = one
    return U


def gridworld_cp_factors(shape, p, one=1):
    """The GridWorld transition model in CP form: for each action a list of
    rank-1 terms (lambda, [U_1, ..., U_D]); the moving dimension gets a
    shift factor and every other dimension the identity (background
    section, Fig. 1: a sum of outer products)."""
    shape = tuple(int(n) for n in shape)
    D = len(shape)
    out = []
    for a in range(2 * D):
        terms = []
        for (dd, step, w) in slip_moves(D, a, p):
            terms.append((w, [shift_matrix(shape[d], step if d == dd else 0, one)
                              for d in range(D)]))
        out.append(terms)
    return out


def expand_cp(terms_per_action, shape, cell):
    """Expand CP terms to P[a, s, s'] (Kronecker sum in Definition 2's
    order), then apply the correction that is not separable per dimension:
    mass landing on an obstacle goes back to s, and rows of obstacle and
    terminal states are zero."""
    cellf = np.asarray(cell).reshape(-1)
    S = cellf.size
    A = len(terms_per_action)
    obst = cellf == OBSTACLE
    out = []
    for a in range(A):
        P = None
        for (w, Us) in terms_per_action[a]:
            K = np.ones((1, 1), dtype=Us[0].dtype)
            for U in Us:
                K = np.kron(K, U)
            P = w * K if P is None else P + w * K
        P = P.copy()
        for s in range(S):
            if cellf[s] != FREE:
                P[s, :] = 0 * P[s, 0]
                continue
            moved = P[s, obst].sum() if obst.any() else 0 * P[s, 0]
            P[s, obst] = 0 * P[s, 0]
            P[s, s] = P[s, s] + moved
        out.append(P)
    return np.stack(out)


def definition3_components(P):
    """Definition 3: for each state s the list of (a, s, s', P(s'|s,a)) with
    P > 0; returns (components, C) where C[s] = number of components of s."""
    A, S, _ = P.shape
    comps, counts = [], np.zeros(S, dtype=np.int64)
    for s in range(S):
        lst = []
        for a in range(A):
            for t in range(S):
                if P[a, s, t] != 0:
                    lst.append((a, s, t, P[a, s, t]))
        comps.append(lst)
        counts[s] = len(lst)
    return comps, counts


def bellman_q(P, R, gamma, V):
    """Q[a, s] = R(s) + gamma * sum_{s'} P(s'|s,a) V(s')  (Eq. 1, inside max)."""
    R = np.asarray(R, dtype=np.float64).reshape(-1)
    V = np.asarray(V, dtype=np.float64).reshape(-1)
    return R[None, :] + gamma * np.einsum("ast,t->as", P, V)


def backup(P, R, gamma, cell, V):
    """One synchronous Bellman backup (Eq. 1) with the scenario's boundary
    rules: free states take max_a Q; terminals keep R(t); obstacles 0.
    Returns (V', greedy policy with lowest index on ties, Q)."""
    cellf = np.asarray(cell).reshape(-1)
    R = np.asarray(R, dtype=np.float64).reshape(-1)
    Q = bellman_q(P, R, gamma, V)
    free = cellf == FREE
    Vn = np.where(free, Q.max(axis=0), np.where(cellf == TERMINAL, R, 0.0))
    pi = np.where(free, Q.argmax(axis=0), 255).astype(np.uint8)
    return Vn, pi, Q


def value_iteration(P, R, gamma, cell, tol=1e-6, max_iter=1000, V0=None):
    """Value iteration (background section): repeat Eq. 1 until the largest
    change over non-obstacle states is below ``tol`` or ``max_iter`` sweeps
    are done. The policy is greedy with respect to the returned V.
    Returns (V, pi, iterations, last residual)."""
    cellf = np.asarray(cell).reshape(-1)
    S = cellf.size
    V = np.zeros(S) if V0 is None else np.asarray(V0, dtype=np.float64).reshape(-1).copy()
    live = cellf != OBSTACLE
    res, k = np.inf, 0
    for k in range(1, max_iter + 1):
        Vn, _, _ = backup(P, R, gamma, cell, V)
        res = float(np.max(np.abs(Vn - V)[live])) if live.any() else 0.0
        V = Vn
        if res < tol:
            break
    _, pi, _ = backup(P, R, gamma, cell, V)
    return V, pi, k, res


def evaluate_policy(P, R, gamma, cell, pi):
    """Exact policy evaluation: solve (I - gamma P_pi) V = R on free states,
    with V(t) = R(t) on terminals and 0 on obstacles (policy evaluation
    step of policy iteration, background section)."""
    cellf = np.asarray(cell).reshape(-1)
    R = np.asarray(R, dtype=np.float64).reshape(-1)
    S = cellf.size
    free = np.flatnonzero(cellf == FREE)
    term = cellf == TERMINAL
    V = np.where(term, R, 0.0)
    if free.size == 0:
        return V
    Ppi = P[np.asarray(pi)[free].astype(np.int64), free, :]          # (F, S)
    rhs = R[free] + gamma * Ppi[:, term] @ R[term]
    M = np.eye(free.size) - gamma * Ppi[:, free]
    V[free] = np.linalg.solve(M, rhs)
    return V


def policy_iteration(P, R, gamma, cell, pi0=None, max_iter=1000, keep_margin=1e-12):
    """Policy iteration (background section): alternate exact evaluation
    and greedy improvement; stop when the improvement changes no action.
    An action is replaced only if another one beats it by more than
    ``keep_margin * (1 + |Q|)`` so that exact ties do not cycle.
    ``pi0`` defaults to the greedy policy of V = 0.
    Returns (V, pi, improvement rounds)."""
    cellf = np.asarray(cell).reshape(-1)
    free = cellf == FREE
    if pi0 is None:
        _, pi, _ = backup(P, R, gamma, cell, np.zeros(cellf.size))
    else:
        pi = np.asarray(pi0, dtype=np.uint8).reshape(-1).copy()
    pi = np.where(free, pi, 255).astype(np.uint8)
    rounds = 0
    for rounds in range(1, max_iter + 1):
        V = evaluate_policy(P, R, gamma, cell, pi)
        Q = bellman_q(P, R, gamma, V)
        best = Q.argmax(axis=0)
        idx = np.arange(cellf.size)
        old = np.where(free, pi, 0).astype(np.int64)
        better = Q[best, idx] > Q[old, idx] + keep_margin * (1.0 + np.abs(Q[old, idx]))
        newpi = np.where(free & better, best, pi).astype(np.uint8)
        if np.array_equal(newpi, pi):
            break
        pi = newpi
    return V, pi, rounds


def brute_force_optimum(P, R, gamma, cell):
    """Enumerate every deterministic policy on the free states, evaluate each
    exactly, and return the state-wise maximum value (= V* for gamma < 1)
    and the list of policies attaining it everywhere. Tiny grids only."""
    cellf = np.asarray(cell).reshape(-1)
    A = P.shape[0]
    free = np.flatnonzero(cellf == FREE)
    pols, vals = [], []
    for choice in itertools.product(range(A), repeat=free.size):
        pi = np.full(cellf.size, 255, dtype=np.uint8)
        pi[free] = choice
        pols.append(pi)
        vals.append(evaluate_policy(P, R, gamma, cell, pi))
    vals = np.asarray(vals)
    best_V = vals.max(axis=0)
    best = [pols[i] for i in range(len(pols)) if np.all(vals[i] >= best_V - 1e-10)]
    return best_V, best


def dense_tabular(factors, lam, shape):
    """P[a] = sum_r lam[a,r] * U_{a,r,1} (x) ... (x) U_{a,r,D} (Kronecker
    product of the per-dimension factors; the CP form of the background
    section's Fig. 1 applied to each action's transition matrix). The
    Kronecker order matches Definition 2's state order."""
    A = len(factors)
    Rk = len(factors[0])
    S = int(np.prod(shape))
    P = np.zeros((A, S, S))
    for a in range(A):
        for r in range(Rk):
            K = np.ones((1, 1))
            for U in factors[a][r]:
                K = np.kron(K, np.asarray(U, dtype=np.float64))
            P[a] += lam[a][r] * K
    return P


def dense_value_iteration(P, R, gamma, tol=1e-6, max_iter=1000, V0=None):
    """Eq. 1 value iteration for a dense model where every state is a free
    state (no obstacles or terminals). Returns (V, pi, iterations, res)."""
    R = np.asarray(R, dtype=np.float64).reshape(-1)
    V = np.zeros(R.size) if V0 is None else np.asarray(V0, dtype=np.float64).reshape(-1).copy()
    res, k = np.inf, 0
    for k in range(1, max_iter + 1):
        Q = bellman_q(P, R, gamma, V)
        Vn = Q.max(axis=0)
        res = float(np.max(np.abs(Vn - V)))
        V = Vn
        if res < tol:
            break
    pi = bellman_q(P, R, gamma, V).argmax(axis=0).astype(np.uint8)
    return V, pi, k, res
