"""Dense CP FP64 oracle: the backup as a chain of mode products.

Test infrastructure only (see the package header).

For action a with rank-R CP transition model
    P_a(s'|s) = sum_r lambda_{a,r} prod_d U_{a,r,d}[s_d, s'_d]
(the CP form of the background section applied per action, with
Definition 2's state tuples), the expected next value is
    E_a[V](s) = sum_r lambda_{a,r} (V x_1 U_{a,r,1} x_2 ... x_D U_{a,r,D})(s)
where (X x_d U)[.., i, ..] = sum_j U[i, j] X[.., j, ..] is the mode-d
product (Kolda and Bader, SIAM Review 2009). Eq. 1 then gives
V'(s) = R(s) + gamma max_a E_a[V](s). Every state is a free state.

Each mode product is one numpy ``tensordot`` (a library matmul used as one
step, no blocking or reordering). ``q_at`` evaluates Q(s, .) for a single
state by contracting V with the rows U[s_d, :] one dimension at a time,
for sampled checks at full size.

Parity pins: tests/test_oracle_pins.py checks these against the Kronecker
expansion of the tabular oracle on small shapes and against the closed
forms for uniform (U = 1/N) and identity factors.
"""
from __future__ import annotations

import numpy as np


def mode_product(X, U, d):
    """(X x_d U): contract X's axis d with U's column index."""
    Y = np.tensordot(np.asarray(U, dtype=np.float64), X, axes=([1], [d]))
    return np.moveaxis(Y, 0, d)


def expectation(dc, V, a):
    """E_a[V] for every state: the sum over ranks of the mode-product chains."""
    V = np.asarray(V, dtype=np.float64).reshape(dc.shape)
    E = np.zeros(dc.shape)
    for r in range(dc.rank):
        T = V
        for d in range(dc.ndim):
            T = mode_product(T, dc.factors[a][r][d], d)
        E += dc.lam[a][r] * T
    return E


def q_values(dc, V):
    """Q[a, s] = R(s) + gamma E_a[V](s), shape (A, |S|)."""
    R = np.asarray(dc.reward, dtype=np.float64).reshape(-1)
    return np.stack([R + dc.gamma * expectation(dc, V, a).reshape(-1)
                     for a in range(dc.nactions)])


def backup(dc, V):
    """One Eq. 1 backup: returns (V', greedy policy (lowest index on ties), residual)."""
    Q = q_values(dc, V)
    Vn = Q.max(axis=0)
    res = float(np.max(np.abs(Vn - np.asarray(V, dtype=np.float64).reshape(-1))))
    return Vn, Q.argmax(axis=0).astype(np.uint8), res


def value_iteration(dc, tol=1e-6, max_iter=1000, V0=None):
    """Value iteration on the dense CP model. Returns (V, pi, sweeps, residual)."""
    V = np.zeros(dc.nstates) if V0 is None else np.asarray(V0, dtype=np.float64).reshape(-1).copy()
    res, k = np.inf, 0
    for k in range(1, max_iter + 1):
        Vn, _, res = backup(dc, V)
        V = Vn
        if res < tol:
            break
    _, pi, _ = backup(dc, V)
    return V, pi, k, res


def q_at(dc, V, coords):
    """Q(s, a) for one state s (tuple of coordinates), all actions."""
    V = np.asarray(V, dtype=np.float64).reshape(dc.shape)
    flat = int(np.ravel_multi_index(tuple(coords), dc.shape))
    R = float(np.asarray(dc.reward).reshape(-1)[flat])
    out = np.empty(dc.nactions)
    for a in range(dc.nactions):
        e = 0.0
        for r in range(dc.rank):
            T = V
            for d in range(dc.ndim):
                T = np.tensordot(np.asarray(dc.factors[a][r][d])[coords[d], :], T, axes=(0, 0))
            e += dc.lam[a][r] * float(T)
        out[a] = R + dc.gamma * e
    return out
