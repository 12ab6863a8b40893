"""Seeded synthetic inputs for CP-MDP GridWorlds and dense CP transition models.

This module is shared by the oracle, the tests and the benchmark. It only
*draws* problem instances: grid shapes, which cells are obstacles or
terminals, rewards, slip probabilities, discount factors and random dense
factor matrices. It contains none of the solver's arithmetic (no transition
expansion, no Bellman backup, no value or policy iteration).

Random numbers come from a counter-based SplitMix64 generator (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
element ``i`` of stream ``k`` under seed ``s`` is ``mix(key(s, k) + (i+1)*G)``
with ``G = 0x9E3779B97F4A7C15``. The value depends only on ``(s, k, i)``, so
instances are identical on every machine and independent of call order.

Cell codes follow the GridWorld scenario of the paper (section "MDP Scenario
and Problem Statement"): ``FREE`` cells are ordinary states, ``OBSTACLE``
cells can never be entered, and ``TERMINAL`` cells end the interaction.
States are enumerated as in Definition 2: the last dimension varies fastest
(C order), so every array here has shape ``(N_1, ..., N_D)`` in C order.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

FREE = 0
OBSTACLE = 1
TERMINAL = 2

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def u64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """``n`` raw 64-bit draws of stream ``stream`` under ``seed``."""
    with np.errstate(over="ignore"):
        key = _mix(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64) * _G
                   ^ _mix(np.array([stream & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64) + _G))
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        return _mix(key + i * _G)


def uniform(seed: int, stream: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """``n`` doubles uniform in ``[lo, hi)`` (53 random bits each)."""
    u = (u64(seed, stream, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def integers(seed: int, stream: int, n: int, lo: int, hi: int) -> np.ndarray:
    """``n`` integers uniform in the closed range ``[lo, hi]``."""
    span = np.uint64(hi - lo + 1)
    return (u64(seed, stream, n) % span).astype(np.int64) + lo


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """``n`` standard normal doubles (Box-Muller on two uniform streams)."""
    u1 = 1.0 - uniform(seed, stream, n)          # (0, 1]
    u2 = uniform(seed, stream + 0x5EED, n)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def _distinct_cells(seed: int, stream: int, count: int, nstates: int,
                    exclude: np.ndarray | None = None) -> np.ndarray:
    """``count`` distinct flat cell indices, drawn in order, skipping repeats."""
    if count > nstates:
        raise ValueError("more distinct cells requested than the grid holds")
    taken = set() if exclude is None else set(int(x) for x in np.flatnonzero(exclude))
    out: list[int] = []
    off = 0
    while len(out) < count:
        draws = (u64(seed, stream, 64, off) % np.uint64(nstates)).astype(np.int64)
        off += 64
        for c in draws:
            c = int(c)
            if c not in taken:
                taken.add(c)
                out.append(c)
                if len(out) == count:
                    break
        if off > 64 * (nstates + 64):
            raise ValueError("could not place distinct cells")
    return np.asarray(out, dtype=np.int64)


@dataclass
class GridWorld:
    """One n-D GridWorld instance: the tuple <S, A, P, R, gamma> of the paper.

    ``shape`` gives the mode sizes N_d (Definition 1), ``cell`` the per-state
    code (FREE / OBSTACLE / TERMINAL), ``reward`` the state reward R(s),
    ``p`` the probability that the intended move happens (the rest slips
    evenly to the 2(D-1) perpendicular moves; for D = 1 it stays put), and
    ``gamma`` the discount. |A| = 2D (two actions per axis).
    """
    shape: tuple
    p: float
    gamma: float
    cell: np.ndarray
    reward: np.ndarray
    seed: int = 0
    label: str = ""

    @property
    def ndim(self) -> int:
        return len(self.shape)

    @property
    def nactions(self) -> int:
        return 2 * len(self.shape)

    @property
    def nstates(self) -> int:
        return int(np.prod(self.shape))


@dataclass
class DenseCP:
    """A dense rank-R CP transition model on an n-D state grid.

    ``factors[a][r][d]`` is the N_d x N_d matrix U_{a,r,d} with rows indexed
    by the current coordinate s_d and columns by the next coordinate s'_d;
    every row sums to one. ``lam[a, r]`` are the rank weights (summing to one
    per action). ``reward`` is R(s) and ``gamma`` the discount.
    """
    shape: tuple
    factors: list
    lam: np.ndarray
    reward: np.ndarray
    gamma: float
    seed: int = 0
    label: str = ""

    @property
    def ndim(self) -> int:
        return len(self.shape)

    @property
    def nactions(self) -> int:
        return len(self.factors)

    @property
    def rank(self) -> int:
        return len(self.factors[0])

    @property
    def nstates(self) -> int:
        return int(np.prod(self.shape))

    def packed_factors(self) -> np.ndarray:
        """Factors flattened as [a][r][d][s_d][s'_d] (row-major per matrix)."""
        return np.concatenate([np.asarray(self.factors[a][r][d], dtype=np.float64).ravel()
                               for a in range(self.nactions)
                               for r in range(self.rank)
                               for d in range(self.ndim)])


# stream ids (any distinct constants)
_S_GOALS, _S_GOALREW, _S_OBST, _S_REW, _S_FACT, _S_META, _S_VALS = 11, 12, 13, 14, 15, 16, 17


def gridworld(shape, *, p: float, gamma: float, step_reward: float,
              goal_rewards, obstacle_rate: float = 0.0, seed: int = 0,
              label: str = "") -> GridWorld:
    """Draw a GridWorld: terminals at distinct seeded cells with the given
    rewards, then each remaining cell an obstacle with probability
    ``obstacle_rate``; every other cell earns ``step_reward``."""
    shape = tuple(int(n) for n in shape)
    if not shape or any(n < 1 for n in shape):
        raise ValueError("every mode size must be >= 1")
    ns = int(np.prod(shape))
    goal_rewards = np.asarray(goal_rewards, dtype=np.float64).ravel()
    cell = np.zeros(ns, dtype=np.uint8)
    reward = np.full(ns, float(step_reward), dtype=np.float64)
    goals = _distinct_cells(seed, _S_GOALS, len(goal_rewards), ns)
    cell[goals] = TERMINAL
    reward[goals] = goal_rewards
    if obstacle_rate > 0.0:
        obst = (uniform(seed, _S_OBST, ns) < obstacle_rate) & (cell != TERMINAL)
        cell[obst] = OBSTACLE
        reward[obst] = 0.0
    return GridWorld(shape=shape, p=float(p), gamma=float(gamma),
                     cell=cell.reshape(shape), reward=reward.reshape(shape),
                     seed=seed, label=label)


def config_small_2d(seed: int = 0) -> GridWorld:
    """2-D 10x10, 4 actions, p = 0.8 (0.1 slip to each side), reward -0.04
    per step, one +1 and one -1 absorbing cell at seeded positions,
    gamma = 0.9, no obstacles."""
    return gridworld((10, 10), p=0.8, gamma=0.9, step_reward=-0.04,
                     goal_rewards=[1.0, -1.0], seed=seed, label="gridworld-10x10")


def config_3d(side: int = 64, seed: int = 0, gamma: float = 0.99) -> GridWorld:
    """3-D side^3 (64^3 = 262,144 states), 6 actions, p = 0.8 (0.05 to each
    of the 4 perpendicular moves), 5 % seeded obstacles, 8 goal cells with
    reward U(0.5, 1), step reward -0.01, gamma = 0.99."""
    goal_r = uniform(seed, _S_GOALREW, 8, 0.5, 1.0)
    return gridworld((side, side, side), p=0.8, gamma=gamma, step_reward=-0.01,
                     goal_rewards=goal_r, obstacle_rate=0.05, seed=seed,
                     label=f"gridworld-{side}^3")


def dense_cp(shape, nactions: int, rank: int, gamma: float, seed: int = 0,
             label: str = "") -> DenseCP:
    """Dense CP model: entries U(0,1), each factor row normalised to sum 1,
    lambda = 1/R, rewards N(0,1) per state."""
    shape = tuple(int(n) for n in shape)
    D = len(shape)
    ns = int(np.prod(shape))
    total = sum(n * n for n in shape) * nactions * rank
    raw = uniform(seed, _S_FACT, total)
    factors, off = [], 0
    for a in range(nactions):
        fa = []
        for r in range(rank):
            fr = []
            for d in range(D):
                n = shape[d]
                m = raw[off:off + n * n].reshape(n, n).copy()
                off += n * n
                m /= m.sum(axis=1, keepdims=True)
                fr.append(m)
            fa.append(fr)
        factors.append(fa)
    lam = np.full((nactions, rank), 1.0 / rank, dtype=np.float64)
    reward = normal(seed, _S_REW, ns).reshape(shape)
    return DenseCP(shape=shape, factors=factors, lam=lam, reward=reward,
                   gamma=float(gamma), seed=seed, label=label or f"dense-cp-{shape}")


def config_dense_4d(side: int = 64, seed: int = 0) -> DenseCP:
    """4-D dense CP model side^4 (64^4 = 16.8M states), 8 actions, rank 8,
    gamma = 0.95."""
    return dense_cp((side,) * 4, 8, 8, 0.95, seed=seed, label=f"dense-cp-{side}^4")


def batch_gridworlds(count: int = 4096, seed: int = 0) -> list:
    """Independent 2-D / 3-D GridWorlds of uneven size (50/50 coin): each 2-D
    side uniform in {8..128}, each 3-D side uniform in {8..48}; p ~ U(0.6,
    0.95), gamma ~ U(0.9, 0.995); reward -0.04 per step, one +1 and one -1
    absorbing cell, 5 % obstacles."""
    coin = integers(seed, _S_META, count, 0, 1)
    pp = uniform(seed, _S_META + 1, count, 0.6, 0.95)
    gg = uniform(seed, _S_META + 2, count, 0.9, 0.995)
    sides2 = integers(seed, _S_META + 3, 2 * count, 8, 128).reshape(count, 2)
    sides3 = integers(seed, _S_META + 4, 3 * count, 8, 48).reshape(count, 3)
    out = []
    for i in range(count):
        shape = tuple(sides2[i]) if coin[i] == 0 else tuple(sides3[i])
        sub = int(u64(seed, _S_META + 5, 1, i)[0] & np.uint64(0x7FFFFFFFFFFFFFFF))
        out.append(gridworld(shape, p=float(pp[i]), gamma=float(gg[i]), step_reward=-0.04,
                             goal_rewards=[1.0, -1.0], obstacle_rate=0.05, seed=sub,
                             label=f"batch-{i}"))
    return out


def random_values(shape, seed: int = 0, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """A random value tensor (float64) for single-sweep parity checks."""
    shape = tuple(int(n) for n in shape)
    return uniform(seed, _S_VALS, int(np.prod(shape)), lo, hi).reshape(shape)
