"""Python wrapper of the plain-C FP64 CP-factor GridWorld oracle.

Test infrastructure only (see the package header). ``build()`` compiles
``cpfactor.c`` with gcc into ``liboracle_cpfactor.so`` next to this file;
nothing here touches CUDA. Functions take a ``cpmdp_inputs.GridWorld`` (or
its fields) and return numpy arrays.

Each function follows the paper as described in ``cpfactor.c``: Eq. 1 for
the backup, the value-iteration and policy-iteration paragraphs of the
background section, and the GridWorld scenario rules. Parity is pinned in
tests/test_oracle_pins.py against the tabular definitions and closed forms.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpfactor.c")
_LIB = os.path.join(_HERE, "liboracle_cpfactor.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc -O2 -fopenmp) if it is missing or stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64p = ctypes.POINTER(ctypes.c_int64)
        u8p = ctypes.c_void_p
        dp = ctypes.c_void_p
        lib.oracle_gw_backup.restype = ctypes.c_double
        lib.oracle_gw_backup.argtypes = [ctypes.c_int, i64p, ctypes.c_double, ctypes.c_double,
                                         u8p, dp, dp, dp, u8p, u8p, dp]
        lib.oracle_gw_value_iteration.restype = ctypes.c_int
        lib.oracle_gw_value_iteration.argtypes = [ctypes.c_int, i64p, ctypes.c_double,
                                                  ctypes.c_double, u8p, dp, dp, u8p,
                                                  ctypes.c_double, ctypes.c_int, dp]
        lib.oracle_gw_evaluate.restype = ctypes.c_int
        lib.oracle_gw_evaluate.argtypes = [ctypes.c_int, i64p, ctypes.c_double, ctypes.c_double,
                                           u8p, dp, u8p, dp, ctypes.c_double, ctypes.c_int, dp]
        lib.oracle_gw_q_states.restype = ctypes.c_int
        lib.oracle_gw_q_states.argtypes = [ctypes.c_int, i64p, ctypes.c_double, ctypes.c_double,
                                           u8p, dp, dp, dp, ctypes.c_int64, dp]
        lib.oracle_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def threads() -> int:
    return _load().oracle_threads()


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _prep(gw):
    shape = np.ascontiguousarray(np.asarray(gw.shape, dtype=np.int64))
    cell = np.ascontiguousarray(np.asarray(gw.cell, dtype=np.uint8).reshape(-1))
    R = np.ascontiguousarray(np.asarray(gw.reward, dtype=np.float64).reshape(-1))
    return shape, cell, R


def backup(gw, V, fixed_pi=None, want_q=False):
    """One FP64 backup (Eq. 1). Returns (V', pi, residual, Q or None)."""
    lib = _load()
    shape, cell, R = _prep(gw)
    S, A = R.size, 2 * len(gw.shape)
    V = np.ascontiguousarray(np.asarray(V, dtype=np.float64).reshape(-1))
    out = np.empty(S)
    pi = np.empty(S, dtype=np.uint8)
    Q = np.empty(A * S) if want_q else None
    fp = None if fixed_pi is None else np.ascontiguousarray(
        np.asarray(fixed_pi, dtype=np.uint8).reshape(-1))
    res = lib.oracle_gw_backup(len(gw.shape), shape.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                               gw.p, gw.gamma, _ptr(cell), _ptr(R), _ptr(V), _ptr(out),
                               _ptr(fp), _ptr(pi), _ptr(Q))
    return out, pi, res, (Q.reshape(A, S) if want_q else None)


def value_iteration(gw, tol=1e-6, max_iter=1000, V0=None):
    """FP64 value iteration to max |dV| < tol. Returns (V, pi, sweeps, residual)."""
    lib = _load()
    shape, cell, R = _prep(gw)
    V = np.zeros(R.size) if V0 is None else np.array(V0, dtype=np.float64).reshape(-1)
    pi = np.empty(R.size, dtype=np.uint8)
    res = ctypes.c_double(0.0)
    k = lib.oracle_gw_value_iteration(len(gw.shape),
                                      shape.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                      gw.p, gw.gamma, _ptr(cell), _ptr(R), _ptr(V), _ptr(pi),
                                      tol, int(max_iter), ctypes.cast(ctypes.pointer(res),
                                                                      ctypes.c_void_p))
    if k < 0:
        raise MemoryError("oracle value iteration: out of memory")
    return V, pi, k, res.value


def evaluate(gw, pi, tol=1e-12, max_iter=100000, V0=None):
    """FP64 iterative evaluation of the fixed policy ``pi``."""
    lib = _load()
    shape, cell, R = _prep(gw)
    V = np.zeros(R.size) if V0 is None else np.array(V0, dtype=np.float64).reshape(-1)
    pi = np.ascontiguousarray(np.asarray(pi, dtype=np.uint8).reshape(-1))
    res = ctypes.c_double(0.0)
    k = lib.oracle_gw_evaluate(len(gw.shape), shape.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                               gw.p, gw.gamma, _ptr(cell), _ptr(R), _ptr(pi), _ptr(V), tol,
                               int(max_iter), ctypes.cast(ctypes.pointer(res), ctypes.c_void_p))
    if k < 0:
        raise MemoryError("oracle policy evaluation: out of memory")
    return V, k, res.value


def policy_iteration(gw, eval_tol=1e-12, max_rounds=1000, keep_margin=1e-12, pi0=None):
    """Policy iteration (background section) with iterative FP64 evaluation
    to ``eval_tol``; an action changes only if another beats it by more than
    ``keep_margin * (1 + |Q|)``. Stops when no action changes.
    Returns (V, pi, rounds)."""
    S = int(np.prod(gw.shape))
    cell = np.asarray(gw.cell, dtype=np.uint8).reshape(-1)
    free = cell == 0
    if pi0 is None:
        _, pi, _, _ = backup(gw, np.zeros(S))
    else:
        pi = np.asarray(pi0, dtype=np.uint8).reshape(-1).copy()
    pi = np.where(free, pi, 255).astype(np.uint8)
    V = np.zeros(S)
    rounds = 0
    idx = np.arange(S)
    for rounds in range(1, max_rounds + 1):
        V, _, _ = evaluate(gw, pi, tol=eval_tol, V0=V)
        _, _, _, Q = backup(gw, V, want_q=True)
        best = Q.argmax(axis=0)
        old = np.where(free, pi, 0).astype(np.int64)
        better = Q[best, idx] > Q[old, idx] + keep_margin * (1.0 + np.abs(Q[old, idx]))
        newpi = np.where(free & better, best, pi).astype(np.uint8)
        if np.array_equal(newpi, pi):
            break
        pi = newpi
    return V, pi, rounds


def q_states(gw, V, states):
    """Q(s, .) in FP64 for the given flat states only: array (len(states), A)."""
    lib = _load()
    shape, cell, R = _prep(gw)
    V = np.ascontiguousarray(np.asarray(V, dtype=np.float64).reshape(-1))
    st = np.ascontiguousarray(np.asarray(states, dtype=np.int64).reshape(-1))
    A = 2 * len(gw.shape)
    Q = np.empty(st.size * A)
    lib.oracle_gw_q_states(len(gw.shape), shape.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                           gw.p, gw.gamma, _ptr(cell), _ptr(R), _ptr(V), _ptr(st), st.size, _ptr(Q))
    return Q.reshape(st.size, A)
