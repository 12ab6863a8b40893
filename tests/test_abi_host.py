"""Host-side tests of libcpmdp: no GPU needed, no kernel launched.

The library loads, exports every function include/cpmdp.h declares, builds
host-only factor objects (device = -1) whose Definition 3 components equal
the oracle's rule-based tabular P, and rejects invalid problems with
CPMDP_EINVAL and a message.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import cpmdp_inputs as ci
from oracle import tabular as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cp():
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2103_00331_gb300 as cp
    return cp


def test_header_symbols_exported(cp):
    hdr = open(os.path.join(ROOT, "include", "cpmdp.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = set(re.findall(r"\b(cpmdp_[a-z0-9_]+)\s*\(", hdr))
    assert {"cpmdp_build_factors", "cpmdp_bellman_backup", "cpmdp_value_iteration",
            "cpmdp_policy_iteration"} <= names
    lib = ctypes.CDLL(cp.LIB_PATH)
    for n in sorted(names):
        assert hasattr(lib, n), f"{n} declared in cpmdp.h but not exported"
    assert set(cp.EXPORTED) == names


def test_version_and_defaults(cp):
    assert "sm_103a" in cp.version()
    o = cp.default_opts()
    assert o.tol == 1e-6 and o.max_iter == 1000 and o.certify == 1 and o.fused == 1
    assert o.partial_eval == -1   # the per-model default evaluation cap


CASES = [
    ((3, 4), 0.8, 0.2, 0), ((2, 3, 4), 0.7, 0.15, 1), ((7,), 0.9, 0.3, 2),
    ((3, 2, 2, 3), 0.6, 0.1, 3), ((2, 2, 2, 2, 2, 2, 2, 2, 2), 0.8, 0.1, 4),
    ((1, 5), 0.8, 0.0, 5), ((4, 1, 3), 0.5, 0.2, 6), ((2, 3, 2, 2, 2), 1.0, 0.2, 7),
]


@pytest.mark.parametrize("shape,p,orate,seed", CASES)
def test_components_match_tabular(cp, shape, p, orate, seed):
    """Definition 3 components from the library's factor object equal the
    oracle's P(s'|s,a), built from the GridWorld rules, for every (s, a)."""
    gw = ci.gridworld(shape, p=p, gamma=0.9, step_reward=-0.04, goal_rewards=[1.0],
                      obstacle_rate=orate, seed=seed)
    P = T.transition_tabular(shape, gw.cell, p)
    f = cp.build_factors(gw, device=-1)
    info = f.info()
    D = len(shape)
    assert info == {"nstates": gw.nstates, "nactions": 2 * D,
                    "rank": 2 if D == 1 else 2 * D - 1, "ndim": D}
    for s in range(gw.nstates):
        for a in range(2 * D):
            comps = cp.components(f, s, a)
            want = [(int(t), float(P[a, s, t])) for t in np.flatnonzero(P[a, s] > 0)]
            assert [c[0] for c in comps] == [w[0] for w in want], (s, a)
            np.testing.assert_allclose([c[1] for c in comps], [w[1] for w in want],
                                       rtol=0, atol=1e-15)
    f.close()


def _bad(cp, **kw):
    gw = ci.gridworld((4, 5), p=0.8, gamma=0.9, step_reward=-0.04, goal_rewards=[1.0], seed=0)
    reward = np.ascontiguousarray(gw.reward.reshape(-1))
    cell = np.ascontiguousarray(gw.cell.reshape(-1))
    args = dict(shape=(4, 5), nactions=4, kind=cp.GRIDWORLD, reward=reward, gamma=0.9,
                p_success=0.8, cell=cell)
    args.update(kw)
    pr = cp.make_problem(**args)
    with pytest.raises(cp.CpmdpError) as ei:
        cp.build_factors(pr, device=-1)
    assert ei.value.status == cp.EINVAL
    assert cp.last_error()
    return cp.last_error()


def test_invalid_problems_rejected(cp):
    assert "nactions" in _bad(cp, nactions=3)
    assert "p_success" in _bad(cp, p_success=1.5)
    assert "gamma" in _bad(cp, gamma=-0.1)
    assert "gamma" in _bad(cp, gamma=1.01)
    r = np.zeros(20)
    r[3] = np.nan
    assert "reward" in _bad(cp, reward=r)
    c = np.zeros(20, dtype=np.uint8)
    c[7] = 3
    assert "cell" in _bad(cp, cell=c)
    assert "shape" in _bad(cp, shape=(4, 0))
    assert "kind" in _bad(cp, kind=7)


def test_dense_validation(cp):
    dc = ci.dense_cp((3, 4), nactions=2, rank=2, gamma=0.9, seed=1)
    f = cp.build_factors(dc, device=-1)
    assert f.info() == {"nstates": 12, "nactions": 2, "rank": 2, "ndim": 2}
    fac = dc.packed_factors().copy()
    fac[0] += 0.01   # row 0 of U_{0,0,0} no longer sums to 1
    reward = np.ascontiguousarray(dc.reward.reshape(-1))
    lam = np.ascontiguousarray(dc.lam.reshape(-1))
    pr = cp.make_problem(dc.shape, 2, cp.DENSE_CP, reward, 0.9, factors=fac, lam=lam, rank=2)
    with pytest.raises(cp.CpmdpError) as ei:
        cp.build_factors(pr, device=-1)
    assert ei.value.status == cp.EINVAL and "sums to" in cp.last_error()
    with pytest.raises(cp.CpmdpError):
        cp.components(f, 0, 0)


def test_solvers_refuse_host_only_factors(cp):
    gw = ci.config_small_2d(0)
    f = cp.build_factors(gw, device=-1)
    V = np.zeros(gw.nstates)
    for call in (lambda: cp.value_iteration(f, cp.F64, V),
                 lambda: cp.bellman_backup(f, cp.F64, V, V.copy()),
                 lambda: cp.policy_iteration(f, cp.F64, V, np.zeros(100, np.uint8))):
        with pytest.raises(cp.CpmdpError) as ei:
            call()
        assert ei.value.status == cp.EINVAL and "host-only" in cp.last_error()


def _c_struct_fields(hdr, name):
    """(field, C type) of `typedef struct { ... } name;` in declaration order."""
    body = re.search(r"typedef struct \{((?:(?!typedef struct).)*?)\}\s*" + name + r";", hdr, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    return [(n, t + p) for t, p, n in re.findall(r"\b(double|int32_t|int64_t)\s*(\*?)\s*(\w+)\s*;", body)]


def test_ctypes_structs_match_header(cp):
    """The binding's SolveOpts / Result mirror cpmdp_solve_opts / cpmdp_result
    field for field (names, order, types), so results are not misread when
    the header grows a field."""
    hdr = open(os.path.join(ROOT, "include", "cpmdp.h")).read()
    ctype = {"double": ctypes.c_double, "int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64,
             "double*": ctypes.c_void_p}
    for cname, pycls in (("cpmdp_solve_opts", cp.SolveOpts), ("cpmdp_result", cp.Result)):
        c = _c_struct_fields(hdr, cname)
        py = list(pycls._fields_)
        assert [n for n, _ in c] == [n for n, _ in py], cname
        for (n, ct), (_, pt) in zip(c, py):
            assert ctype[ct] is pt, (cname, n)
