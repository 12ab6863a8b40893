"""The dense solvers run their loops as recorded CUDA graphs (conditional
nodes), recorded once per buffers and options and replayed. These tests
change the options, buffers, precision and method between calls on one
factors object and check every call against the FP64 oracle's value
iteration of the same model (Eq. 1 iterated from V = 0), so that a replay of
a graph recorded for other options would show.

Collected with the other GPU tests (`-m gpu`)."""
import numpy as np
import pytest

import cpmdp_inputs as ci

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2103_00331_gb300 as cpm
    return cpm


def test_simt_graphs_follow_options(cp):
    import torch
    from oracle import dense as od
    dc = ci.dense_cp((6, 7, 5), 4, 3, 0.9, seed=8)
    f = cp.build_factors(dc, device=0)
    V = torch.zeros(dc.nstates, dtype=torch.float64, device="cuda")
    pi = torch.zeros(dc.nstates, dtype=torch.uint8, device="cuda")

    # a sweep limit: exactly that many sweeps, not converged, the oracle's iterate after them
    V5, _, _, res5 = od.value_iteration(dc, tol=0.0, max_iter=5)
    r = cp.value_iteration(f, cp.F64, V, pi, opts=cp.default_opts(max_iter=5), raise_on_noconv=False)
    assert r["iterations"] == 5 and r["status"] == cp.ENOCONV
    assert np.abs(V.cpu().numpy() - V5).max() <= 1e-12
    assert abs(r["residual"] - res5) <= 1e-12

    # the default options again (another graph): the oracle's sweep count and
    # values, and a per-sweep trace equal to the oracle's residuals
    Vo, pio, ko, _ = od.value_iteration(dc, tol=1e-6)
    trace_o, W = [], np.zeros(dc.nstates)
    for _ in range(ko):
        Wn, _, res = od.backup(dc, W)
        trace_o.append(res)
        W = Wn
    o = cp.default_opts()
    tr = torch.full((o.max_iter,), -1.0, dtype=torch.float64, device="cuda")   # max_iter doubles
    o.trace = tr.data_ptr()
    V.zero_()
    r = cp.value_iteration(f, cp.F64, V, pi, opts=o)
    assert r["iterations"] == ko and r["status"] == cp.OK
    assert np.abs(V.cpu().numpy() - Vo).max() <= 1e-12
    t = tr.cpu().numpy()
    assert np.allclose(t[:ko], trace_o, rtol=0, atol=1e-12)

    # policy iteration on the same factors, then value iteration once more
    Vs, _, _, _ = od.value_iteration(dc, tol=1e-13, max_iter=5000)
    Q = od.q_values(dc, Vs)
    Qs = np.sort(Q, axis=0)
    sure = (Qs[-1] - Qs[-2]) > 1e-6
    V.zero_()
    r = cp.policy_iteration(f, cp.F64, V, pi)
    assert r["status"] == cp.OK and r["rounds"] >= 1
    assert np.abs(V.cpu().numpy() - Vs).max() <= 1e-8
    assert np.array_equal(pi.cpu().numpy()[sure], Q.argmax(axis=0)[sure])
    V.zero_()
    r = cp.value_iteration(f, cp.F64, V, pi)
    assert r["iterations"] == ko
    assert np.abs(V.cpu().numpy() - Vo).max() <= 1e-12

    # FP32 on other buffers: the FP32 loop stops on its own residual, within
    # a sweep of the oracle's count, and lands within its bound of V*
    V32 = torch.zeros(dc.nstates, dtype=torch.float32, device="cuda")
    pi32 = torch.zeros(dc.nstates, dtype=torch.uint8, device="cuda")
    r = cp.value_iteration(f, cp.F32, V32, pi32)
    assert abs(r["iterations"] - ko) <= 1
    bound = (r["residual"] + 1e-5 * max(1.0, np.abs(Vs).max())) / (1 - dc.gamma)
    assert np.abs(V32.double().cpu().numpy() - Vs).max() <= bound
    V32.zero_()
    r = cp.policy_iteration(f, cp.F32, V32, pi32)
    assert r["status"] == cp.OK
    assert np.abs(V32.double().cpu().numpy() - Vs).max() <= bound
    # policies compared where the gap exceeds what the value error and the
    # FP32 keep margin (1e-6 (1 + |Q|)) can move
    sure32 = (Qs[-1] - Qs[-2]) > 2 * dc.gamma * bound + 2e-6 * (1 + np.abs(Q).max())
    assert sure32.sum() > 0
    assert np.array_equal(pi32.cpu().numpy()[sure32], Q.argmax(axis=0)[sure32])
