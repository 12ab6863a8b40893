"""GPU parity of the dense CP path (mode-product chains) against the FP64 oracle.

Tolerances: one FP64 sweep 1e-12 (max|R| + max|V|); one FP32 sweep: each of
the D mode products sums N_d non-negative-weight terms (row-stochastic
factors), so its rounding error is at most about (N_d + 2) u times the
largest |value|, and the lambda-weighted sum over R ranks adds R u:
|V32' - V64'| <= (sum_d (N_d + 2) + R + 4) u (max|R| + max|V|), u = 2^-24.
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


def _tol32(dc, V):
    n = sum(s + 2 for s in dc.shape) + dc.rank + 4
    return n * U32 * (np.abs(dc.reward).max() + np.abs(V).max())


@pytest.mark.parametrize("shape,A,R", [((6, 5, 4), 3, 2), ((8, 8, 8, 8), 4, 3), ((70, 33), 2, 5),
                                       ((130,), 3, 2), ((3, 65, 2, 7), 2, 1)])
@pytest.mark.parametrize("prec", [0, 1])
def test_dense_one_sweep(cp, shape, A, R, prec):
    import torch
    from oracle import dense as od
    dc = ci.dense_cp(shape, A, R, 0.95, seed=3)
    f = cp.build_factors(dc, device=0)
    dt = torch.float64 if prec == cp.F64 else torch.float32
    Vd = torch.as_tensor(ci.random_values(shape, seed=1, lo=-2, hi=2).reshape(-1)).to("cuda", dt)
    Vh = Vd.double().cpu().numpy()
    out = torch.empty_like(Vd)
    pi = torch.empty(dc.nstates, dtype=torch.uint8, device="cuda")
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    cp.bellman_backup(f, prec, Vd, out, pi, res)
    torch.cuda.synchronize()
    Q = od.q_values(dc, Vh)
    want = Q.max(axis=0)
    tol = _tol32(dc, Vh) if prec == cp.F32 else 1e-12 * (np.abs(dc.reward).max() + np.abs(Vh).max())
    got = out.double().cpu().numpy()
    assert np.abs(got - want).max() <= tol
    Qs = np.sort(Q, axis=0)
    sure = (Qs[-1] - Qs[-2]) > 2 * tol
    assert np.array_equal(pi.cpu().numpy()[sure], Q.argmax(axis=0)[sure])
    assert abs(res.item() - np.abs(want - Vh).max()) <= 2 * tol


def test_dense_vi_pi_small(cp):
    """FP64 VI and PI on a 6x7x5 dense model, 4 actions, rank 3: the VI
    sweep count and values match the oracle's VI; PI's policy equals the
    greedy policy of the oracle's V* where the gap exceeds 1e-6."""
    import torch
    from oracle import dense as od
    dc = ci.dense_cp((6, 7, 5), 4, 3, 0.9, seed=8)
    Vo, pio, ko, _ = od.value_iteration(dc, tol=1e-6)
    f = cp.build_factors(dc, device=0)
    V = torch.zeros(dc.nstates, dtype=torch.float64, device="cuda")
    pi = torch.zeros(dc.nstates, dtype=torch.uint8, device="cuda")
    r = cp.value_iteration(f, cp.F64, V, pi)
    assert r["iterations"] == ko
    assert np.abs(V.cpu().numpy() - Vo).max() <= 1e-12
    Vs, _, _, _ = od.value_iteration(dc, tol=1e-13, max_iter=5000)
    Q = od.q_values(dc, Vs)
    Qs = np.sort(Q, axis=0)
    sure = (Qs[-1] - Qs[-2]) > 1e-6
    assert np.array_equal(pi.cpu().numpy()[sure], Q.argmax(axis=0)[sure])
    V.zero_()
    r = cp.policy_iteration(f, cp.F64, V, pi)
    assert np.abs(V.cpu().numpy() - Vs).max() <= 1e-8
    assert np.array_equal(pi.cpu().numpy()[sure], Q.argmax(axis=0)[sure])


def test_dense_64_4_sampled(cp):
    """64^4 (16.8M states), 8 actions, rank 8, gamma 0.95: one FP32 sweep
    through the C ABI, checked on sampled states against the oracle's
    per-state FP64 Q (contraction of V with the factor rows)."""
    import torch
    from oracle import dense as od
    dc = ci.config_dense_4d(side=64, seed=0)
    f = cp.build_factors(dc, device=0)
    Vh = ci.random_values(dc.shape, seed=2, lo=-3, hi=3).reshape(-1).astype(np.float32)
    Vd = torch.as_tensor(Vh).cuda()
    out = torch.empty_like(Vd)
    pi = torch.empty(dc.nstates, dtype=torch.uint8, device="cuda")
    cp.bellman_backup(f, cp.F32, Vd, out, pi, None)
    torch.cuda.synchronize()
    tol = _tol32(dc, Vh)
    picks = [(0, 0, 0, 0), (63, 63, 63, 63), (5, 40, 17, 63), (31, 0, 62, 8), (12, 12, 50, 33), (63, 1, 0, 30)]
    Vt = Vh.astype(np.float64)
    for c in picks:
        s = int(np.ravel_multi_index(c, dc.shape))
        q = od.q_at(dc, Vt, c)
        assert abs(out[s].item() - q.max()) <= tol, (c, out[s].item(), q.max(), tol)
        qs = np.sort(q)
        if qs[-1] - qs[-2] > 2 * tol:
            assert pi[s].item() == int(q.argmax())
    f.close()
    del Vd, out, pi
    torch.cuda.empty_cache()
