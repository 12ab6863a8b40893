"""GPU parity of the dense BF16x3 tensor-core path (64^4) against the FP64 oracle.

BF16x3 error bound (derived): an operand x is held as hi + lo with
|x - hi - lo| <= 2^-18 |x|; the product drops lo_a lo_b (<= 2^-18 |ab|), so
each product is off by at most 3 2^-18 |ab|, and a 64-term sum with
row-stochastic weights by 3 2^-18 max|x| plus FP32 accumulation
(192 products: <= 192 2^-24 of the magnitude). The intermediate is rounded
to hi + lo again (2^-18). Four mode products and the rank sum give
|E_bf16x3 - E| <= 4 (3 2^-18 + 192 2^-24 + 2^-18) max|V| < 1.2e-4 max|V|,
so one backup is within gamma * 1.2e-4 * max|V| + FP32 rounding of Eq. 1.
"""
import numpy as np
import pytest

import cpmdp_inputs as ci

pytestmark = pytest.mark.gpu

BF16X3_REL = 4 * (3 * 2.0 ** -18 + 192 * 2.0 ** -24 + 2.0 ** -18)


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2103_00331_gb300 as cp
    dc = ci.config_dense_4d(side=64, seed=0)
    f = cp.build_factors(dc, device=0)
    yield cp, dc, f
    f.close()
    torch.cuda.empty_cache()


PICKS = [(0, 0, 0, 0), (63, 63, 63, 63), (5, 40, 17, 63), (31, 0, 62, 8), (12, 12, 50, 33),
         (63, 1, 0, 30), (7, 59, 3, 44)]


def test_bf16x3_one_sweep(setup):
    import torch
    from oracle import dense as od
    cp, dc, f = setup
    Vh = ci.random_values(dc.shape, seed=2, lo=-3, hi=3).reshape(-1).astype(np.float32)
    Vd = torch.as_tensor(Vh).cuda()
    out = torch.empty_like(Vd)
    pi = torch.empty(dc.nstates, dtype=torch.uint8, device="cuda")
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    cp.bellman_backup(f, cp.BF16X3, Vd, out, pi, res)
    torch.cuda.synchronize()
    tol = dc.gamma * BF16X3_REL * np.abs(Vh).max() + 1e-5
    Vt = Vh.astype(np.float64)
    for c in PICKS:
        s = int(np.ravel_multi_index(c, dc.shape))
        q = od.q_at(dc, Vt, c)
        assert abs(out[s].item() - q.max()) <= tol, (c, out[s].item(), q.max(), tol)
        qs = np.sort(q)
        if qs[-1] - qs[-2] > 2 * tol:
            assert pi[s].item() == int(q.argmax())
    # against the FP32 SIMT sweep on every state (a GPU-internal consistency check)
    out32 = torch.empty_like(Vd)
    cp.bellman_backup(f, cp.F32, Vd, out32, None, None)
    torch.cuda.synchronize()
    d = (out - out32).abs().max().item()
    assert d <= tol, d
    assert abs(res.item() - (out.double() - Vd.double()).abs().max().item()) <= 1e-6


def test_bf16x3_value_iteration(setup):
    """VI to max|dV| < 1e-6 with BF16x3 sweeps and FP32-base defect
    correction, stopped by the FP64 residual. The oracle's own FP64 backup
    of the returned V over all 16.8M states (Eq. 1 by mode products)
    re-derives the certified residual, which must be below tol, and the
    greedy policy, which must equal the GPU's FP64 argmax wherever the
    oracle's best and second-best Q differ by more than FP64 rounding. The
    certified residual bounds max|V - V*| by certified / (1 - gamma)."""
    import torch
    from oracle import dense as od
    cp, dc, f = setup
    V = torch.zeros(dc.nstates, dtype=torch.float32, device="cuda")
    pi = torch.zeros(dc.nstates, dtype=torch.uint8, device="cuda")
    r = cp.value_iteration(f, cp.BF16X3, V, pi, opts=cp.default_opts(max_iter=2000))
    assert r["status"] == cp.OK and r["eval_sweeps"] >= 1
    assert 0 <= r["certified_residual"] < 1e-6
    assert abs(r["error_bound"] - r["certified_residual"] / (1 - dc.gamma)) <= 1e-15
    Vt = V.double().cpu().numpy()
    pg = pi.cpu().numpy()
    Q = od.q_values(dc, Vt)
    TV = Q.max(axis=0)
    cert = float(np.abs(TV - Vt).max())
    # FP64 with different summation orders: agreement to a few ulps of |V|
    assert abs(cert - r["certified_residual"]) <= 1e-12, (cert, r["certified_residual"])
    top2 = np.partition(Q, -2, axis=0)[-2:]
    gap = np.abs(top2[1] - top2[0])
    sure = gap > 1e-10
    assert sure.mean() > 0.99
    assert np.array_equal(pg[sure], Q.argmax(axis=0)[sure].astype(np.uint8))


def test_bf16x3_vi_against_oracle_vi(setup):
    """The GPU's value iteration against the FP64 oracle's own value
    iteration of the same model from V = 0 (stored at 4096 seeded states by
    tests/golden/make_dense64_vi.py, which calls only the oracle). Both stop
    with an FP64 residual below 1e-6, so each is within its residual /
    (1 - gamma) of V*: the two agree within the sum of those bounds, and
    their policies agree wherever the oracle's Q gap exceeds twice gamma
    times that."""
    import os
    import torch
    path = os.path.join(os.path.dirname(__file__), "golden", "dense64_vi_samples.npz")
    if not os.path.exists(path):
        pytest.skip("golden samples not generated")
    g = np.load(path)
    cp, dc, f = setup
    V = torch.zeros(dc.nstates, dtype=torch.float32, device="cuda")
    pi = torch.zeros(dc.nstates, dtype=torch.uint8, device="cuda")
    r = cp.value_iteration(f, cp.BF16X3, V, pi, opts=cp.default_opts(max_iter=2000))
    idx = torch.as_tensor(g["state"]).cuda()
    got = V[idx].double().cpu().numpy()
    bound = (r["certified_residual"] + float(g["certified_residual"])) / (1 - dc.gamma)
    assert float(g["certified_residual"]) < 1e-6
    assert np.abs(got - g["value"]).max() <= bound
    sure = g["gap"] > 2 * dc.gamma * bound
    assert np.array_equal(pi[idx].cpu().numpy()[sure], g["policy"][sure])


def test_bf16x3_policy_iteration(setup):
    """Policy iteration on the tensor cores (BF16x3 evaluation sweeps with
    the defect correction, improvement by an evaluation-mode sweep, a max
    sweep and the keep-margin compare). The oracle's FP64 backup of all
    16.8M states of the returned V re-derives the certified residual; the
    returned policy equals the oracle's greedy policy of V wherever the
    oracle's Q gap exceeds twice gamma times the distance bound
    certified / (1 - gamma) plus the keep margin; the values agree with the
    FP32 SIMT policy iteration within the two results' bounds."""
    import torch
    from oracle import dense as od
    cp, dc, f = setup
    V = torch.zeros(dc.nstates, dtype=torch.float32, device="cuda")
    pi = torch.zeros(dc.nstates, dtype=torch.uint8, device="cuda")
    r = cp.policy_iteration(f, cp.BF16X3, V, pi, opts=cp.default_opts(max_iter=2000))
    assert r["status"] == cp.OK and r["rounds"] >= 1 and r["solver"] == cp.SOLVER_DENSE
    cert = r["certified_residual"]
    assert 0 <= cert < 1e-5
    Vt = V.double().cpu().numpy()
    pg = pi.cpu().numpy()
    Q = od.q_values(dc, Vt)
    assert abs(float(np.abs(Q.max(axis=0) - Vt).max()) - cert) <= 1e-12
    bound = cert / (1 - dc.gamma)
    top2 = np.partition(Q, -2, axis=0)[-2:]
    sure = np.abs(top2[1] - top2[0]) > 2 * dc.gamma * bound + 2e-6 * (1 + np.abs(Q).max(axis=0))
    assert sure.sum() > 100000
    assert np.array_equal(pg[sure], Q.argmax(axis=0)[sure].astype(np.uint8))
