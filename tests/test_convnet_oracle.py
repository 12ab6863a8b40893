"""Pins of the warm-start network oracle (FP64, CPU)."""
import numpy as np
import pytest

import cpmdp_inputs as ci
from oracle import convnet as N


def _rand(shape, seed):
    return ci.random_values(shape, seed=seed).reshape(shape)


def test_conv_forward_against_loops():
    x = _rand((2, 3, 4, 5, 3), 1)
    w = _rand((27, 2, 3), 2)
    b = _rand((2,), 3).reshape(-1)
    for d in (1, 2):
        y = N.conv_forward(x, w, b, d)
        ref = np.zeros(y.shape)
        for n in range(2):
            for z in range(3):
                for yy in range(4):
                    for xx in range(5):
                        for co in range(2):
                            acc = b[co]
                            for t, (oz, oy, ox) in enumerate(N.offsets()):
                                zz, y2, x2 = z + d * oz, yy + d * oy, xx + d * ox
                                if 0 <= zz < 3 and 0 <= y2 < 4 and 0 <= x2 < 5:
                                    acc += sum(x[n, zz, y2, x2, ci] * w[t, co, ci] for ci in range(3))
                            ref[n, z, yy, xx, co] = acc
        np.testing.assert_allclose(y, ref, rtol=0, atol=1e-12)


def test_identity_kernel():
    x = _rand((1, 4, 3, 5, 4), 4)
    w = np.zeros((27, 4, 4))
    w[13] = np.eye(4)
    np.testing.assert_array_equal(N.conv_forward(x, w, np.zeros(4), 3), x)


def test_backward_against_finite_differences():
    rng = np.random.default_rng(0)
    params = [(rng.normal(size=(27, 5, 3)) * 0.3, rng.normal(size=5) * 0.1, 1),
              (rng.normal(size=(27, 4, 5)) * 0.3, rng.normal(size=4) * 0.1, 2),
              (rng.normal(size=(27, 2, 4)) * 0.3, rng.normal(size=2) * 0.1, 1)]
    x = rng.normal(size=(2, 4, 3, 5, 3))
    target = rng.normal(size=(2, 4, 3, 5))
    mask = (rng.random(size=(2, 4, 3, 5)) > 0.2).astype(float)
    acts = N.net_forward(x, params)
    grads = N.net_backward(acts, params, target, mask)

    def loss(ps):
        return N.net_loss(N.net_forward(x, ps)[-1], target, mask)

    eps = 1e-6
    for li in range(3):
        w, b, d = params[li]
        for idx in [(0, 0, 0), (13, 1, 2), (26, len(b) - 1, w.shape[2] - 1), (5, 0, 1)]:
            wp, wm = w.copy(), w.copy()
            wp[idx] += eps
            wm[idx] -= eps
            pp = [p if i != li else (wp, b, d) for i, p in enumerate(params)]
            pm = [p if i != li else (wm, b, d) for i, p in enumerate(params)]
            fd = (loss(pp) - loss(pm)) / (2 * eps)
            assert abs(fd - grads[li][0][idx]) <= 1e-6 * max(1.0, abs(fd)), (li, idx, fd, grads[li][0][idx])
        bp, bm = b.copy(), b.copy()
        bp[0] += eps
        bm[0] -= eps
        fd = (loss([p if i != li else (w, bp, d) for i, p in enumerate(params)]) -
              loss([p if i != li else (w, bm, d) for i, p in enumerate(params)])) / (2 * eps)
        assert abs(fd - grads[li][1][0]) <= 1e-6 * max(1.0, abs(fd))


def test_features_target_upsample():
    gw = ci.gridworld((9, 8, 5), p=0.8, gamma=0.95, step_reward=-0.01, goal_rewards=[0.7, 0.9],
                      obstacle_rate=0.2, seed=4)
    f = N.features(gw)
    assert f.shape == (3, 2, 2, 4)
    assert np.allclose(f[..., 3], -np.log(0.05) / 5)
    # a cell's obstacle fraction counts only the states inside the grid
    blk = gw.cell[8:9, 4:8, 4:5]
    assert f[2, 1, 1, 1] == pytest.approx((blk == 1).mean())
    V = ci.random_values(gw.shape, seed=5)
    t, m = N.coarse_target(gw, V)
    live = gw.cell[0:4, 0:4, 0:4] != 1
    assert t[0, 0, 0] == pytest.approx(V[0:4, 0:4, 0:4][live].mean())
    V0 = N.upsample(gw, t)
    assert V0.shape == gw.shape
    free = gw.cell == 0
    assert np.all(V0[(gw.cell == 1)] == 0) and np.all(V0[gw.cell == 2] == gw.reward[gw.cell == 2])
    assert V0[5, 6, 3] == (t[1, 1, 0] if free[5, 6, 3] else V0[5, 6, 3])


def test_bf16_round_against_torch():
    torch = pytest.importorskip("torch")
    vals = np.concatenate([ci.random_values((4096,), seed=30, lo=-50, hi=50),
                           [1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 0.0, 1e-30, 3.0e38]])
    want = torch.as_tensor(vals.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(N.bf16_round(vals), want)
    assert N.bf16_round([1.0 + 2.0 ** -8])[0] == 1.0          # tie to even
    assert N.bf16_round([1.0 + 3 * 2.0 ** -8])[0] == 1.0 + 2.0 ** -6
