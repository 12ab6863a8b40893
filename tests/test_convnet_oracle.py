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
    assert np.all(V0[(gw.cell == 1)] == 0) and np.all(V0[gw.cell == 2] == gw.reward[gw.cell == 2])


def test_trilinear_upsample_closed_forms():
    """Trilinear interpolation between cell centres: a constant coarse array
    gives that constant everywhere; a coarse array linear in the cell index
    (a z_c + b y_c + c x_c + d) gives, between the outermost centres, the
    same linear function of the fine coordinate in cell units
    (x + 0.5) / 4 - 0.5, and is clamped to the edge centres outside them."""
    shape = (13, 9, 10)
    gw = ci.GridWorld(shape=shape, p=0.8, gamma=0.9, cell=np.zeros(shape, np.uint8), reward=np.zeros(shape))
    cs = (4, 3, 3)
    assert np.allclose(N.upsample(gw, np.full(cs, 0.37)), 0.37)
    a, b, c, d = 0.5, -1.25, 2.0, 0.1
    C = np.fromfunction(lambda z, y, x: a * z + b * y + c * x + d, cs)
    V0 = N.upsample(gw, C)

    def u(p, n):
        return min(max((p + 0.5) / 4 - 0.5, 0.0), n - 1.0)
    for z, y, x in [(0, 0, 0), (5, 4, 7), (12, 8, 9), (7, 1, 3), (2, 6, 8)]:
        want = a * u(z, 4) + b * u(y, 3) + c * u(x, 3) + d
        assert V0[z, y, x] == pytest.approx(want, abs=1e-12)


def test_coarse_gridworld_rules_and_closed_form():
    """The coarse copy: cells with at least half obstacles are obstacles,
    cells holding terminals are terminals with the largest terminal reward;
    and with a constant reward r, no obstacles and no terminals, the coarse
    value r (1 + ... + gamma^3) / (1 - gamma^4) equals the fine closed form
    r / (1 - gamma) exactly (geometric series)."""
    from oracle import cpfactor as oc
    shape = (8, 8, 6)
    cell = np.zeros(shape, np.uint8)
    cell[0:4, 0:4, 0:2] = 1                      # 32 of 64: an obstacle cell
    cell[4:8, 0:4, 0:1] = 1                      # 16 of 64: stays free
    cell[5, 6, 5] = 2
    cell[6, 7, 4] = 2
    R = np.full(shape, -0.02)
    R[cell == 1] = 0.0
    R[5, 6, 5], R[6, 7, 4] = 0.4, 0.9
    gw = ci.GridWorld(shape=shape, p=0.8, gamma=0.95, cell=cell, reward=R)
    cg, kind = N.coarse_gridworld(gw)
    assert cg.shape == (2, 2, 2) and kind[0, 0, 0] == 1 and kind[1, 0, 0] == 0
    assert kind[1, 1, 1] == 2 and cg.reward[1, 1, 1] == 0.9
    assert cg.gamma == pytest.approx(0.95 ** 4)
    free = (cell[4:8, 0:4, 0:4] == 0)
    assert cg.reward[1, 0, 0] == pytest.approx(-0.02 * sum(0.95 ** j for j in range(4)))
    assert free.sum() == 48
    r, g = -0.03, 0.97
    flat = ci.GridWorld(shape=(12, 8, 8), p=0.8, gamma=g, cell=np.zeros((12, 8, 8), np.uint8),
                        reward=np.full((12, 8, 8), r))
    cf, _ = N.coarse_gridworld(flat)
    Vc, _, _, _ = oc.value_iteration(cf, tol=1e-13, max_iter=100000)
    assert np.allclose(Vc, r / (1 - g), atol=1e-10)


def test_bf16_round_against_torch():
    torch = pytest.importorskip("torch")
    vals = np.concatenate([ci.random_values((4096,), seed=30, lo=-50, hi=50),
                           [1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 0.0, 1e-30, 3.0e38]])
    want = torch.as_tensor(vals.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(N.bf16_round(vals), want)
    assert N.bf16_round([1.0 + 2.0 ** -8])[0] == 1.0          # tie to even
    assert N.bf16_round([1.0 + 3 * 2.0 ** -8])[0] == 1.0 + 2.0 ** -6


def test_fine_loss_gradient_against_finite_differences():
    """The fine-level loss is quadratic in the coarse estimate, so central
    differences give its gradient exactly up to rounding: every cell's
    derivative is checked, including cells at the clamped edges, on a grid
    whose sides are not multiples of 4. The loss vanishes when the target
    is the upsampling itself, and the gradient then too."""
    gw = ci.gridworld((9, 7, 6), p=0.8, gamma=0.95, step_reward=-0.01, goal_rewards=[0.7, 0.9],
                      obstacle_rate=0.15, seed=8)
    cs = (3, 2, 2)
    rng = np.random.default_rng(3)
    C = rng.normal(size=cs)
    Vt = ci.random_values(gw.shape, seed=9)
    loss, grad = N.fine_loss_grad(gw, Vt, C)
    assert loss > 0
    eps = 1e-4
    for c in np.ndindex(cs):
        Cp, Cm = C.copy(), C.copy()
        Cp[c] += eps
        Cm[c] -= eps
        fd = (N.fine_loss_grad(gw, Vt, Cp)[0] - N.fine_loss_grad(gw, Vt, Cm)[0]) / (2 * eps)
        assert grad[c] == pytest.approx(fd, rel=1e-7, abs=1e-10)
    l0, g0 = N.fine_loss_grad(gw, N.upsample(gw, C), C)
    assert l0 == 0.0 and np.all(g0 == 0.0)
