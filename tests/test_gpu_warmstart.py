"""Warm-start network on the GPU against the FP64 oracle (oracle/convnet.py).

Inputs and weights are rounded to bf16 on the host (round to nearest even,
torch CPU) and the oracle evaluates the same rounded values in float64, so
the only differences are FP32 accumulation and the bf16 rounding of outputs
and intermediate activations:
* one convolution: |y - y_ref| <= 2^-8 |y_ref| + 1e-5 sum|x||w| (bf16 output);
* weight / bias gradients (FP32 outputs): <= 1e-4 of sum|dy||x|;
* whole-network gradients against the oracle with the network's bf16
  storage points (activations and inter-layer gradients rounded to bf16,
  oracle/convnet.py bf16=True): what remains is FP32 vs FP64 accumulation
  (about 1e-6) and the few elements whose accumulated value lands on the
  other side of a bf16 rounding boundary (a 2^-8 relative step each, on a
  small fraction f of elements, amplified through the remaining layers):
  per-layer relative error (Frobenius) <= 5e-3, and element by element
  within 2^-5 of the element plus 2^-5 of the layer's largest gradient.
"""
import numpy as np
import pytest

import cpmdp_inputs as ci

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2103_00331_gb300 as cp
    from paper_2103_00331_gb300 import warmstart as ws
    return cp, ws, torch


def _bf16(a, torch):
    """Round float64 values to bf16 on the host; returns (bf16 tensor, float64 values)."""
    t = torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t, t.to(torch.float64).numpy()


@pytest.mark.parametrize("dims,dils", [((2, 3, 4, 5), (1, 2)), ((3, 7, 9, 11), (1, 4)), ((5, 8, 8, 8), (1, 3)),
                                       ((2, 16, 16, 16), (2, 4)), ((40, 16, 16, 16), (1,))])
def test_conv_kernels_match_oracle(env, dims, dils):
    """Tensor-core convolutions fed by tensor copies (tiles of 128 voxels,
    batches of 4 tiles per CTA): tiles larger than the grid (8 x 4 x 4 boxes
    on a 5 x 4 x 3 grid), ragged one-plane tiles whose three oy taps share
    one tall box (dilations 1 and 4, taps that leave the grid), two-plane
    tiles with three boxes per tap group (8^3, odd dilation 3), the 16^3
    coarse grid of the 64^3 instances (tall boxes of 12 and 16 rows), and
    320 batches over the SMs, so every CTA reuses both accumulator sets."""
    cp, ws, torch = env
    from oracle import convnet as N
    shp = dims + (64,)
    xb, x = _bf16(ci.random_values(shp, seed=1), torch)
    dyb, dy = _bf16(ci.random_values(shp, seed=2), torch)
    w32 = (ci.random_values((27, 64, 64), seed=3) * 0.1).astype(np.float32)
    wq = torch.as_tensor(w32).to(torch.bfloat16).to(torch.float64).numpy()
    b = (ci.random_values((64,), seed=4) * 0.1).astype(np.float32)
    dev = torch.device("cuda")
    wt = torch.as_tensor(w32).to(dev)
    wf = torch.empty((27, 64, 64), dtype=torch.bfloat16, device=dev)
    wb = torch.empty_like(wf)
    cp.ws_cast_weights(wt, wf, wb, 1)
    xg, dyg = xb.to(dev).reshape(-1, 64), dyb.to(dev).reshape(-1, 64)
    for dil in dils:
        y = torch.empty_like(xg)
        y0 = torch.empty(xg.shape[0], dtype=torch.float32, device=dev)
        cp.conv3d_forward(xg, wf, torch.as_tensor(b).to(dev), y, y0, dims, dil, relu=False)
        cp.ws_sync()
        ref = N.conv_forward(x, wq, b.astype(np.float64), dil).reshape(-1, 64)
        mag = N.conv_forward(np.abs(x), np.abs(wq), np.zeros(64), dil).reshape(-1, 64)
        got = y.to(torch.float64).cpu().numpy()
        assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-5 * mag + 1e-6)
        np.testing.assert_allclose(y0.cpu().numpy(), ref[:, 0], rtol=1e-5, atol=1e-5)
        # data gradient with the ReLU mask of an input activation
        act = torch.as_tensor(np.asarray(ci.random_values(shp, seed=5), np.float32)).to(torch.bfloat16).to(dev)
        act_mask = act.to(torch.float64).cpu().numpy().reshape(shp) > 0
        dx = torch.empty_like(dyg)
        cp.conv3d_backward_data(dyg, wb, act.reshape(-1, 64), dx, dims, dil)
        cp.ws_sync()
        dref, dWref, dbref = N.conv_backward(x, wq, dy, dil)
        dref = (dref * act_mask).reshape(-1, 64)
        dmag = N.conv_backward(np.abs(x), np.abs(wq), np.abs(dy), dil)[0].reshape(-1, 64)
        got = dx.to(torch.float64).cpu().numpy()
        assert np.all(np.abs(got - dref) <= 2.0 ** -8 * np.abs(dref) + 1e-5 * dmag + 1e-6)
        dW = torch.zeros((27, 64, 64), dtype=torch.float32, device=dev)
        db = torch.zeros(64, dtype=torch.float32, device=dev)
        cp.conv3d_backward_weight(xg, dyg, dW, db, dims, dil)
        wmag = N.conv_backward(np.abs(x), np.abs(wq), np.abs(dy), dil)[1]
        assert np.all(np.abs(dW.cpu().numpy() - dWref) <= 1e-4 * wmag + 1e-6)
        np.testing.assert_allclose(db.cpu().numpy(), dbref, rtol=1e-4, atol=1e-4)


def test_network_gradient_matches_oracle(env):
    cp, ws, torch = env
    from oracle import convnet as N
    net = ws.WarmStartNet(device=0, seed=3)
    dims = (2, 6, 5, 6)
    nv = int(np.prod(dims))
    f = np.zeros(dims + (64,))
    f[..., :net.n_feat] = ci.random_values(dims + (net.n_feat,), seed=8)
    fb, fq = _bf16(f, torch)
    tgt = ci.random_values(dims, seed=9).astype(np.float32)
    msk = (ci.uniform(0, 10, nv, 0, 1) > 0.2).astype(np.float32).reshape(dims)
    dev = net.dev
    feat = fb.to(dev).reshape(nv, 64)
    t = torch.as_tensor(tgt.reshape(-1)).to(dev)
    m = torch.as_tensor(msk.reshape(-1)).to(dev)
    w_before, b_before = net.numpy_params()
    net.train_step(feat, t, m, dims, lr=0.0)
    wq = [torch.as_tensor(w_before[i]).to(torch.bfloat16).to(torch.float64).numpy() for i in range(net.layers)]
    params = [(wq[i], b_before[i].astype(np.float64), net.dil[i]) for i in range(net.layers)]
    acts = N.net_forward(fq, params, bf16=True)
    acts[-1] = acts[-1].astype(np.float32).astype(np.float64)
    grads = N.net_backward(acts, params, tgt.astype(np.float64), msk.astype(np.float64), bf16=True)
    dW = net.dw.cpu().numpy()
    dB = net.db.cpu().numpy()
    for i in range(net.layers):
        gw, gb = grads[i]
        nrm = np.linalg.norm(gw)
        if nrm > 0:
            assert np.linalg.norm(dW[i] - gw) <= 5e-3 * nrm, (i, np.linalg.norm(dW[i] - gw) / nrm)
            # element by element: every weight gradient within 2^-5 of its own
            # value plus 2^-5 of the layer's largest (a wrong tap, channel or
            # sign moves whole groups of elements by their full size)
            top = np.abs(gw).max()
            err = np.abs(dW[i] - gw)
            assert np.all(err <= 2.0 ** -5 * (np.abs(gw) + top)), (i, float((err / (np.abs(gw) + top)).max()))
        assert np.linalg.norm(dB[i] - gb) <= 5e-3 * max(np.linalg.norm(gb), 1e-12), i
        assert np.all(np.abs(dB[i] - gb) <= 2.0 ** -5 * (np.abs(gb) + np.abs(gb).max() + 1e-12)), i


def test_features_targets_upsample(env):
    cp, ws, torch = env
    from oracle import convnet as N
    inst = [ci.gridworld((9, 8, 5), p=0.8, gamma=g, step_reward=-0.01, goal_rewards=[0.7, 0.9],
                         obstacle_rate=0.2, seed=s) for s, g in ((4, 0.95), (5, 0.9), (6, 0.99))]
    B = cp.batch_build(inst, device=0)
    dims = ws.coarse_dims(3, (9, 8, 5))
    cells = int(np.prod(dims[1:]))
    dev = torch.device("cuda")
    feat = torch.empty((3 * cells, 64), dtype=torch.bfloat16, device=dev)
    cp.ws_features(B, 0, 3, feat)
    Vh = np.concatenate([ci.random_values(g.shape, seed=11 + i).reshape(-1) for i, g in enumerate(inst)])
    V = torch.zeros(int(B.total_states), dtype=torch.float32, device=dev)
    for i, g in enumerate(inst):
        lo = int(B.offsets[i])
        V[lo:lo + g.nstates] = torch.as_tensor(Vh[i * 360:(i + 1) * 360].astype(np.float32))
    tgt = torch.empty(3 * cells, dtype=torch.float32, device=dev)
    msk = torch.empty_like(tgt)
    base = torch.as_tensor(ci.random_values((3 * cells,), seed=22).astype(np.float32)).to(dev)
    cp.ws_targets(B, V, 0, 3, tgt, msk, base=base)
    coarse = torch.as_tensor(ci.random_values((3 * cells,), seed=21).astype(np.float32)).to(dev)
    V0 = torch.zeros_like(V)
    cp.ws_upsample(B, coarse, 0, 3, V0, base=base)
    bh = base.cpu().numpy().astype(np.float64)
    fh = feat.to(torch.float64).cpu().numpy().reshape(3, cells, 64)
    for i, g in enumerate(inst):
        fo = N.features(g).reshape(cells, 4)
        assert np.all(np.abs(fh[i, :, :4] - fo) <= 2.0 ** -8 * np.abs(fo) + 1e-6)
        assert np.all(fh[i, :, 4:] == 0)
        Vi = Vh[i * 360:(i + 1) * 360].astype(np.float32).astype(np.float64)
        to, mo = N.coarse_target(g, Vi)
        bi = bh[i * cells:(i + 1) * cells]
        np.testing.assert_allclose(tgt.cpu().numpy()[i * cells:(i + 1) * cells], to.reshape(-1) - bi, rtol=1e-5,
                                   atol=1e-6)
        assert np.array_equal(msk.cpu().numpy()[i * cells:(i + 1) * cells], mo.reshape(-1))
        lo = int(B.offsets[i])
        ch = coarse.cpu().numpy()[i * cells:(i + 1) * cells].astype(np.float64)
        up = N.upsample(g, (ch + bi).reshape(dims[1:]))
        np.testing.assert_allclose(V0.cpu().numpy()[lo:lo + g.nstates], up.reshape(-1), rtol=1e-5, atol=1e-6)
    B.close()


def test_coarse_value_iteration_matches_oracle(env):
    """cpmdp_ws_coarse_vi (one CTA per instance, shared memory) against the
    oracle's value iteration of the coarse GridWorld it defines (cells of
    4^3 states, gamma^4, rewards of four fine steps), on 32^3 benchmark
    instances and ragged shapes: both stop below their tolerance, so they
    agree within (gamma_c tol + FP32 rounding) / (1 - gamma_c); channel 4 of
    the features holds the bf16 copy."""
    cp, ws, torch = env
    from oracle import convnet as N
    from oracle import cpfactor as oc
    groups = [ws.training_instances(6, 32, seed=31),
              [ci.gridworld((9, 8, 5), p=0.7, gamma=g, step_reward=-0.02, goal_rewards=[0.7, -0.3],
                            obstacle_rate=0.3, seed=s) for s, g in ((8, 0.93), (9, 0.99))]]
    for inst in groups:
        n = len(inst)
        B = cp.batch_build(inst, device=0)
        dims = ws.coarse_dims(n, inst[0].shape)
        cells = int(np.prod(dims[1:]))
        cv = torch.empty(n * cells, dtype=torch.float32, device="cuda")
        feat = torch.zeros((n * cells, 64), dtype=torch.bfloat16, device="cuda")
        tol = 1e-5
        cp.ws_coarse_vi(B, 0, n, cv, feat, tol=tol, max_sweeps=100000)
        got = cv.cpu().numpy().astype(np.float64).reshape(n, cells)
        f4 = feat[:, 4].float().cpu().numpy().reshape(n, cells)
        for i, g in enumerate(inst):
            cg, kind = N.coarse_gridworld(g)
            Vo, _, _, _ = oc.value_iteration(cg, tol=1e-12, max_iter=1000000)
            gc = cg.gamma
            bound = (gc * tol + 8 * 2.0 ** -24 * (np.abs(Vo).max() + np.abs(cg.reward).max())) / (1 - gc)
            assert np.abs(got[i] - Vo.reshape(-1)).max() <= bound, (i, np.abs(got[i] - Vo.reshape(-1)).max(), bound)
            assert np.all(np.abs(f4[i] - got[i]) <= 2.0 ** -8 * np.abs(got[i]) + 1e-30)
        B.close()


def test_fine_loss_grad_matches_oracle(env):
    """ws_fine_loss_grad against oracle/convnet.fine_loss_grad on three
    instances of a shape that is not a multiple of 4 (clamped edge cells):
    residuals and loss within FP32 rounding, the gradient (bf16 in dy
    channel 0) within 2^-8 of each element plus 1e-6 of the largest, and
    channels 1..63 zero."""
    cp, ws, torch = env
    from oracle import convnet as N
    shape = (10, 9, 7)
    inst = [ci.gridworld(shape, p=0.8, gamma=0.95, step_reward=-0.01, goal_rewards=[0.6, 0.9],
                         obstacle_rate=0.15, seed=60 + i) for i in range(3)]
    B = cp.batch_build(inst, device=0)
    dev = torch.device("cuda", 0)
    cs = (3, 3, 2)
    cells = int(np.prod(cs))
    pred = ci.random_values((3,) + cs, seed=61).astype(np.float32)
    base = ci.random_values((3,) + cs, seed=62).astype(np.float32)
    Vt = np.concatenate([ci.random_values(shape, seed=70 + i).astype(np.float32).reshape(-1) for i in range(3)])
    n = 3 * int(np.prod(shape))
    vt_dev = torch.zeros(int(B.total_states), dtype=torch.float32, device=dev)
    for i in range(3):
        o = int(B.offsets[i])
        vt_dev[o:o + int(np.prod(shape))] = torch.as_tensor(Vt[i * int(np.prod(shape)):(i + 1) * int(np.prod(shape))])
    p_dev = torch.as_tensor(pred.reshape(-1)).to(dev)
    b_dev = torch.as_tensor(base.reshape(-1)).to(dev)
    resid = torch.empty(n, dtype=torch.float32, device=dev)
    dy = torch.full((3 * cells, 64), 7.0, dtype=torch.bfloat16, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    cp.ws_fine_loss_grad(B, vt_dev, 0, 3, p_dev, b_dev, resid, dy, loss)
    ws.ws_sync()
    got_r = resid.cpu().numpy().reshape(3, -1)
    got_g = dy[:, 0].float().cpu().numpy().reshape((3,) + cs)
    assert np.all(dy[:, 1:].float().cpu().numpy() == 0.0)
    want_loss = 0.0
    for i, gw in enumerate(inst):
        coarse = pred[i].astype(np.float64) + base[i].astype(np.float64)
        vt = Vt[i * int(np.prod(shape)):(i + 1) * int(np.prod(shape))].astype(np.float64)
        li, gi = N.fine_loss_grad(gw, vt, coarse, n=n)
        want_loss += li
        want_r = np.where(np.asarray(gw.cell) == 0, N.upsample(gw, coarse) - vt.reshape(shape), 0.0).reshape(-1)
        np.testing.assert_allclose(got_r[i], want_r, rtol=0, atol=1e-5)
        top = np.abs(gi).max()
        assert np.all(np.abs(got_g[i] - gi) <= 2.0 ** -8 * np.abs(gi) + 1e-6 * top), i
    assert float(loss.item()) == pytest.approx(want_loss, rel=1e-4)
    B.close()


def test_trained_network_saves_sweeps(env):
    """Train on 256 solved 32^3 instances with the full-grid loss, then
    warm-start value iteration on 24 held-out 32^3 instances: every instance
    still converges to |dV|inf < 1e-6 and ends at the zero start's fixed
    point; training lowers the loss; the coarse start alone and the
    network's start both need fewer sweeps in total than zero
    initialisation on the same instances."""
    cp, ws, torch = env
    chunk = ws.solved_chunk(ws.training_instances(256, 32, seed=1))
    net = ws.WarmStartNet(device=0, seed=0)
    losses = ws.train(net, [chunk], (32, 32, 32), epochs=30, batch=16, lr=1e-3, lr_final=5e-5)
    chunk[0].close()
    assert losses[-1] < losses[0], losses
    test_inst = ws.training_instances(24, 32, seed=777)
    B = cp.batch_build(test_inst, device=0)
    V = torch.zeros(int(B.total_states), dtype=torch.float32, device=net.dev)
    _, it_zero, res0 = cp.batch_value_iteration(B, V, opts=cp.default_opts(max_iter=5000))
    Vz = V.clone()
    ws.warm_start_values(None, B, 24, (32, 32, 32), V)
    _, it_coarse, resc = cp.batch_value_iteration(B, V, opts=cp.default_opts(max_iter=5000))
    ws.warm_start_values(net, B, 24, (32, 32, 32), V)
    _, it_warm, res1 = cp.batch_value_iteration(B, V, opts=cp.default_opts(max_iter=5000))
    assert np.all(res0 < 1e-6) and np.all(resc < 1e-6) and np.all(res1 < 1e-6)
    assert it_coarse.sum() < it_zero.sum(), (it_coarse.sum(), it_zero.sum())
    assert it_warm.sum() < it_zero.sum(), (it_warm.sum(), it_coarse.sum(), it_zero.sum())
    # both end at the same fixed point (within the stopping bound)
    g = max(x.gamma for x in test_inst)
    assert (V - Vz).abs().max().item() <= (2 * g * 1e-6 + 4e-6) / (1 - g)
    B.close()


def test_committed_network_saves_sweeps_at_64(env):
    """The committed weights (trained on 64^3 instances with the full-grid
    loss) on 8 held-out 64^3 instances of the config-5 recipe: the warm start
    needs fewer sweeps in total than zero initialisation, and both
    converge."""
    import os
    cp, ws, torch = env
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2103_00331_gb300",
                        "data", "warmstart_weights.npz")
    net = ws.WarmStartNet.load(path, device=0)
    test_inst = ws.training_instances(8, 64, seed=424243)
    B = cp.batch_build(test_inst, device=0)
    V = torch.zeros(int(B.total_states), dtype=torch.float32, device=net.dev)
    _, it_zero, res0 = cp.batch_value_iteration(B, V, opts=cp.default_opts(max_iter=5000))
    V.zero_()
    ws.warm_start_values(net, B, 8, (64, 64, 64), V)
    _, it_warm, res1 = cp.batch_value_iteration(B, V, opts=cp.default_opts(max_iter=5000))
    B.close()
    assert np.all(res0 < 1e-6) and np.all(res1 < 1e-6)
    assert it_warm.sum() < it_zero.sum(), (it_warm.sum(), it_zero.sum())
