"""Learned warm start for value iteration (driver over the library's kernels).

The start is built in two stages, both on the coarse grid of 4 x 4 x 4
cells. First, value iteration of the coarsened copy of each instance
(``ws_coarse_vi``: a cheap solve of a 64-times smaller GridWorld) gives a
coarse value per cell. Then a fully convolutional 3-D network reads the
cell features together with that coarse value and predicts a correction to
it. Value iteration starts from the corrected coarse values, upsampled
trilinearly to the full grid. Value iteration itself is unchanged: it still
runs to the same residual, and zero initialisation stays the fallback
against which the warm start is judged.

Network: dilated 3 x 3 x 3 convolutions (default dilations 1, 2, 1), 64
channels, ReLU after all but the last, output channel 0. The first layer
reads the 5 input channels (mean reward of the non-obstacle states, obstacle
fraction, largest terminal reward, -log(1 - gamma) / 5, the coarse value);
its other input weights stay zero, and the last layer writes only channel 0.
Weights are FP32 masters with bf16 copies for the convolution kernels;
activations are bf16 with FP32 accumulation; training uses Adam.

Training loss: the squared error of the upsampled start against V* on every
free state of the full grid (``ws_fine_loss_grad``), so the network learns
the coarse values whose interpolation is closest to V* state by state, not
the cell means (whose interpolation starts value iteration farther away).
Every arithmetic step runs in a libcpmdp kernel; this module only allocates
buffers and sequences the calls.
"""
from __future__ import annotations

import numpy as np

from . import (BF16X3, adam_step, batch_build, batch_value_iteration, conv3d_backward_data,  # noqa: F401
               conv3d_backward_weight, conv3d_forward, default_opts, ws_cast_weights, ws_coarse_vi, ws_features,
               ws_fine_loss_grad, ws_loss_grad, ws_sync, ws_targets, ws_upsample)

C = 64
FACTOR = 4
N_FEAT = 5
DILATIONS = (1, 2, 1)
COARSE_TOL = 1e-4


def coarse_dims(count, shape):
    return (int(count),) + tuple((int(n) + FACTOR - 1) // FACTOR for n in shape)


class WarmStartNet:
    def __init__(self, device=0, seed=0, init=None, dilations=DILATIONS, n_feat=N_FEAT):
        import torch
        import cpmdp_inputs as ci
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.dil = tuple(int(d) for d in dilations)
        self.layers = len(self.dil)
        self.n_feat = int(n_feat)
        L = self.layers
        if init is None:
            w = np.zeros((L, 27, C, C), dtype=np.float32)
            for layer in range(L):
                cin = self.n_feat if layer == 0 else C
                cout = 1 if layer == L - 1 else C
                std = np.sqrt(2.0 / (27 * cin)) * (0.5 if layer == L - 1 else 1.0)
                draw = ci.normal(seed * 100 + layer, 3, 27 * cout * cin).reshape(27, cout, cin) * std
                w[layer, :, :cout, :cin] = draw
            b = np.zeros((L, C), dtype=np.float32)
        else:
            w, b = init
        self.w = torch.as_tensor(np.ascontiguousarray(w, dtype=np.float32)).to(self.dev)
        self.b = torch.as_tensor(np.ascontiguousarray(b, dtype=np.float32)).to(self.dev)
        self.wf = torch.empty((L, 27, C, C), dtype=torch.bfloat16, device=self.dev)
        self.wb = torch.empty_like(self.wf)
        self.dw = torch.zeros_like(self.w)
        self.db = torch.zeros_like(self.b)
        self.mw, self.vw = torch.zeros_like(self.w), torch.zeros_like(self.w)
        self.mb, self.vb = torch.zeros_like(self.b), torch.zeros_like(self.b)
        self.step = 0
        self._cast()

    def _cast(self):
        ws_cast_weights(self.w, self.wf, self.wb, self.layers)

    def numpy_params(self):
        return self.w.cpu().numpy(), self.b.cpu().numpy()

    def save(self, path):
        w, b = self.numpy_params()
        np.savez(path, w=w, b=b, step=self.step, dilations=np.array(self.dil), n_feat=self.n_feat)

    @classmethod
    def load(cls, path, device=0):
        d = np.load(path)
        net = cls(device=device, init=(d["w"], d["b"]), dilations=tuple(d["dilations"]), n_feat=int(d["n_feat"]))
        net.step = int(d["step"])
        return net

    def forward(self, feat, dims):
        """Activations [feat, a1, ..., out] (bf16) and the FP32 output channel 0."""
        torch = self.torch
        nvox = int(np.prod(dims))
        acts = [feat]
        pred = torch.empty(nvox, dtype=torch.float32, device=self.dev)
        for layer in range(self.layers):
            last = layer == self.layers - 1
            y = torch.empty((nvox, C), dtype=torch.bfloat16, device=self.dev)
            conv3d_forward(acts[-1], self.wf[layer], self.b[layer], y, pred if last else None, dims,
                           self.dil[layer], relu=not last)
            acts.append(y)
        return acts, pred

    def predict(self, feat, dims):
        return self.forward(feat, dims)[1]

    def train_step(self, feat, target, mask, dims, lr=1e-3, loss_acc=None, fine=None):
        """One Adam step on a minibatch; adds the minibatch loss to loss_acc
        (device). The loss is the masked per-cell squared error against
        ``target``, or, with ``fine = (batch, V_target, first, base, resid)``,
        the full-grid error of upsample(prediction + base) against V_target
        for instances first..first+dims[0]-1 of that batch (``resid`` is
        scratch of one float per state)."""
        torch = self.torch
        nvox = int(np.prod(dims))
        acts, pred = self.forward(feat, dims)
        dy = torch.empty((nvox, C), dtype=torch.bfloat16, device=self.dev)
        if fine is None:
            ws_loss_grad(pred, target, mask, nvox, dy, loss_acc)
        else:
            b, vt, first, base, resid = fine
            ws_fine_loss_grad(b, vt, first, dims[0], pred, base, resid, dy, loss_acc)
        self.dw.zero_()
        self.db.zero_()
        for layer in range(self.layers - 1, -1, -1):
            conv3d_backward_weight(acts[layer], dy, self.dw[layer], self.db[layer], dims, self.dil[layer])
            if layer > 0:
                dx = torch.empty_like(dy)
                conv3d_backward_data(dy, self.wb[layer], acts[layer], dx, dims, self.dil[layer])
                dy = dx
        self.step += 1
        adam_step(self.w, self.dw, self.mw, self.vw, self.w.numel(), lr, 0.9, 0.999, 1e-8, self.step)
        adam_step(self.b, self.db, self.mb, self.vb, self.b.numel(), lr, 0.9, 0.999, 1e-8, self.step)
        self._cast()


def training_instances(count, side, seed, gamma_lo=0.9, gamma_hi=0.995):
    """3-D GridWorlds side^3 with the 64^3 benchmark recipe (p = 0.8, 5 %
    obstacles, 8 goals U(0.5, 1), step -0.01) and gamma ~ U(gamma_lo, gamma_hi)."""
    import cpmdp_inputs as ci
    g = ci.uniform(seed, 901, count, gamma_lo, gamma_hi)
    return [ci.config_3d(side=side, seed=seed * 1000003 + i, gamma=float(g[i])) for i in range(count)]


def coarse_inputs(batch_obj, count, shape, device_obj, features=True):
    """Cell features with the coarse value iteration's value in channel 4
    (None without ``features``), and that coarse value (FP32), for
    instances 0..count-1 of a batch."""
    import torch
    cells = int(np.prod(coarse_dims(count, shape)[1:]))
    feat = torch.empty((count * cells, C), dtype=torch.bfloat16, device=device_obj) if features else None
    cv = torch.empty(count * cells, dtype=torch.float32, device=device_obj)
    if features:
        ws_features(batch_obj, 0, count, feat)
    ws_coarse_vi(batch_obj, 0, count, cv, feat, tol=COARSE_TOL, max_sweeps=4000)
    return feat, cv


def solved_chunk(instances, device=0, tol=1e-6):
    """Solve instances (one shape) with the batched solver; returns
    (batch, V*, feat, coarse value) on the device."""
    import torch
    B = batch_build(instances, device=device)
    dev = torch.device("cuda", device)
    V = torch.zeros(int(B.total_states), dtype=torch.float32, device=dev)
    batch_value_iteration(B, V, opts=default_opts(tol=tol, max_iter=5000))
    feat, cv = coarse_inputs(B, len(instances), instances[0].shape, dev)
    return B, V, feat, cv


def train(net, chunks, shape, epochs=10, batch=32, lr=1e-3, lr_final=1e-4, log=None):
    """Minibatch Adam on the full-grid loss over solved chunks (each from
    ``solved_chunk``, instances drawn i.i.d.); minibatches of ``batch``
    instances taken in turn from each chunk; the learning rate decays
    geometrically from lr to lr_final. Returns the mean loss of each epoch."""
    torch = net.torch
    dims = coarse_dims(batch, shape)
    cells = int(np.prod(dims[1:]))
    per = int(np.prod(shape))
    order = sorted(((lo, j) for j, ch in enumerate(chunks) for lo in range(0, int(ch[0].count) - batch + 1, batch)))
    resid = torch.empty(batch * per, dtype=torch.float32, device=net.dev)
    total = epochs * len(order)
    losses = []
    acc = torch.zeros(1, dtype=torch.float32, device=net.dev)
    k = 0
    for ep in range(epochs):
        acc.zero_()
        for lo, j in order:
            B, V, feat, cv = chunks[j]
            rate = lr * (lr_final / lr) ** (k / max(1, total - 1))
            net.train_step(feat[lo * cells:(lo + batch) * cells], None, None, dims, lr=rate, loss_acc=acc,
                           fine=(B, V, lo, cv[lo * cells:(lo + batch) * cells], resid))
            k += 1
        ws_sync()
        losses.append(acc.item() / len(order))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.3e}")
    return losses


def warm_start_values(net, batch_obj, count, shape, V):
    """Coarse value iteration, the network's correction (``net`` None: none)
    and the upsampled start written into V (packed). Returns (correction or
    None, coarse value): the start interpolates their sum."""
    dev = net.dev if net is not None else V.device
    feat, cv = coarse_inputs(batch_obj, count, shape, dev, features=net is not None)
    if net is None:
        ws_upsample(batch_obj, cv, 0, count, V)
        return None, cv
    pred = net.predict(feat, coarse_dims(count, shape))
    ws_upsample(batch_obj, pred, 0, count, V, base=cv)
    return pred, cv


def evaluate(net, count=512, side=64, seed=424242, device=0, log=None, reps=3):
    """Held-out instances (seeds disjoint from training): batched value
    iteration to |dV|inf < 1e-6 from zeros, from the coarse value iteration
    alone, and from the network's corrected start. Times come from CUDA
    events around each stage (median of ``reps``); returns a dict."""
    import statistics
    import torch
    inst = training_instances(count, side, seed=seed)
    B = batch_build(inst, device=device)
    dev = torch.device("cuda", device)
    V = torch.zeros(int(B.total_states), dtype=torch.float32, device=dev)
    opts = default_opts(tol=1e-6, max_iter=5000)
    batch_value_iteration(B, V, opts=opts)                 # autotune and record the graph
    shape = (side,) * 3

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        r = fn()
        e1.record()
        ws_sync()
        return r, e0.elapsed_time(e1)

    def run(start):
        """start() writes V0 into V; returns (start ms, VI ms, sweeps, residuals, V0)."""
        start()                                            # warm-up of the start's kernels
        _, s_ms = timed(start)
        V0 = V.clone()
        vi = []
        for _ in range(reps):
            V.copy_(V0)
            (r, it, res), ms = timed(lambda: batch_value_iteration(B, V, opts=opts))
            vi.append(ms)
        return s_ms, statistics.median(vi), it, res, r

    z_ms, zvi, it0, res0, r0 = run(lambda: V.zero_())
    Vz = V.clone()
    c_ms, cvi, itc, resc, _ = run(lambda: warm_start_values(None, B, count, shape, V))
    n_ms, nvi, it1, res1, r1 = run(lambda: warm_start_values(net, B, count, shape, V))
    diff = (V - Vz).abs().max().item()
    out = {"instances": count, "side": side, "zero_init_ms": zvi,
           "coarse_start_ms": c_ms, "coarse_vi_ms": cvi, "coarse_total_ms": c_ms + cvi,
           "speedup_coarse_only": zvi / (c_ms + cvi), "mean_sweeps_coarse": float(itc.mean()),
           "net_ms": n_ms, "warm_vi_ms": nvi, "warm_total_ms": n_ms + nvi, "speedup_total": zvi / (n_ms + nvi),
           "mean_sweeps_zero": float(it0.mean()), "mean_sweeps_warm": float(it1.mean()),
           "sweeps_saved_frac": float(1 - it1.sum() / it0.sum()),
           "sweeps_saved_frac_coarse_only": float(1 - itc.sum() / it0.sum()),
           "launch_sweeps_zero": r0["iterations"], "launch_sweeps_warm": r1["iterations"],
           "all_converged": bool((res0 < 1e-6).all() and (resc < 1e-6).all() and (res1 < 1e-6).all()),
           "max_abs_diff_warm_vs_zero": diff, "network": {"dilations": list(net.dil), "layers": net.layers},
           "timing": f"CUDA events; start = features + coarse value iteration (+ network) + upsampling; "
                     f"value iteration median of {reps}"}
    B.close()
    if log:
        log(str(out))
    return out


def main(argv=None):
    import argparse
    import json
    import time
    ap = argparse.ArgumentParser(description="train / evaluate the learned warm start")
    ap.add_argument("mode", choices=["train", "eval"])
    ap.add_argument("--instances", type=int, default=2048)
    ap.add_argument("--side", type=int, default=64)
    ap.add_argument("--chunk", type=int, default=512)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-final", type=float, default=5e-5)
    ap.add_argument("--dilations", default="1,2,1")
    ap.add_argument("--weights", default=None)
    ap.add_argument("--eval-instances", type=int, default=512)
    ap.add_argument("--eval-side", type=int, default=64)
    args = ap.parse_args(argv)
    t0 = time.time()
    if args.mode == "train":
        chunks = []
        for lo in range(0, args.instances, args.chunk):
            part = training_instances(min(args.chunk, args.instances - lo), args.side, seed=1 + lo // args.chunk)
            chunks.append(solved_chunk(part))
            print(f"solved {lo + len(part)} / {args.instances} instances, {time.time() - t0:.1f} s", flush=True)
        net = WarmStartNet(device=0, seed=0, dilations=tuple(int(d) for d in args.dilations.split(",")))
        losses = train(net, chunks, (args.side,) * 3, epochs=args.epochs, batch=args.batch, lr=args.lr,
                       lr_final=args.lr_final, log=lambda s: print(s, flush=True))
        if args.weights:
            net.save(args.weights)
        for B, *_ in chunks:
            B.close()
        print(json.dumps({"train_instances": args.instances, "side": args.side, "epochs": args.epochs,
                          "dilations": list(net.dil), "losses": losses, "seconds": time.time() - t0}), flush=True)
        if args.eval_instances > 0:
            print(json.dumps(evaluate(net, count=args.eval_instances, side=args.eval_side)), flush=True)
    else:
        net = WarmStartNet.load(args.weights)
        out = evaluate(net, count=args.eval_instances, side=args.eval_side)
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
