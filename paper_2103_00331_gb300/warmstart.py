"""Learned warm start for value iteration (driver over the library's kernels).

A fully convolutional 3-D network reads the coarse features of GridWorld
instances (4 x 4 x 4 cells) and predicts the mean of V* per coarse cell;
value iteration then starts from that estimate upsampled to the full grid.
Value iteration itself is unchanged: it still runs to the same residual,
and zero initialisation stays the fallback against which the warm start is
judged.

Network: six dilated 3 x 3 x 3 convolutions (dilations 1, 2, 4, 2, 1, 1;
receptive field 23 coarse cells; every tap stays inside the 8^3 coarse
grids of 32^3 training instances), 64 channels, ReLU after all but the last,
output channel 0. The first layer reads the 4 feature channels (its other
input weights stay zero) and the last layer writes only channel 0, so the
trainable weights number 27 (4 * 64 + 4 * 64 * 64 + 64) + 5 * 64 + 1 ~ 0.45M.
Weights are FP32 masters with bf16 copies for the convolution kernels;
activations are bf16 with FP32 accumulation; training uses Adam. Every
arithmetic step runs in a libcpmdp kernel; this module only allocates
buffers and sequences the calls.
"""
from __future__ import annotations

import numpy as np

from . import (BF16X3, adam_step, batch_build, batch_value_iteration, conv3d_backward_data,  # noqa: F401
               conv3d_backward_weight, conv3d_forward, default_opts, ws_cast_weights, ws_features,
               ws_loss_grad, ws_sync, ws_targets, ws_upsample)

C = 64
FACTOR = 4
N_FEAT = 4
DILATIONS = (1, 2, 4, 2, 1, 1)
LAYERS = len(DILATIONS)


def coarse_dims(count, shape):
    return (int(count),) + tuple((int(n) + FACTOR - 1) // FACTOR for n in shape)


class WarmStartNet:
    def __init__(self, device=0, seed=0, init=None):
        import torch
        import cpmdp_inputs as ci
        self.torch = torch
        self.dev = torch.device("cuda", device)
        if init is None:
            w = np.zeros((LAYERS, 27, C, C), dtype=np.float32)
            for layer in range(LAYERS):
                cin = N_FEAT if layer == 0 else C
                cout = 1 if layer == LAYERS - 1 else C
                std = np.sqrt(2.0 / (27 * cin)) * (0.5 if layer == LAYERS - 1 else 1.0)
                draw = ci.normal(seed * 100 + layer, 3, 27 * cout * cin).reshape(27, cout, cin) * std
                w[layer, :, :cout, :cin] = draw
            b = np.zeros((LAYERS, C), dtype=np.float32)
        else:
            w, b = init
        self.w = torch.as_tensor(np.ascontiguousarray(w, dtype=np.float32)).to(self.dev)
        self.b = torch.as_tensor(np.ascontiguousarray(b, dtype=np.float32)).to(self.dev)
        self.wf = torch.empty((LAYERS, 27, C, C), dtype=torch.bfloat16, device=self.dev)
        self.wb = torch.empty_like(self.wf)
        self.dw = torch.zeros_like(self.w)
        self.db = torch.zeros_like(self.b)
        self.mw, self.vw = torch.zeros_like(self.w), torch.zeros_like(self.w)
        self.mb, self.vb = torch.zeros_like(self.b), torch.zeros_like(self.b)
        self.step = 0
        self._cast()

    def _cast(self):
        ws_cast_weights(self.w, self.wf, self.wb, LAYERS)

    def numpy_params(self):
        return self.w.cpu().numpy(), self.b.cpu().numpy()

    def save(self, path):
        w, b = self.numpy_params()
        np.savez(path, w=w, b=b, step=self.step)

    @classmethod
    def load(cls, path, device=0):
        d = np.load(path)
        net = cls(device=device, init=(d["w"], d["b"]))
        net.step = int(d["step"])
        return net

    def forward(self, feat, dims):
        """Activations [feat, a1, ..., out] (bf16) and the FP32 output channel 0."""
        torch = self.torch
        nvox = int(np.prod(dims))
        acts = [feat]
        pred = torch.empty(nvox, dtype=torch.float32, device=self.dev)
        for layer in range(LAYERS):
            last = layer == LAYERS - 1
            y = torch.empty((nvox, C), dtype=torch.bfloat16, device=self.dev)
            conv3d_forward(acts[-1], self.wf[layer], self.b[layer], y, pred if last else None, dims,
                           DILATIONS[layer], relu=not last)
            acts.append(y)
        return acts, pred

    def predict(self, feat, dims):
        return self.forward(feat, dims)[1]

    def train_step(self, feat, target, mask, dims, lr=1e-3, loss_acc=None):
        """One Adam step on a minibatch; adds the minibatch loss to loss_acc (device)."""
        torch = self.torch
        nvox = int(np.prod(dims))
        acts, pred = self.forward(feat, dims)
        dy = torch.empty((nvox, C), dtype=torch.bfloat16, device=self.dev)
        ws_loss_grad(pred, target, mask, nvox, dy, loss_acc)
        self.dw.zero_()
        self.db.zero_()
        for layer in range(LAYERS - 1, -1, -1):
            conv3d_backward_weight(acts[layer], dy, self.dw[layer], self.db[layer], dims, DILATIONS[layer])
            if layer > 0:
                dx = torch.empty_like(dy)
                conv3d_backward_data(dy, self.wb[layer], acts[layer], dx, dims, DILATIONS[layer])
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


def solved_dataset(instances, device=0, tol=1e-6):
    """Solve the instances with the batched solver and return (batch, V, feat,
    target, mask, dims) on the device."""
    import torch
    B = batch_build(instances, device=device)
    dev = torch.device("cuda", device)
    V = torch.zeros(int(B.total_states), dtype=torch.float32, device=dev)
    batch_value_iteration(B, V, opts=default_opts(tol=tol, max_iter=5000))
    dims = coarse_dims(len(instances), instances[0].shape)
    cells = int(np.prod(dims[1:]))
    feat = torch.empty((len(instances) * cells, C), dtype=torch.bfloat16, device=dev)
    target = torch.empty(len(instances) * cells, dtype=torch.float32, device=dev)
    mask = torch.empty_like(target)
    ws_features(B, 0, len(instances), feat)
    ws_targets(B, V, 0, len(instances), target, mask)
    return B, V, feat, target, mask, dims


def train(net, feat, target, mask, dims, epochs=10, batch=64, lr=1e-3, lr_final=1e-4, log=None):
    """Minibatch Adam over the instances in order (they are drawn i.i.d.);
    learning rate decays geometrically from lr to lr_final. Returns the
    mean training loss of each epoch."""
    torch = net.torch
    n, cells = dims[0], int(np.prod(dims[1:]))
    steps_per_epoch = max(1, n // batch)
    total = epochs * steps_per_epoch
    losses = []
    acc = torch.zeros(1, dtype=torch.float32, device=net.dev)
    k = 0
    for ep in range(epochs):
        acc.zero_()
        for s in range(steps_per_epoch):
            lo = s * batch * cells
            hi = lo + batch * cells
            rate = lr * (lr_final / lr) ** (k / max(1, total - 1))
            net.train_step(feat[lo:hi], target[lo:hi], mask[lo:hi], (batch,) + tuple(dims[1:]), lr=rate,
                           loss_acc=acc)
            k += 1
        ws_sync()
        losses.append(acc.item() / steps_per_epoch)
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.3e}")
    return losses


def warm_start_values(net, batch_obj, count, shape, V):
    """Features -> network -> upsampled estimate written into V (packed)."""
    torch = net.torch
    dims = coarse_dims(count, shape)
    cells = int(np.prod(dims[1:]))
    feat = torch.empty((count * cells, C), dtype=torch.bfloat16, device=net.dev)
    ws_features(batch_obj, 0, count, feat)
    pred = net.predict(feat, dims)
    ws_upsample(batch_obj, pred, 0, count, V)
    return pred


def evaluate(net, count=512, side=64, seed=424242, device=0, log=None):
    """Held-out instances (seeds disjoint from training): batched value
    iteration to |dV|inf < 1e-6 from zeros and from the network's estimate.
    Times come from CUDA events around each stage; returns a dict."""
    import time
    import torch
    inst = training_instances(count, side, seed=seed)
    B = batch_build(inst, device=device)
    dev = net.dev
    V = torch.zeros(int(B.total_states), dtype=torch.float32, device=dev)
    opts = default_opts(tol=1e-6, max_iter=5000)
    batch_value_iteration(B, V, opts=opts)                 # autotune and record the graph
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    V.zero_()
    torch.cuda.synchronize()
    ev[0].record()
    r0, it0, res0 = batch_value_iteration(B, V, opts=opts)
    ev[1].record()
    torch.cuda.synchronize()
    Vz = V.clone()
    warm_start_values(net, B, count, (side,) * 3, V)      # warm-up of the network kernels
    ws_sync()
    ev[2].record()
    warm_start_values(net, B, count, (side,) * 3, V)
    ev[3].record()
    r1, it1, res1 = batch_value_iteration(B, V, opts=opts)
    ev[4].record()
    ws_sync()
    zero_ms = ev[0].elapsed_time(ev[1])
    net_ms = ev[2].elapsed_time(ev[3])
    vi_ms = ev[3].elapsed_time(ev[4])
    diff = (V - Vz).abs().max().item()
    out = {"instances": count, "side": side, "zero_init_ms": zero_ms, "net_ms": net_ms, "warm_vi_ms": vi_ms,
           "warm_total_ms": net_ms + vi_ms, "speedup_total": zero_ms / (net_ms + vi_ms),
           "mean_sweeps_zero": float(it0.mean()), "mean_sweeps_warm": float(it1.mean()),
           "sweeps_saved_frac": float(1 - it1.sum() / it0.sum()),
           "launch_sweeps_zero": r0["iterations"], "launch_sweeps_warm": r1["iterations"],
           "all_converged": bool((res0 < 1e-6).all() and (res1 < 1e-6).all()),
           "max_abs_diff_warm_vs_zero": diff}
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
    ap.add_argument("--instances", type=int, default=20000)
    ap.add_argument("--side", type=int, default=32)
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--lr-final", type=float, default=1e-4)
    ap.add_argument("--weights", default=None)
    ap.add_argument("--eval-instances", type=int, default=512)
    ap.add_argument("--eval-side", type=int, default=64)
    args = ap.parse_args(argv)
    t0 = time.time()
    if args.mode == "train":
        inst = []
        chunk = 2000
        feats, targets, masks = [], [], []
        dims = None
        for lo in range(0, args.instances, chunk):
            part = training_instances(min(chunk, args.instances - lo), args.side, seed=1 + lo // chunk)
            B, V, f, t, m, d = solved_dataset(part)
            feats.append(f)
            targets.append(t)
            masks.append(m)
            dims = d
            B.close()
            del V
            print(f"solved {lo + len(part)} / {args.instances} instances, {time.time() - t0:.1f} s", flush=True)
        import torch
        feat = torch.cat(feats)
        target = torch.cat(targets)
        mask = torch.cat(masks)
        dims = (args.instances,) + tuple(dims[1:])
        net = WarmStartNet(device=0, seed=0)
        losses = train(net, feat, target, mask, dims, epochs=args.epochs, batch=args.batch, lr=args.lr,
                       lr_final=args.lr_final, log=lambda s: print(s, flush=True))
        if args.weights:
            net.save(args.weights)
        print(json.dumps({"train_instances": args.instances, "side": args.side, "epochs": args.epochs,
                          "losses": losses, "seconds": time.time() - t0}), flush=True)
    else:
        net = WarmStartNet.load(args.weights)
        out = evaluate(net, count=args.eval_instances, side=args.eval_side)
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
