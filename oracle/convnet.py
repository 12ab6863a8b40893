"""FP64 oracle of the learned warm start (test infrastructure only).

The warm start maps a GridWorld instance to an estimate of V* on a grid
coarsened by 4 in every dimension, through a fully convolutional 3-D
network; value iteration then starts from that estimate upsampled to the
full grid (the solver's semantics are unchanged: it only starts elsewhere).

Tensors are channels-last, float64: activations (N, Z, Y, X, C), weights
(27, C_out, C_in) with tap t = (dz+1)*9 + (dy+1)*3 + (dx+1) for offsets
d * (dz, dy, dx), dz, dy, dx in {-1, 0, 1} and dilation d; zero padding keeps
the spatial size ("same" convolution).

Definitions (written out, no library convolution):
    y[n, v, co] = b[co] + sum_t sum_ci x[n, v + d*off(t), ci] w[t, co, ci]
    dW[t, co, ci] = sum_{n, v} dy[n, v, co] x[n, v + d*off(t), ci]
    dx[n, u, ci] = sum_t sum_co dy[n, u - d*off(t), co] w[t, co, ci]
    db[co] = sum_{n, v} dy[n, v, co]

Parity pins (tests/test_convnet_oracle.py): forward against scalar loops,
backward against central finite differences of the forward loss, identity
kernels, pooling and upsampling against direct per-cell definitions.
"""
from __future__ import annotations

import numpy as np

FACTOR = 4
N_FEAT = 4


def offsets():
    return [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _shift(x, dz, dy, dx):
    """s[n, z, y, x_] = x[n, z+dz, y+dy, x_+dx] (zero outside)."""
    N, Z, Y, X, C = x.shape
    out = np.zeros_like(x)
    zs, ze = max(0, -dz), min(Z, Z - dz)
    ys, ye = max(0, -dy), min(Y, Y - dy)
    xs, xe = max(0, -dx), min(X, X - dx)
    if zs < ze and ys < ye and xs < xe:
        out[:, zs:ze, ys:ye, xs:xe, :] = x[:, zs + dz:ze + dz, ys + dy:ye + dy, xs + dx:xe + dx, :]
    return out


def conv_forward(x, w, b, dilation):
    """'Same' dilated 3x3x3 convolution, channels last."""
    y = np.zeros(x.shape[:4] + (w.shape[1],))
    for t, (dz, dy, dx) in enumerate(offsets()):
        xs = _shift(x, dilation * dz, dilation * dy, dilation * dx)
        y += xs @ w[t].T
    return y + b


def conv_backward(x, w, dy, dilation):
    """(dx, dW, db) of conv_forward for the upstream gradient dy."""
    dW = np.zeros_like(w)
    dxa = np.zeros_like(x)
    for t, (oz, oy, ox) in enumerate(offsets()):
        xs = _shift(x, dilation * oz, dilation * oy, dilation * ox)
        dW[t] = np.einsum("nzyxo,nzyxi->oi", dy, xs)
        dxa += _shift(dy, -dilation * oz, -dilation * oy, -dilation * ox) @ w[t]
    db = dy.sum(axis=(0, 1, 2, 3))
    return dxa, dW, db


def relu(x):
    return np.maximum(x, 0.0)


DILATIONS = (1, 2, 4, 2, 1, 1)


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), via float32: keep the top
    16 bits of the float32 pattern after adding 0x7FFF plus the lowest kept
    bit. The network stores activations and gradients this way."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def net_forward(x, params, bf16=False):
    """Layers conv -> ReLU (all but the last); params = [(w, b, dilation)].
    Returns the list of activations [x, a1, ..., out]. With bf16=True every
    hidden activation is stored rounded to bf16 (the last output stays
    unrounded, as the loss reads it in FP32)."""
    acts = [x]
    h = x
    for i, (w, b, d) in enumerate(params):
        z = conv_forward(h, w, b, d)
        h = z if i == len(params) - 1 else relu(z)
        if bf16 and i < len(params) - 1:
            h = bf16_round(h)
        acts.append(h)
    return acts


def net_loss(out, target, mask):
    """Squared error of output channel 0 on the masked coarse cells, averaged
    over all coarse cells of the batch."""
    diff = (out[..., 0] - target) * mask
    return float((diff ** 2).sum() / diff.size)


def net_backward(acts, params, target, mask, bf16=False):
    """Gradients [(dW, db)] of net_loss, by the chain rule layer by layer.
    With bf16=True the gradient passed between layers is stored rounded to
    bf16, as in the network's kernels."""
    out = acts[-1]
    g = np.zeros_like(out)
    g[..., 0] = 2.0 * (out[..., 0] - target) * mask / mask.size
    if bf16:
        g = bf16_round(g)
    grads = []
    for i in range(len(params) - 1, -1, -1):
        w, b, d = params[i]
        dxa, dW, db = conv_backward(acts[i], w, g, d)
        grads.append((dW, db))
        if i > 0:
            g = dxa * (acts[i] > 0)
            if bf16:
                g = bf16_round(g)
    return grads[::-1]


def features(gw):
    """Coarse input features of a GridWorld (cells of FACTOR^3 fine states,
    partial cells at the far edges): mean reward of the non-obstacle cells,
    obstacle fraction, largest terminal reward (0 if none), and
    -log(1 - gamma) / 5. Shape (Zc, Yc, Xc, 4)."""
    shape = gw.shape
    cs = tuple((n + FACTOR - 1) // FACTOR for n in shape)
    R = np.asarray(gw.reward, dtype=np.float64)
    cell = np.asarray(gw.cell)
    f = np.zeros(cs + (N_FEAT,))
    g = -np.log(1.0 - gw.gamma) / 5.0
    for cz in range(cs[0]):
        for cy in range(cs[1]):
            for cx in range(cs[2]):
                blk = (slice(cz * FACTOR, min((cz + 1) * FACTOR, shape[0])),
                       slice(cy * FACTOR, min((cy + 1) * FACTOR, shape[1])),
                       slice(cx * FACTOR, min((cx + 1) * FACTOR, shape[2])))
                c, r = cell[blk], R[blk]
                live = c != 1
                f[cz, cy, cx, 0] = r[live].mean() if live.any() else 0.0
                f[cz, cy, cx, 1] = (c == 1).mean()
                f[cz, cy, cx, 2] = r[c == 2].max() if (c == 2).any() else 0.0
                f[cz, cy, cx, 3] = g
    return f


def coarse_target(gw, V):
    """Mean of V over the non-obstacle fine states of each coarse cell, and
    the mask of cells that have any."""
    shape = gw.shape
    cs = tuple((n + FACTOR - 1) // FACTOR for n in shape)
    V = np.asarray(V, dtype=np.float64).reshape(shape)
    cell = np.asarray(gw.cell)
    t = np.zeros(cs)
    m = np.zeros(cs)
    for cz in range(cs[0]):
        for cy in range(cs[1]):
            for cx in range(cs[2]):
                blk = (slice(cz * FACTOR, min((cz + 1) * FACTOR, shape[0])),
                       slice(cy * FACTOR, min((cy + 1) * FACTOR, shape[1])),
                       slice(cx * FACTOR, min((cx + 1) * FACTOR, shape[2])))
                live = cell[blk] != 1
                if live.any():
                    t[cz, cy, cx] = V[blk][live].mean()
                    m[cz, cy, cx] = 1.0
    return t, m


def _corners(p3, cshape):
    """The eight (cell, weight) pairs of the trilinear interpolation at fine
    coordinate p3: a coordinate p sits at (p + 0.5) / FACTOR - 0.5 in cell
    units, clamped to the outermost centres (where the clamp folds two
    corners onto one cell both pairs name it)."""
    lo, hi, t = [], [], []
    for p, n in zip(p3, cshape):
        u = min(max((p + 0.5) / FACTOR - 0.5, 0.0), n - 1.0)
        a = int(np.floor(u))
        lo.append(a)
        hi.append(min(a + 1, n - 1))
        t.append(u - a)
    out = []
    for k in range(8):
        pick = tuple((hi if (k >> (2 - d)) & 1 else lo)[d] for d in range(3))
        w = np.prod([t[d] if (k >> (2 - d)) & 1 else 1.0 - t[d] for d in range(3)])
        out.append((pick, w))
    return out


def upsample(gw, coarse):
    """Warm start on the full grid: the coarse values sit at the cell
    centres; a free state at fine coordinate x is at (x + 0.5) / FACTOR - 0.5
    in cell units (clamped to the outermost centres) and takes the trilinear
    interpolation of the eight surrounding centres; terminals R(t),
    obstacles 0."""
    shape = gw.shape
    C = np.asarray(coarse, dtype=np.float64)
    V0 = np.zeros(shape)
    for z in range(shape[0]):
        for y in range(shape[1]):
            for x in range(shape[2]):
                V0[z, y, x] = sum(w * C[c] for c, w in _corners((z, y, x), C.shape))
    cell = np.asarray(gw.cell)
    V0 = np.where(cell == 2, np.asarray(gw.reward), V0)
    return np.where(cell == 1, 0.0, V0)


def fine_loss_grad(gw, V_target, coarse, n=None):
    """Loss of a coarse estimate on the full grid and its gradient:
    r = upsample(coarse) - V_target on the free states (terminals and
    obstacles are exact), loss = sum r^2 / n, and d loss / d coarse[c] =
    2 / n * sum over free states of (interpolation weight of c) * r (the
    transpose of the interpolation). n defaults to the instance's state
    count."""
    shape = gw.shape
    C = np.asarray(coarse, dtype=np.float64)
    Vt = np.asarray(V_target, dtype=np.float64).reshape(shape)
    n = float(np.prod(shape)) if n is None else float(n)
    Vh = upsample(gw, C)
    free = np.asarray(gw.cell) == 0
    r = np.where(free, Vh - Vt, 0.0)
    grad = np.zeros(C.shape)
    for z in range(shape[0]):
        for y in range(shape[1]):
            for x in range(shape[2]):
                if r[z, y, x] != 0.0:
                    for c, w in _corners((z, y, x), C.shape):
                        grad[c] += 2.0 / n * w * r[z, y, x]
    return float((r * r).sum() / n), grad


def coarse_gridworld(gw):
    """The coarsened copy of a 3-D GridWorld on which the warm start's coarse
    value iteration runs, written out as an ordinary GridWorld: cells of
    FACTOR^3 states; a cell is an obstacle when at least half of its states
    are, else a terminal of reward max R(t) when it holds terminals, else a
    free cell whose reward is the mean reward of its free states times
    1 + gamma + ... + gamma^(FACTOR-1) (FACTOR fine steps); discount
    gamma^FACTOR and the same slip probability. Returns (GridWorld, kind)
    with kind 0 free, 1 obstacle, 2 terminal."""
    import cpmdp_inputs as ci
    shape = gw.shape
    cs = tuple((n + FACTOR - 1) // FACTOR for n in shape)
    R = np.asarray(gw.reward, dtype=np.float64)
    cell = np.asarray(gw.cell)
    kind = np.zeros(cs, dtype=np.uint8)
    rew = np.zeros(cs)
    steps = sum(gw.gamma ** j for j in range(FACTOR))
    for cz in range(cs[0]):
        for cy in range(cs[1]):
            for cx in range(cs[2]):
                blk = (slice(cz * FACTOR, min((cz + 1) * FACTOR, shape[0])),
                       slice(cy * FACTOR, min((cy + 1) * FACTOR, shape[1])),
                       slice(cx * FACTOR, min((cx + 1) * FACTOR, shape[2])))
                c, r = cell[blk], R[blk]
                if 2 * (c == 1).sum() >= c.size:
                    kind[cz, cy, cx] = 1
                elif (c == 2).any():
                    kind[cz, cy, cx] = 2
                    rew[cz, cy, cx] = r[c == 2].max()
                else:
                    free = c == 0
                    rew[cz, cy, cx] = r[free].mean() * steps if free.any() else 0.0
    return ci.GridWorld(shape=cs, p=gw.p, gamma=gw.gamma ** FACTOR, cell=kind, reward=rew), kind
