"""Plain FP64 restatement of the learned warm start's network.  TEST INFRASTRUCTURE ONLY.

The paper has no network: it solves Prob. (S3TTV_denoising) by Alg. 1 from
u = v, s = t = 0.  The warm start is an addition beside the method: a small
3-D convolutional U-Net maps the noisy cube v to an estimate of Alg. 1's primal
variables (u, s, t), which then initialise the solver; the solver still decides
the result.  This module is the reference the CUDA forward and backward kernels
are checked against, written as the plain definitions:

* volumes are (B, D, H, W, C) float64 arrays (channels last); a cube
  (N1, N2, N3) is the volume D = N1, H = N2, W = N3 with B = C = 1;
* ``conv3``: y[p, o] = b[o] + sum_{tap, c} x[p + delta_tap, c] w[o, tap, c] over
  the 27 offsets delta in {-1, 0, 1}^3, tap = 9 (dz + 1) + 3 (dy + 1) + (dx + 1),
  with x = 0 outside the volume (zero padding, "same" size);
* ``avg_pool``: the mean of each 2 x 2 x 2 cell; ``upsample``: nearest, x2 on
  D, H and W; ``relu``: max(x, 0);
* the network (3 levels, 32 / 64 / 128 channels; channel counts in ``LAYERS``):
  e1a = relu(conv3(v)), e1b = relu(conv3(e1a)); e2a = relu(conv3(pool(e1b))),
  e2b = relu(conv3(e2a)); ba = relu(conv3(pool(e2b))), bb = relu(conv3(ba));
  d2a = relu(conv3(cat[up(bb), e2b])), d2b = relu(conv3(d2a));
  d1a = relu(conv3(cat[up(d2b), e1b])), d1b = relu(conv3(d1a));
  h = Wh d1b + bh (a 1 x 1 x 1 convolution to 3 channels);
  prediction (u, s, t) = (v + h_0, h_1, h_2);
* loss: the mean over all voxels and the three outputs of the squared error
  against a target (u*, s*, t*);
* ``adam_step``: Adam (Kingma and Ba) with bias correction.

The backward pass is written by hand, layer by layer (the transposes of the
operations above), and is pinned by finite differences and adjoint identities
in ``tests/test_oracle_unet.py``.

Parameters travel as one flat vector: for each of ``LAYERS`` in order, the
weight w[o, tap, c] (o slowest) and then the bias b[o]; last the head
Wh[j, c] and bh[j].
"""
from __future__ import annotations

import numpy as np

__all__ = ["LAYERS", "HEAD", "param_shapes", "param_count", "unpack", "conv3", "conv3_backward",
           "avg_pool", "avg_pool_adjoint", "upsample", "upsample_adjoint", "forward", "loss_and_grad",
           "adam_step", "ADAM_BETA1", "ADAM_BETA2", "ADAM_EPS"]

# (name, input channels, output channels); inputs of d2a and d1a are
# [upsampled deeper features, skip] in that channel order.
LAYERS = (
    ("e1a", 1, 32), ("e1b", 32, 32),
    ("e2a", 32, 64), ("e2b", 64, 64),
    ("ba", 64, 128), ("bb", 128, 128),
    ("d2a", 128 + 64, 64), ("d2b", 64, 64),
    ("d1a", 64 + 32, 32), ("d1b", 32, 32),
)
HEAD = (32, 3)
ADAM_BETA1, ADAM_BETA2, ADAM_EPS = 0.9, 0.999, 1e-8


def param_shapes():
    shapes = []
    for _, ci, co in LAYERS:
        shapes += [(co, 27, ci), (co,)]
    shapes += [(HEAD[1], HEAD[0]), (HEAD[1],)]
    return shapes


def param_count():
    return sum(int(np.prod(s)) for s in param_shapes())


def unpack(theta):
    """Flat vector -> list of arrays in ``param_shapes()`` order (views)."""
    out, off = [], 0
    for s in param_shapes():
        n = int(np.prod(s))
        out.append(np.asarray(theta[off:off + n]).reshape(s))
        off += n
    assert off == theta.size
    return out


def _taps():
    return [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _shifted(x, dz, dy, dx):
    """s[b, z, y, x, c] = x[b, z + dz, y + dy, x + dx, c], zero outside."""
    B, D, H, W, C = x.shape
    xp = np.zeros((B, D + 2, H + 2, W + 2, C), dtype=x.dtype)
    xp[:, 1:-1, 1:-1, 1:-1] = x
    return xp[:, 1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W]


def conv3(x, w, b):
    """3 x 3 x 3 convolution (cross-correlation), zero padding, same size."""
    y = np.zeros(x.shape[:4] + (w.shape[0],))
    for t, (dz, dy, dx) in enumerate(_taps()):
        y += _shifted(x, dz, dy, dx) @ w[:, t, :].T
    return y + b


def conv3_backward(x, w, gy):
    """Gradients of <conv3(x, w, b), gy> with respect to x, w and b.

    gx[p, c] = sum_{tap, o} gy[p - delta_tap, o] w[o, tap, c];
    gw[o, tap, c] = sum_p gy[p, o] x[p + delta_tap, c];  gb[o] = sum_p gy[p, o].
    """
    gx = np.zeros_like(x)
    gw = np.zeros_like(w)
    for t, (dz, dy, dx) in enumerate(_taps()):
        gx += _shifted(gy, -dz, -dy, -dx) @ w[:, t, :]
        gw[:, t, :] = np.einsum("bzyxo,bzyxc->oc", gy, _shifted(x, dz, dy, dx))
    return gx, gw, gy.sum(axis=(0, 1, 2, 3))


def avg_pool(x):
    B, D, H, W, C = x.shape
    return x.reshape(B, D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4, 6))


def avg_pool_adjoint(g):
    return upsample(g) / 8.0


def upsample(x):
    return x.repeat(2, axis=1).repeat(2, axis=2).repeat(2, axis=3)


def upsample_adjoint(g):
    B, D, H, W, C = g.shape
    return g.reshape(B, D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4, 6))


def _relu(x):
    return np.maximum(x, 0.0)


def forward(theta, v, keep=False):
    """Prediction (u, s, t), each (B, D, H, W), from v (B, D, H, W); D, H, W
    must be multiples of 4.  With keep=True also returns the activations."""
    P = unpack(np.asarray(theta, dtype=np.float64))
    W = {name: (P[2 * i], P[2 * i + 1]) for i, (name, _, _) in enumerate(LAYERS)}
    x = np.asarray(v, dtype=np.float64)[..., None]
    a = {"v": x}
    a["e1a"] = _relu(conv3(x, *W["e1a"]))
    a["e1b"] = _relu(conv3(a["e1a"], *W["e1b"]))
    a["p1"] = avg_pool(a["e1b"])
    a["e2a"] = _relu(conv3(a["p1"], *W["e2a"]))
    a["e2b"] = _relu(conv3(a["e2a"], *W["e2b"]))
    a["p2"] = avg_pool(a["e2b"])
    a["ba"] = _relu(conv3(a["p2"], *W["ba"]))
    a["bb"] = _relu(conv3(a["ba"], *W["bb"]))
    a["c2"] = np.concatenate([upsample(a["bb"]), a["e2b"]], axis=-1)
    a["d2a"] = _relu(conv3(a["c2"], *W["d2a"]))
    a["d2b"] = _relu(conv3(a["d2a"], *W["d2b"]))
    a["c1"] = np.concatenate([upsample(a["d2b"]), a["e1b"]], axis=-1)
    a["d1a"] = _relu(conv3(a["c1"], *W["d1a"]))
    a["d1b"] = _relu(conv3(a["d1a"], *W["d1b"]))
    Wh, bh = P[-2], P[-1]
    h = a["d1b"] @ Wh.T + bh
    pred = (x[..., 0] + h[..., 0], h[..., 1], h[..., 2])
    return (pred, a) if keep else pred


def loss_and_grad(theta, v, target):
    """(loss, flat gradient) for the mean squared error of forward(theta, v)
    against target = (u*, s*, t*)."""
    theta = np.asarray(theta, dtype=np.float64)
    P = unpack(theta)
    W = {name: (P[2 * i], P[2 * i + 1]) for i, (name, _, _) in enumerate(LAYERS)}
    pred, a = forward(theta, v, keep=True)
    n = 3 * pred[0].size
    err = [pred[j] - np.asarray(target[j], dtype=np.float64) for j in range(3)]
    loss = sum(float((e * e).sum()) for e in err) / n
    gh = np.stack([2.0 * e / n for e in err], axis=-1)  # d loss / d h (u = v + h_0)
    G = {}
    Wh = P[-2]
    G["head_w"] = np.einsum("bzyxj,bzyxc->jc", gh, a["d1b"])
    G["head_b"] = gh.sum(axis=(0, 1, 2, 3))
    g = (gh @ Wh) * (a["d1b"] > 0)

    def back(name, x_in, g_out):
        gx, gw, gb = conv3_backward(x_in, W[name][0], g_out)
        G[name] = (gw, gb)
        return gx

    g = back("d1b", a["d1a"], g) * (a["d1a"] > 0)
    gc1 = back("d1a", a["c1"], g)
    c_up = a["d2b"].shape[-1]  # channels of up(d2b) at the front of c1
    g_d2b = upsample_adjoint(gc1[..., :c_up]) * (a["d2b"] > 0)
    g_skip1 = gc1[..., c_up:]
    g = back("d2b", a["d2a"], g_d2b) * (a["d2a"] > 0)
    gc2 = back("d2a", a["c2"], g)
    c_up = a["bb"].shape[-1]  # channels of up(bb) at the front of c2
    g_bb = upsample_adjoint(gc2[..., :c_up]) * (a["bb"] > 0)
    g_skip2 = gc2[..., c_up:]
    g = back("bb", a["ba"], g_bb) * (a["ba"] > 0)
    gp2 = back("ba", a["p2"], g)
    g = (avg_pool_adjoint(gp2) + g_skip2) * (a["e2b"] > 0)
    g = back("e2b", a["e2a"], g) * (a["e2a"] > 0)
    gp1 = back("e2a", a["p1"], g)
    g = (avg_pool_adjoint(gp1) + g_skip1) * (a["e1b"] > 0)
    g = back("e1b", a["e1a"], g) * (a["e1a"] > 0)
    back("e1a", a["v"], g)
    flat = []
    for name, _, _ in LAYERS:
        flat += [G[name][0].ravel(), G[name][1].ravel()]
    flat += [G["head_w"].ravel(), G["head_b"].ravel()]
    return loss, np.concatenate(flat)


def adam_step(theta, grad, m, s, step, lr):
    """One Adam update (step counts from 1); returns new (theta, m, s)."""
    m = ADAM_BETA1 * m + (1 - ADAM_BETA1) * grad
    s = ADAM_BETA2 * s + (1 - ADAM_BETA2) * grad * grad
    mhat = m / (1 - ADAM_BETA1 ** step)
    shat = s / (1 - ADAM_BETA2 ** step)
    return theta - lr * mhat / (np.sqrt(shat) + ADAM_EPS), m, s
