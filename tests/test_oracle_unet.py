"""Pins of the FP64 warm-start network oracle (oracle/unet.py) against things other
than itself: brute-force loops, a library correlation, adjoint identities, finite
differences of the whole network, and Adam's closed-form first step."""
import numpy as np
import pytest

from oracle import unet
from synthetic import network_params

rng = np.random.default_rng(7)


def brute_conv3(x, w, b):
    """y[b, z, y, x, o] written as six nested loops with explicit bounds."""
    B, D, H, W, C = x.shape
    O = w.shape[0]
    y = np.zeros((B, D, H, W, O))
    for bi in range(B):
        for z in range(D):
            for yy in range(H):
                for xx in range(W):
                    for o in range(O):
                        acc = b[o]
                        for dz in (-1, 0, 1):
                            for dy in (-1, 0, 1):
                                for dx in (-1, 0, 1):
                                    zz, y2, x2 = z + dz, yy + dy, xx + dx
                                    if 0 <= zz < D and 0 <= y2 < H and 0 <= x2 < W:
                                        tap = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)
                                        for c in range(C):
                                            acc += x[bi, zz, y2, x2, c] * w[o, tap, c]
                        y[bi, z, yy, xx, o] = acc
    return y


def test_param_count_by_hand():
    # 27 * sum(c_in * c_out) + sum(c_out) + head 3 * 32 + 3
    assert unet.param_count() == 27 * 52256 + 640 + 99 == 1411651


def test_conv3_matches_brute_force():
    x = rng.standard_normal((2, 3, 4, 5, 2))
    w = rng.standard_normal((3, 27, 2))
    b = rng.standard_normal(3)
    np.testing.assert_allclose(unet.conv3(x, w, b), brute_conv3(x, w, b), rtol=1e-12, atol=1e-12)


def test_conv3_single_channel_matches_scipy_correlate():
    ndimage = pytest.importorskip("scipy.ndimage")
    x = rng.standard_normal((1, 6, 5, 7, 1))
    w = rng.standard_normal((1, 27, 1))
    ref = ndimage.correlate(x[0, ..., 0], w[0, :, 0].reshape(3, 3, 3), mode="constant", cval=0.0)
    np.testing.assert_allclose(unet.conv3(x, w, np.zeros(1))[0, ..., 0], ref, rtol=1e-12, atol=1e-12)


def test_conv3_backward_adjoint_identities():
    x = rng.standard_normal((2, 4, 3, 5, 3))
    w = rng.standard_normal((4, 27, 3))
    b = rng.standard_normal(4)
    gy = rng.standard_normal((2, 4, 3, 5, 4))
    gx, gw, gb = unet.conv3_backward(x, w, gy)
    lhs = float((unet.conv3(x, w, np.zeros(4)) * gy).sum())
    assert abs(lhs - float((x * gx).sum())) < 1e-10 * max(1.0, abs(lhs))   # linear in x
    assert abs(lhs - float((w * gw).sum())) < 1e-10 * max(1.0, abs(lhs))   # linear in w
    bias_only = float(((unet.conv3(x, w, b) - unet.conv3(x, w, np.zeros(4))) * gy).sum())
    assert abs(bias_only - float((b * gb).sum())) < 1e-10 * max(1.0, abs(bias_only))


def test_pool_and_upsample_adjoints():
    x = rng.standard_normal((2, 4, 6, 8, 3))
    g = rng.standard_normal((2, 2, 3, 4, 3))
    assert abs(float((unet.avg_pool(x) * g).sum()) - float((x * unet.avg_pool_adjoint(g)).sum())) < 1e-12
    assert abs(float((unet.upsample(g) * x).sum()) - float((g * unet.upsample_adjoint(x)).sum())) < 1e-12
    const = np.full((1, 4, 4, 4, 2), 3.25)
    np.testing.assert_allclose(unet.avg_pool(const), 3.25)
    # an 8-voxel cell averages its entries
    cell = np.arange(8.0).reshape(1, 2, 2, 2, 1)
    assert unet.avg_pool(cell)[0, 0, 0, 0, 0] == 3.5


def _tiny_problem(seed, shape=(1, 4, 4, 4)):
    r = np.random.default_rng(seed)
    theta = network_params(unet.param_shapes(), seed=seed, head_scale=1.0).astype(np.float64)
    # nonzero biases so the bias gradients are exercised away from zero
    off = 0
    for s in unet.param_shapes():
        n = int(np.prod(s))
        if len(s) == 1:
            theta[off:off + n] = 0.1 * r.standard_normal(n)
        off += n
    v = r.uniform(0, 1, size=shape)
    target = tuple(r.standard_normal(shape) for _ in range(3))
    return theta, v, target


def test_forward_shapes_and_residual_form():
    theta, v, _ = _tiny_problem(1, (2, 4, 8, 4))
    u, s, t = unet.forward(theta, v)
    assert u.shape == s.shape == t.shape == v.shape
    # a zero head makes the prediction (v, 0, 0)
    th = theta.copy()
    th[-99:] = 0.0
    u0, s0, t0 = unet.forward(th, v)
    np.testing.assert_array_equal(u0, v)
    assert not s0.any() and not t0.any()


def test_loss_and_grad_match_finite_differences():
    theta, v, target = _tiny_problem(3)
    loss, g = unet.loss_and_grad(theta, v, target)
    pred = unet.forward(theta, v)
    assert abs(loss - sum(float(((p - q) ** 2).sum()) for p, q in zip(pred, target)) / (3 * v.size)) < 1e-14
    f = lambda th: unet.loss_and_grad(th, v, target)[0]
    h = 1e-5
    r = np.random.default_rng(11)
    # random directions through every parameter at once
    gn = float(np.linalg.norm(g))
    for _ in range(3):
        d = r.standard_normal(theta.size)
        d /= np.linalg.norm(d)  # a step of length h, so no ReLU unit changes side
        fd = (f(theta + h * d) - f(theta - h * d)) / (2 * h)
        assert abs(fd - float(g @ d)) <= 1e-6 * gn
    # single coordinates inside every parameter array (a transposed or
    # misplaced gradient block fails here)
    off = 0
    for s in unet.param_shapes():
        n = int(np.prod(s))
        for j in r.choice(n, size=min(2, n), replace=False):
            e = np.zeros(theta.size)
            e[off + j] = 1.0
            fd = (f(theta + h * e) - f(theta - h * e)) / (2 * h)
            assert abs(fd - g[off + j]) <= 1e-6 * max(1e-3 * gn, abs(fd)), (s, j, fd, g[off + j])
        off += n


def test_gradient_vanishes_at_a_perfect_fit():
    theta, v, _ = _tiny_problem(5)
    target = unet.forward(theta, v)
    loss, g = unet.loss_and_grad(theta, v, target)
    assert loss == 0.0 and not g.any()


def test_adam_first_step_closed_form():
    theta = rng.standard_normal(50)
    grad = rng.standard_normal(50)
    grad[3] = 0.0
    new, m, s = unet.adam_step(theta, grad, np.zeros(50), np.zeros(50), 1, 1e-3)
    # bias correction makes the first step -lr * g / (|g| + eps)
    np.testing.assert_allclose(new - theta, -1e-3 * grad / (np.abs(grad) + unet.ADAM_EPS), rtol=1e-9, atol=0)
    assert new[3] == theta[3]
