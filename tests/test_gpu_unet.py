"""GPU parity of the learned warm start's network (s3ttv_net_*, through the C ABI)
against the FP64 oracle (oracle/unet.py), and its training and use as a warm start.

Tolerances.  Both sides get the same BF16-representable parameters, so the
differences come from where the GPU stores BF16: every activation (12 stored
tensors on the longest path) and every activation gradient (as many again).  A
BF16 rounding has relative error at most u = 2^-8 and about u / sqrt(3) = 2.3e-3
in RMS; independent roundings add in quadrature, so the prediction's RMS
relative error is about sqrt(12) * 2.3e-3 = 8e-3 and a gradient's about
sqrt(24) * 2.3e-3 = 1.1e-2.  The tests allow four times that: relative L2
3e-2 for the network output h and 5e-2 for each parameter array's gradient.
"""
import numpy as np
import pytest

from oracle import unet as OU
from synthetic import network_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H_TOL = 3e-2
GRAD_TOL = 5e-2


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2404_03313_gb300 as P
    P.library()
    return P


def bf16_params(seed):
    """Seeded parameters with random biases, rounded to BF16 values (so the
    GPU's BF16 weights equal the oracle's exactly)."""
    theta = network_params(OU.param_shapes(), seed=seed, head_scale=1.0)
    r = np.random.default_rng(seed + 1)
    off = 0
    for s in OU.param_shapes():
        n = int(np.prod(s))
        if len(s) == 1:
            theta[off:off + n] = 0.05 * r.standard_normal(n)
        off += n
    return torch.from_numpy(theta).to(torch.bfloat16).to(torch.float32).numpy()


def inputs(shape, seed):
    r = np.random.default_rng(seed)
    v = r.uniform(0.0, 1.0, size=shape).astype(np.float32)
    tgt = tuple((0.3 * r.standard_normal(shape)).astype(np.float32) for _ in range(3))
    return v, tgt


# (B, D, H, W): a multiple of the 128-voxel tile, a ragged last tile, a single
# cell at the coarsest level, and non-cubic sides
SHAPES = [(2, 8, 12, 16), (1, 12, 4, 20), (1, 4, 4, 4), (3, 4, 8, 12)]


def test_param_count_matches_oracle(P):
    assert int(P.library().s3ttv_net_param_count()) == OU.param_count()


@pytest.mark.parametrize("shape", SHAPES)
def test_forward_matches_oracle(P, shape):
    theta = bf16_params(1)
    v, _ = inputs(shape, 2)
    with P.WarmStartNet(0) as net:
        net.set_params(torch.from_numpy(theta).cuda())
        vd = torch.from_numpy(v).cuda()
        u, s, t = (x.cpu().numpy() for x in net.forward(vd))
    ou, os_, ot = OU.forward(theta.astype(np.float64), v.astype(np.float64))
    h_gpu = np.stack([u - v, s, t])
    h_ref = np.stack([ou - v, os_, ot])
    assert rel(h_gpu, h_ref) <= H_TOL, rel(h_gpu, h_ref)
    assert np.isfinite(h_gpu).all()


def test_forward_host_buffers_equal_device_buffers(P):
    theta = bf16_params(3)
    v, _ = inputs((1, 8, 8, 8), 4)
    with P.WarmStartNet(0) as net:
        net.set_params(theta)
        host = net.forward(v)
        dev = net.forward(torch.from_numpy(v).cuda())
    for a, b in zip(host, dev):
        np.testing.assert_array_equal(a, b.cpu().numpy())


@pytest.mark.parametrize("shape", SHAPES[:2])
def test_gradient_matches_oracle(P, shape):
    theta = bf16_params(5)
    v, tgt = inputs(shape, 6)
    with P.WarmStartNet(0) as net:
        net.set_params(torch.from_numpy(theta).cuda())
        loss, g = net.gradient(*(torch.from_numpy(x).cuda() for x in (v,) + tgt))
    oloss, og = OU.loss_and_grad(theta.astype(np.float64), v.astype(np.float64), tgt)
    assert abs(loss - oloss) <= H_TOL * oloss
    off = 0
    worst = 0.0
    for shp in OU.param_shapes():
        n = int(np.prod(shp))
        e = rel(g[off:off + n], og[off:off + n])
        worst = max(worst, e)
        assert e <= GRAD_TOL, (shp, e)
        off += n
    assert rel(g, og) <= GRAD_TOL / 2, rel(g, og)


def test_adam_step_matches_oracle(P):
    """One Adam step from zero moments moves every parameter by -lr g / (|g| + eps):
    by lr times the sign of the gradient wherever |g| >> eps.  The GPU's step is
    compared with the oracle's step taken with the oracle's own gradient."""
    theta = bf16_params(7)
    v, tgt = inputs((1, 8, 8, 8), 8)
    lr = 1e-3
    with P.WarmStartNet(0) as net:
        net.set_params(theta)
        loss = net.train_step(v, *tgt, lr)
        after = net.get_params()
    oloss, og = OU.loss_and_grad(theta.astype(np.float64), v.astype(np.float64), tgt)
    onew, _, _ = OU.adam_step(theta.astype(np.float64), og, np.zeros_like(og), np.zeros_like(og), 1, lr)
    d_gpu = after.astype(np.float64) - theta
    d_ref = onew - theta
    assert abs(loss - oloss) <= H_TOL * oloss
    assert np.all(np.abs(d_gpu) <= lr * (1 + 1e-3))
    # where the oracle gradient is not tiny the two steps agree (a sign decided
    # by a near-zero gradient may differ within the gradient tolerance)
    big = np.abs(og) > 1e-2 * np.abs(og).max()
    assert big.sum() > 1000
    assert np.mean(np.abs(d_gpu[big] - d_ref[big]) <= 1e-2 * lr) >= 0.99


def test_training_lowers_the_loss(P):
    """Twenty Adam steps on one fixed batch lower its loss."""
    theta = bf16_params(9)
    v, tgt = inputs((2, 8, 8, 8), 10)
    with P.WarmStartNet(0) as net:
        net.set_params(theta)
        args = [torch.from_numpy(x).cuda() for x in (v,) + tgt]
        losses = [net.train_step(*args, 3e-4) for _ in range(20)]
    assert losses[-1] < 0.7 * losses[0], losses


def test_invalid_shapes_rejected(P):
    with P.WarmStartNet(0) as net:
        with pytest.raises(P.S3TTVError):
            net.forward(np.zeros((4, 4, 4), np.float32))  # parameters not set
        net.set_params(bf16_params(1))
        with pytest.raises(P.S3TTVError):
            net.forward(np.zeros((6, 8, 8), np.float32))  # side not a multiple of 4


def test_trained_network_as_warm_start(P):
    """What the trained network gains over the plain solver, as measured.
    Train on six 64x64x32 cubes solved by the library, then on a held-out cube:
    (1) the prediction alone (one forward pass, milliseconds) restores far more
    than the noisy input holds (> 6 dB); (2) the solver started from it reaches
    the minimiser the cold start reaches (MPSNR within 0.01 dB after a tight stop
    rule, 1e-7, or 20000 passes), so the network never changes the result;
    (3) with the paper's printed step sizes, where the stop rule does not fire,
    the warm start is more than 3 dB ahead after 200 passes.  What it does not
    gain: passes to the stop rule with the PC_EXACT step sizes (the duals, not
    u, set that count; measured at 256x256x128, a warm start took 1025 and 1568
    passes against 972 and 1714 cold, and starting the block duals from the
    prediction saved 1-2% more), so that count is printed, not asserted."""
    import oracle as O
    from paper_2404_03313_gb300 import warmstart as WS
    from synthetic import make_cube, warm_start_specs

    shape = (64, 64, 32)
    cubes, radii = [], []
    for sp in warm_start_specs(6, 10000, shape):
        _, v = make_cube(sp)
        cubes.append(torch.from_numpy(v).cuda())
        radii.append(P.radii(v.size, sp.sigma, sp.p_s, sp.p_t))
    targets = WS.solver_targets(cubes, radii, 5, 5000, 1e-5, P.STEP_PC_EXACT)
    with P.WarmStartNet(0) as net:
        net.set_params(network_params(OU.param_shapes(), seed=0, head_scale=0.1))
        losses = WS.train(net, cubes, [x[:3] for x in targets], 300, crop=(32, 32, 32), batch=4, lr=1e-3,
                          lr_final=1e-4)
        assert np.mean(losses[-20:]) < 0.5 * np.mean(losses[:5])
        net_params = net.get_params()
        sp = warm_start_specs(1, 20000, shape)[0]
        clean, v = make_cube(sp)
        vd = torch.from_numpy(v).cuda()
        e, a, b = P.radii(v.size, sp.sigma, sp.p_s, sp.p_t)
        pred = net.forward(vd)[0].cpu().numpy()
        cold = WS.solve(vd, e, a, b, 5, None, 20000, 1e-7, P.STEP_PC_EXACT)
        warm = WS.solve(vd, e, a, b, 5, net, 20000, 1e-7, P.STEP_PC_EXACT)
    m_obs, m_net = O.mpsnr(v, clean), O.mpsnr(pred, clean)
    m_cold, m_warm = O.mpsnr(cold["u"].cpu().numpy(), clean), O.mpsnr(warm["u"].cpu().numpy(), clean)
    print(f"MPSNR observed {m_obs:.3f} network {m_net:.3f} cold {m_cold:.4f} ({cold['info']['iters']} passes) "
          f"warm {m_warm:.4f} ({warm['info']['iters']} passes)")
    assert m_net > m_obs + 6.0
    # both runs end at the stop rule or at the same cap, at the same minimiser
    assert cold["info"]["iters"] <= 20000 and warm["info"]["iters"] <= 20000
    assert abs(m_warm - m_cold) <= 0.01
    # with the paper's printed step sizes the stop rule does not fire and u moves
    # slowly: after a fixed budget of passes the warm start is far ahead
    with P.WarmStartNet(0) as net2:
        net2.set_params(net_params)
        cold_p = WS.solve(vd, e, a, b, 5, None, 200, 0.0, P.STEP_PAPER)
        warm_p = WS.solve(vd, e, a, b, 5, net2, 200, 0.0, P.STEP_PAPER)
    mc, mw = O.mpsnr(cold_p["u"].cpu().numpy(), clean), O.mpsnr(warm_p["u"].cpu().numpy(), clean)
    print(f"paper steps, 200 passes: MPSNR cold {mc:.3f} warm {mw:.3f}")
    assert mw > mc + 3.0
