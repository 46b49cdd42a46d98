"""Parity at full size, in the launch configuration bench.py times.

After a few warm passes of Alg. 1 on the 256x256x128 (k = 5) and 304x304x191
(k = 5, odd band count) cubes and a 100x100x198 cube with the paper's 10 x 10
blocks, with the block-dual products on tensor cores and on CUDA cores (the
same FP32 path for k = 10), one more pass on the GPU is compared with the FP64
oracle applied to the same state: whole arrays where the oracle can afford them
(both l1-ball projections, y2, y3 over every voxel), sampled blocks for the block
duals, sampled voxels for u; plus the constraints each projection guarantees.
"""
import math

import numpy as np
import pytest

import oracle as O
from synthetic import WORKLOADS, make_cube

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OP_TOL = 1e-5


def op_tol(k):
    """1e-5 for every block size (the per-operator bound of the parity tests)."""
    return OP_TOL


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


class BlockCache:
    """Host copies of single blocks of a device-resident Y, fetched on demand."""

    def __init__(self, Yd):
        self.Yd = Yd
        self.cache = {}

    def block(self, l):
        if l not in self.cache:
            self.cache[l] = self.Yd[l].double().cpu().numpy()
        return self.cache[l]

    def __getitem__(self, idx):
        l, r, c = idx
        return self.block(int(l))[r, c]


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2404_03313_gb300 as P
    P.library()
    return P


@pytest.mark.parametrize("form", [pytest.param(1, id="tc"), pytest.param(2, id="tc_stream"), pytest.param(0, id="fp32")])
@pytest.mark.parametrize("name,warm_passes", [("s3ttv_256x256x128_k5", 3), ("s3ttv_304x304x191_k5", 2),
                                              ("paper_100x100x198_k10", 2)])
def test_one_full_size_pass(P, name, warm_passes, form):
    spec = WORKLOADS[name]
    k = spec.k
    clean, v = make_cube(spec)
    shape = v.shape
    N1, N2, N3 = shape
    eps, alpha, beta = O.radii(v.size, spec.sigma, spec.p_s, spec.p_t)
    g = O.step_sizes(N1, N2, k, "paper")
    s = P.Solver(0)
    s.set_option(P.OPT_TENSOR_CORES, form)
    try:
        vd = torch.from_numpy(v).cuda()
        s.setup(vd, eps, alpha, beta, k)
        s.iterate(warm_passes)
        before = {key: s.get_state(key).astype(np.float64) for key in ("u", "s", "t", "y2", "y3")}
        Yb = s.get_state("Y", like=vd)  # device tensor (L, k*k, 2*N3)
        info = s.iterate(1)
        assert info["iters"] == 1 and info["jacobi_nonconverged"] == 0
        after = {key: s.get_state(key).astype(np.float64) for key in ("u", "s", "t", "y2", "y3")}
        Ya = s.get_state("Y", like=vd)
    finally:
        s.close()
    v64 = v.astype(np.float64)

    # steps 3-4: both l1-ball projections over every voxel
    zs = before["s"] - g["s"] * before["y3"]
    zt = before["t"] - g["t"] * (O.diff_adj(before["y2"], O.AXIS_V) + before["y3"])
    s_ref = O.proj_l1_ball(zs, alpha)
    t_ref = O.proj_l1_ball(zt, beta)
    assert rel(after["s"], s_ref) <= OP_TOL
    assert rel(after["t"], t_ref) <= OP_TOL
    assert np.abs(after["s"]).sum() <= alpha * (1 + 1e-5)
    assert np.abs(after["t"]).sum() <= beta * (1 + 1e-5)

    # step 2 at sampled voxels (the pointwise adjoint of the block extraction)
    rng = np.random.default_rng(7)
    vox = [(0, 0, 0), (N1 - 1, N2 - 1, N3 - 1), (0, N2 - 1, 1)]
    vox += [tuple(int(x) for x in (rng.integers(N1), rng.integers(N2), rng.integers(N3))) for _ in range(13)]
    Yc = BlockCache(Yb)
    for (i, j, b) in vox:
        grad = O.linear_op_adjoint_u_at(Yc, k, shape, i, j, b)
        u_ref = min(max(before["u"][i, j, b] - g["u"] * (grad + before["y3"][i, j, b]), 0.0), 1.0)
        assert abs(after["u"][i, j, b] - u_ref) <= 1e-6, (i, j, b)
    assert after["u"].min() >= 0.0 and after["u"].max() <= 1.0

    # steps 8-11 on sampled blocks
    ubar = 2.0 * after["u"] - before["u"]
    blocks = [0, N2 - 1, (N1 - 1) * N2, N1 * N2 - 1] + [int(x) for x in rng.integers(N1 * N2, size=28)]
    for l in blocks:
        p, q = divmod(l, N2)
        X = O.structure_tensor_block(ubar, k, p, q)
        ref = O.block_dual_update(Yb[l].double().cpu().numpy(), X, g["Y"])
        got = Ya[l].double().cpu().numpy()
        assert rel(got, ref) <= op_tol(k), l
        assert np.linalg.norm(got, 2) <= 1 + 1e-4

    # steps 5-7, 12-14 over every voxel, from the oracle's own s+, t+
    sb, tb = 2 * s_ref - before["s"], 2 * t_ref - before["t"]
    y2_ref = before["y2"] + g["y2"] * O.diff(tb, O.AXIS_V)
    assert rel(after["y2"], y2_ref) <= OP_TOL
    y3p = before["y3"] + g["y3"] * (ubar + sb + tb)
    y3_ref = y3p - g["y3"] * O.proj_l2_ball(y3p / g["y3"], v64, eps)
    # outside the ball y3+ = g3 (1 - eps/||d||) d, d = y3'/g3 - v: the factor
    # amplifies relative errors of ||d|| by (eps/||d||) / (1 - eps/||d||)
    ratio = eps / max(np.linalg.norm(y3p / g["y3"] - v64), 1e-300)
    amp = ratio / (1.0 - ratio) if ratio < 1 else 0.0
    assert rel(after["y3"], y3_ref) <= OP_TOL * max(1.0, amp)
    assert math.isfinite(info["rel_change"])
