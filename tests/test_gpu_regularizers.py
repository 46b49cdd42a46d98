"""GPU parity of the comparison regularisers the paper runs through the same
P-PDS (Sec. IV): STV (block nuclear norms of first-order spatial differences),
SSTV (l1 norm of D D_s u), HSSTV1 / HSSTV2 (SSTV plus omega-weighted
first-order differences, l1 or per-voxel l1,2) and SSST (block nuclear norms of
first-order spatial and spectral differences, k^2 x 3N3 blocks), against the
FP64 oracle through the C ABI.

Tolerances as in test_gpu_parity: one pass from a random state, relative L2
1e-5 per state (SSTV's clip is exact; STV's blocks have k^2 = 9 rows); after
300 passes relative L2 1e-3 of the iterates and MPSNR within 0.01 dB; the FP64
objective 1e-5 relative."""
import numpy as np
import pytest

import oracle as O
from synthetic import WORKLOADS, make_cube, random_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REGS = ["stv", "sstv", "hsstv1", "hsstv2", "ssst"]


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


def solver_for(P, reg):
    s = P.Solver(0)
    s.set_option(P.OPT_REGULARIZER, {"stv": P.REG_STV, "sstv": P.REG_SSTV, "hsstv1": P.REG_HSSTV1,
                                      "hsstv2": P.REG_HSSTV2, "ssst": P.REG_SSST}[reg])
    return s


@pytest.mark.parametrize("reg", REGS)
def test_one_pass_from_a_random_state(P, reg):
    N1, N2, N3, k = 12, 11, 9, 3
    st = random_state(N1, N2, N3, k, seed=5)
    r = np.random.default_rng(6)
    v = r.uniform(0, 1, (N1, N2, N3)).astype(np.float32)
    if reg in ("sstv", "hsstv1", "hsstv2"):
        st["Y"] = (0.3 * r.standard_normal((2 if reg == "sstv" else 4, N1, N2, N3))).astype(np.float32)
    if reg == "ssst":
        st["Y"] = (0.3 * r.standard_normal((N1 * N2, k * k, 3 * N3))).astype(np.float32)
    eps, alpha, beta = 3.0, 20.0, 10.0
    ref_state = {key: val.astype(np.float64) for key, val in st.items()}
    gam = O.step_sizes(N1, N2, k, "paper", reg)
    ref, _ = O.iterate(ref_state, v, k, eps, alpha, beta, 0.0, 1.0, gam, reg=reg)
    with solver_for(P, reg) as s:
        s.setup(v, eps, alpha, beta, k)
        for name in ("u", "s", "t", "y2", "y3", "Y"):
            s.set_state(name, st[name])
        s.iterate(1)
        for name in ("u", "s", "t", "y2", "y3", "Y"):
            got = s.get_state(name)
            assert rel(got, ref[name].reshape(got.shape)) <= 1e-5, (name, rel(got, ref[name].reshape(got.shape)))


@pytest.mark.parametrize("reg", REGS)
def test_300_passes(P, reg):
    spec = WORKLOADS["parity_32x32x16_k3"]
    clean, v = make_cube(spec)
    eps, alpha, beta = O.radii(v.size, spec.sigma, spec.p_s, spec.p_t)
    ref, _, _ = O.solve(v, spec.k, eps, alpha, beta, max_iter=300, tol=0.0, reg=reg)
    with solver_for(P, reg) as s:
        u, sp, t, info = s.solve(torch.from_numpy(v).cuda(), eps, alpha, beta, spec.k, max_iter=300, tol=0.0)
        u, sp, t = (x.cpu().numpy() for x in (u, sp, t))
    assert info["iters"] == 300
    for name, got in (("u", u), ("s", sp), ("t", t)):
        assert rel(got, ref[name]) <= 1e-3, (name, rel(got, ref[name]))
    assert abs(O.mpsnr(u, clean) - O.mpsnr(ref["u"], clean)) <= 0.01
    with P.Solver(0) as s:  # a different problem from S3TTV's
        us, _, _, _ = s.solve(torch.from_numpy(v).cuda(), eps, alpha, beta, spec.k, max_iter=300, tol=0.0)
    assert rel(us.cpu().numpy(), u) > 1e-4


@pytest.mark.parametrize("reg", REGS)
def test_objective(P, reg):
    spec = WORKLOADS["parity_32x32x16_k3"]
    _, v = make_cube(spec)
    with solver_for(P, reg) as s:
        got = s.objective(v, 3)
    ref = O.objective(v.astype(np.float64), 3, reg=reg)
    assert abs(got - ref) <= 1e-5 * ref, (got, ref)


@pytest.mark.parametrize("shape,k", [((9, 8, 7), 1), ((12, 11, 10), 5), ((10, 9, 6), 8)])
def test_ssst_one_pass_block_sizes(P, shape, k):
    """SSST's k^2 x 3N3 blocks at the smallest block (one row), at k = 5 and at
    the largest supported k = 8 (64 rows, 4 lanes per Jacobi pair), one pass
    from a random state against the oracle."""
    N1, N2, N3 = shape
    st = random_state(N1, N2, N3, k, seed=11)
    r = np.random.default_rng(12)
    v = r.uniform(0, 1, (N1, N2, N3)).astype(np.float32)
    scale = r.uniform(0.02, 3.0, size=(N1 * N2, 1, 1)) / np.sqrt(k * k + 3 * N3)
    st["Y"] = (r.standard_normal((N1 * N2, k * k, 3 * N3)) * scale).astype(np.float32)
    eps, alpha, beta = 3.0, 20.0, 10.0
    ref_state = {key: val.astype(np.float64) for key, val in st.items()}
    gam = O.step_sizes(N1, N2, k, "paper", "ssst")
    ref, _ = O.iterate(ref_state, v, k, eps, alpha, beta, 0.0, 1.0, gam, reg="ssst")
    with solver_for(P, "ssst") as s:
        s.setup(v, eps, alpha, beta, k)
        for name in ("u", "s", "t", "y2", "y3", "Y"):
            s.set_state(name, st[name])
        s.iterate(1)
        for name in ("u", "s", "t", "y2", "y3", "Y"):
            got = s.get_state(name)
            tol = 1e-5
            assert rel(got, ref[name].reshape(got.shape)) <= tol, (name, rel(got, ref[name].reshape(got.shape)))


def test_ssst_unsupported_settings(P):
    """SSST takes the paper layout, the periodic D_s and k <= 8; it has no
    stand-alone block-dual entry point."""
    v = np.random.default_rng(0).uniform(0, 1, (12, 12, 6)).astype(np.float32)
    with solver_for(P, "ssst") as s:
        with pytest.raises(P.S3TTVError):
            s.setup(v, 1.0, 1.0, 1.0, 9)
        s.set_option(P.OPT_LAYOUT, P.LAYOUT_STACKED)
        with pytest.raises(P.S3TTVError):
            s.setup(v, 1.0, 1.0, 1.0, 3)
        s.set_option(P.OPT_LAYOUT, P.LAYOUT_PAPER)
        s.set_option(P.OPT_SPECTRAL_BOUNDARY, P.SPECTRAL_OPEN)
        with pytest.raises(P.S3TTVError):
            s.setup(v, 1.0, 1.0, 1.0, 3)
        s.set_option(P.OPT_SPECTRAL_BOUNDARY, P.SPECTRAL_PERIODIC)
        s.setup(v, 1.0, 1.0, 1.0, 3)
        info = s.iterate(2)
        assert info["iters"] == 2
        Y = np.zeros((144, 9, 12), np.float32)
        with pytest.raises(P.S3TTVError):
            s.block_dual(torch.from_numpy(Y).cuda(), torch.from_numpy(v).cuda(), 3)
