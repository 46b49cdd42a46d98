"""The FP64 re-solve of blocks whose FP32 eigen-solve reaches its sweep cap
(S3TTV_OPT_FP64_FALLBACK), through the C ABI against the FP64 oracle.

A sweep cap of 1 from a cold start leaves the FP32 Jacobi of random blocks
unconverged, so every such block goes to the FP64 re-solve; its result must
then match the oracle's SVD form at the per-operator tolerance (the FP32 Y'
is the only FP32 rounding left), with the blocks counted in
info.jacobi_fallbacks and none left in info.jacobi_nonconverged.  With the
re-solve switched off the same blocks are reported unconverged."""
import numpy as np
import pytest

import oracle as O
from synthetic import random_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def random_blocks(shape, k, seed, width=2):
    N1, N2, N3 = shape
    rng = np.random.default_rng(seed)
    L = N1 * N2
    scale = rng.uniform(0.5, 3.0, size=(L, 1, 1)) / np.sqrt(k * k + width * N3)
    Y = (rng.standard_normal((L, k * k, width * N3)) * scale).astype(np.float32)
    ubar = rng.uniform(-0.5, 1.5, size=shape).astype(np.float32)
    return Y, ubar


# k <= 5 (both product forms) and the per-CTA kernel (k = 6, 10)
CASES = [((9, 8, 16), 3, 1), ((9, 8, 16), 3, 0), ((10, 11, 7), 5, 1), ((9, 8, 7), 6, 1), ((11, 10, 20), 10, 1)]


@pytest.mark.parametrize("shape,k,tc", CASES)
def test_unconverged_blocks_are_resolved_in_fp64(P, shape, k, tc):
    Y, ubar = random_blocks(shape, k, seed=k * 100 + tc)
    X = O.structure_tensors(ubar.astype(np.float64), k)
    Yref = O.block_dual_update(Y.astype(np.float64), X, 0.25)
    Zvr, Zhr = O.structure_tensors_adjoint(Yref, k, shape)
    tol = 1e-5
    with P.Solver(0) as s:
        s.set_option(P.OPT_TENSOR_CORES, tc)
        s.set_option(P.OPT_JACOBI_MAX_SWEEPS, 1)
        Yd = torch.from_numpy(Y.copy()).cuda()
        Zv, Zh, info = s.block_dual(Yd, torch.from_numpy(ubar).cuda(), k)
        assert info["jacobi_fallbacks"] > 0.5 * Y.shape[0], info
        assert info["jacobi_nonconverged"] == 0, info
        assert rel(Yd.cpu().numpy(), Yref) <= tol, rel(Yd.cpu().numpy(), Yref)
        assert rel(Zv.cpu().numpy(), Zvr) <= tol
        assert rel(Zh.cpu().numpy(), Zhr) <= tol
        # switched off: the same blocks stay unconverged and are applied as they stand
        s.set_option(P.OPT_FP64_FALLBACK, 0)
        Yd = torch.from_numpy(Y.copy()).cuda()
        _, _, info0 = s.block_dual(Yd, torch.from_numpy(ubar).cuda(), k)
        assert info0["jacobi_fallbacks"] == 0
        assert info0["jacobi_nonconverged"] == info["jacobi_fallbacks"], (info0, info)


@pytest.mark.parametrize("layout,reg,k", [("paper", "s3ttv", 3), ("stacked", "s3ttv", 2), ("paper", "ssst", 3)])
def test_one_pass_with_resolved_blocks(P, layout, reg, k):
    """One pass of Alg. 1 from a random state with a sweep cap of 1: the queued
    blocks are re-solved inside the pass (every state to 1e-5), and the pass
    after it starts those blocks cold."""
    N1, N2, N3 = 10, 9, 8
    st = random_state(N1, N2, N3, k, seed=21)
    r = np.random.default_rng(22)
    v = r.uniform(0, 1, (N1, N2, N3)).astype(np.float32)
    rows, width = (2 * k * k, 1) if layout == "stacked" else (k * k, 3 if reg == "ssst" else 2)
    scale = r.uniform(0.5, 3.0, size=(N1 * N2, 1, 1)) / np.sqrt(rows + width * N3)
    st["Y"] = (r.standard_normal((N1 * N2, rows, width * N3)) * scale).astype(np.float32)
    eps, alpha, beta = 3.0, 20.0, 10.0
    ref_state = {key: val.astype(np.float64) for key, val in st.items()}
    gam = O.step_sizes(N1, N2, k, "paper", reg)
    ref, _ = O.iterate(ref_state, v, k, eps, alpha, beta, 0.0, 1.0, gam, layout=layout, reg=reg)
    with P.Solver(0) as s:
        s.set_option(P.OPT_LAYOUT, P.LAYOUT_STACKED if layout == "stacked" else P.LAYOUT_PAPER)
        s.set_option(P.OPT_REGULARIZER, P.REG_SSST if reg == "ssst" else P.REG_S3TTV)
        s.set_option(P.OPT_JACOBI_MAX_SWEEPS, 1)
        s.setup(v, eps, alpha, beta, k)
        for name in ("u", "s", "t", "y2", "y3", "Y"):
            s.set_state(name, st[name])
        info = s.iterate(1)
        assert info["jacobi_fallbacks"] > 0 and info["jacobi_nonconverged"] == 0, info
        for name in ("u", "s", "t", "y2", "y3", "Y"):
            got = s.get_state(name)
            assert rel(got, ref[name].reshape(got.shape)) <= 1e-5, (name, rel(got, ref[name].reshape(got.shape)))
        info2 = s.iterate(1)
        assert info2["jacobi_nonconverged"] == 0, info2
