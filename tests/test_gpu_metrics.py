"""GPU parity of the evaluation entry points against the FP64 oracle:
s3ttv_objective (S3TTV(u)) and s3ttv_quality (MPSNR, MSSIM, SAM).

Tolerances: MPSNR, MSSIM and SAM are FP64 sums of the same FP32 inputs on both
sides, so they agree to rounding (1e-9 relative, 1e-9 rad).  The objective is an
FP64 Gram and Jacobi on the GPU and an FP64 SVD in the oracle: an eigenvalue of
the Gram carries an absolute error of about n 2^-52 lambda_max, so a zero
singular value can come out as up to sqrt(n 2^-52) sigma_max (1.5e-7 sigma_max
at n = 100); with up to n of them in a block, relative error <= 1e-5.
"""
import numpy as np
import pytest

import oracle as O
from synthetic import CubeSpec, make_cube

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2404_03313_gb300 as P
    s = P.Solver(0)
    yield s
    s.close()


@pytest.mark.parametrize("shape,k", [((12, 13, 9), 3), ((16, 16, 20), 5), ((11, 12, 7), 1), ((14, 13, 6), 10)])
def test_objective_matches_oracle(solver, shape, k):
    r = np.random.default_rng(sum(shape) + k)
    u = r.uniform(0, 1, shape).astype(np.float32)
    got = solver.objective(torch.from_numpy(u).cuda(), k)
    ref = O.objective(u.astype(np.float64), k)
    assert abs(got - ref) <= 1e-5 * ref, (got, ref)


def test_objective_of_a_denoised_cube_and_of_a_flat_one(solver):
    spec = CubeSpec(24, 24, 16, regions=4, endmembers=3, sigma=0.05, p_s=0.0, p_t=0.0, k=3, seed=4)
    clean, v = make_cube(spec)
    for cube in (clean, v):
        got = solver.objective(cube, 3)
        ref = O.objective(cube.astype(np.float64), 3)
        assert abs(got - ref) <= 1e-5 * ref
    flat = np.repeat(np.random.default_rng(1).uniform(0, 1, (10, 10, 1)), 8, axis=2).astype(np.float32)
    assert solver.objective(flat, 3) == 0.0


@pytest.mark.parametrize("shape,trim", [((32, 32, 16), 3), ((13, 40, 9), 0), ((20, 11, 5), 3)])
def test_quality_matches_oracle(solver, shape, trim):
    r = np.random.default_rng(shape[0] * 7 + trim)
    ref = r.uniform(0.05, 0.95, shape).astype(np.float32)
    u = np.clip(ref + 0.05 * r.standard_normal(shape), 0, 1).astype(np.float32)
    u[0, 0, :] = 0.0  # a zero spectrum: angle pi / 2
    q = solver.quality(torch.from_numpy(u).cuda(), torch.from_numpy(ref).cuda(), trim=trim, sam_map=True)
    u64, r64 = u.astype(np.float64), ref.astype(np.float64)
    assert q["mpsnr"] == pytest.approx(O.mpsnr(u64, r64, trim), rel=1e-9)
    assert q["mssim"] == pytest.approx(O.mssim(u64, r64, trim), rel=1e-9)
    smap = O.sam_map(u64, r64)
    assert q["sam"] == pytest.approx(smap.mean(), abs=1e-9)
    np.testing.assert_allclose(q["sam_map"].cpu().numpy(), smap, atol=1e-6)


def test_quality_host_buffers_and_identity(solver):
    r = np.random.default_rng(5)
    ref = r.uniform(0.05, 0.95, (12, 12, 8)).astype(np.float32)
    q = solver.quality(ref, ref.copy(), trim=1, sam_map=True)
    assert q["mpsnr"] == float("inf") and q["mssim"] == pytest.approx(1.0, abs=1e-12) and q["sam"] < 1e-6
    assert isinstance(q["sam_map"], np.ndarray) and q["sam_map"].shape == (12, 12)


def test_objective_refuses_blocks_above_12(solver):
    """The solver takes k = 13..16; the FP64 objective keeps each block's
    k^2 x k^2 Gram in shared memory and refuses those sizes with a status."""
    import paper_2404_03313_gb300 as P
    u = np.random.default_rng(3).uniform(0, 1, (14, 14, 4)).astype(np.float32)
    with pytest.raises(P.S3TTVError) as e:
        solver.objective(torch.from_numpy(u).cuda(), 13)
    assert e.value.status == P.EUNSUPPORTED
    assert solver.objective(u, 2) > 0.0  # the context stays usable
