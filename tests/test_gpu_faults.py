"""Host-side fault handling of the C ABI on a GPU context: an injected
allocation cap (S3TTV_OPT_ALLOC_LIMIT) gives S3TTV_ENOMEM and leaves the context
usable; an iteration cap reached before the stop rule gives S3TTV_MAXITER with
valid iterates; NVTX ranges (S3TTV_OPT_NVTX) leave the results as they are.
No kernel is made to fault: every failure here is made on the host."""
import numpy as np
import pytest

from synthetic import WORKLOADS, make_cube

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2404_03313_gb300 as P
    P.library()
    return P


@pytest.fixture(scope="module")
def cube(P):
    spec = WORKLOADS["parity_32x32x16_k3"]
    _, v = make_cube(spec)
    return spec, v, P.radii(v.size, spec.sigma, spec.p_s, spec.p_t)


def test_allocation_cap_gives_enomem_and_the_context_recovers(P, cube):
    spec, v, (eps, alpha, beta) = cube
    with P.Solver(0) as s:
        s.set_option(P.OPT_ALLOC_LIMIT, 1 << 20)  # far below the workspace of this problem
        with pytest.raises(P.S3TTVError) as e:
            s.setup(v, eps, alpha, beta, spec.k)
        assert e.value.status == P.ENOMEM
        with pytest.raises(P.S3TTVError):
            s.iterate(1)  # nothing is set up
        s.set_option(P.OPT_ALLOC_LIMIT, 0)
        u, _, _, info = s.solve(v, eps, alpha, beta, spec.k, max_iter=5, tol=0.0)
        assert info["iters"] == 5 and np.isfinite(u).all()
        with pytest.raises(P.S3TTVError):
            s.set_option(P.OPT_ALLOC_LIMIT, -1)


def test_iteration_cap_gives_maxiter_with_valid_iterates(P, cube):
    spec, v, (eps, alpha, beta) = cube
    with P.Solver(0) as s:
        u, sp, t, info = s.solve(v, eps, alpha, beta, spec.k, max_iter=7, tol=1e-12)
    assert info["status"] == P.MAXITER and info["iters"] == 7 and not info["converged"]
    assert np.isfinite(u).all() and np.isfinite(sp).all() and np.isfinite(t).all()
    assert u.min() >= 0.0 and u.max() <= 1.0  # the box of step 2 holds at every pass


def test_nvtx_ranges_leave_results_unchanged(P, cube):
    spec, v, (eps, alpha, beta) = cube
    out = []
    for flag in (0, 1):
        with P.Solver(0) as s:
            s.set_option(P.OPT_NVTX, flag)
            u, _, _, info = s.solve(v, eps, alpha, beta, spec.k, max_iter=10, tol=0.0)
            out.append(u)
    # the Z scatter adds with atomics, so two runs agree to FP32 rounding, not bitwise
    np.testing.assert_allclose(out[0], out[1], rtol=1e-5, atol=1e-6)
