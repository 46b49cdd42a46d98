"""Batched solves (s3ttv_solve_batched): several uneven cubes at once give what
each cube gives alone, each with its own stop rule, and what the FP64 oracle
gives for the same passes of Alg. 1."""
import numpy as np
import pytest

import oracle as O
from synthetic import CubeSpec, make_cube

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


SPECS = [CubeSpec(20, 24, 13, regions=4, k=3, seed=1), CubeSpec(16, 18, 8, regions=3, k=5, seed=2),
         CubeSpec(12, 12, 33, regions=2, k=2, seed=3), CubeSpec(9, 10, 7, regions=2, k=1, seed=4)]


def _problems(specs, device=True):
    probs = []
    for sp in specs:
        _, v = make_cube(sp)
        eps, alpha, beta = O.radii(v.size, sp.sigma, sp.p_s, sp.p_t)
        probs.append({"v": torch.from_numpy(v).cuda() if device else v, "eps": eps, "alpha": alpha,
                      "beta": beta, "k": sp.k})
    return probs


# form 2 (streaming) with the work list batches every problem's block duals
# into one launch per block side; otherwise each problem's own launches are
# recorded
@pytest.mark.parametrize("form,worklist", [pytest.param(2, 1, id="tc_stream_worklist"),
                                           pytest.param(2, 0, id="tc_stream"), pytest.param(1, 0, id="tc"),
                                           pytest.param(0, 0, id="fp32")])
def test_batch_matches_each_cube_alone_and_the_oracle(P, form, worklist):
    probs = _problems(SPECS)
    with P.Solver(0) as s:
        s.set_option(P.OPT_TENSOR_CORES, form)
        s.set_option(P.OPT_BATCH_WORKLIST, worklist)
        out = s.solve_batched(probs, max_iter=30, tol=0.0)  # one recorded chunk of 16 plus 14 more
        alone = []
        for p in probs:
            alone.append(s.solve(p["v"], p["eps"], p["alpha"], p["beta"], p["k"], max_iter=30, tol=0.0))
    for (u, sp_, t, info), (ua, sa, ta, ia), p in zip(out, alone, probs):
        assert info["iters"] == 30 and info["status"] == 1 and info["jacobi_nonconverged"] == 0
        # same kernels in the same order; Z is accumulated with float atomics
        assert rel(u.cpu().numpy(), ua.cpu().numpy()) <= 1e-6
        assert rel(sp_.cpu().numpy(), sa.cpu().numpy()) <= 1e-6
        assert rel(t.cpu().numpy(), ta.cpu().numpy()) <= 1e-6
    for (u, sp_, t, info), p in list(zip(out, probs))[2:]:  # the two smallest against the oracle
        ref, it, _ = O.solve(p["v"].cpu().numpy(), p["k"], p["eps"], p["alpha"], p["beta"], max_iter=30, tol=0.0)
        assert rel(u.cpu().numpy(), ref["u"]) <= 1e-4
        assert rel(t.cpu().numpy(), ref["t"]) <= 1e-4


def test_each_problem_has_its_own_stop_rule(P):
    probs = _problems(SPECS[:2])
    # a constant cube is a fixed point: its relative change is 0 after one pass
    probs.append({"v": torch.full((10, 11, 6), 0.4, dtype=torch.float32, device="cuda"), "eps": 1.0,
                  "alpha": 1.0, "beta": 1.0, "k": 3})
    with P.Solver(0) as s:
        s.set_option(P.OPT_CHECK_EVERY, 7)  # chunks of 8 passes
        out = s.solve_batched(probs, max_iter=20, tol=1e-5)
    infos = [o[3] for o in out]
    assert infos[2]["converged"] == 1 and infos[2]["status"] == 0 and infos[2]["iters"] == 1
    assert np.allclose(out[2][0].cpu().numpy(), 0.4)
    for info in infos[:2]:
        assert info["iters"] == 20 and info["status"] == 1


def test_host_buffers_and_repeated_calls(P):
    probs = _problems(SPECS[:3], device=False)
    with P.Solver(0) as s:
        first = s.solve_batched(probs, max_iter=12, tol=0.0)
        second = s.solve_batched(probs[::-1], max_iter=12, tol=0.0)  # members reused, other shapes
    for (u1, _, _, _), (u2, _, _, _) in zip(first, second[::-1]):
        assert isinstance(u1, np.ndarray)
        assert rel(u1, u2) <= 1e-6


def test_invalid_problem_is_named(P):
    probs = _problems(SPECS[:2])
    probs[1]["k"] = 40  # larger than the cube
    with P.Solver(0) as s:
        with pytest.raises(P.S3TTVError) as e:
            s.solve_batched(probs, max_iter=5)
    assert e.value.status == P.EINVAL and "problem 1" in str(e.value)


def test_problems_that_need_different_shared_memory(P):
    """Cubes whose block-dual CTAs need different amounts of shared memory (band
    counts 191 and 8, the smaller set up last) launch side by side."""
    specs = [CubeSpec(10, 9, 191, regions=2, k=5, seed=5), CubeSpec(11, 10, 8, regions=2, k=5, seed=6)]
    probs = _problems(specs)
    with P.Solver(0) as s:
        out = s.solve_batched(probs, max_iter=4, tol=0.0)
        alone = [s.solve(p["v"], p["eps"], p["alpha"], p["beta"], p["k"], max_iter=4, tol=0.0) for p in probs]
    for o, a in zip(out, alone):
        assert rel(o[0].cpu().numpy(), a[0].cpu().numpy()) <= 1e-6


def test_batch_with_blocks_of_10_and_14(P):
    """Members whose block side takes the per-CTA kernel: k = 10 (rows in
    shared memory) and k = 14 (196 rows: the n x n matrices in the member's own
    global row scratch, allocated after its workspace) batched with a k = 5
    cube give what each gives alone."""
    specs = [CubeSpec(14, 15, 10, regions=3, k=14, seed=6), CubeSpec(12, 11, 12, regions=3, k=10, seed=7),
             CubeSpec(16, 18, 8, regions=3, k=5, seed=2)]
    probs = _problems(specs)
    with P.Solver(0) as s:
        out = s.solve_batched(probs, max_iter=20, tol=0.0)
        alone = [s.solve(p["v"], p["eps"], p["alpha"], p["beta"], p["k"], max_iter=20, tol=0.0) for p in probs]
    for (u, sp_, t, info), (ua, sa, ta, ia) in zip(out, alone):
        assert info["iters"] == 20 and info["jacobi_nonconverged"] == 0
        assert rel(u.cpu().numpy(), ua.cpu().numpy()) <= 1e-6
        assert rel(t.cpu().numpy(), ta.cpu().numpy()) <= 1e-6
