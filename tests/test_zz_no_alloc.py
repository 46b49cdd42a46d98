"""The allocation-free l1-ball entry point (s3ttv_l1_ball_static) against the
context-based one (s3ttv_l1_ball).

It serves callers that cannot call cudaMalloc (an arena or pool that owns all
device memory, a host that forbids allocation after start-up, a real-time loop):
its scratch is a fixed array in the library's device memory.  This file is
collected last so that a failure here leaves every other test already run; it
also passes on its own in a fresh process, where its first call does the
once-per-device set-up.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5  # the per-operator tolerance of the GPU parity tests


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


def test_static_matches_context_entry_point_twice(P):
    """Two calls in a row: the second must not see state left by the first."""
    rng = np.random.default_rng(2024)
    with P.Solver(0) as s:
        for n, frac in ((300_001, 0.3), (77_777, 0.05)):
            x = (rng.standard_normal(n) * rng.uniform(0.01, 3.0, size=n)).astype(np.float32)
            xd = torch.from_numpy(x).cuda()
            r = frac * float(np.abs(x.astype(np.float64)).sum())
            ref, tau_ref = s.l1_ball(xd, r)
            got, tau = P.l1_ball_static(xd, r)
            torch.cuda.synchronize()
            assert rel(got.cpu().numpy(), ref.cpu().numpy()) <= TOL
            assert tau == pytest.approx(tau_ref, rel=TOL)
            assert float(np.abs(got.cpu().numpy().astype(np.float64)).sum()) == pytest.approx(r, rel=1e-5)


def test_static_rejects_what_it_cannot_take(P):
    lib = P.library()
    import ctypes
    buf = torch.zeros(16, device="cuda")
    tau = ctypes.c_double()
    # larger than the 32-bit bin counters of the fixed scratch: rejected before any work
    rc = lib.s3ttv_l1_ball_static(buf.data_ptr(), buf.data_ptr(), P.L1_STATIC_MAX_N + 1, 1.0,
                                  ctypes.byref(tau), None)
    assert rc == P.ETOOBIG
    host = np.zeros(16, np.float32)  # host buffers would need staging, i.e. an allocation
    rc = lib.s3ttv_l1_ball_static(host.ctypes.data, host.ctypes.data, 16, 1.0, ctypes.byref(tau), None)
    assert rc == P.EINVAL


def test_static_edge_cases_back_to_back(P):
    """The branches outside the three-level search, called back to back after a
    full search so that state the array keeps from one call would show: a
    radius at or above ||x||_1 (the identity, tau = 0), radius 0 (all zero),
    n = 0, and an in-place call (out = x).  Each is checked against the context
    entry point and the oracle's sort-based projection."""
    import oracle as O
    rng = np.random.default_rng(77)
    n = 123_457
    x = (rng.standard_normal(n) * rng.uniform(0.01, 2.0, size=n)).astype(np.float32)
    l1 = float(np.abs(x.astype(np.float64)).sum())
    xd = torch.from_numpy(x).cuda()
    with P.Solver(0) as s:
        for r in (0.4 * l1, 1.5 * l1, 0.0, 0.1 * l1, l1 * 2.0, 0.0):
            got, tau = P.l1_ball_static(xd, r)
            ref, tau_ref = s.l1_ball(xd, r)
            torch.cuda.synchronize()
            orc = O.proj_l1_ball(x.astype(np.float64), r)
            g = got.cpu().numpy()
            assert rel(g, ref.cpu().numpy()) <= TOL, r
            assert rel(g, orc) <= TOL, r
            if r >= l1:
                assert tau == 0.0 and np.array_equal(g, x)
            if r == 0.0:
                assert np.all(g == 0.0)
        empty = torch.zeros(0, device="cuda")
        got, tau = P.l1_ball_static(empty, 1.0)
        assert got.numel() == 0 and tau == 0.0
        # in place: out is x itself
        r = 0.25 * l1
        ref, _ = s.l1_ball(xd, r)
        xin = xd.clone()
        got, tau = P.l1_ball_static(xin, r, out=xin)
        torch.cuda.synchronize()
        assert got.data_ptr() == xin.data_ptr()
        assert rel(xin.cpu().numpy(), ref.cpu().numpy()) <= TOL
        assert rel(xin.cpu().numpy(), O.proj_l1_ball(x.astype(np.float64), r)) <= TOL
