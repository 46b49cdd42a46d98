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
