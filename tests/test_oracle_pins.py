"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each oracle function is checked against something other than itself: brute force
on tiny inputs built from the index definitions, optimality conditions of the
proximity operators, closed forms, invariances, and values the paper prints
(``tests/golden/``).  A plausible mistake (a dropped term, a wrong sign or index,
a transposed operand) fails at least one of these.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------------------
# Sec. II-A difference operators.
# ---------------------------------------------------------------------------
def _brute_diff(x, axis):
    N1, N2, N3 = x.shape
    y = np.zeros_like(x)
    for i in range(N1):
        for j in range(N2):
            for b in range(N3):
                nxt = [((i + 1) % N1, j, b), (i, (j + 1) % N2, b), (i, j, (b + 1) % N3)][axis]
                y[i, j, b] = x[nxt] - x[i, j, b]
    return y


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_diff_matches_brute_force_and_adjoint(axis):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 4, 5))
    y = rng.standard_normal((3, 4, 5))
    np.testing.assert_allclose(O.diff(x, axis), _brute_diff(x, axis), rtol=0, atol=1e-14)
    lhs = np.sum(O.diff(x, axis) * y)
    rhs = np.sum(x * O.diff_adj(y, axis))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1)
    # a constant has no differences
    assert np.all(O.diff(np.full((3, 4, 5), 0.7), axis) == 0)


def test_vertical_stripe_has_no_vertical_difference():
    """C1 reading: a vertical stripe (constant down a column i) has D_v t = 0 (Sec. III-B)."""
    t = np.zeros((6, 7, 3))
    t[:, 2, :] = 0.4
    t[:, 5, 1] = -0.3
    assert np.all(O.diff(t, O.AXIS_V) == 0)
    assert np.any(O.diff(t, O.AXIS_H) != 0)


# ---------------------------------------------------------------------------
# Sec. III-A structure tensors.
# ---------------------------------------------------------------------------
def _brute_tensors(u, k):
    """Expanded second-order difference, element by element (no composition)."""
    N1, N2, N3 = u.shape
    X = np.zeros((N1 * N2, k * k, 2 * N3))
    for p in range(N1):
        for q in range(N2):
            for a in range(k):
                for c in range(k):
                    i, j = (p + a) % N1, (q + c) % N2
                    for b in range(N3):
                        b1, i1, j1 = (b + 1) % N3, (i + 1) % N1, (j + 1) % N2
                        fv = u[i1, j, b1] - u[i1, j, b] - u[i, j, b1] + u[i, j, b]
                        fh = u[i, j1, b1] - u[i, j1, b] - u[i, j, b1] + u[i, j, b]
                        X[p * N2 + q, a * k + c, 2 * b] = fv
                        X[p * N2 + q, a * k + c, 2 * b + 1] = fh
    return X


@pytest.mark.parametrize("shape,k", [((4, 5, 3), 2), ((3, 3, 4), 3), ((5, 4, 2), 1), ((4, 4, 3), 4)])
def test_structure_tensors_brute_force(shape, k):
    rng = np.random.default_rng(2)
    u = rng.standard_normal(shape)
    Xb = _brute_tensors(u, k)
    np.testing.assert_allclose(O.structure_tensors(u, k), Xb, rtol=0, atol=1e-13)
    N1, N2, _ = shape
    for p, q in [(0, 0), (N1 - 1, N2 - 1), (1 % N1, 2 % N2)]:
        np.testing.assert_allclose(O.structure_tensor_block(u, k, p, q), Xb[p * N2 + q], atol=1e-13)


@pytest.mark.parametrize("shape,k", [((4, 5, 3), 2), ((6, 5, 4), 3), ((5, 5, 2), 5)])
def test_structure_tensor_adjoint_identity(shape, k):
    rng = np.random.default_rng(3)
    u = rng.standard_normal(shape)
    Y = rng.standard_normal((shape[0] * shape[1], k * k, 2 * shape[2]))
    lhs = np.sum(O.structure_tensors(u, k) * Y)
    rhs = np.sum(u * O.linear_op_adjoint_u(Y, k, shape))
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + 1)


def test_pointwise_adjoint_matches_whole_cube():
    rng = np.random.default_rng(16)
    shape, k = (5, 6, 4), 3
    Y = rng.standard_normal((30, 9, 8))
    full = O.linear_op_adjoint_u(Y, k, shape)
    for (i, j, b) in [(0, 0, 0), (4, 5, 3), (2, 3, 1), (0, 5, 2)]:
        assert O.linear_op_adjoint_u_at(Y, k, shape, i, j, b) == pytest.approx(full[i, j, b], abs=1e-12)


def test_assembled_operator_agrees_with_oracle_operators():
    """The sparse operator built from index definitions equals the oracle's
    forward map and its transpose equals the oracle's adjoint (Alg. 1 step 2)."""
    shape, k = (4, 3, 3), 2
    A = O.assemble_operator(*shape, k)
    rng = np.random.default_rng(4)
    u = rng.standard_normal(shape)
    Y = rng.standard_normal((12, k * k, 2 * shape[2]))
    np.testing.assert_allclose(A[("Y", "u")] @ u.ravel(), O.structure_tensors(u, k).ravel(), atol=1e-13)
    np.testing.assert_allclose(A[("Y", "u")].T @ Y.ravel(),
                               O.linear_op_adjoint_u(Y, k, shape).ravel(), atol=1e-12)
    t = rng.standard_normal(shape)
    np.testing.assert_allclose(A[("y2", "t")] @ t.ravel(), O.diff(t, O.AXIS_V).ravel(), atol=1e-14)


def test_low_rank_spectra_give_low_rank_tensors():
    """Appendix A direction: a cube whose spectra span r vectors has structure
    tensors of rank <= r (the differences are linear in the spectra)."""
    rng = np.random.default_rng(5)
    N1, N2, N3, k, r = 7, 6, 12, 3, 2
    A = rng.standard_normal((N1, N2, r))
    E = rng.standard_normal((r, N3))
    u = A @ E
    X = O.structure_tensors(u, k)
    rk = lambda M: np.linalg.matrix_rank(M, tol=1e-9)
    # the vertical and the horizontal halves each lie in the span of the r
    # differenced spectra; side by side (eq. SSST) at most 2r
    assert max(rk(X[l][:, 0::2]) for l in range(X.shape[0])) == r
    assert max(rk(X[l][:, 1::2]) for l in range(X.shape[0])) == r
    assert max(rk(X[l]) for l in range(X.shape[0])) <= 2 * r


def test_appendix_a_rank_inequality():
    """Appendix A: rank(U) <= rank(D'_v U D'_s) + 2 for a block U (k^2 x N3), with
    D' the (non-periodic) difference matrices; checked on random low-rank U."""
    rng = np.random.default_rng(6)
    k2, N3 = 9, 10
    Dv = np.eye(k2, k=1)[:-1] - np.eye(k2)[:-1]       # (k2-1) x k2, rank k2-1
    Ds = (np.eye(N3, k=1)[:-1] - np.eye(N3)[:-1]).T    # N3 x (N3-1), rank N3-1
    for r in range(1, 6):
        U = rng.standard_normal((k2, r)) @ rng.standard_normal((r, N3))
        assert np.linalg.matrix_rank(U) <= np.linalg.matrix_rank(Dv @ U @ Ds) + 2


# ---------------------------------------------------------------------------
# Step sizes: eq. (stepsize_denoising), Lemma 1, convergence condition.
# ---------------------------------------------------------------------------
def test_lemma1_reproduces_printed_step_sizes():
    g = _gold("stepsizes.json")
    N1, N2, N3, k = 4, 5, 3, 2
    lem = O.lemma1_step_sizes(O.assemble_operator(N1, N2, N3, k))
    for key, gold in (("s", g["gamma_s"]), ("t", g["gamma_t"]), ("Y", g["gamma_Y"]),
                      ("y2", g["gamma_y2"]), ("y3", g["gamma_y3"])):
        val, uniform = lem[key]
        assert uniform
        assert val == pytest.approx(gold, rel=1e-15)
    # u: Lemma 1 gives 1/(8k^2+1) exactly; the printed 1/(8L+1) is never larger
    val, uniform = lem["u"]
    assert uniform and val == pytest.approx(1.0 / (8 * k * k + 1), rel=1e-15)
    gp = O.step_sizes(N1, N2, k, "paper")
    ge = O.step_sizes(N1, N2, k, "pc_exact")
    assert gp["u"] == pytest.approx(1.0 / (8 * N1 * N2 + 1)) and gp["u"] <= val
    assert ge["u"] == pytest.approx(val)
    for key, gkey in (("s", "gamma_s"), ("t", "gamma_t"), ("Y", "gamma_Y"), ("y2", "gamma_y2"), ("y3", "gamma_y3")):
        assert gp[key] == pytest.approx(g[gkey]) and ge[key] == pytest.approx(g[gkey])


@pytest.mark.parametrize("policy", ["paper", "pc_exact"])
def test_convergence_condition_holds(policy):
    """Theorem 1 condition: ||Gamma_2^1/2 A Gamma_1^1/2||_op^2 < 1."""
    import scipy.sparse as sp
    N1, N2, N3, k = 4, 4, 3, 2
    B = O.assemble_operator(N1, N2, N3, k)
    A = sp.bmat([[B[(d, p)] for p in ("u", "s", "t")] for d in ("Y", "y2", "y3")]).toarray()
    g = O.step_sizes(N1, N2, k, policy)
    N = N1 * N2 * N3
    g1 = np.concatenate([np.full(N, g["u"]), np.full(N, g["s"]), np.full(N, g["t"])])
    nY = B[("Y", "u")].shape[0]
    g2 = np.concatenate([np.full(nY, g["Y"]), np.full(N, g["y2"]), np.full(N, g["y3"])])
    M = np.sqrt(g2)[:, None] * A * np.sqrt(g1)[None, :]
    nrm2 = np.linalg.norm(M, 2) ** 2
    assert nrm2 < 1.0


# ---------------------------------------------------------------------------
# Proximity operators.
# ---------------------------------------------------------------------------
def test_prox_nuclear_hand_examples():
    for case in _gold("nuclear_prox_hand.json")["cases"]:
        out = O.prox_nuclear(np.array(case["A"]), case["gamma"])
        np.testing.assert_allclose(out, np.array(case["out"]), atol=1e-14)


@pytest.mark.parametrize("m,n", [(4, 7), (9, 4), (5, 5), (1, 6)])
def test_prox_nuclear_optimality(m, n):
    """P = prox_{g||.||_*}(A) iff (A-P)/g is a subgradient of ||.||_* at P:
    ||(A-P)/g||_2 <= 1 and <(A-P)/g, P> = ||P||_*."""
    rng = np.random.default_rng(7)
    for g in (0.1, 1.0, 3.0):
        A = rng.standard_normal((m, n))
        P = O.prox_nuclear(A, g)
        W = (A - P) / g
        assert np.linalg.norm(W, 2) <= 1 + 1e-12
        assert np.sum(W * P) == pytest.approx(np.linalg.svd(P, compute_uv=False).sum(), rel=1e-12, abs=1e-12)


def _is_spectral_projection(Yp, Yn, rng, trials=200):
    """Yn = argmin_{||Z||_2 <= 1} ||Z - Yp||_F: feasible, and the variational
    inequality <Yp - Yn, Z - Yn> <= 0 holds for every feasible Z."""
    assert np.linalg.norm(Yn, 2) <= 1 + 1e-12
    for _ in range(trials):
        Z = rng.standard_normal(Yp.shape)
        Z /= max(1.0, np.linalg.norm(Z, 2)) * rng.uniform(1.0, 3.0)
        assert np.sum((Yp - Yn) * (Z - Yn)) <= 1e-10


@pytest.mark.parametrize("k2,cols", [(9, 32), (25, 16), (9, 4), (4, 40)])
def test_block_dual_update_is_projection_on_spectral_ball(k2, cols):
    """Steps 9-10 through Moreau's identity (eq. ProxConjugate) equal the
    projection onto the spectral-norm unit ball: clip singular values at 1."""
    rng = np.random.default_rng(8)
    for scale in (0.05, 0.5, 3.0):
        Y = scale * rng.standard_normal((k2, cols))
        X = scale * rng.standard_normal((k2, cols))
        Yn = O.block_dual_update(Y, X, 0.25)
        _is_spectral_projection(Y + 0.25 * X, Yn, rng)
        # idempotent
        np.testing.assert_allclose(O.block_dual_update(Yn, np.zeros_like(X), 0.25), Yn, atol=1e-12)


def test_block_dual_update_special_cases():
    rng = np.random.default_rng(9)
    # all singular values below 1: identity
    Y = rng.standard_normal((9, 20))
    Y *= 0.9 / np.linalg.norm(Y, 2)
    np.testing.assert_allclose(O.block_dual_update(Y, np.zeros_like(Y), 0.25), Y, atol=1e-13)
    # k = 1: each block is one row, projected onto the unit l2 ball (textbook)
    rows = rng.standard_normal((50, 1, 12)) * rng.uniform(0.1, 3.0, size=(50, 1, 1))
    out = O.block_dual_update(rows, np.zeros_like(rows), 0.25)
    nrm = np.linalg.norm(rows, axis=2, keepdims=True)
    np.testing.assert_allclose(out, rows / np.maximum(nrm, 1.0), atol=1e-13)
    # rank-deficient block with one singular value exactly 1 and one at 2
    u1, u2 = np.eye(5)[0], np.eye(5)[3]
    v1, v2 = np.eye(8)[1], np.eye(8)[6]
    B = 1.0 * np.outer(u1, v1) + 2.0 * np.outer(u2, v2)
    np.testing.assert_allclose(O.block_dual_update(B, np.zeros_like(B), 0.25),
                               np.outer(u1, v1) + np.outer(u2, v2), atol=1e-13)
    # non-expansive
    A1, A2 = rng.standard_normal((2, 9, 10)) * 2
    P1 = O.block_dual_update(A1, 0 * A1, 0.25)
    P2 = O.block_dual_update(A2, 0 * A2, 0.25)
    assert np.linalg.norm(P1 - P2) <= np.linalg.norm(A1 - A2) + 1e-12


def test_gram_route_equals_svd_route():
    """The reading used by the GPU path: with G = Y'Y'^T = V diag(lam) V^T,
    clip(Y') = V diag(min(1, lam^-1/2)) V^T Y'.  Pinned here in FP64."""
    rng = np.random.default_rng(10)
    for _ in range(20):
        Yp = rng.standard_normal((25, 64)) * rng.uniform(0.01, 0.5)
        lam, V = np.linalg.eigh(Yp @ Yp.T)
        f = np.where(lam > 1, 1.0 / np.sqrt(np.maximum(lam, 1e-300)), 1.0)
        np.testing.assert_allclose((V * f) @ V.T @ Yp, O.block_dual_update(Yp, 0 * Yp, 0.25), atol=1e-12)


def _bisect_tau(a, r):
    lo, hi = 0.0, float(a.max())
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if np.maximum(a - mid, 0).sum() > r:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def test_l1_ball_hand_examples():
    for case in _gold("l1_ball_hand.json")["cases"]:
        out = O.proj_l1_ball(np.array(case["x"]), case["radius"])
        np.testing.assert_allclose(out, np.array(case["out"]), atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 7, 100, 5000])
def test_l1_ball_vs_bisection_and_kkt(n):
    rng = np.random.default_rng(11 + n)
    x = rng.standard_normal(n) * rng.uniform(0.1, 5, size=n)
    x[rng.uniform(size=n) < 0.1] = 0.0
    l1 = np.abs(x).sum()
    for r in (0.0, 1e-3 * l1, 0.3 * l1, 0.999 * l1, l1, 2 * l1):
        y = O.proj_l1_ball(x, r)
        if r >= l1:
            np.testing.assert_array_equal(y, x)
            continue
        if r == 0:
            assert np.all(y == 0)
            continue
        tau = _bisect_tau(np.abs(x), r)
        np.testing.assert_allclose(y, np.sign(x) * np.maximum(np.abs(x) - tau, 0), atol=1e-9 * (1 + np.abs(x).max()))
        # KKT: on the sphere, signs kept, one common shrink tau on the support
        assert np.abs(y).sum() == pytest.approx(r, rel=1e-12)
        assert np.all(np.sign(y[y != 0]) == np.sign(x[y != 0]))
        sup = y != 0
        shr = np.abs(x[sup]) - np.abs(y[sup])
        assert np.ptp(shr) <= 1e-9 * (1 + np.abs(x).max())
        assert np.all(np.abs(x[~sup]) <= shr[0] + 1e-9)


def test_l1_ball_enumeration_tiny():
    """Brute force over supports and sign patterns for n <= 5."""
    import itertools
    rng = np.random.default_rng(12)
    for _ in range(40):
        n = int(rng.integers(1, 6))
        x = rng.standard_normal(n) * 2
        r = float(rng.uniform(0.05, np.abs(x).sum()))
        best, bestd = None, np.inf
        # candidates: for each support S, y_S = sign(x_S)(|x_S| - tau) with tau = (sum|x_S| - r)/|S|
        for m in range(1, n + 1):
            for S in itertools.combinations(range(n), m):
                S = list(S)
                tau = (np.abs(x[S]).sum() - r) / m
                y = np.zeros(n)
                y[S] = np.sign(x[S]) * (np.abs(x[S]) - tau)
                if np.any(np.abs(x[S]) - tau < -1e-15):
                    continue
                d = np.sum((y - x) ** 2)
                if d < bestd and np.abs(y).sum() <= r + 1e-12:
                    best, bestd = y, d
        np.testing.assert_allclose(O.proj_l1_ball(x, r), best, atol=1e-12)


def test_box_and_l2_ball():
    x = np.array([-0.5, 0.25, 1.5, 1.0, 0.0])
    np.testing.assert_array_equal(O.proj_box(x, 0.0, 1.0), [0.0, 0.25, 1.0, 1.0, 0.0])
    v = np.array([1.0, 2.0])
    np.testing.assert_allclose(O.proj_l2_ball(np.array([4.0, 6.0]), v, 2.5), [2.5, 4.0])  # 3-4-5 triangle
    np.testing.assert_array_equal(O.proj_l2_ball(np.array([1.5, 2.0]), v, 2.5), [1.5, 2.0])
    rng = np.random.default_rng(13)
    for _ in range(20):
        c = rng.standard_normal(30)
        z = rng.standard_normal(30) * 3
        eps = float(rng.uniform(0.1, 5))
        p = O.proj_l2_ball(z, c, eps)
        assert np.linalg.norm(p - c) <= eps * (1 + 1e-14)
        for _ in range(20):
            w = c + rng.standard_normal(30)
            w = c + (w - c) * min(1.0, eps / np.linalg.norm(w - c)) * rng.uniform(0, 1)
            assert np.dot(z - p, w - p) <= 1e-10


# ---------------------------------------------------------------------------
# Experiment rules and metrics (Sec. IV-A).
# ---------------------------------------------------------------------------
def test_radii_parity_cube():
    g = _gold("radii_parity_cube.json")
    eps, alpha, beta = O.radii(g["N"], g["sigma"], g["p_s"], g["p_t"], g["rho"])
    assert alpha == pytest.approx(g["alpha"], rel=1e-14)
    assert beta == pytest.approx(g["beta"], rel=1e-14)
    assert eps == pytest.approx(g["eps"], rel=1e-14)
    assert O.radii(100, 0.0, 0.0, 0.0)[0] == 0.01


def test_mpsnr_hand():
    g = _gold("mpsnr_hand.json")
    ref = np.random.default_rng(14).uniform(size=g["shape"])
    u = ref + np.array(g["band_delta"])[None, None, :]
    assert O.mpsnr(u, ref) == pytest.approx(g["mpsnr"], abs=1e-12)


# ---------------------------------------------------------------------------
# Alg. 1 as a whole: fixed points, invariances, convergence.
# ---------------------------------------------------------------------------
def _run(v, k, iters, policy="paper", eps=1.0, alpha=2.0, beta=1.0, **kw):
    st, it, rel = O.solve(v, k, eps, alpha, beta, max_iter=iters, tol=0.0, policy=policy, **kw)
    return st


@pytest.mark.parametrize("kind", ["constant", "spectrally_flat"])
def test_fixed_points(kind):
    """v inside the box with D_s v = 0 is a solution (objective 0, feasible);
    Alg. 1 started there stays there: u = v, s = t = 0, all duals 0."""
    rng = np.random.default_rng(15)
    if kind == "constant":
        v = np.full((5, 6, 4), 0.37)
    else:
        v = np.repeat(rng.uniform(0.1, 0.9, size=(5, 6, 1)), 4, axis=2)
    st = _run(v, 2, 7)
    np.testing.assert_allclose(st["u"], v, atol=1e-15)
    for key in ("s", "t", "y2", "y3", "Y"):
        assert np.abs(st[key]).max() <= 1e-15


def test_zero_radii_keep_noise_components_zero():
    from synthetic import CubeSpec, make_cube
    _, v = make_cube(CubeSpec(8, 8, 6, regions=3, endmembers=2, seed=3))
    st = _run(v, 2, 10, alpha=0.0, beta=0.0)
    assert np.all(st["s"] == 0) and np.all(st["t"] == 0)


@pytest.mark.parametrize("shift", [(2, 0, 0), (0, 3, 0), (0, 0, 1), (1, -2, 2)])
def test_circular_shift_equivariance(shift):
    """All boundaries are periodic, so shifting v circularly shifts u, s, t."""
    from synthetic import CubeSpec, make_cube
    _, v = make_cube(CubeSpec(8, 7, 6, regions=3, endmembers=2, seed=4))
    v = v.astype(np.float64)
    a = _run(v, 3, 6)
    b = _run(np.roll(v, shift, axis=(0, 1, 2)), 3, 6)
    for key in ("u", "s", "t", "y2", "y3"):
        np.testing.assert_allclose(b[key], np.roll(a[key], shift, axis=(0, 1, 2)), atol=1e-11)


def test_convergence_feasibility_and_residuals():
    """P-PDS converges (Theorem 1): at the end the constraints of Prob.
    (S3TTV_denoising) hold and successive differences vanish."""
    from synthetic import CubeSpec, make_cube
    spec = CubeSpec(8, 8, 6, regions=3, endmembers=2, sigma=0.05, p_s=0.05, p_t=0.1, seed=5)
    clean, v = make_cube(spec)
    v = v.astype(np.float64)
    eps, alpha, beta = O.radii(v.size, spec.sigma, spec.p_s, spec.p_t)
    trace = []
    st, it, rel = O.solve(v, 2, eps, alpha, beta, max_iter=3000, tol=0.0, policy="pc_exact", trace=trace)
    assert st["u"].min() >= 0.0 and st["u"].max() <= 1.0
    assert np.abs(st["s"]).sum() <= alpha * (1 + 1e-12)
    assert np.abs(st["t"]).sum() <= beta * (1 + 1e-12)
    assert np.linalg.norm(O.diff(st["t"], O.AXIS_V)) <= 1e-3 * (1 + np.linalg.norm(st["t"]))
    assert np.linalg.norm(st["u"] + st["s"] + st["t"] - v) <= eps * (1 + 1e-3)
    assert trace[-1] < 1e-4 * max(trace[:10])
    # one more pass barely moves anything
    st2, _ = O.iterate(st, v, 2, eps, alpha, beta, 0.0, 1.0, O.step_sizes(8, 8, 2, "pc_exact"))
    assert np.linalg.norm(st2["u"] - st["u"]) <= 1e-4 * np.linalg.norm(st["u"])


def test_parity_cube_improves_mpsnr():
    """Fig. 11 behaviour on the 32x32x16 parity cube: the restored cube is
    closer to the clean one than the observation after 300 passes."""
    from synthetic import WORKLOADS, make_cube
    spec = WORKLOADS["parity_32x32x16_k3"]
    clean, v = make_cube(spec)
    eps, alpha, beta = O.radii(v.size, spec.sigma, spec.p_s, spec.p_t)
    trace = []
    st, it, rel = O.solve(v, spec.k, eps, alpha, beta, max_iter=300, tol=0.0, trace=trace)
    assert it == 300
    assert O.mpsnr(st["u"], clean) > O.mpsnr(v, clean) + 1.0
    assert np.median(trace[-20:]) < np.median(trace[1:21])


# ---------------------------------------------------------------------------
# Evaluation metrics: objective S3TTV(u), MSSIM (eq. MSSIM), SAM (eq. 2D_SAM)
# ---------------------------------------------------------------------------
def test_objective_k1_is_a_sum_of_row_norms():
    """With 1 x 1 blocks each structure tensor is one row (the 2 N3 second
    differences of one pixel), whose only singular value is its l2 norm."""
    r = np.random.default_rng(21)
    u = r.standard_normal((5, 6, 4))
    dvs = np.roll(np.roll(u, -1, 0) - u, -1, 2) - (np.roll(u, -1, 0) - u)
    dhs = np.roll(np.roll(u, -1, 1) - u, -1, 2) - (np.roll(u, -1, 1) - u)
    expect = np.sqrt((dvs ** 2).sum(axis=2) + (dhs ** 2).sum(axis=2)).sum()
    assert O.objective(u, 1) == pytest.approx(expect, rel=1e-12)


def test_objective_invariances():
    r = np.random.default_rng(22)
    u = r.uniform(0, 1, (6, 7, 5))
    f = O.objective(u, 3)
    assert f > 0
    assert O.objective(u + 0.37, 3) == pytest.approx(f, rel=1e-12)  # differences remove constants
    assert O.objective(-2.5 * u, 3) == pytest.approx(2.5 * f, rel=1e-12)  # absolute homogeneity
    flat = np.repeat(r.uniform(0, 1, (6, 7, 1)), 5, axis=2)  # spectrally flat: D_s u = 0
    assert O.objective(flat, 3) == 0.0


def _ssim_loops(x, y):
    """SSIM written pixel by pixel with explicit window loops."""
    w = O.ssim_window()
    H, W = x.shape
    C1, C2 = 1e-4, 9e-4
    vals = []
    for i in range(5, H - 5):
        for j in range(5, W - 5):
            mx = my = sxx = syy = sxy = 0.0
            for a in range(11):
                for b in range(11):
                    xv, yv, wt = x[i + a - 5, j + b - 5], y[i + a - 5, j + b - 5], w[a, b]
                    mx += wt * xv
                    my += wt * yv
                    sxx += wt * xv * xv
                    syy += wt * yv * yv
                    sxy += wt * xv * yv
            sxx -= mx * mx
            syy -= my * my
            sxy -= mx * my
            vals.append(((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2)))
    return float(np.mean(vals))


def test_ssim_window_is_the_standard_gaussian():
    w = O.ssim_window()
    assert w.shape == (11, 11) and abs(w.sum() - 1.0) < 1e-15
    assert w[5, 6] / w[5, 5] == pytest.approx(np.exp(-1 / 4.5), rel=1e-13)


def test_ssim_against_loops_and_closed_forms():
    r = np.random.default_rng(23)
    x = r.uniform(0, 1, (13, 14))
    y = np.clip(x + 0.1 * r.standard_normal((13, 14)), 0, 1)
    assert O.ssim_band(x, y) == pytest.approx(_ssim_loops(x, y), rel=1e-12)
    assert O.ssim_band(x, x) == pytest.approx(1.0, abs=1e-15)
    assert O.ssim_band(x, y) == pytest.approx(O.ssim_band(y, x), rel=1e-14)
    # constant images a, b: variances vanish, SSIM = (2ab + C1) / (a^2 + b^2 + C1)
    a, b = 0.3, 0.7
    cx, cy = np.full((12, 12), a), np.full((12, 12), b)
    assert O.ssim_band(cx, cy) == pytest.approx((2 * a * b + 1e-4) / (a * a + b * b + 1e-4), rel=1e-12)
    u = np.stack([x, y, x], axis=2)
    assert O.mssim(u, u, trim=0) == pytest.approx(1.0, abs=1e-15)


def test_sam_hand_cases():
    ref = np.zeros((1, 5, 2))
    u = np.zeros((1, 5, 2))
    ref[0, 0], u[0, 0] = (1, 0), (0, 1)        # orthogonal: pi / 2
    ref[0, 1], u[0, 1] = (1, 1), (1, 0)        # 45 degrees
    ref[0, 2], u[0, 2] = (0.2, 0.4), (1, 2)    # parallel, scaled: 0
    ref[0, 3], u[0, 3] = (1, 0), (-1, 0)       # opposite: pi
    ref[0, 4] = (0, 0)                         # both zero: 0
    np.testing.assert_allclose(O.sam_map(u, ref)[0], [np.pi / 2, np.pi / 4, 0.0, np.pi, 0.0], atol=1e-7)


# ---------------------------------------------------------------------------
# The stacked (2k^2) x (N3 or N3 - 1) block matrices and the open D_s
# ---------------------------------------------------------------------------
def _stacked_loops(u, k, periodic_s):
    N1, N2, N3 = u.shape
    M = N3 if periodic_s else N3 - 1
    X = np.zeros((N1 * N2, 2 * k * k, M))
    for p in range(N1):
        for q in range(N2):
            for a in range(k):
                for c in range(k):
                    i, j = (p + a) % N1, (q + c) % N2
                    for b in range(M):
                        b1 = (b + 1) % N3
                        ds = lambda ii, jj: u[ii, jj, b1] - u[ii, jj, b]
                        X[p * N2 + q, 2 * (a * k + c), b] = ds((i + 1) % N1, j) - ds(i, j)
                        X[p * N2 + q, 2 * (a * k + c) + 1, b] = ds(i, (j + 1) % N2) - ds(i, j)
    return X


@pytest.mark.parametrize("periodic_s", [True, False])
def test_stacked_tensors_match_loops(periodic_s):
    u = np.random.default_rng(31).standard_normal((4, 5, 6))
    np.testing.assert_allclose(O.structure_tensors(u, 2, "stacked", periodic_s), _stacked_loops(u, 2, periodic_s),
                               rtol=0, atol=1e-13)


def test_stacked_and_paper_forms_share_entries_not_singular_values():
    u = np.random.default_rng(32).standard_normal((5, 6, 7))
    Xp = O.structure_tensors(u, 3)
    Xs = O.structure_tensors(u, 3, "stacked")
    # the same second differences, arranged differently
    np.testing.assert_allclose(np.sort(Xp.ravel()), np.sort(Xs.ravel()), atol=1e-14)
    assert O.objective(u, 3, "stacked") != pytest.approx(O.objective(u, 3), rel=1e-3)
    # the open D_s drops exactly the wrap-around band
    np.testing.assert_allclose(O.structure_tensors(u, 3, "stacked", False), Xs[:, :, :-1], atol=1e-14)


@pytest.mark.parametrize("layout,periodic_s", [("stacked", True), ("stacked", False), ("paper", False)])
def test_stacked_and_open_adjoint_identities(layout, periodic_s):
    r = np.random.default_rng(33)
    u = r.standard_normal((4, 5, 6))
    X = O.structure_tensors(u, 2, layout, periodic_s)
    Y = r.standard_normal(X.shape)
    lhs = float((X * Y).sum())
    rhs = float((u * O.linear_op_adjoint_u(Y, 2, u.shape, layout, periodic_s)).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


# ---------------------------------------------------------------------------
# Comparison regularisers through the same P-PDS (Sec. IV): STV and SSTV
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("reg,k", [("stv", 2), ("stv", 1), ("sstv", 2)])
def test_comparison_step_sizes_are_lemma1_on_assembled_operators(reg, k):
    got = O.lemma1_step_sizes(O.assemble_operator(4, 5, 3, k, reg))
    want = O.step_sizes(4, 5, k, "paper", reg)
    for key in ("u", "s", "t", "Y", "y2", "y3"):
        assert got[key][0] == pytest.approx(want[key], rel=1e-12), key
        assert got[key][1], key  # every column (row) has the same abs-sum


def test_sstv_dual_prox_is_the_clip_to_the_unit_box():
    """Moreau (eq. ProxConjugate) with prox of gamma^-1 ||.||_1 (soft threshold)
    reduces to clipping every entry of Y' to [-1, 1]."""
    r = np.random.default_rng(41)
    v = r.uniform(0, 1, (5, 6, 4))
    st = O.init_state(v, 1, reg="sstv")
    st["Y"] = 2.0 * r.standard_normal(st["Y"].shape)
    gam = O.step_sizes(5, 6, 1, "paper", "sstv")
    new, _ = O.iterate(st, v, 1, 1.0, 5.0, 3.0, 0.0, 1.0, gam, reg="sstv")
    ub = 2.0 * new["u"] - st["u"]
    Yp = st["Y"] + gam["Y"] * np.stack(O.spectral_diffs(ub, True))
    np.testing.assert_allclose(new["Y"], np.clip(Yp, -1.0, 1.0), atol=1e-14)


def test_stv_tensors_adjoint_and_k1_closed_form():
    r = np.random.default_rng(42)
    u = r.standard_normal((4, 5, 6))
    X = O.structure_tensors(u, 2, second_order=False)
    Y = r.standard_normal(X.shape)
    lhs = float((X * Y).sum())
    rhs = float((u * O.linear_op_adjoint_u(Y, 2, u.shape, second_order=False)).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))
    dv = np.roll(u, -1, 0) - u
    dh = np.roll(u, -1, 1) - u
    expect = np.sqrt((dv ** 2).sum(axis=2) + (dh ** 2).sum(axis=2)).sum()
    assert O.objective(u, 1, reg="stv") == pytest.approx(expect, rel=1e-12)
    flat = np.ones((4, 5, 6))
    assert O.objective(flat, 2, reg="stv") == 0.0 and O.objective(flat, 2, reg="sstv") == 0.0
    Fv, Fh = O.spectral_diffs(u, True)
    assert O.objective(u, 2, reg="sstv") == pytest.approx(np.abs(Fv).sum() + np.abs(Fh).sum(), rel=1e-14)


@pytest.mark.parametrize("reg", ["hsstv1", "hsstv2"])
def test_hsstv_step_sizes_and_dual_prox(reg):
    """Lemma 1 on the assembled operator: gamma_u is the exact column bound; the
    dual rows' bound is 4 for the second-order and 2 omega for the first-order
    parts, and the common gamma_Y = 1/4 respects both.  The conjugate prox is
    the projection onto the unit l_inf ball (HSSTV1) or onto each voxel's unit
    l2 ball of its four differences (HSSTV2)."""
    got = O.lemma1_step_sizes(O.assemble_operator(4, 5, 3, 1, reg))
    want = O.step_sizes(4, 5, 1, "paper", reg)
    assert got["u"][0] == pytest.approx(want["u"], rel=1e-12) and got["u"][1]
    assert want["Y"] <= got["Y"][0] + 1e-15  # the smallest row bound is 1/4
    r = np.random.default_rng(51)
    v = r.uniform(0, 1, (5, 6, 4))
    st = O.init_state(v, 1, reg=reg)
    st["Y"] = 2.0 * r.standard_normal(st["Y"].shape)
    new, _ = O.iterate(st, v, 1, 1.0, 5.0, 3.0, 0.0, 1.0, want, reg=reg)
    ub = 2.0 * new["u"] - st["u"]
    w = O.HSSTV_OMEGA
    A = np.stack(O.spectral_diffs(ub, True) + (w * O.diff(ub, O.AXIS_V), w * O.diff(ub, O.AXIS_H)))
    Yp = st["Y"] + want["Y"] * A
    if reg == "hsstv1":
        expect = np.clip(Yp, -1.0, 1.0)
    else:
        expect = Yp / np.maximum(1.0, np.sqrt((Yp * Yp).sum(axis=0, keepdims=True)))
    np.testing.assert_allclose(new["Y"], expect, atol=1e-13)


def test_hsstv_objectives_and_adjoint():
    r = np.random.default_rng(52)
    u = r.standard_normal((4, 5, 6))
    w = O.HSSTV_OMEGA
    F2v, F2h = O.spectral_diffs(u, True)
    F1v, F1h = O.diff(u, O.AXIS_V), O.diff(u, O.AXIS_H)
    l1 = np.abs(F2v).sum() + np.abs(F2h).sum() + w * (np.abs(F1v).sum() + np.abs(F1h).sum())
    l12 = np.sqrt(F2v ** 2 + F2h ** 2 + (w * F1v) ** 2 + (w * F1h) ** 2).sum()
    assert O.objective(u, 1, reg="hsstv1") == pytest.approx(l1, rel=1e-13)
    assert O.objective(u, 1, reg="hsstv2") == pytest.approx(l12, rel=1e-13)
    # the primal term is the adjoint of the stacked operator
    Y = r.standard_normal((4,) + u.shape)
    st = {"u": u, "s": np.zeros_like(u), "t": np.zeros_like(u), "y2": np.zeros_like(u), "y3": np.zeros_like(u),
          "Y": Y}
    g = dict(O.step_sizes(4, 5, 1, "paper", "hsstv1"))
    # one pass with a tiny gamma_u and a wide box: u+ - u = -gamma_u (A^T Y)
    g["u"] = 1e-6
    new, _ = O.iterate(st, np.zeros_like(u), 1, 1e9, 1e9, 1e9, -1e9, 1e9, g, reg="hsstv1")
    ATY = -(new["u"] - u) / g["u"]
    A = np.stack((F2v, F2h, w * F1v, w * F1h))
    lhs, rhs = float((A * Y).sum()), float((u * ATY).sum())
    assert abs(lhs - rhs) <= 1e-6 * max(1.0, abs(lhs))


def test_ssst_step_sizes_adjoint_and_k1_closed_form():
    """SSST (structure tensors of first-order spatial and spectral differences):
    Lemma 1 on the assembled operator gives gamma_u = 1/(6k^2 + 1), gamma_Y = 1/2;
    the adjoint identity; with k = 1 each tensor is one row, its norm the
    nuclear norm."""
    got = O.lemma1_step_sizes(O.assemble_operator(4, 5, 3, 2, "ssst"))
    want = O.step_sizes(4, 5, 2, "paper", "ssst")
    for key in ("u", "s", "t", "Y", "y2", "y3"):
        assert got[key][0] == pytest.approx(want[key], rel=1e-12) and got[key][1], key
    r = np.random.default_rng(61)
    u = r.standard_normal((4, 5, 6))
    X = O.structure_tensors(u, 2, spectral_part=True)
    Y = r.standard_normal(X.shape)
    lhs, rhs = float((X * Y).sum()), float((u * O.ssst_adjoint_u(Y, 2, u.shape)).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))
    dv, dh, ds = (np.roll(u, -1, ax) - u for ax in (0, 1, 2))
    expect = np.sqrt((dv ** 2 + dh ** 2 + ds ** 2).sum(axis=2)).sum()
    assert O.objective(u, 1, reg="ssst") == pytest.approx(expect, rel=1e-12)


# ---------------------------------------------------------------------------
# Alg. 1, one whole pass written out by hand (steps 2-14 and the stop rule).
#
# Every step is an explicit index loop over the cube, in the order Alg. 1 prints
# them; the block operator comes from assemble_operator (built entry by entry
# from the index definitions), step 10 is the clip of the singular values of Y'
# at 1 (the Moreau form of eq. ProxConjugate, not the oracle's prox route), and
# the l1-ball projections are a bisection on the threshold (not the oracle's
# sort).  Steps 12-14 must read the extrapolated t_bar, u_bar, s_bar; the
# variants that read t+, u+, s+ instead are built too, and must disagree.
# ---------------------------------------------------------------------------
def _l1_bisect(x, r):
    """argmin ||y - x|| over ||y||_1 <= r: soft threshold at the tau with
    sum max(|x| - tau, 0) = r, found by bisection (r = 0 gives 0)."""
    a = np.abs(x)
    if a.sum() <= r:
        return x.copy()
    if r <= 0.0:
        return np.zeros_like(x)
    lo, hi = 0.0, float(a.max())
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if np.maximum(a - mid, 0.0).sum() > r:
            lo = mid
        else:
            hi = mid
    tau = 0.5 * (lo + hi)
    return np.sign(x) * np.maximum(a - tau, 0.0)


def _pass_by_hand(st, v, k, eps, alpha, beta, mu_min, mu_max, g, AY, read_bar=(True, True, True)):
    """One pass of Alg. 1 from state ``st``; ``read_bar`` = whether steps 12-14
    read (u_bar, s_bar, t_bar) (Alg. 1) or (u+, s+, t+) (a planted mistake)."""
    N1, N2, N3 = v.shape
    u, s, t, y2, y3, Y = (st[n] for n in ("u", "s", "t", "y2", "y3", "Y"))
    # step 2: u+ = P_[mu_min, mu_max](u - gamma_u (L^T Y + y3)), L^T from the assembled operator
    LtY = (AY.T @ Y.ravel()).reshape(v.shape)
    u_new = np.empty_like(u)
    for i in range(N1):
        for j in range(N2):
            for b in range(N3):
                x = u[i, j, b] - g["u"] * (LtY[i, j, b] + y3[i, j, b])
                u_new[i, j, b] = min(max(x, mu_min), mu_max)
    # step 3: s+ = P_{B1, alpha}(s - gamma_s y3)
    zs = np.empty_like(s)
    for i in range(N1):
        for j in range(N2):
            for b in range(N3):
                zs[i, j, b] = s[i, j, b] - g["s"] * y3[i, j, b]
    s_new = _l1_bisect(zs, alpha)
    # step 4: t+ = P_{B1, beta}(t - gamma_t (D_v^T y2 + y3)), (D_v^T y)[i] = y[i-1] - y[i]
    zt = np.empty_like(t)
    for i in range(N1):
        for j in range(N2):
            for b in range(N3):
                dvt = y2[(i - 1) % N1, j, b] - y2[i, j, b]
                zt[i, j, b] = t[i, j, b] - g["t"] * (dvt + y3[i, j, b])
    t_new = _l1_bisect(zt, beta)
    # steps 5-7: extrapolation
    ub, sb, tb = np.empty_like(u), np.empty_like(s), np.empty_like(t)
    for i in range(N1):
        for j in range(N2):
            for b in range(N3):
                ub[i, j, b] = 2.0 * u_new[i, j, b] - u[i, j, b]
                sb[i, j, b] = 2.0 * s_new[i, j, b] - s[i, j, b]
                tb[i, j, b] = 2.0 * t_new[i, j, b] - t[i, j, b]
    # steps 8-11: Y' = Y + gamma_Y P_l D D_s u_bar; Y+ = U min(Sigma, 1) V^T of Y'
    X = (AY @ ub.ravel()).reshape(Y.shape)
    Y_new = np.empty_like(Y)
    for l in range(Y.shape[0]):
        Yp = Y[l] + g["Y"] * X[l]
        U, sv, Vt = np.linalg.svd(Yp, full_matrices=False)
        Y_new[l] = (U * np.minimum(sv, 1.0)) @ Vt
    ru, rs, rt = (ub if read_bar[0] else u_new), (sb if read_bar[1] else s_new), (tb if read_bar[2] else t_new)
    # step 12: y2+ = y2 + gamma_2 D_v t_bar, (D_v x)[i] = x[i+1] - x[i]
    y2_new = np.empty_like(y2)
    for i in range(N1):
        for j in range(N2):
            for b in range(N3):
                y2_new[i, j, b] = y2[i, j, b] + g["y2"] * (rt[(i + 1) % N1, j, b] - rt[i, j, b])
    # step 13: y3' = y3 + gamma_3 (u_bar + s_bar + t_bar)
    y3p = np.empty_like(y3)
    for i in range(N1):
        for j in range(N2):
            for b in range(N3):
                y3p[i, j, b] = y3[i, j, b] + g["y3"] * (ru[i, j, b] + rs[i, j, b] + rt[i, j, b])
    # step 14: y3+ = y3' - gamma_3 P_{B2, eps}^v(y3' / gamma_3)
    ss = 0.0
    for i in range(N1):
        for j in range(N2):
            for b in range(N3):
                ss += (y3p[i, j, b] / g["y3"] - v[i, j, b]) ** 2
    nrm = math.sqrt(ss)
    y3_new = np.empty_like(y3)
    for i in range(N1):
        for j in range(N2):
            for b in range(N3):
                w = y3p[i, j, b] / g["y3"]
                pw = w if nrm <= eps else v[i, j, b] + eps * (w - v[i, j, b]) / nrm
                y3_new[i, j, b] = y3p[i, j, b] - g["y3"] * pw
    # eq. StopCri_simulated with the previous iterate's norm (||u+ - u|| alone if ||u|| = 0)
    du2, nu2 = 0.0, 0.0
    for i in range(N1):
        for j in range(N2):
            for b in range(N3):
                du2 += (u_new[i, j, b] - u[i, j, b]) ** 2
                nu2 += u[i, j, b] ** 2
    relc = math.sqrt(du2) / math.sqrt(nu2) if nu2 > 0 else math.sqrt(du2)
    return {"u": u_new, "s": s_new, "t": t_new, "y2": y2_new, "y3": y3_new, "Y": Y_new}, relc


def _hand_case(policy):
    from synthetic import CubeSpec, make_cube, random_state
    N1, N2, N3, k = 4, 5, 3, 2
    _, v = make_cube(CubeSpec(N1, N2, N3, regions=2, endmembers=2, seed=31))
    v = v.astype(np.float64)
    st = {key: val.astype(np.float64) for key, val in random_state(N1, N2, N3, k, seed=32, scale=0.6).items()}
    st["u"] = st["u"] * 1.4 - 0.2  # some entries outside the box, so step 2's clamp acts
    g = O.step_sizes(N1, N2, k, policy)
    AY = O.assemble_operator(N1, N2, N3, k)[("Y", "u")]
    # radii that make every projection of the pass active: half the l1 norms of
    # the arguments of steps 3-4, half the distance of step 14's argument
    big, _ = _pass_by_hand(st, v, k, 1e30, 1e30, 1e30, 0.0, 1.0, g, AY)
    zs = st["s"] - g["s"] * st["y3"]
    zt = st["t"] - g["t"] * (np.roll(st["y2"], 1, axis=0) - st["y2"] + st["y3"])
    alpha, beta = 0.5 * np.abs(zs).sum(), 0.5 * np.abs(zt).sum()
    probe, _ = _pass_by_hand(st, v, k, 1e30, alpha, beta, 0.0, 1.0, g, AY)
    bars = [2 * probe[x] - st[x] for x in ("u", "s", "t")]
    eps = 0.5 * np.linalg.norm((st["y3"] + g["y3"] * sum(bars)) / g["y3"] - v)
    return st, v, k, eps, alpha, beta, g, AY


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("policy", ["paper", "pc_exact"])
def test_one_pass_by_hand(policy):
    st, v, k, eps, alpha, beta, g, AY = _hand_case(policy)
    want, rel_want = _pass_by_hand(st, v, k, eps, alpha, beta, 0.0, 1.0, g, AY)
    got, rel_got = O.iterate(st, v, k, eps, alpha, beta, 0.0, 1.0, g)
    for key in ("u", "s", "t", "y2", "y3", "Y"):
        assert _rel(got[key], want[key]) <= 1e-11, key
    assert rel_got == pytest.approx(rel_want, rel=1e-12)
    # the case is not degenerate: every projection is active and the
    # extrapolated values differ from the new ones
    assert np.any(want["u"] == 0.0) or np.any(want["u"] == 1.0)
    assert np.abs(want["s"]).sum() == pytest.approx(alpha, rel=1e-9)
    assert np.abs(want["t"]).sum() == pytest.approx(beta, rel=1e-9)
    for x in ("u", "s", "t"):
        assert _rel(2 * want[x] - st[x], want[x]) > 0.1


@pytest.mark.parametrize("planted", [(False, True, True), (True, False, True), (True, True, False)])
def test_one_pass_by_hand_detects_unextrapolated_reads(planted):
    """Steps 12-14 reading u+, s+ or t+ instead of the extrapolated values is a
    plausible slip; the hand pass built that way must be far from the oracle,
    so the pin above would catch it."""
    st, v, k, eps, alpha, beta, g, AY = _hand_case("pc_exact")
    wrong, _ = _pass_by_hand(st, v, k, eps, alpha, beta, 0.0, 1.0, g, AY, read_bar=planted)
    got, _ = O.iterate(st, v, k, eps, alpha, beta, 0.0, 1.0, g)
    keys = ("y3",) if planted[2] else ("y2", "y3")
    for key in keys:
        assert _rel(got[key], wrong[key]) > 1e-3, key


def test_relative_change_uses_the_previous_iterate():
    """C7: ||u+ - u|| / ||u|| with u the iterate before the pass.  All duals 0
    and u = 2 everywhere (outside the box [0, 1]): step 2 only clamps, u+ = 1,
    so the relative change is |1 - 2| / |2| = 1/2 exactly (1 if the new
    iterate's norm were used)."""
    shape = (3, 4, 3)
    v = np.full(shape, 0.5)
    st = O.init_state(v, 2)
    st["u"] = np.full(shape, 2.0)
    g = O.step_sizes(3, 4, 2, "pc_exact")
    new, rel = O.iterate(st, v, 2, 1e6, 1e6, 1e6, 0.0, 1.0, g)
    assert np.all(new["u"] == 1.0)
    assert rel == 0.5


def test_relative_change_at_zero_iterate():
    """C7 with ||u|| = 0: the change itself.  u = 0, y3 = -c everywhere, all
    other duals 0: u+ = gamma_u c (inside the box), so the relative change is
    gamma_u c sqrt(N)."""
    shape = (3, 4, 3)
    v = np.full(shape, 0.5)
    st = O.init_state(v, 2)
    st["u"] = np.zeros(shape)
    c = 0.75
    st["y3"] = np.full(shape, -c)
    g = O.step_sizes(3, 4, 2, "pc_exact")
    new, rel = O.iterate(st, v, 2, 1e6, 1e6, 1e6, 0.0, 1.0, g)
    np.testing.assert_allclose(new["u"], g["u"] * c, rtol=1e-15)
    assert rel == pytest.approx(g["u"] * c * math.sqrt(v.size), rel=1e-14)


def test_solve_counts_completed_passes_and_stops_on_the_first_crossing():
    """C7: the test runs after every pass; the count is the passes completed."""
    v = np.full((4, 4, 3), 0.37)  # a fixed point: the first pass already changes nothing
    st, it, rel = O.solve(v, 2, 1.0, 1.0, 1.0, max_iter=50, tol=1e-5)
    assert it == 1 and rel == 0.0
    from synthetic import CubeSpec, make_cube
    _, v = make_cube(CubeSpec(6, 6, 4, regions=2, endmembers=2, seed=33))
    trace = []
    O.solve(v, 2, 0.5, 1.0, 1.0, max_iter=40, tol=0.0, policy="pc_exact", trace=trace)
    tol = trace[25] * 1.0000001  # first crossing at pass 26 unless an earlier pass is lower
    first = next(i for i, r in enumerate(trace) if r < tol) + 1
    st, it, rel = O.solve(v, 2, 0.5, 1.0, 1.0, max_iter=40, tol=tol, policy="pc_exact")
    assert it == first and rel == trace[first - 1]
    st, it, rel = O.solve(v, 2, 0.5, 1.0, 1.0, max_iter=7, tol=1e-30, policy="pc_exact")
    assert it == 7
