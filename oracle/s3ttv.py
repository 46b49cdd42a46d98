"""Plain FP64 restatement of S3TTV denoising / destriping (Takemoto, Naganuma, Ono).

TEST INFRASTRUCTURE ONLY: the oracle the CUDA path is checked against.  Nothing
in the product imports this module.

Everything follows the paper's notation and the order of its steps:

* Sec. II-A: forward differences D_v, D_h, D_s with periodic boundaries.
* Sec. II-B: prox, conjugate prox (Moreau, eq. ProxConjugate), projections.
* Sec. II-C: P-PDS and Lemma 1 (diagonal preconditioners, eq. Preconditioners).
* Sec. III-A: spatio-spectral structure tensors (eq. SSST, eq. rewrite_Lu).
* Sec. III-C: Alg. 1 and the proximity operators it uses (eq. prox_box_constraint,
  eq. prox_zeroset, eq. prox_l2ball_constraint, eq. prox_nuclear_norm, the
  l1-ball projection) and the step sizes (eq. stepsize_denoising).
* Sec. IV-A: radii rule (eq. RadiusSet), stopping rule (eq. StopCri_simulated),
  MPSNR (eq. MPSNR), MSSIM (eq. MSSIM), 2-D SAM (eq. 2D_SAM), the objective of
  Prob. (S3TTV_denoising).
* Sec. IV: the comparison regularisers run through the same P-PDS (``reg=``):
  STV, SSTV, HSSTV1/2 and SSST, with their Lemma 1 step sizes.
* Layout variants (``layout="stacked"``, ``periodic_s=False``): the (2k^2) x N3
  stacking of the vertical and horizontal rows and the open spectral boundary.

Readings of passages the paper leaves open:
D_v differences along the first (vertical, i) axis and D_h along the second (j);
blocks are all N1*N2 stride-1 k x k windows with periodic wrap, one per anchor
(p, q) covering pixels (p+a, q+c), a, c in [0, k); block row r = a*k + c; column
2b is the vertical and 2b+1 the horizontal difference of band b; initial values
u = v, s = t = 0, all duals 0; the stop test uses ||u^(t)|| of the previous
iterate (||u+ - u|| alone when ||u|| = 0).

Arrays are (N1, N2, N3) float64, element (i, j, b).
"""
from __future__ import annotations

import math
import numpy as np

__all__ = [
    "AXIS_V", "AXIS_H", "AXIS_S", "HSSTV_OMEGA", "diff", "diff_adj", "spectral_diffs", "spectral_diff_adjoint", "structure_tensors",
    "structure_tensors_adjoint", "structure_tensor_block", "linear_op_adjoint_u",
    "linear_op_adjoint_u_at",
    "prox_nuclear", "ssst_adjoint_u", "block_dual_update", "proj_box", "proj_l2_ball",
    "proj_l1_ball", "step_sizes", "assemble_operator", "lemma1_step_sizes",
    "radii", "init_state", "iterate", "solve", "mpsnr", "objective", "ssim_window", "ssim_band", "mssim",
    "sam_map",
]

AXIS_V, AXIS_H, AXIS_S = 0, 1, 2
# HSSTV's weight of the first-order spatial differences (a reading: the paper
# names HSSTV [Takeyama et al. 2020] without its parameters)
HSSTV_OMEGA = 0.05


# ----------------------------------------------------------------------------
# Sec. II-A: difference operators (forward, periodic boundary).
# ----------------------------------------------------------------------------
def diff(x: np.ndarray, axis: int) -> np.ndarray:
    """Forward difference with periodic boundary: (D x)[i] = x[i+1] - x[i] (Sec. II-A)."""
    return np.roll(x, -1, axis=axis) - x


def diff_adj(y: np.ndarray, axis: int) -> np.ndarray:
    """Adjoint of :func:`diff`: (D^T y)[i] = y[i-1] - y[i] (periodic)."""
    return np.roll(y, 1, axis=axis) - y


# ----------------------------------------------------------------------------
# Sec. III-A: spatio-spectral structure tensors T_u^(l) = P_l D D_s u.
# ----------------------------------------------------------------------------
def spectral_diffs(u: np.ndarray, periodic_s: bool = True):
    """(D_v D_s u, D_h D_s u).  With periodic_s (Sec. II-A) D_s wraps from the
    last band to the first and both have N3 bands; otherwise D_s stops at the
    last band (x[b+1] - x[b], b < N3 - 1) and both have N3 - 1 bands."""
    Ds = diff(u, AXIS_S) if periodic_s else u[..., 1:] - u[..., :-1]
    return diff(Ds, AXIS_V), diff(Ds, AXIS_H)


def structure_tensors(u: np.ndarray, k: int, layout: str = "paper", periodic_s: bool = True,
                      second_order: bool = True, spectral_part: bool = False) -> np.ndarray:
    """All structure tensors of eq. (SSST) / eq. (rewrite_Lu).

    Block l = p*N2 + q holds the second-order differences D_v D_s u and D_h D_s u
    of the k x k window whose pixels are ((p+a) mod N1, (q+c) mod N2) (the
    footnote of Sec. III-A pads a window at the border with pixels from the
    opposite side); window pixel r = a*k + c.
    layout "paper" (eq. SSST): shape (L, k*k, 2*M), row r, columns
    [v_1 h_1 ... v_M h_M].  layout "stacked": shape (L, 2*k*k, M), row 2r the
    vertical and row 2r + 1 the horizontal differences of pixel r, one column per
    band.  M = N3 with the periodic D_s, N3 - 1 without.  second_order=False
    builds STV's tensors instead: first-order spatial differences D_v u, D_h u
    (no D_s; M = N3); with spectral_part as well, SSST's: a third part D_s u,
    columns [v_1 h_1 s_1 ... v_N3 h_N3 s_N3] (paper layout only).
    """
    N1, N2, N3 = u.shape
    if spectral_part:
        parts = (diff(u, AXIS_V), diff(u, AXIS_H), diff(u, AXIS_S))
        X = np.empty((N1, N2, k * k, 3 * N3))
        for a in range(k):
            for c in range(k):
                for o in range(3):
                    X[:, :, a * k + c, o::3] = np.roll(parts[o], shift=(-a, -c), axis=(0, 1))
        return X.reshape(N1 * N2, k * k, 3 * N3)
    Fv, Fh = spectral_diffs(u, periodic_s) if second_order else (diff(u, AXIS_V), diff(u, AXIS_H))
    M = Fv.shape[2]
    if layout == "paper":
        X = np.empty((N1, N2, k * k, 2 * M))
        for a in range(k):
            for c in range(k):
                r = a * k + c
                X[:, :, r, 0::2] = np.roll(Fv, shift=(-a, -c), axis=(0, 1))
                X[:, :, r, 1::2] = np.roll(Fh, shift=(-a, -c), axis=(0, 1))
        return X.reshape(N1 * N2, k * k, 2 * M)
    if layout == "stacked":
        X = np.empty((N1, N2, 2 * k * k, M))
        for a in range(k):
            for c in range(k):
                r = a * k + c
                X[:, :, 2 * r] = np.roll(Fv, shift=(-a, -c), axis=(0, 1))
                X[:, :, 2 * r + 1] = np.roll(Fh, shift=(-a, -c), axis=(0, 1))
        return X.reshape(N1 * N2, 2 * k * k, M)
    raise ValueError(f"unknown layout {layout!r}")


def structure_tensor_block(u: np.ndarray, k: int, p: int, q: int) -> np.ndarray:
    """One structure tensor T_u^(l) of eq. (SSST), anchor (p, q); shape (k*k, 2*N3)."""
    N1, N2, N3 = u.shape
    X = np.empty((k * k, 2 * N3))
    for a in range(k):
        for c in range(k):
            i, j = (p + a) % N1, (q + c) % N2
            i1, j1 = (i + 1) % N1, (j + 1) % N2
            ds = lambda ii, jj: np.roll(u[ii, jj], -1) - u[ii, jj]  # D_s along bands
            X[a * k + c, 0::2] = ds(i1, j) - ds(i, j)
            X[a * k + c, 1::2] = ds(i, j1) - ds(i, j)
    return X


def structure_tensors_adjoint(Y: np.ndarray, k: int, shape, layout: str = "paper",
                              periodic_s: bool = True) -> tuple[np.ndarray, np.ndarray]:
    """sum_l P_l^T Y_l split into its vertical and horizontal parts (Zv, Zh),
    each (N1, N2, M) with M as in :func:`structure_tensors`."""
    N1, N2, N3 = shape
    M = Y.shape[-1] // 2 if layout == "paper" else Y.shape[-1]
    Zv = np.zeros((N1, N2, M))
    Zh = np.zeros((N1, N2, M))
    if layout == "paper":
        Y = Y.reshape(N1, N2, k * k, 2 * M)
        parts = lambda r: (Y[:, :, r, 0::2], Y[:, :, r, 1::2])
    else:
        Y = Y.reshape(N1, N2, 2 * k * k, M)
        parts = lambda r: (Y[:, :, 2 * r], Y[:, :, 2 * r + 1])
    for a in range(k):
        for c in range(k):
            yv, yh = parts(a * k + c)
            Zv += np.roll(yv, shift=(a, c), axis=(0, 1))
            Zh += np.roll(yh, shift=(a, c), axis=(0, 1))
    return Zv, Zh


def spectral_diff_adjoint(w: np.ndarray, periodic_s: bool = True) -> np.ndarray:
    """Adjoint of the D_s of :func:`spectral_diffs`: (D_s^T w)[b] = w[b-1] - w[b],
    with w[-1] = w[N3-1] (periodic) or w[-1] = w[N3-1] = 0 (open; w has N3 - 1
    bands and the result N3)."""
    if periodic_s:
        return diff_adj(w, AXIS_S)
    pad = np.zeros(w.shape[:-1] + (w.shape[-1] + 2,))
    pad[..., 1:-1] = w
    return pad[..., :-1] - pad[..., 1:]


def ssst_adjoint_u(Y: np.ndarray, k: int, shape) -> np.ndarray:
    """SSST's dual-to-primal term: sum_l [D_v; D_h; D_s]^T P_l^T Y_l."""
    N1, N2, N3 = shape
    Y = Y.reshape(N1, N2, k * k, 3 * N3)
    Z = [np.zeros((N1, N2, N3)) for _ in range(3)]
    for a in range(k):
        for c in range(k):
            for o in range(3):
                Z[o] += np.roll(Y[:, :, a * k + c, o::3], shift=(a, c), axis=(0, 1))
    return diff_adj(Z[0], AXIS_V) + diff_adj(Z[1], AXIS_H) + diff_adj(Z[2], AXIS_S)


def linear_op_adjoint_u(Y: np.ndarray, k: int, shape, layout: str = "paper", periodic_s: bool = True,
                        second_order: bool = True) -> np.ndarray:
    """sum_l D_s^T D^T P_l^T Y_l, the dual-to-primal term of Alg. 1 step 2
    (sum_l D^T P_l^T Y_l for STV's first-order tensors)."""
    Zv, Zh = structure_tensors_adjoint(Y, k, shape, layout, periodic_s)
    w = diff_adj(Zv, AXIS_V) + diff_adj(Zh, AXIS_H)
    return spectral_diff_adjoint(w, periodic_s) if second_order else w


def linear_op_adjoint_u_at(Y: np.ndarray, k: int, shape, i: int, j: int, b: int) -> float:
    """One entry (i, j, b) of sum_l D_s^T D^T P_l^T Y_l, from the definitions.

    (D^T z)(i, j) = z_v(i-1, j) - z_v(i, j) + z_h(i, j-1) - z_h(i, j), then
    (D_s^T w)(b) = w(b-1) - w(b); z = sum_l P_l^T Y_l gathers, for pixel (x, y),
    row a*k + c of the block anchored at (x - a, y - c).  ``Y`` may be any array
    indexable as Y[l, r, col] (for example a GPU tensor moved block by block).
    """
    N1, N2, N3 = shape

    def z(x, y, o, bb):
        tot = 0.0
        for a in range(k):
            for c in range(k):
                l = ((x - a) % N1) * N2 + (y - c) % N2
                tot += float(Y[l, a * k + c, 2 * (bb % N3) + o])
        return tot

    def w(bb):
        return (z(i - 1, j, 0, bb) - z(i, j, 0, bb)) + (z(i, j - 1, 1, bb) - z(i, j, 1, bb))

    return w(b - 1) - w(b)


# ----------------------------------------------------------------------------
# Sec. II-B / III-C: proximity operators and projections.
# ----------------------------------------------------------------------------
def prox_nuclear(A: np.ndarray, gamma: float) -> np.ndarray:
    """prox of gamma*||.||_* by eq. (prox_nuclear_norm): U diag(max(s - gamma, 0)) V^T.

    ``A`` may be a stack (..., m, n); the SVD is numpy's (LAPACK gesdd).
    """
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    return U @ (np.maximum(s - gamma, 0.0)[..., :, None] * Vt)


def block_dual_update(Y: np.ndarray, X: np.ndarray, gamma_Y: float) -> np.ndarray:
    """Alg. 1 steps 9-10 for a stack of blocks.

    Y' = Y + gamma_Y X, then Y+ = Y' - gamma_Y prox_{gamma_Y^-1 ||.||_*}(gamma_Y^-1 Y'),
    which is the conjugate prox of eq. (ProxConjugate) applied to the nuclear norm.
    """
    Yp = Y + gamma_Y * X
    return Yp - gamma_Y * prox_nuclear(Yp / gamma_Y, 1.0 / gamma_Y)


def proj_box(x: np.ndarray, lo: float, hi: float) -> np.ndarray:
    """Projection onto [mu_min, mu_max]^N, eq. (prox_box_constraint)."""
    return np.minimum(np.maximum(x, lo), hi)


def proj_l2_ball(x: np.ndarray, center: np.ndarray, eps: float) -> np.ndarray:
    """Projection onto {x : ||x - v||_2 <= eps}, eq. (prox_l2ball_constraint)."""
    d = x - center
    nrm = math.sqrt(float(np.sum(d * d)))
    if nrm <= eps:
        return x.copy()
    return center + eps * d / nrm


def proj_l1_ball(x: np.ndarray, radius: float) -> np.ndarray:
    """Projection onto {x : ||x||_1 <= radius} (Sec. III-C, the l1-ball projection
    the paper cites from Condat 2016, in its sort-based form, O(N log N) as in
    Table II).

    With a_1 >= a_2 >= ... the sorted |x|: rho = max{j : a_j > (sum_{i<=j} a_i - r)/j},
    tau = (sum_{i<=rho} a_i - r)/rho, result sign(x) max(|x| - tau, 0).
    """
    a = np.abs(x).ravel()
    if a.sum() <= radius:
        return x.copy()
    if radius <= 0.0:
        return np.zeros_like(x)
    srt = np.sort(a)[::-1]
    cs = np.cumsum(srt)
    j = np.arange(1, srt.size + 1)
    rho = int(np.nonzero(srt > (cs - radius) / j)[0][-1]) + 1
    tau = (cs[rho - 1] - radius) / rho
    return np.sign(x) * np.maximum(np.abs(x) - tau, 0.0)


# ----------------------------------------------------------------------------
# Step sizes: eq. (stepsize_denoising) and Lemma 1 (eq. Preconditioners).
# ----------------------------------------------------------------------------
def step_sizes(N1: int, N2: int, k: int, policy: str = "paper", reg: str = "s3ttv") -> dict:
    """Step sizes of Alg. 1.

    For the comparison regularisers the paper runs through the same P-PDS (Sec.
    IV: the regularisation function of Prob. (S3TTV_denoising) replaced), the
    exact Lemma 1 values of their operators (``policy`` is ignored): STV
    (nuclear norms of P_l D u): gamma_u = 1/(4k^2 + 1), gamma_Y = 1/2; SSTV
    (l1 norm of D D_s u): gamma_u = 1/9, gamma_Y = 1/4.

    ``policy="paper"``: eq. (stepsize_denoising) as printed, gamma_u = 1/(8L + 1)
    with L = N1*N2 blocks.  ``policy="pc_exact"``: gamma_u = 1/(8k^2 + 1), the exact
    column abs-sum of Lemma 1 when every entry of D D_s u lies in k^2 blocks.
    The other five are the same in both (Lemma 1 reproduces them exactly).
    """
    L = N1 * N2
    if reg == "stv":
        return {"u": 1.0 / (4.0 * k * k + 1.0), "s": 1.0, "t": 1.0 / 3.0, "Y": 0.5, "y2": 0.5, "y3": 1.0 / 3.0}
    if reg == "sstv":
        return {"u": 1.0 / 9.0, "s": 1.0, "t": 1.0 / 3.0, "Y": 0.25, "y2": 0.5, "y3": 1.0 / 3.0}
    if reg == "ssst":
        # first-order D_v, D_h, D_s: column abs-sum 6 per block, in k^2 blocks; rows 2
        return {"u": 1.0 / (6.0 * k * k + 1.0), "s": 1.0, "t": 1.0 / 3.0, "Y": 0.5, "y2": 0.5, "y3": 1.0 / 3.0}
    if reg in ("hsstv1", "hsstv2"):
        # column abs-sum 8 + 4 omega (+1 for y3); the dual rows' sums are 4 and
        # 2 omega, and one gamma_Y = 1/4 serves all four parts (omega <= 2)
        return {"u": 1.0 / (9.0 + 4.0 * HSSTV_OMEGA), "s": 1.0, "t": 1.0 / 3.0, "Y": 0.25, "y2": 0.5,
                "y3": 1.0 / 3.0}
    if reg != "s3ttv":
        raise ValueError(reg)
    if policy == "paper":
        gu = 1.0 / (8.0 * L + 1.0)
    elif policy == "pc_exact":
        gu = 1.0 / (8.0 * k * k + 1.0)
    else:
        raise ValueError(policy)
    return {"u": gu, "s": 1.0, "t": 1.0 / 3.0, "Y": 0.25, "y2": 0.5, "y3": 1.0 / 3.0}


def assemble_operator(N1: int, N2: int, N3: int, k: int, reg: str = "s3ttv"):
    """The linear operator of Prob. (denoising2PPDS) as scipy.sparse blocks.

    Built entry by entry from the index definitions (not from :func:`diff`), so it
    is an independent construction.  Returns a dict of blocks A[(dual, primal)]
    with duals 'Y' (all L blocks stacked, row order (l, r, column) of eq. SSST),
    'y2', 'y3' and primals 'u', 's', 't'.
    """
    import scipy.sparse as sp

    N = N1 * N2 * N3

    def idx(i, j, b):
        return ((i % N1) * N2 + (j % N2)) * N3 + (b % N3)

    def dmat(axis):
        rows, cols, vals = [], [], []
        for i in range(N1):
            for j in range(N2):
                for b in range(N3):
                    r = idx(i, j, b)
                    nxt = [(i + 1, j, b), (i, j + 1, b), (i, j, b + 1)][axis]
                    rows += [r, r]
                    cols += [idx(*nxt), r]
                    vals += [1.0, -1.0]
        return sp.csr_matrix((vals, (rows, cols)), shape=(N, N))

    Dv, Dh, Ds = dmat(0), dmat(1), dmat(2)
    DvDs = (Dv @ Ds).tocsr()
    DhDs = (Dh @ Ds).tocsr()
    if reg == "stv":  # first-order spatial differences in the blocks
        DvDs, DhDs = Dv, Dh
    L = N1 * N2
    if reg == "ssst":  # blocks of [D_v u, D_h u, D_s u], columns 3b + o
        rows, cols, vals = [], [], []
        for p in range(N1):
            for q in range(N2):
                l = p * N2 + q
                for a in range(k):
                    for c in range(k):
                        r = a * k + c
                        for b in range(N3):
                            for o, M in ((0, Dv), (1, Dh), (2, Ds)):
                                row = (l * k * k + r) * 3 * N3 + 3 * b + o
                                src = M.getrow(idx(p + a, q + c, b))
                                rows += [row] * src.nnz
                                cols += list(src.indices)
                                vals += list(src.data)
        AY = sp.csr_matrix((vals, (rows, cols)), shape=(L * k * k * 3 * N3, N))
        I = sp.identity(N, format="csr")
        Z = sp.csr_matrix((N, N))
        return {("Y", "u"): AY, ("Y", "s"): sp.csr_matrix((AY.shape[0], N)),
                ("Y", "t"): sp.csr_matrix((AY.shape[0], N)), ("y2", "u"): Z, ("y2", "s"): Z, ("y2", "t"): Dv,
                ("y3", "u"): I, ("y3", "s"): I, ("y3", "t"): I}
    rows, cols, vals = [], [], []
    for p in range(N1):
        for q in range(N2):
            l = p * N2 + q
            for a in range(k):
                for c in range(k):
                    r = a * k + c
                    for b in range(N3):
                        for o, M in ((0, DvDs), (1, DhDs)):
                            row = (l * k * k + r) * 2 * N3 + 2 * b + o
                            src = M.getrow(idx(p + a, q + c, b))
                            rows += [row] * src.nnz
                            cols += list(src.indices)
                            vals += list(src.data)
    AY = sp.csr_matrix((vals, (rows, cols)), shape=(L * k * k * 2 * N3, N))
    if reg == "sstv":  # no blocks: the dual is (D_v D_s u, D_h D_s u) itself
        AY = sp.vstack([DvDs, DhDs]).tocsr()
    if reg in ("hsstv1", "hsstv2"):
        AY = sp.vstack([DvDs, DhDs, HSSTV_OMEGA * Dv, HSSTV_OMEGA * Dh]).tocsr()
    I = sp.identity(N, format="csr")
    Z = sp.csr_matrix((N, N))
    return {
        ("Y", "u"): AY, ("Y", "s"): sp.csr_matrix((AY.shape[0], N)),
        ("Y", "t"): sp.csr_matrix((AY.shape[0], N)),
        ("y2", "u"): Z, ("y2", "s"): Z, ("y2", "t"): Dv,
        ("y3", "u"): I, ("y3", "s"): I, ("y3", "t"): I,
    }


def lemma1_step_sizes(blocks) -> dict:
    """Lemma 1 (eq. Preconditioners): primal gamma = 1 / column abs-sum, dual
    gamma = 1 / row abs-sum, of the stacked operator; returns the per-variable
    value together with whether every column (row) of the variable agrees."""
    out = {}
    for prim in ("u", "s", "t"):
        colsum = sum(np.asarray(abs(blocks[(d, prim)]).sum(axis=0)).ravel() for d in ("Y", "y2", "y3"))
        out[prim] = (1.0 / colsum.max(), bool(np.allclose(colsum, colsum[0])))
    for dual in ("Y", "y2", "y3"):
        rowsum = sum(np.asarray(abs(blocks[(dual, p)]).sum(axis=1)).ravel() for p in ("u", "s", "t"))
        out[dual] = (1.0 / rowsum.max(), bool(np.allclose(rowsum, rowsum[0])))
    return out


def radii(N: int, sigma: float, p_s: float, p_t: float, rho: float = 0.95):
    """eq. (RadiusSet): alpha = rho N p_s / 2, beta = rho 0.5 N p_t (1 - p_s) / 2,
    eps = rho sqrt(sigma^2 N (1 - p_s)); with sigma = 0 the paper fixes eps = 0.01."""
    alpha = rho * N * p_s / 2.0
    beta = rho * 0.5 * N * p_t * (1.0 - p_s) / 2.0
    eps = rho * math.sqrt(sigma * sigma * N * (1.0 - p_s)) if sigma > 0 else 0.01
    return eps, alpha, beta


# ----------------------------------------------------------------------------
# Alg. 1: the P-PDS solver.
# ----------------------------------------------------------------------------
def init_state(v: np.ndarray, k: int, layout: str = "paper", periodic_s: bool = True, reg: str = "s3ttv") -> dict:
    """Initial values (Alg. 1 leaves them open): u = v, s = t = 0, duals 0.  For
    SSTV the dual Y is the pair (Y_v, Y_h) of cubes, shape (2, N1, N2, N3)."""
    v = np.asarray(v, dtype=np.float64)
    z = np.zeros_like(v)
    if reg == "sstv":
        Y = np.zeros((2,) + v.shape)
    elif reg in ("hsstv1", "hsstv2"):
        Y = np.zeros((4,) + v.shape)
    elif reg == "ssst":
        Y = np.zeros_like(structure_tensors(v, k, spectral_part=True))
    else:
        Y = np.zeros_like(structure_tensors(v, k, layout, periodic_s, reg != "stv"))
    return {"u": v.copy(), "s": z.copy(), "t": z.copy(), "y2": z.copy(), "y3": z.copy(), "Y": Y}


def iterate(state: dict, v: np.ndarray, k: int, eps: float, alpha: float, beta: float,
            mu_min: float, mu_max: float, gammas: dict, layout: str = "paper",
            periodic_s: bool = True, reg: str = "s3ttv") -> tuple[dict, float]:
    """One pass of Alg. 1 (steps 2-14); returns (new state, relative change).

    The relative change is eq. (StopCri_simulated): ||u+ - u||_2 / ||u||_2.
    ``layout`` and ``periodic_s`` choose the block matrices (see
    :func:`structure_tensors`); the paper's are the defaults.  ``reg`` replaces
    the regularisation function as Sec. IV does for the comparison methods:
    "stv" (block nuclear norms of first-order spatial differences) or "sstv"
    (l1 norm of D D_s u, whose conjugate prox is the projection onto the unit
    l_inf ball, computed here through eq. ProxConjugate and soft thresholding).
    """
    v = np.asarray(v, dtype=np.float64)
    u, s, t, y2, y3, Y = (state[n] for n in ("u", "s", "t", "y2", "y3", "Y"))
    g = gammas
    # Step 2: u update, box projection.
    if reg == "sstv":
        lin = spectral_diff_adjoint(diff_adj(Y[0], AXIS_V) + diff_adj(Y[1], AXIS_H), True)
    elif reg == "ssst":
        lin = ssst_adjoint_u(Y, k, u.shape)
    elif reg in ("hsstv1", "hsstv2"):
        lin = (spectral_diff_adjoint(diff_adj(Y[0], AXIS_V) + diff_adj(Y[1], AXIS_H), True)
               + HSSTV_OMEGA * (diff_adj(Y[2], AXIS_V) + diff_adj(Y[3], AXIS_H)))
    else:
        lin = linear_op_adjoint_u(Y, k, u.shape, layout, periodic_s, reg != "stv")
    u_new = proj_box(u - g["u"] * (lin + y3), mu_min, mu_max)
    # Step 3: sparse noise, l1 ball of radius alpha.
    s_new = proj_l1_ball(s - g["s"] * y3, alpha)
    # Step 4: stripe noise, l1 ball of radius beta.
    t_new = proj_l1_ball(t - g["t"] * (diff_adj(y2, AXIS_V) + y3), beta)
    # Steps 5-7: extrapolation.
    ub, sb, tb = 2.0 * u_new - u, 2.0 * s_new - s, 2.0 * t_new - t
    # Steps 8-11: every block dual, through the nuclear-norm conjugate prox.
    if reg == "sstv":
        Yp = Y + g["Y"] * np.stack(spectral_diffs(ub, True))
        w = Yp / g["Y"]  # Y+ = Y' - gamma prox_{||.||_1 / gamma}(Y' / gamma)
        Y_new = Yp - g["Y"] * np.sign(w) * np.maximum(np.abs(w) - 1.0 / g["Y"], 0.0)
    elif reg in ("hsstv1", "hsstv2"):
        A = np.stack(spectral_diffs(ub, True) + (HSSTV_OMEGA * diff(ub, AXIS_V), HSSTV_OMEGA * diff(ub, AXIS_H)))
        Yp = Y + g["Y"] * A
        w = Yp / g["Y"]  # Y+ = Y' - gamma prox_{||.|| / gamma}(Y' / gamma)
        if reg == "hsstv1":  # l1: soft thresholding entry by entry
            prox = np.sign(w) * np.maximum(np.abs(w) - 1.0 / g["Y"], 0.0)
        else:  # l1,2 over the four differences of each voxel: group soft thresholding
            nrm = np.sqrt((w * w).sum(axis=0, keepdims=True))
            prox = w * np.maximum(1.0 - (1.0 / g["Y"]) / np.maximum(nrm, 1e-300), 0.0)
        Y_new = Yp - g["Y"] * prox
    elif reg == "ssst":
        Y_new = block_dual_update(Y, structure_tensors(ub, k, spectral_part=True), g["Y"])
    else:
        Y_new = block_dual_update(Y, structure_tensors(ub, k, layout, periodic_s, reg != "stv"), g["Y"])
    # Step 12: prox of the conjugate of iota_{0} is the identity (eq. prox_zeroset).
    y2_new = y2 + g["y2"] * diff(tb, AXIS_V)
    # Steps 13-14: fidelity dual through the l2-ball projection.
    y3p = y3 + g["y3"] * (ub + sb + tb)
    y3_new = y3p - g["y3"] * proj_l2_ball(y3p / g["y3"], v, eps)
    du = math.sqrt(float(np.sum((u_new - u) ** 2)))
    nu = math.sqrt(float(np.sum(u * u)))
    rel = du / nu if nu > 0 else du
    return {"u": u_new, "s": s_new, "t": t_new, "y2": y2_new, "y3": y3_new, "Y": Y_new}, rel


def solve(v: np.ndarray, k: int, eps: float, alpha: float, beta: float, mu_min: float = 0.0,
          mu_max: float = 1.0, max_iter: int = 5000, tol: float = 1e-5, policy: str = "paper",
          state: dict | None = None, trace: list | None = None, layout: str = "paper", periodic_s: bool = True,
          reg: str = "s3ttv"):
    """Run Alg. 1 until the relative change is below ``tol`` or ``max_iter`` passes.

    Returns (state, iterations completed, last relative change).
    """
    v = np.asarray(v, dtype=np.float64)
    N1, N2, _ = v.shape
    gam = step_sizes(N1, N2, k, policy, reg)
    st = init_state(v, k, layout, periodic_s, reg) if state is None else state
    rel = float("inf")
    it = 0
    while it < max_iter:
        st, rel = iterate(st, v, k, eps, alpha, beta, mu_min, mu_max, gam, layout, periodic_s, reg)
        it += 1
        if trace is not None:
            trace.append(rel)
        if rel < tol:
            break
    return st, it, rel


# ----------------------------------------------------------------------------
# Sec. IV-A: evaluation.
# ----------------------------------------------------------------------------
def mpsnr(u: np.ndarray, ref: np.ndarray, trim: int = 3) -> float:
    """eq. (MPSNR) with peak 1, averaged over bands, the first and last ``trim``
    bands dropped (the paper cuts three because of the circulant boundary)."""
    u = np.asarray(u, np.float64)
    ref = np.asarray(ref, np.float64)
    N1, N2, N3 = u.shape
    bands = range(trim, N3 - trim) if N3 > 2 * trim else range(N3)
    vals = []
    for b in bands:
        err = float(np.sum((u[:, :, b] - ref[:, :, b]) ** 2))
        vals.append(10.0 * math.log10(N1 * N2 / err) if err > 0 else float("inf"))
    return float(np.mean(vals))


def objective(u: np.ndarray, k: int, layout: str = "paper", periodic_s: bool = True, reg: str = "s3ttv") -> float:
    """S3TTV(u) = sum_l ||T_u^(l)||_*, eq. (S3TTV_Lu) (for the chosen block
    matrices); STV's block nuclear norms of first-order differences; SSTV's
    ||D D_s u||_1."""
    u = np.asarray(u, np.float64)
    if reg == "sstv":
        Fv, Fh = spectral_diffs(u, True)
        return float(np.abs(Fv).sum() + np.abs(Fh).sum())
    if reg in ("hsstv1", "hsstv2"):
        A = np.stack(spectral_diffs(u, True) + (HSSTV_OMEGA * diff(u, AXIS_V), HSSTV_OMEGA * diff(u, AXIS_H)))
        return float(np.abs(A).sum() if reg == "hsstv1" else np.sqrt((A * A).sum(axis=0)).sum())
    if reg == "ssst":
        X = structure_tensors(u, k, spectral_part=True)
    else:
        X = structure_tensors(u, k, layout, periodic_s, reg != "stv")
    return float(np.linalg.svd(X, compute_uv=False).sum())


def ssim_window(radius: int = 5, sigma: float = 1.5) -> np.ndarray:
    """The (2 radius + 1)^2 Gaussian window of [Wang et al. 2004] (standard
    deviation 1.5, 11 x 11), normalized to sum 1."""
    x = np.arange(-radius, radius + 1, dtype=np.float64)
    g = np.exp(-(x[:, None] ** 2 + x[None, :] ** 2) / (2.0 * sigma * sigma))
    return g / g.sum()


def ssim_band(x: np.ndarray, y: np.ndarray, L: float = 1.0) -> float:
    """SSIM of two images [Wang et al. 2004] as eq. (MSSIM) cites it: local
    Gaussian-weighted means mu, variances sigma^2 and covariance sigma_xy at
    every pixel whose whole 11 x 11 window lies inside the image ("valid"
    windows), the map ((2 mu_x mu_y + C1)(2 sigma_xy + C2)) /
    ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 + sigma_y^2 + C2)) with C1 = (0.01 L)^2 and
    C2 = (0.03 L)^2, averaged over those pixels."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    w = ssim_window()
    r = w.shape[0] // 2
    H, W = x.shape
    C1, C2 = (0.01 * L) ** 2, (0.03 * L) ** 2

    def filt(img):
        out = np.zeros((H - 2 * r, W - 2 * r))
        for a in range(2 * r + 1):
            for b in range(2 * r + 1):
                out += w[a, b] * img[a:a + H - 2 * r, b:b + W - 2 * r]
        return out

    mx, my = filt(x), filt(y)
    sxx = filt(x * x) - mx * mx
    syy = filt(y * y) - my * my
    sxy = filt(x * y) - mx * my
    m = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    return float(m.mean())


def mssim(u: np.ndarray, ref: np.ndarray, trim: int = 3) -> float:
    """eq. (MSSIM): the SSIM of every band, averaged over the bands left after
    dropping the first and last ``trim`` (as for MPSNR)."""
    u = np.asarray(u, np.float64)
    ref = np.asarray(ref, np.float64)
    N3 = u.shape[2]
    bands = range(trim, N3 - trim) if N3 > 2 * trim else range(N3)
    return float(np.mean([ssim_band(ref[:, :, b], u[:, :, b]) for b in bands]))


def sam_map(u: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """eq. (2D_SAM): the angle (radians) between the spectra of u and ref at
    every pixel, arccos of the normalized inner product clipped to [-1, 1]; a
    pixel where either spectrum is zero gets pi / 2 (0 if both are zero)."""
    u = np.asarray(u, np.float64)
    ref = np.asarray(ref, np.float64)
    dot = (u * ref).sum(axis=2)
    nu = np.sqrt((u * u).sum(axis=2))
    nr = np.sqrt((ref * ref).sum(axis=2))
    out = np.empty(dot.shape)
    both = (nu > 0) & (nr > 0)
    out[both] = np.arccos(np.clip(dot[both] / (nu[both] * nr[both]), -1.0, 1.0))
    out[~both] = np.where((nu[~both] == 0) & (nr[~both] == 0), 0.0, np.pi / 2)
    return out
