"""Seeded synthetic hyperspectral cubes shaped like the scenes of the S3TTV paper.

This module is the one piece shared by the FP64 oracle (``oracle/``) and the CUDA
path (``paper_2404_03313_gb300``).  It draws random numbers and builds inputs; it
holds none of the denoising method's arithmetic (no differences, no projections,
no radii rule).

Recipe (the paper's real scenes are not available, so seeded synthetic cubes of
the same kind stand in for them; the noise model is the paper's, Sec. IV-A,
cases 1-8):

* endmembers: ``M`` spectra, each a sum of three Gaussian bumps over
  ``x_b = (b + 0.5) / N3`` with centres ~ U(0, 1), widths ~ U(0.05, 0.25) and
  amplitudes ~ U(0.2, 1), then min-max scaled to [0.05, 0.95];
* regions: ``R`` Voronoi sites ~ U over the N1 x N2 grid (Euclidean distance,
  no wrap, ties to the lowest site index); each region gets abundances
  ~ Dirichlet(1_M);
* clean cube: ``clean[i, j, :] = sum_m A[r(i, j), m] * E[m]`` (values in [0.05, 0.95]);
* noise, in this order: white Gaussian noise of standard deviation ``sigma``;
  vertical stripes (per band, ``round(p_t * N2)`` columns drawn without
  replacement, each shifted by one constant ~ U(-0.5, 0.5) over the whole
  column); salt-and-pepper on ``round(p_s * N)`` entries drawn without
  replacement, each set to 0 or 1 with probability 1/2 (applied last, so it
  overwrites the other noise).

Arrays are C-contiguous ``[N1][N2][N3]`` (band fastest): element (i, j, b) sits at
``(i * N2 + j) * N3 + b``.  Random draws use numpy's PCG64 ``default_rng(seed)`` in a
fixed order, so a seed fixes the cube on every machine.
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = ["CubeSpec", "make_cube", "WORKLOADS", "random_state", "batch_specs", "network_params",
           "warm_start_specs"]


@dataclasses.dataclass(frozen=True)
class CubeSpec:
    """Shape, scene structure and noise levels of one synthetic cube."""

    N1: int
    N2: int
    N3: int
    regions: int = 6
    endmembers: int = 3
    sigma: float = 0.1
    p_s: float = 0.05
    p_t: float = 0.05
    k: int = 3
    seed: int = 0


# The workloads: a parity case small enough for the FP64 oracle to finish in
# seconds, the 256x256x128 headline cube, the larger 304x304x191 cube, and
# cubes of the paper's scene sizes with its 10 x 10 blocks.
WORKLOADS = {
    "parity_32x32x16_k3": CubeSpec(32, 32, 16, regions=6, endmembers=3, sigma=0.1,
                                   p_s=0.05, p_t=0.05, k=3, seed=0),
    "s3ttv_256x256x128_k5": CubeSpec(256, 256, 128, regions=32, endmembers=5, sigma=0.05,
                                     p_s=0.05, p_t=0.10, k=5, seed=0),
    "s3ttv_304x304x191_k5": CubeSpec(304, 304, 191, regions=32, endmembers=5, sigma=0.1,
                                     p_s=0.05, p_t=0.05, k=5, seed=0),
    # a quarter of the headline cube's pixels, for profiler captures that must stay small
    "profile_128x128x128_k5": CubeSpec(128, 128, 128, regions=16, endmembers=5, sigma=0.05,
                                       p_s=0.05, p_t=0.10, k=5, seed=0),
    # the paper's own scene sizes (Sec. IV) with its 10 x 10 blocks
    "profile_64x64x64_k10": CubeSpec(64, 64, 64, regions=8, endmembers=5, sigma=0.1, p_s=0.05, p_t=0.05,
                                     k=10, seed=0),
    "paper_100x100x198_k10": CubeSpec(100, 100, 198, regions=8, endmembers=5, sigma=0.1,
                                      p_s=0.05, p_t=0.05, k=10, seed=0),
    "paper_120x120x98_k10": CubeSpec(120, 120, 98, regions=8, endmembers=5, sigma=0.1,
                                     p_s=0.05, p_t=0.05, k=10, seed=0),
    "paper_100x100x128_k10": CubeSpec(100, 100, 128, regions=8, endmembers=5, sigma=0.1,
                                      p_s=0.05, p_t=0.05, k=10, seed=0),
    "paper_120x120x198_k10": CubeSpec(120, 120, 198, regions=8, endmembers=5, sigma=0.1,
                                      p_s=0.05, p_t=0.05, k=10, seed=0),
    "paper_100x100x360_k10": CubeSpec(100, 100, 360, regions=8, endmembers=5, sigma=0.1,
                                      p_s=0.05, p_t=0.05, k=10, seed=0),
}


def batch_specs(count: int = 64, seed: int = 0, size_range=(64, 256)):
    """An uneven batch of cubes: the shape and noise of cube i come from one
    batch generator seeded with `seed`, its contents from seed 1000 + i.

    N1, N2 ~ U{lo..hi} (size_range), N3 from {31, 64, 128, 191}, sigma from
    {0.05, 0.1}, p_s = 0.05, p_t from {0, 0.05, 0.10}, k from {3, 5},
    R = max(4, N1 N2 // 2048) regions, M = 5 endmembers.
    """
    rng = np.random.default_rng(seed)
    lo, hi = size_range
    specs = []
    for i in range(count):
        N1, N2 = (int(x) for x in rng.integers(lo, hi + 1, size=2))
        N3 = int(rng.choice([31, 64, 128, 191]))
        sigma = float(rng.choice([0.05, 0.1]))
        p_t = float(rng.choice([0.0, 0.05, 0.10]))
        k = int(rng.choice([3, 5]))
        specs.append(CubeSpec(N1, N2, N3, regions=max(4, N1 * N2 // 2048), endmembers=5, sigma=sigma,
                              p_s=0.05, p_t=p_t, k=k, seed=1000 + i))
    return specs


def _endmembers(rng: np.random.Generator, M: int, N3: int) -> np.ndarray:
    x = (np.arange(N3, dtype=np.float64) + 0.5) / N3
    E = np.zeros((M, N3), dtype=np.float64)
    for m in range(M):
        centres = rng.uniform(0.0, 1.0, size=3)
        widths = rng.uniform(0.05, 0.25, size=3)
        amps = rng.uniform(0.2, 1.0, size=3)
        for c, w, a in zip(centres, widths, amps):
            E[m] += a * np.exp(-0.5 * ((x - c) / w) ** 2)
        lo, hi = E[m].min(), E[m].max()
        if hi > lo:
            E[m] = 0.05 + 0.9 * (E[m] - lo) / (hi - lo)
        else:
            E[m] = 0.5
    return E


def _labels(rng: np.random.Generator, N1: int, N2: int, R: int) -> np.ndarray:
    sites = np.stack([rng.uniform(0, N1, size=R), rng.uniform(0, N2, size=R)], axis=1)
    ii, jj = np.meshgrid(np.arange(N1) + 0.5, np.arange(N2) + 0.5, indexing="ij")
    best = np.full((N1, N2), np.inf)
    lab = np.zeros((N1, N2), dtype=np.int64)
    for r in range(R):  # strict '<' keeps the lowest index on ties
        d = (ii - sites[r, 0]) ** 2 + (jj - sites[r, 1]) ** 2
        closer = d < best
        lab[closer] = r
        best[closer] = d[closer]
    return lab


def make_cube(spec: CubeSpec):
    """Return ``(clean, v)`` as float32 arrays of shape (N1, N2, N3).

    ``v`` is the noisy observation that both the oracle and the GPU solver read.
    Both are rounded to float32 once here, so the two sides start from the same
    bits (the oracle widens them to float64).
    """
    N1, N2, N3 = spec.N1, spec.N2, spec.N3
    rng = np.random.default_rng(spec.seed)
    E = _endmembers(rng, spec.endmembers, N3)
    lab = _labels(rng, N1, N2, spec.regions)
    A = rng.dirichlet(np.ones(spec.endmembers), size=spec.regions)  # (R, M)
    clean = (A @ E)[lab]  # (N1, N2, N3)

    v = clean + rng.normal(0.0, spec.sigma, size=clean.shape) if spec.sigma > 0 else clean.copy()
    n_cols = int(round(spec.p_t * N2))
    if n_cols > 0:
        for b in range(N3):
            cols = rng.choice(N2, size=n_cols, replace=False)
            offs = rng.uniform(-0.5, 0.5, size=n_cols)
            v[:, cols, b] += offs[None, :]
    N = N1 * N2 * N3
    n_sp = int(round(spec.p_s * N))
    if n_sp > 0:
        flat = v.reshape(-1)
        idx = rng.choice(N, size=n_sp, replace=False)
        flat[idx] = (rng.uniform(0.0, 1.0, size=n_sp) < 0.5).astype(np.float64)
    return clean.astype(np.float32), v.astype(np.float32)


def random_state(N1: int, N2: int, N3: int, k: int, seed: int, scale: float = 0.3):
    """Random P-PDS state (u, s, t, y2, y3, Y, ubar) for one-step parity tests.

    ``Y`` has shape (N1*N2, k*k, 2*N3) in the paper's column order (eq. SSST):
    column 2b holds the vertical and column 2b+1 the horizontal difference of
    band b.  Values are plain Gaussians; nothing here is a solver iterate.
    """
    rng = np.random.default_rng(seed)
    shp = (N1, N2, N3)
    st = {
        "u": rng.uniform(0.0, 1.0, size=shp),
        "s": scale * rng.standard_normal(shp),
        "t": scale * rng.standard_normal(shp),
        "y2": scale * rng.standard_normal(shp),
        "y3": scale * rng.standard_normal(shp),
        "Y": scale * rng.standard_normal((N1 * N2, k * k, 2 * N3)),
    }
    return {key: val.astype(np.float32) for key, val in st.items()}


def network_params(shapes, seed: int, head_scale: float = 0.1) -> np.ndarray:
    """Seeded initial parameters of a convolutional network, flat float32.

    ``shapes`` lists the parameter arrays in order: a 3-D weight (out, taps, in)
    draws He-normal values, N(0, 2 / (taps * in)); a 2-D weight (out, in) draws
    N(0, head_scale^2 / in); a 1-D bias is zero.  Only random draws happen here.
    """
    rng = np.random.default_rng(seed)
    parts = []
    for shp in shapes:
        if len(shp) == 3:
            parts.append(rng.standard_normal(shp) * np.sqrt(2.0 / (shp[1] * shp[2])))
        elif len(shp) == 2:
            parts.append(rng.standard_normal(shp) * (head_scale / np.sqrt(shp[1])))
        else:
            parts.append(np.zeros(shp))
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def warm_start_specs(count: int, seed: int, shape=(128, 128, 64)):
    """Training or evaluation cubes for the learned warm start: ``count`` cubes
    of one shape with cube i seeded ``seed + i``; noise levels cycle through
    sigma in {0.05, 0.1} and stripe rates in {0.05, 0.10}, sparse rate 0.05,
    k = 5, 32 regions of 5 endmembers (fewer regions on small cubes)."""
    N1, N2, N3 = shape
    R = max(4, min(32, (N1 * N2) // 2048))
    out = []
    for i in range(count):
        out.append(CubeSpec(N1, N2, N3, regions=R, endmembers=5, sigma=(0.05, 0.1)[i % 2], p_s=0.05,
                            p_t=(0.05, 0.10)[(i // 2) % 2], k=5, seed=seed + i))
    return out
