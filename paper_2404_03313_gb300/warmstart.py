"""Learned warm start for Alg. 1, on the library's kernels.

The paper has none: Alg. 1 starts from u = v, s = t = 0.  Here a 3-D U-Net
(``WarmStartNet``, ``s3ttv_net_*`` in include/s3ttv.h) is trained on pairs
(noisy cube, converged solver output) and its prediction (u, s, t) becomes the
solver's starting point through ``s3ttv_set_state``; every dual starts at zero
as usual.  The solver alone decides the result; the network can only change how
many passes the stop rule needs.

Arrays are float32 CUDA tensors shaped (N1, N2, N3).  PyTorch only slices and
stacks training crops here; every arithmetic step runs in the library.
"""
from __future__ import annotations

import time

import numpy as np

from ._binding import OPT_STEP_POLICY, STEP_PAPER, Solver, WarmStartNet

__all__ = ["solver_targets", "train", "solve"]


def solver_targets(cubes, radii, k, max_iter, tol, policy=STEP_PAPER, device=0):
    """Solve every cube from the usual cold start; returns [(u, s, t, info)].

    cubes: list of (N1, N2, N3) CUDA tensors; radii: list of (eps, alpha, beta)."""
    out = []
    with Solver(device) as sv:
        sv.set_option(OPT_STEP_POLICY, policy)
        for v, (eps, alpha, beta) in zip(cubes, radii):
            u, s, t, info = sv.solve(v, eps, alpha, beta, k, max_iter=max_iter, tol=tol)
            out.append((u, s, t, info))
    return out


def train(net: WarmStartNet, inputs, targets, steps, crop=(32, 32, 32), batch=4, lr=1e-3, lr_final=1e-4, seed=0,
          log_every=0):
    """Adam on random crops: each step stacks `batch` crops of shape `crop` (each
    side a multiple of 4, at most the cube's) drawn from random training cubes.
    inputs: list of noisy cubes v; targets: list of (u, s, t).  The learning rate
    decays geometrically from lr to lr_final.  Returns the per-step losses."""
    import torch
    rng = np.random.default_rng(seed)
    losses = []
    for step in range(steps):
        f = step / max(1, steps - 1)
        rate = lr * (lr_final / lr) ** f
        vs, us, ss, ts = [], [], [], []
        for _ in range(batch):
            i = int(rng.integers(len(inputs)))
            v = inputs[i]
            o = [int(rng.integers(v.shape[a] - crop[a] + 1)) for a in range(3)]
            sl = tuple(slice(o[a], o[a] + crop[a]) for a in range(3))
            vs.append(v[sl])
            us.append(targets[i][0][sl])
            ss.append(targets[i][1][sl])
            ts.append(targets[i][2][sl])
        stack = [torch.stack(x).contiguous() for x in (vs, us, ss, ts)]
        losses.append(net.train_step(*stack, rate))
        if log_every and (step % log_every == 0 or step == steps - 1):
            print(f"step {step} loss {losses[-1]:.3e} lr {rate:.2e}", flush=True)
    return losses


def solve(v, eps, alpha, beta, k, net: WarmStartNet | None = None, max_iter=5000, tol=1e-5, policy=STEP_PAPER,
          solver: Solver | None = None, device=0, settle=32):
    """Alg. 1 on v from the cold start (net None) or from the network's
    prediction.  Returns a dict with u, s, t, the solver info (`iters` counts
    every pass), `seconds` (all of it: inference, set-up and passes) and
    `net_seconds` (inference alone).

    A warm start first runs `settle` passes without the stop test: the duals
    start at zero, so the first passes leave u almost where the network put it
    (exactly there if the prediction lies inside [mu_min, mu_max]), and the stop
    rule of eq. (StopCri_simulated), a relative change of u, would otherwise
    fire before the solver has done any work."""
    import torch
    own = solver is None
    sv = solver if solver is not None else Solver(device)
    try:
        sv.set_option(OPT_STEP_POLICY, policy)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        init = None
        if net is not None:
            init = net.forward(v)
        t1 = time.perf_counter()
        sv.setup(v, eps, alpha, beta, k)
        if init is not None:
            for name, x in zip(("u", "s", "t"), init):
                sv.set_state(name, x)
        if init is not None and settle > 0:
            first = sv.iterate(min(settle, max_iter), 0.0)
            info = first
            if first["iters"] < max_iter:
                info = sv.iterate(max_iter - first["iters"], tol)
                info["iters"] += first["iters"]
        else:
            info = sv.iterate(max_iter, tol)
        u = sv.get_state("u", like=v)
        s = sv.get_state("s", like=v)
        t = sv.get_state("t", like=v)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
    finally:
        if own:
            sv.close()
    return {"u": u, "s": s, "t": t, "info": info, "seconds": t2 - t0, "net_seconds": t1 - t0}
