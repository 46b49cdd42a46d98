"""Learned warm start for Alg. 1, on the library's kernels.

The paper has none: Alg. 1 starts from u = v, s = t = 0.  Here a 3-D U-Net
(``WarmStartNet``, ``s3ttv_net_*`` in include/s3ttv.h) is trained on pairs
(noisy cube, converged solver output) and its prediction (u, s, t) becomes the
solver's starting point through ``s3ttv_set_state``; the duals start at zero as
usual, or the block duals from the prediction (``dual_scale``).  The solver
alone decides the result; the network can only change how many passes the
stop rule needs.

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
          solver: Solver | None = None, device=0, settle=32, dual_scale=0.0, trace_ref=None, trace_every=16):
    """Alg. 1 on v from the cold start (net None) or from the network's
    prediction.  Returns a dict with u, s, t, the solver info (`iters` counts
    every pass), `seconds` (all of it: inference, set-up and passes) and
    `net_seconds` (inference alone).

    dual_scale > 0 also starts the block duals from the network's u: Y =
    the singular values of dual_scale * X(u_pred) clipped at 1 (one block-dual
    step from Y = 0 with gamma_Y = dual_scale).  With trace_ref (the clean cube)
    the MPSNR of u is recorded every trace_every passes as `trace`: [(passes,
    MPSNR)] (the traced run's `seconds` include the measurements).

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
            if dual_scale > 0:
                N1, N2, N3 = v.shape
                Y = torch.zeros(N1 * N2, k * k, 2 * N3, dtype=torch.float32, device=v.device)
                with Solver(device) as aux:
                    aux.block_dual(Y, init[0].contiguous(), k, gamma_Y=float(dual_scale))
                sv.set_state("Y", Y)
                del Y
        trace = [] if trace_ref is not None else None

        def run(n, stop_tol):
            if trace is None:
                return sv.iterate(n, stop_tol)
            done, last = 0, None
            while done < n:
                last = sv.iterate(min(trace_every, n - done), stop_tol)
                done += last["iters"]
                base = trace[-1][0] if trace else 0
                trace.append((base + last["iters"], sv.quality(sv.get_state("u", like=v), trace_ref)["mpsnr"]))
                if last["converged"]:
                    break
            last["iters"] = done
            return last

        if init is not None and settle > 0:
            first = run(min(settle, max_iter), 0.0)
            info = first
            if first["iters"] < max_iter:
                info = run(max_iter - first["iters"], tol)
                info["iters"] += first["iters"]
        else:
            info = run(max_iter, tol)
        u = sv.get_state("u", like=v)
        s = sv.get_state("s", like=v)
        t = sv.get_state("t", like=v)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
    finally:
        if own:
            sv.close()
    return {"u": u, "s": s, "t": t, "info": info, "seconds": t2 - t0, "net_seconds": t1 - t0, "trace": trace}
