"""Convergence traces of Alg. 1, the quantities Fig. 11 of the paper plots:
the relative change ||u^(t+1) - u^(t)|| / ||u^(t)|| (the stop rule's value),
the objective S3TTV(u), and MPSNR and MSSIM of u against a reference cube,
recorded every few passes.  Every number comes from the library
(``s3ttv_iterate``, ``s3ttv_objective``, ``s3ttv_quality``)."""
from __future__ import annotations

from ._binding import OPT_STEP_POLICY, STEP_PAPER, Solver

__all__ = ["convergence_trace"]


def convergence_trace(v, ref, eps, alpha, beta, k, passes, every=10, policy=STEP_PAPER, mu_min=0.0, mu_max=1.0,
                      solver: Solver | None = None, device=0, objective=True, trim=3):
    """Run ``passes`` passes of Alg. 1 on v from the usual start and return one
    record per ``every`` passes: {"iter", "rel_change", "objective", "mpsnr",
    "mssim", "sam"} (objective None when not asked for; mssim None on cubes
    narrower than 11 pixels)."""
    own = solver is None
    sv = solver if solver is not None else Solver(device)
    try:
        sv.set_option(OPT_STEP_POLICY, policy)
        sv.setup(v, eps, alpha, beta, k, mu_min, mu_max)
        rows, done = [], 0
        while done < passes:
            n = min(every, passes - done)
            info = sv.iterate(n, 0.0)
            done += info["iters"]
            u = sv.get_state("u", like=v)
            q = sv.quality(u, ref, trim=trim)
            rows.append({"iter": done, "rel_change": info["rel_change"],
                         "objective": sv.objective(u, k) if objective else None,
                         "mpsnr": q["mpsnr"], "mssim": q["mssim"], "sam": q["sam"]})
        return rows
    finally:
        if own:
            sv.close()
