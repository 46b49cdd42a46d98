"""GB300-native S3TTV hyperspectral denoising and destriping.

The solver (Alg. 1 of the paper, P-PDS) runs in hand-written sm_103a CUDA kernels
behind the C ABI of ``include/s3ttv.h`` (``libs3ttv.so``); this package is the
thin ctypes binding over it plus the build script.  ``warmstart`` trains and
applies the learned warm start (a 3-D U-Net, also on the library's kernels).  Nothing here computes on the
CPU: if the library is not built, calls raise ``S3TTVError``.
"""
from ._binding import (  # noqa: F401
    Info, S3TTVError, Solver, WarmStartNet, library, radii, step_sizes, l1_ball_static, fp32_peak, LIB_PATH, SIGNATURES, STATE,
    L1_STATIC_MAX_N, ETOOBIG,
    STEP_PAPER, STEP_PC_EXACT, OPT_STEP_POLICY, OPT_CHECK_EVERY, OPT_JACOBI_MAX_SWEEPS, OPT_JACOBI_TOL,
    OPT_PROFILE, OPT_WARM_START, OPT_TENSOR_CORES, OPT_LAYOUT, OPT_SPECTRAL_BOUNDARY, LAYOUT_PAPER,
    LAYOUT_STACKED, SPECTRAL_PERIODIC, SPECTRAL_OPEN, OPT_REGULARIZER, OPT_AUTOTUNE, OPT_HSSTV_OMEGA, OPT_FP64_FALLBACK, OPT_ALLOC_LIMIT, OPT_NVTX, OPT_JACOBI_POLISH_TOL, OPT_FIRST_ORDER, OPT_BATCH_WORKLIST, REG_S3TTV, REG_STV, REG_SSTV, REG_HSSTV1,
    REG_HSSTV2, REG_SSST, KERNEL_CLASSES,
    OK, MAXITER, EINVAL, ENOMEM, ECUDA, ENUMERIC, EUNSUPPORTED, ESTATE,
)
