"""ctypes binding of libs3ttv.so (include/s3ttv.h): argument marshalling only.

Every step of the solver runs in the library's CUDA kernels.  Arrays may be torch
tensors (CUDA or CPU) or numpy arrays; they must be float32 and C-contiguous.
If the shared library is missing, every call raises S3TTVError: there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libs3ttv.so")

# status codes (s3ttv_status)
OK, MAXITER, EINVAL, ENOMEM, ECUDA, ENUMERIC, EUNSUPPORTED, ESTATE, ETOOBIG = 0, 1, -1, -2, -3, -4, -5, -6, -7
L1_STATIC_MAX_N = 4294967295
STEP_PAPER, STEP_PC_EXACT = 0, 1
OPT_STEP_POLICY, OPT_CHECK_EVERY, OPT_JACOBI_MAX_SWEEPS, OPT_JACOBI_TOL, OPT_PROFILE, OPT_WARM_START = 1, 2, 3, 4, 5, 6
OPT_TENSOR_CORES = 7
OPT_LAYOUT, OPT_SPECTRAL_BOUNDARY = 8, 9
LAYOUT_PAPER, LAYOUT_STACKED = 0, 1
SPECTRAL_PERIODIC, SPECTRAL_OPEN = 0, 1
OPT_REGULARIZER = 10
OPT_AUTOTUNE = 11
OPT_HSSTV_OMEGA = 12
OPT_FP64_FALLBACK = 13
OPT_ALLOC_LIMIT = 14
OPT_NVTX = 15
OPT_JACOBI_POLISH_TOL = 16
OPT_FIRST_ORDER = 17
OPT_BATCH_WORKLIST = 18
REG_S3TTV, REG_STV, REG_SSTV, REG_HSSTV1, REG_HSSTV2, REG_SSST = 0, 1, 2, 3, 4, 5
KERNEL_CLASSES = ("primal", "l1_search", "block_dual", "dual", "finalize")
STATE = {"u": 0, "s": 1, "t": 2, "y2": 3, "y3": 4, "Y": 5}

# Every symbol include/s3ttv.h declares, with (restype, argtypes).
_c_int, _c_ll, _c_f, _c_d, _vp = ctypes.c_int, ctypes.c_longlong, ctypes.c_float, ctypes.c_double, ctypes.c_void_p


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("converged", ctypes.c_int),
                ("jacobi_nonconverged", ctypes.c_int), ("rel_change", ctypes.c_double),
                ("seconds", ctypes.c_double), ("jacobi_sweeps", ctypes.c_double),
                ("jacobi_fallbacks", ctypes.c_int), ("first_order", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Problem(ctypes.Structure):
    """s3ttv_problem: one cube of a batched solve."""
    _fields_ = [("v", _vp), ("N1", ctypes.c_int), ("N2", ctypes.c_int), ("N3", ctypes.c_int),
                ("eps", ctypes.c_float), ("alpha", ctypes.c_float), ("beta", ctypes.c_float),
                ("mu_min", ctypes.c_float), ("mu_max", ctypes.c_float), ("k", ctypes.c_int),
                ("u", _vp), ("s", _vp), ("t", _vp)]


_P = ctypes.POINTER
SIGNATURES = {
    "s3ttv_create": (_c_int, [_P(_vp), _c_int, _vp]),
    "s3ttv_fp32_peak": (_c_int, [_c_int, _c_int, _P(_c_d)]),
    "s3ttv_destroy": (None, [_vp]),
    "s3ttv_strerror": (ctypes.c_char_p, [_c_int]),
    "s3ttv_last_error": (ctypes.c_char_p, [_vp]),
    "s3ttv_set_option": (_c_int, [_vp, _c_int, _c_d]),
    "s3ttv_workspace_bytes": (_c_ll, [_vp]),
    "s3ttv_launch_count": (_c_ll, [_vp]),
    "s3ttv_kernel_stats": (_c_int, [_vp, _P(_c_d), _P(_c_ll)]),
    "s3ttv_solve": (_c_int, [_vp, _vp, _c_int, _c_int, _c_int, _c_f, _c_f, _c_f, _c_f, _c_f, _c_int, _c_int,
                             _c_f, _vp, _vp, _vp, _P(Info)]),
    "s3ttv_solve_batched": (_c_int, [_vp, _c_int, _P(Problem), _c_int, _c_f, _P(Info)]),
    "s3ttv_setup": (_c_int, [_vp, _vp, _c_int, _c_int, _c_int, _c_f, _c_f, _c_f, _c_f, _c_f, _c_int]),
    "s3ttv_iterate": (_c_int, [_vp, _c_int, _c_f, _P(Info)]),
    "s3ttv_get_state": (_c_int, [_vp, _c_int, _vp]),
    "s3ttv_set_state": (_c_int, [_vp, _c_int, _vp]),
    "s3ttv_l1_ball": (_c_int, [_vp, _vp, _vp, _c_ll, _c_d, _P(_c_d)]),
    "s3ttv_block_dual": (_c_int, [_vp, _vp, _vp, _vp, _vp, _c_int, _c_int, _c_int, _c_int, _c_f, _P(Info)]),
    "s3ttv_l1_ball_static": (_c_int, [_vp, _vp, _c_ll, _c_d, _P(_c_d), _vp]),
    "s3ttv_radii": (_c_int, [_c_ll, _c_d, _c_d, _c_d, _c_d, _P(_c_d), _P(_c_d), _P(_c_d)]),
    "s3ttv_step_sizes": (_c_int, [_c_int, _c_int, _c_int, _c_int, _P(_c_d)]),
    "s3ttv_objective": (_c_int, [_vp, _vp, _c_int, _c_int, _c_int, _c_int, _P(_c_d)]),
    "s3ttv_tuned_form": (_c_int, [_vp, _P(_c_int), _P(_c_int)]),
    "s3ttv_quality": (_c_int, [_vp, _vp, _vp, _c_int, _c_int, _c_int, _c_int, _P(_c_d), _P(_c_d), _P(_c_d), _vp]),
    "s3ttv_net_param_count": (_c_ll, []),
    "s3ttv_net_create": (_c_int, [_P(_vp), _c_int, _vp]),
    "s3ttv_net_destroy": (None, [_vp]),
    "s3ttv_net_last_error": (ctypes.c_char_p, [_vp]),
    "s3ttv_net_set_params": (_c_int, [_vp, _vp]),
    "s3ttv_net_get_params": (_c_int, [_vp, _vp]),
    "s3ttv_net_forward": (_c_int, [_vp, _vp, _c_int, _c_int, _c_int, _c_int, _vp, _vp, _vp]),
    "s3ttv_net_gradient": (_c_int, [_vp, _vp, _vp, _vp, _vp, _c_int, _c_int, _c_int, _c_int, _P(_c_d), _vp]),
    "s3ttv_net_train_step": (_c_int, [_vp, _vp, _vp, _vp, _vp, _c_int, _c_int, _c_int, _c_int, _c_f, _P(_c_d)]),
}


class S3TTVError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"s3ttv status {status}: {msg}")
        self.status = status


_LIB = None


def library():
    """Load libs3ttv.so (once) and declare its signatures."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise S3TTVError(ECUDA, f"{LIB_PATH} is not built; run paper_2404_03313_gb300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, n=None, name="array"):
    """Device or host address of a float32 C-contiguous array (torch or numpy)."""
    if x is None:
        return None
    if _is_torch(x):
        import torch
        if x.dtype != torch.float32 or not x.is_contiguous():
            raise S3TTVError(EINVAL, f"{name} must be a contiguous float32 tensor")
        if n is not None and x.numel() != n:
            raise S3TTVError(EINVAL, f"{name} has {x.numel()} elements, expected {n}")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if x.dtype != np.float32 or not x.flags["C_CONTIGUOUS"]:
            raise S3TTVError(EINVAL, f"{name} must be a C-contiguous float32 array")
        if n is not None and x.size != n:
            raise S3TTVError(EINVAL, f"{name} has {x.size} elements, expected {n}")
        return x.ctypes.data
    raise S3TTVError(EINVAL, f"{name}: unsupported array type {type(x)}")


def _empty_like(x, shape):
    if _is_torch(x):
        import torch
        return torch.empty(shape, dtype=torch.float32, device=x.device)
    return np.empty(shape, dtype=np.float32)


def _sync_torch(*arrays):
    """Make torch's pending work on CUDA inputs visible to the library's stream."""
    for x in arrays:
        if x is not None and _is_torch(x) and x.is_cuda:
            import torch
            torch.cuda.current_stream(x.device).synchronize()
            return


def radii(N, sigma, p_s, p_t, rho=0.95):
    """eq. (RadiusSet) as implemented by the library: returns (eps, alpha, beta)."""
    e, a, b = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rc = library().s3ttv_radii(int(N), float(sigma), float(p_s), float(p_t), float(rho),
                               ctypes.byref(e), ctypes.byref(a), ctypes.byref(b))
    if rc:
        raise S3TTVError(rc, "s3ttv_radii")
    return e.value, a.value, b.value


def l1_ball_static(x, radius, out=None, stream=None):
    """Allocation-free l1-ball projection (s3ttv_l1_ball_static) for callers that
    cannot allocate device memory: x and out must be CUDA tensors on the current
    device; returns (out, tau).  Its fixed scratch is shared by every call, so
    calls must not overlap on the GPU."""
    n = int(np.prod(x.shape))
    out = _empty_like(x, x.shape) if out is None else out
    if _is_torch(x) and _is_torch(out) and x.is_cuda and out.is_cuda:
        import torch
        cur = torch.cuda.current_device()
        if x.device.index != cur or out.device.index != cur:
            raise S3TTVError(EINVAL, "s3ttv_l1_ball_static: x and out must be on the current CUDA device")
    tau = ctypes.c_double()
    st = None
    if stream is not None:
        st = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    _sync_torch(x)
    rc = library().s3ttv_l1_ball_static(_ptr(x, n, "x"), _ptr(out, n, "out"), n, float(radius),
                                        ctypes.byref(tau), st)
    if rc < 0:
        raise S3TTVError(rc, "s3ttv_l1_ball_static: " + library().s3ttv_strerror(rc).decode())
    return out, tau.value


def step_sizes(N1, N2, k, policy=STEP_PAPER):
    g = (ctypes.c_double * 6)()
    rc = library().s3ttv_step_sizes(N1, N2, k, policy, g)
    if rc:
        raise S3TTVError(rc, "s3ttv_step_sizes")
    return dict(zip(("u", "s", "t", "Y", "y2", "y3"), list(g)))


def fp32_peak(device=0, packed=False):
    """Measured FP32 rate of the device in TFLOP/s (s3ttv_fp32_peak): scalar or
    packed FP32x2 FMA chains over a full grid."""
    t = ctypes.c_double()
    rc = library().s3ttv_fp32_peak(int(device), 1 if packed else 0, ctypes.byref(t))
    if rc:
        raise S3TTVError(rc, "s3ttv_fp32_peak")
    return t.value


class Solver:
    """One s3ttv_ctx: a device, a stream, and the workspace of one problem."""

    def __init__(self, device: int = 0, stream=None):
        self._lib = library()
        h = ctypes.c_void_p()
        st = None
        if stream is not None:
            st = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        rc = self._lib.s3ttv_create(ctypes.byref(h), int(device), st)
        if rc:
            raise S3TTVError(rc, f"s3ttv_create(device={device}) failed")
        self._h = h
        self.device = device
        self.shape = None
        self.k = None

    def close(self):
        if getattr(self, "_h", None):
            self._lib.s3ttv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc, what):
        if rc < 0:
            msg = self._lib.s3ttv_last_error(self._h).decode(errors="replace")
            raise S3TTVError(rc, f"{what}: {msg}")
        return rc

    def set_option(self, key, value):
        self._check(self._lib.s3ttv_set_option(self._h, key, float(value)), "set_option")
        if key == OPT_LAYOUT:
            self.layout = int(value)
        if key == OPT_REGULARIZER:
            self.reg = int(value)

    def workspace_bytes(self):
        return int(self._lib.s3ttv_workspace_bytes(self._h))

    def launch_count(self):
        return int(self._lib.s3ttv_launch_count(self._h))

    def kernel_stats(self):
        """{class: (total ms, launches)} since profiling was switched on."""
        ms = (ctypes.c_double * len(KERNEL_CLASSES))()
        n = (ctypes.c_longlong * len(KERNEL_CLASSES))()
        self._check(self._lib.s3ttv_kernel_stats(self._h, ms, n), "kernel_stats")
        return {name: (ms[i], n[i]) for i, name in enumerate(KERNEL_CLASSES)}

    def solve(self, v, eps, alpha, beta, k, mu_min=0.0, mu_max=1.0, max_iter=5000, tol=1e-5,
              out=None):
        """Run Alg. 1 on v (N1, N2, N3); returns (u, s, t, info dict)."""
        N1, N2, N3 = v.shape
        n = N1 * N2 * N3
        u, s, t = out if out is not None else (_empty_like(v, v.shape) for _ in range(3))
        info = Info()
        _sync_torch(v)
        rc = self._lib.s3ttv_solve(self._h, _ptr(v, n, "v"), N1, N2, N3, eps, alpha, beta, mu_min, mu_max, k,
                                   max_iter, tol, _ptr(u, n, "u"), _ptr(s, n, "s"), _ptr(t, n, "t"),
                                   ctypes.byref(info))
        self._check(rc, "s3ttv_solve")
        self.shape, self.k = (N1, N2, N3), k
        return u, s, t, info.as_dict()

    def solve_batched(self, problems, max_iter=5000, tol=1e-5):
        """Solve several cubes at once (s3ttv_solve_batched).  problems: a list of
        dicts with keys v (N1, N2, N3), eps, alpha, beta, k and optionally mu_min,
        mu_max.  Returns a list of (u, s, t, info dict), outputs shaped and placed
        like each v."""
        n = len(problems)
        arr = (Problem * n)()
        outs = []
        for i, p in enumerate(problems):
            v = p["v"]
            N1, N2, N3 = v.shape
            m = N1 * N2 * N3
            u, s, t = (_empty_like(v, v.shape) for _ in range(3))
            outs.append((u, s, t))
            arr[i] = Problem(_ptr(v, m, "v"), N1, N2, N3, p["eps"], p["alpha"], p["beta"],
                             p.get("mu_min", 0.0), p.get("mu_max", 1.0), p["k"],
                             _ptr(u, m, "u"), _ptr(s, m, "s"), _ptr(t, m, "t"))
        infos = (Info * n)()
        _sync_torch(*[p["v"] for p in problems])
        rc = self._lib.s3ttv_solve_batched(self._h, n, arr, int(max_iter), float(tol), infos)
        self._check(rc, "s3ttv_solve_batched")
        return [(u, s, t, infos[i].as_dict()) for i, (u, s, t) in enumerate(outs)]

    def setup(self, v, eps, alpha, beta, k, mu_min=0.0, mu_max=1.0):
        N1, N2, N3 = v.shape
        _sync_torch(v)
        rc = self._lib.s3ttv_setup(self._h, _ptr(v, N1 * N2 * N3, "v"), N1, N2, N3, eps, alpha, beta,
                                   mu_min, mu_max, k)
        self._check(rc, "s3ttv_setup")
        self.shape, self.k = (N1, N2, N3), k
        self._problem = {"v": v, "eps": float(eps), "alpha": float(alpha), "beta": float(beta), "k": int(k),
                         "mu_min": float(mu_min), "mu_max": float(mu_max)}

    def save(self, path):
        """Write the problem and the whole P-PDS state (u, s, t, y2, y3 and the
        block duals Y) to a .npz file, so that a later ``load`` continues the
        iteration where it stopped (the eigen-solves then start cold once)."""
        p = getattr(self, "_problem", None)
        if p is None:
            raise S3TTVError(ESTATE, "save before setup")
        v = p["v"].cpu().numpy() if _is_torch(p["v"]) else np.asarray(p["v"])
        arrays = {name: self.get_state(name) for name in STATE}
        np.savez(path, v=v, **arrays, **{key: np.asarray(p[key]) for key in
                                        ("eps", "alpha", "beta", "k", "mu_min", "mu_max")})

    def load(self, path, device_arrays=True):
        """Set up the problem stored by ``save`` and restore its state."""
        z = np.load(path)
        v = np.ascontiguousarray(z["v"], dtype=np.float32)
        if device_arrays:
            import torch
            v = torch.from_numpy(v).to(f"cuda:{self.device}")
        self.setup(v, float(z["eps"]), float(z["alpha"]), float(z["beta"]), int(z["k"]), float(z["mu_min"]),
                   float(z["mu_max"]))
        for name in STATE:
            self.set_state(name, np.ascontiguousarray(z[name], dtype=np.float32))

    def iterate(self, n, tol=0.0):
        info = Info()
        rc = self._lib.s3ttv_iterate(self._h, int(n), float(tol), ctypes.byref(info))
        self._check(rc, "s3ttv_iterate")
        return info.as_dict()

    def _state_size(self, which):
        N1, N2, N3 = self.shape
        if which == "Y":
            if getattr(self, "reg", REG_S3TTV) == REG_SSTV:
                return (2, N1, N2, N3)
            if getattr(self, "reg", REG_S3TTV) in (REG_HSSTV1, REG_HSSTV2):
                return (4, N1, N2, N3)
            if getattr(self, "reg", REG_S3TTV) == REG_SSST:
                return (N1 * N2, self.k * self.k, 3 * N3)
            if getattr(self, "layout", LAYOUT_PAPER) == LAYOUT_STACKED:
                return (N1 * N2, 2 * self.k * self.k, N3)
            return (N1 * N2, self.k * self.k, 2 * N3)
        return (N1, N2, N3)

    def get_state(self, which, like=None):
        shp = self._state_size(which)
        dst = _empty_like(like, shp) if like is not None else np.empty(shp, np.float32)
        self._check(self._lib.s3ttv_get_state(self._h, STATE[which], _ptr(dst, int(np.prod(shp)), which)),
                    "get_state")
        return dst

    def set_state(self, which, src):
        shp = self._state_size(which)
        _sync_torch(src)
        self._check(self._lib.s3ttv_set_state(self._h, STATE[which], _ptr(src, int(np.prod(shp)), which)),
                    "set_state")

    def l1_ball(self, x, radius, out=None):
        """Projection onto the l1 ball of the given radius; returns (out, tau)."""
        n = int(np.prod(x.shape))
        out = _empty_like(x, x.shape) if out is None else out
        tau = ctypes.c_double()
        _sync_torch(x)
        self._check(self._lib.s3ttv_l1_ball(self._h, _ptr(x, n, "x"), _ptr(out, n, "out"), n, float(radius),
                                            ctypes.byref(tau)), "s3ttv_l1_ball")
        return out, tau.value

    def tuned_form(self):
        """(tensor_cores, ctas_per_sm) the autotuner chose, or (-1, 0)."""
        tc, cp = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.s3ttv_tuned_form(self._h, ctypes.byref(tc), ctypes.byref(cp)), "s3ttv_tuned_form")
        return tc.value, cp.value

    def objective(self, u, k):
        """S3TTV(u), the sum of the nuclear norms of the structure tensors of all blocks."""
        N1, N2, N3 = u.shape
        val = ctypes.c_double()
        _sync_torch(u)
        self._check(self._lib.s3ttv_objective(self._h, _ptr(u, N1 * N2 * N3, "u"), N1, N2, N3, int(k),
                                              ctypes.byref(val)), "s3ttv_objective")
        return val.value

    def quality(self, u, ref, trim=3, sam_map=False):
        """{mpsnr, mssim, sam} of u against ref (MSSIM needs N1, N2 >= 11), plus
        the 2-D SAM map (N1, N2) when sam_map is true."""
        N1, N2, N3 = u.shape
        n = N1 * N2 * N3
        ps, ss, sm = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        want_ssim = N1 >= 11 and N2 >= 11
        m = _empty_like(u, (N1, N2)) if sam_map else None
        _sync_torch(u, ref)
        self._check(self._lib.s3ttv_quality(self._h, _ptr(u, n, "u"), _ptr(ref, n, "ref"), N1, N2, N3, int(trim),
                                            ctypes.byref(ps), ctypes.byref(ss) if want_ssim else None,
                                            ctypes.byref(sm), _ptr(m, N1 * N2, "sam_map") if sam_map else None),
                    "s3ttv_quality")
        out = {"mpsnr": ps.value, "mssim": ss.value if want_ssim else None, "sam": sm.value}
        if sam_map:
            out["sam_map"] = m
        return out

    def block_dual(self, Y, ubar, k, gamma_Y=0.25):
        """Alg. 1 steps 8-11 on every block; Y (L, k*k, 2*N3) is updated in place.
        Returns (Zv, Zh, info)."""
        N1, N2, N3 = ubar.shape
        n = N1 * N2 * N3
        Zv, Zh = _empty_like(ubar, ubar.shape), _empty_like(ubar, ubar.shape)
        info = Info()
        _sync_torch(Y, ubar)
        rc = self._lib.s3ttv_block_dual(self._h, _ptr(Y, N1 * N2 * k * k * 2 * N3, "Y"), _ptr(ubar, n, "ubar"),
                                        _ptr(Zv, n, "Zv"), _ptr(Zh, n, "Zh"), N1, N2, N3, k, gamma_Y,
                                        ctypes.byref(info))
        self._check(rc, "s3ttv_block_dual")
        return Zv, Zh, info.as_dict()


def _vol_shape(x):
    """(B, D, H, W) of a cube (N1, N2, N3) or a batch (B, N1, N2, N3)."""
    shp = tuple(x.shape)
    if len(shp) == 3:
        return (1,) + shp
    if len(shp) == 4:
        return shp
    raise S3TTVError(EINVAL, f"expected a cube (N1, N2, N3) or a batch (B, N1, N2, N3), got {shp}")


class WarmStartNet:
    """The learned warm start's 3-D U-Net (s3ttv_net_*): forward, gradient and
    Adam training steps on the library's kernels.  Arrays are float32 cubes
    (N1, N2, N3) or batches (B, N1, N2, N3), torch (CUDA or CPU) or numpy."""

    def __init__(self, device: int = 0, stream=None):
        self._lib = library()
        h = ctypes.c_void_p()
        st = None
        if stream is not None:
            st = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        rc = self._lib.s3ttv_net_create(ctypes.byref(h), int(device), st)
        if rc:
            raise S3TTVError(rc, f"s3ttv_net_create(device={device}) failed")
        self._h = h
        self.device = device
        self.param_count = int(self._lib.s3ttv_net_param_count())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.s3ttv_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc, what):
        if rc < 0:
            msg = self._lib.s3ttv_net_last_error(self._h).decode(errors="replace")
            raise S3TTVError(rc, f"{what}: {msg}")
        return rc

    def set_params(self, theta):
        _sync_torch(theta)
        self._check(self._lib.s3ttv_net_set_params(self._h, _ptr(theta, self.param_count, "theta")), "set_params")

    def get_params(self, like=None):
        out = _empty_like(like, (self.param_count,)) if like is not None else np.empty(self.param_count, np.float32)
        self._check(self._lib.s3ttv_net_get_params(self._h, _ptr(out, self.param_count, "theta")), "get_params")
        return out

    def forward(self, v):
        """Predicted (u, s, t), shaped and placed like v."""
        B, D, H, W = _vol_shape(v)
        n = B * D * H * W
        u, s, t = (_empty_like(v, v.shape) for _ in range(3))
        _sync_torch(v)
        self._check(self._lib.s3ttv_net_forward(self._h, _ptr(v, n, "v"), B, D, H, W, _ptr(u, n, "u"),
                                                _ptr(s, n, "s"), _ptr(t, n, "t")), "s3ttv_net_forward")
        return u, s, t

    def gradient(self, v, u_ref, s_ref, t_ref, grad=None):
        """(loss, flat gradient) of the mean squared error against (u_ref, s_ref, t_ref)."""
        B, D, H, W = _vol_shape(v)
        n = B * D * H * W
        g = grad if grad is not None else np.empty(self.param_count, np.float32)
        loss = ctypes.c_double()
        _sync_torch(v, u_ref, s_ref, t_ref)
        self._check(self._lib.s3ttv_net_gradient(self._h, _ptr(v, n, "v"), _ptr(u_ref, n, "u_ref"),
                                                 _ptr(s_ref, n, "s_ref"), _ptr(t_ref, n, "t_ref"), B, D, H, W,
                                                 ctypes.byref(loss), _ptr(g, self.param_count, "grad")),
                    "s3ttv_net_gradient")
        return loss.value, g

    def train_step(self, v, u_ref, s_ref, t_ref, lr):
        """One Adam step; returns the loss before it."""
        B, D, H, W = _vol_shape(v)
        n = B * D * H * W
        loss = ctypes.c_double()
        _sync_torch(v, u_ref, s_ref, t_ref)
        self._check(self._lib.s3ttv_net_train_step(self._h, _ptr(v, n, "v"), _ptr(u_ref, n, "u_ref"),
                                                   _ptr(s_ref, n, "s_ref"), _ptr(t_ref, n, "t_ref"), B, D, H, W,
                                                   float(lr), ctypes.byref(loss)), "s3ttv_net_train_step")
        return loss.value
