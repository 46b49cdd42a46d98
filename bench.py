#!/usr/bin/env python3
"""Throughput of the S3TTV P-PDS solver (Alg. 1) on GB300.

One "step" is one full pass of Alg. 1 (steps 2-14: primal update, both l1-ball
projections, every block dual with its singular-value clip, both dual updates,
the fidelity projection and the stop test) over the whole cube.  The headline
workload is the seeded synthetic 256x256x128 cube with k = 5 blocks.

``value``  P-PDS passes per second over all ranks, inputs resident in HBM, timed
           with CUDA events on the solver's stream (max over ranks).
``e2e``    the same rate through the public C ABI call s3ttv_solve with pinned
           HOST buffers: setup, host->device copy of v, the passes and the
           device->host copy of u, s, t inside the timed region.
``roofline`` the dominant kernel (block dual, steps 8-11): algorithmic bytes per
           launch / its average CUDA-event duration in the timed region.
``cpu_baseline`` the FP64 oracle timed on this host: one pass over the whole
           cube (not scaled), the cores it really used (CPU seconds / wall
           seconds) and the CPU model, plus a one-thread run on a crop (a
           reported baseline, not a target).
``forms``  the same passes with the block-dual products on the tensor cores
           (three TF32 products per FP32 product) and as plain FP32 FMAs on
           the CUDA cores: passes/s and the block dual's roofline fraction.
``to_tol`` seconds and passes to the paper's stop rule (||u+ - u||/||u|| <
           1e-5, cap 5000) with the printed step sizes, and under PC_EXACT
           (gamma_u = 1/(8k^2 + 1), where the rule fires) for both product
           forms, with the restored cube's MPSNR.
``precision_form`` the 304x304x191 cube to the stop rule (PC_EXACT) with both
           product forms: seconds, passes and MPSNR side by side.

``--impl reference`` times the FP64 oracle instead (host cores, rank 0 only):
one step is one oracle pass over a crop of the cube, so ms_per_step x steps
is the time it really spends; value scales that rate to the full cube.
Multi-GPU: the method has no exchange step at one cube, so N ranks run N
independent replicas (weak scaling); only the timing is reduced over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "S3TTV seconds-to-tol at 256×256×128; P-PDS iters/s; % of roofline"
UNIT = "iter/s"
DEFAULT_WORKLOAD = "s3ttv_256x256x128_k5"
# block-dual forms (S3TTV_OPT_TENSOR_CORES)
FORM_NAMES = {2: "tensor_cores_3xtf32_stream", 1: "tensor_cores_3xtf32_group", 0: "cuda_cores_fp32"}
FORM_TEXT = {2: "tensor cores, each FP32 operand split into two TF32 parts; every warp streams a block of its own",
             1: "tensor cores, each FP32 operand split into two TF32 parts; four warps share each block",
             0: "CUDA cores, FP32 FMA"}
FALLBACK_HBM_GBS = 6800.0
# DRAM bytes (read + write) per voxel of one block-dual launch (the streaming
# form), from an ncu capture of the kernel whose source hashes to `sha`
# (profiles/block_dual_stream_k5_128x128x128.md); traffic is reported only
# while the kernel source is unchanged.
BLOCK_DUAL_TRAFFIC = {"sha": "8e1bfef7d4d9cdec", "k": 5, "bytes_per_voxel": (526.2528e6 + 495.520768e6) / 2097152}


# ---------------------------------------------------------------------------
# distributed helpers (replicas only)
# ---------------------------------------------------------------------------
def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def dist_init(backend):
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def dist_barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def dist_max(x, world, device=None):
    """Max of a float over ranks (identity at world size 1)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu_id)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def nvsmi_id(device_index):
    import torch
    try:
        props = torch.cuda.get_device_properties(device_index)
        bus = getattr(props, "pci_bus_id", None)
        dom = getattr(props, "pci_domain_id", None)
        dev = getattr(props, "pci_device_id", None)
        if bus is not None and dom is not None and dev is not None:
            return f"{dom:08x}:{bus:02x}:{dev:02x}.0"
    except Exception:
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [x for x in vis.split(",") if x.strip()]
    if ids and all(x.strip().isdigit() for x in ids) and device_index < len(ids):
        return ids[device_index].strip()
    return str(device_index)


def block_dual_source_sha():
    """sha256 prefix of the streaming block-dual kernel's sources (block_dual.cu
    and the internal header holding its shared device helpers)."""
    import hashlib
    h = hashlib.sha256()
    try:
        for name in ("block_dual.cu", "s3ttv_internal.cuh"):
            h.update(open(os.path.join(ROOT, "paper_2404_03313_gb300", "csrc", name), "rb").read())
    except OSError:
        return None
    return h.hexdigest()[:16]


def block_dual_traffic(k, N):
    """DRAM bytes of one block-dual launch, scaled by voxels from the ncu capture
    of the 128x128x128 case; None once the kernel's sources have changed."""
    if block_dual_source_sha() != BLOCK_DUAL_TRAFFIC["sha"] or k != BLOCK_DUAL_TRAFFIC["k"]:
        return None
    return BLOCK_DUAL_TRAFFIC["bytes_per_voxel"] * N


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded crop of the same workload
# ---------------------------------------------------------------------------
def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or "unknown"


def cpu_seconds():
    """User + system CPU seconds of this process so far (all its threads)."""
    import resource
    r = resource.getrusage(resource.RUSAGE_SELF)
    return r.ru_utime + r.ru_stime


def oracle_rate(spec, crop, seconds_budget, min_steps=2, max_steps=None, warmup=0, policy="paper"):
    """Time oracle passes on the top-left crop x crop x N3 of the workload cube
    (same generator, same noise model).  Returns a dict: full-cube passes/s
    (the crop's rate scaled by pixels), passes, seconds, seconds per crop pass,
    the crop's share of the cube, the cores actually used (CPU seconds / wall
    seconds over the timed passes) and a description of the sample."""
    import numpy as np
    import oracle as O
    from synthetic import CubeSpec, make_cube
    sub = CubeSpec(crop, crop, spec.N3, regions=max(2, spec.regions * crop * crop // (spec.N1 * spec.N2)),
                   endmembers=spec.endmembers, sigma=spec.sigma, p_s=spec.p_s, p_t=spec.p_t, k=spec.k,
                   seed=spec.seed)
    _, v = make_cube(sub)
    v = v.astype(np.float64)
    eps, alpha, beta = O.radii(v.size, sub.sigma, sub.p_s, sub.p_t)
    g = O.step_sizes(spec.N1, spec.N2, spec.k, policy)  # the full cube's step sizes
    st = O.init_state(v, spec.k)
    for _ in range(warmup):
        st, _ = O.iterate(st, v, spec.k, eps, alpha, beta, 0.0, 1.0, g)
    n, c0, t0 = 0, cpu_seconds(), time.perf_counter()
    while True:
        st, _ = O.iterate(st, v, spec.k, eps, alpha, beta, 0.0, 1.0, g)
        n += 1
        el = time.perf_counter() - t0
        if max_steps is not None and n >= max_steps:
            break
        if max_steps is None and n >= min_steps and el >= seconds_budget:
            break
    cores = (cpu_seconds() - c0) / el if el > 0 else 1.0
    frac = (crop * crop) / (spec.N1 * spec.N2)
    per_pass_full = el / n / frac
    sample = (f"{n} oracle passes (FP64, numpy/LAPACK SVD per block) on a {crop}x{crop}x{spec.N3} crop, "
              f"k={spec.k}, scaled by {spec.N1 * spec.N2}/{crop * crop} pixels to one full-cube pass")
    return {"rate": 1.0 / per_pass_full, "passes": n, "seconds": el, "seconds_per_pass": el / n,
            "fraction": frac, "cores": cores, "sample": sample}


def oracle_full_pass(spec, policy="paper"):
    """One oracle pass over the whole workload cube, timed (not scaled): returns
    (seconds, cores actually used)."""
    import numpy as np
    import oracle as O
    from synthetic import make_cube
    _, v = make_cube(spec)
    v = v.astype(np.float64)
    eps, alpha, beta = O.radii(v.size, spec.sigma, spec.p_s, spec.p_t)
    g = O.step_sizes(spec.N1, spec.N2, spec.k, policy)
    st = O.init_state(v, spec.k)
    c0, t0 = cpu_seconds(), time.perf_counter()
    st, _ = O.iterate(st, v, spec.k, eps, alpha, beta, 0.0, 1.0, g)
    el = time.perf_counter() - t0
    return el, (cpu_seconds() - c0) / el


def oracle_one_thread(workload, crop, seconds_budget, policy):
    """oracle_rate in a child process whose BLAS / LAPACK / OpenMP pools are
    limited to one thread."""
    env = dict(os.environ)
    for key in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[key] = "1"
    code = ("import json, sys; sys.path.insert(0, %r); import bench; from synthetic import WORKLOADS; "
            "print(json.dumps(bench.oracle_rate(WORKLOADS[%r], %d, %r, policy=%r)))"
            % (ROOT, workload, crop, float(seconds_budget), policy))
    try:
        p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        return json.loads(p.stdout.strip().splitlines()[-1])
    except (OSError, subprocess.SubprocessError, ValueError, IndexError):
        return None


def run_reference(args, spec):
    """The oracle arm: one step = one oracle pass over a crop of the workload
    cube (the bounded sample), so ms_per_step x steps is the time really spent;
    value = full-cube passes/s, the crop's rate scaled by its share of the
    pixels."""
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    total = args.steps + args.warmup
    crop = 32 if total > 40 else 64
    r = oracle_rate(spec, crop, 0.0, max_steps=args.steps, warmup=args.warmup, policy=args.policy)
    rate = r["rate"]
    out = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * r["seconds_per_pass"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "N1": spec.N1, "N2": spec.N2, "N3": spec.N3, "k": spec.k,
                   "policy": args.policy,
                   "step": f"one oracle pass over a {crop}x{crop}x{spec.N3} crop "
                           f"({r['fraction']:.4f} of the cube's pixels); value scales its rate to the full cube"},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": round(r["cores"], 2),
                         "cores_available": os.cpu_count(), "cpu_model": cpu_model(), "kind": "oracle",
                         "sample": r["sample"]},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def mpsnr(u, ref, trim=3):
    import numpy as np
    u = np.asarray(u, np.float64)
    ref = np.asarray(ref, np.float64)
    N1, N2, N3 = u.shape
    bands = range(trim, N3 - trim) if N3 > 2 * trim else range(N3)
    err = ((u - ref) ** 2).sum(axis=(0, 1))
    return float(np.mean([10 * math.log10(N1 * N2 / err[b]) for b in bands]))


def run_ours(args, spec):
    import numpy as np
    import torch
    import paper_2404_03313_gb300 as P
    from synthetic import make_cube

    rank, local_rank, world = dist_env()
    if world > 1:
        dist_init("nccl")
    dev = local_rank if world > 1 else 0
    torch.cuda.set_device(dev)
    P.library()
    clean, v = make_cube(spec)
    N = v.size
    eps, alpha, beta = P.radii(N, spec.sigma, spec.p_s, spec.p_t, 0.95)
    policy = P.STEP_PC_EXACT if args.policy == "pc_exact" else P.STEP_PAPER
    stream = torch.cuda.Stream(device=dev)
    solver = P.Solver(dev, stream=stream)
    solver.set_option(P.OPT_STEP_POLICY, policy)
    solver.set_option(P.OPT_TENSOR_CORES, args.tensor_cores)
    solver.set_option(P.OPT_LAYOUT, P.LAYOUT_STACKED if args.layout == "stacked" else P.LAYOUT_PAPER)
    solver.set_option(P.OPT_SPECTRAL_BOUNDARY, P.SPECTRAL_OPEN if args.spectral == "open" else P.SPECTRAL_PERIODIC)
    solver.set_option(P.OPT_REGULARIZER, {"s3ttv": P.REG_S3TTV, "stv": P.REG_STV, "sstv": P.REG_SSTV,
                                          "hsstv1": P.REG_HSSTV1, "hsstv2": P.REG_HSSTV2,
                                          "ssst": P.REG_SSST}[args.reg])
    if args.autotune:
        solver.set_option(P.OPT_AUTOTUNE, 1)
    vd = torch.from_numpy(v).to(f"cuda:{dev}")
    torch.cuda.synchronize()

    # ---- device-resident timing ----
    solver.setup(vd, eps, alpha, beta, spec.k)
    solver.set_option(P.OPT_CHECK_EVERY, max(args.steps, args.warmup, 1))
    solver.iterate(max(args.warmup, 12) if args.autotune else args.warmup)  # the tuner needs 2 + 2 x forms passes
    tuned = solver.tuned_form() if args.autotune else None
    solver.set_option(P.OPT_PROFILE, 1)
    launches0 = solver.launch_count()
    sampler = ClockSampler(nvsmi_id(dev)).start()
    time.sleep(0.3)
    dist_barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    info = solver.iterate(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    dist_barrier(world)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    ms_max = dist_max(ms, world, device=f"cuda:{dev}")
    launches = solver.launch_count() - launches0
    stats = solver.kernel_stats()
    solver.set_option(P.OPT_PROFILE, 0)
    value = world * args.steps / (ms_max / 1000.0)

    # ---- roofline of the dominant kernel (block dual, steps 8-11) ----
    k2 = spec.k * spec.k
    bd_ms, bd_n = stats["block_dual"]
    bd_avg_s = bd_ms / max(bd_n, 1) / 1000.0
    # Y read + write, ubar read, Z written once (SSST: three parts of Y and Z)
    bytes_per_voxel = 24 * k2 + 4 + 12 if args.reg == "ssst" else 16 * k2 + 4 + 8
    alg_bytes = bytes_per_voxel * N
    peak, peak_src = measured_peaks()
    stacked = args.layout == "stacked"
    if args.reg in ("sstv", "hsstv1", "hsstv2"):
        # SSTV / HSSTV: the dual step is one elementwise kernel (the block_dual
        # class): ubar read, Y (2 or 4 cubes) read and written, Z written
        sb = (28 if args.reg == "sstv" else 44) * N
        achieved = sb / bd_avg_s / 1e9 if bd_avg_s > 0 else 0.0
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": None, "kernel": "sstv_dual_kernel" if args.reg == "sstv" else "hsstv_dual_kernel",
                    "peak_source": peak_src,
                    "algorithmic_bytes_per_launch": sb, "avg_launch_ms": bd_avg_s * 1000.0}
    elif spec.k <= 5 and not stacked and args.reg != "ssst":
        achieved = alg_bytes / bd_avg_s / 1e9 if bd_avg_s > 0 else 0.0
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": block_dual_traffic(spec.k, N), "kernel": f"block_dual_kernel<{spec.k}, *>",
                    "peak_source": peak_src,
                    "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": bd_avg_s * 1000.0}
    else:
        # k = 6..12, the stacked layout and SSST: the eigen-solve binds, not
        # HBM.  Algorithmic FP32 work per block: Gram and apply 2 n^2 cols each
        # (n rows, cols = N3, 2 N3 or SSST's 3 N3), a symmetric eigen-solve with
        # vectors ~9 n^3.  peak = the measured FP32 rate (s3ttv_fp32_peak: FMA
        # chains over a full grid, scalar and packed FP32x2, the larger); the
        # figure derived from the unit counts (152 SMs x 128 FP32 lanes x 2
        # flops x max SM clock) is reported beside it.
        n = 2 * k2 if stacked else k2
        cols = spec.N3 if stacked else (3 if args.reg == "ssst" else 2) * spec.N3
        flops = (4.0 * n * n * cols + 9.0 * n ** 3) * spec.N1 * spec.N2
        sm_mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
        derived_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        fp32_scalar, fp32_packed = P.fp32_peak(dev, False), P.fp32_peak(dev, True)
        alu_peak = max(fp32_scalar, fp32_packed)
        achieved = flops / bd_avg_s / 1e12 if bd_avg_s > 0 else 0.0
        roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": achieved / alu_peak, "traffic": None,
                    "kernel": f"block_dual_large_kernel<{spec.k}, {'true' if stacked else 'false'}, "
                              f"{3 if args.reg == 'ssst' else 2}>",
                    "peak_source": f"measured (s3ttv_fp32_peak): FP32 FMA chains over a full grid, scalar "
                                   f"{fp32_scalar:.1f}, packed FP32x2 {fp32_packed:.1f} TFLOP/s, the larger",
                    "derived_peak": derived_peak,
                    "algorithmic_flops_per_launch": flops, "avg_launch_ms": bd_avg_s * 1000.0,
                    "hbm_frac": alg_bytes / bd_avg_s / 1e9 / peak if bd_avg_s > 0 else 0.0}
    pass_bytes = (16 * k2 + 120) * N
    kernel_ms = {name: (t / max(c, 1)) for name, (t, c) in stats.items()}

    # ---- end to end through the C ABI with pinned host buffers ----
    vh = torch.from_numpy(v).pin_memory()
    outs = [torch.empty(v.shape, dtype=torch.float32).pin_memory() for _ in range(3)]
    dist_barrier(world)
    t0 = time.perf_counter()
    solver.solve(vh.numpy(), eps, alpha, beta, spec.k, max_iter=args.steps, tol=0.0,
                 out=[o.numpy() for o in outs])
    e2e_s = time.perf_counter() - t0
    e2e_s = dist_max(e2e_s, world, device=f"cuda:{dev}")
    e2e = {"value": world * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 4 * N / args.steps,
           "d2h_bytes_per_step": 12 * N / args.steps, "seconds": e2e_s}

    # ---- the other forms of the block duals on the same passes ----
    # (k <= 5, paper layout, S3TTV: tensor cores with three TF32 products per
    # FP32 product, a warp streaming each block or four warps sharing it, or
    # plain FP32 FMAs on the CUDA cores)
    forms = None
    if spec.k <= 5 and not stacked and args.reg == "s3ttv":
        forms = {}
        for tc in (args.tensor_cores,) + tuple(x for x in (2, 1, 0) if x != args.tensor_cores):
            if tc != args.tensor_cores:
                solver.set_option(P.OPT_TENSOR_CORES, tc)
                solver.iterate(args.warmup)
                solver.set_option(P.OPT_PROFILE, 1)
                f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                f0.record(stream)
                solver.iterate(args.steps)
                f1.record(stream)
                torch.cuda.synchronize()
                fms = dist_max(f0.elapsed_time(f1), world, device=f"cuda:{dev}")
                fbd_ms, fbd_n = solver.kernel_stats()["block_dual"]
                solver.set_option(P.OPT_PROFILE, 0)
                solver.set_option(P.OPT_TENSOR_CORES, args.tensor_cores)
            else:
                fms, fbd_ms, fbd_n = ms_max, bd_ms, bd_n
            fbd_s = fbd_ms / max(fbd_n, 1) / 1000.0
            forms[FORM_NAMES[tc]] = {
                "value": world * args.steps / (fms / 1000.0), "unit": UNIT, "ms_per_step": fms / args.steps,
                "block_dual_ms": fbd_s * 1000.0,
                "block_dual_frac": (alg_bytes / fbd_s / 1e9 / peak) if fbd_s > 0 else 0.0}

    # ---- seconds to the paper's stop rule (||u+ - u|| / ||u|| < 1e-5, cap 5000) ----
    def to_tol(slv, vin, cln, e, a, b, k, policy_id, tc, max_iter=5000, tol=1e-5):
        slv.set_option(P.OPT_STEP_POLICY, policy_id)
        slv.set_option(P.OPT_TENSOR_CORES, tc)
        slv.set_option(P.OPT_CHECK_EVERY, 16)
        u, _, _, inf = slv.solve(vin, e, a, b, k, max_iter=max_iter, tol=tol)
        torch.cuda.synchronize()
        return {"seconds": inf["seconds"], "iters": inf["iters"], "converged": bool(inf["converged"]),
                "rel_change": inf["rel_change"], "mpsnr_restored": mpsnr(u.cpu().numpy(), cln),
                "iters_per_s": inf["iters"] / inf["seconds"] if inf["seconds"] > 0 else None}

    tol_run = None
    if not args.no_tol_run:
        tol_run = to_tol(solver, vd, clean, eps, alpha, beta, spec.k, policy, args.tensor_cores)
        tol_run.update({"policy": args.policy, "mpsnr_observed": mpsnr(v, clean), "stop_tol": 1e-5,
                        "max_iter": 5000})
        if args.policy == "paper" and args.reg == "s3ttv" and not stacked:
            # PC_EXACT (gamma_u = 1/(8k^2 + 1), the exact Lemma 1 column sum):
            # the stop rule fires; both product forms where both exist
            pc = {}
            pair = (args.tensor_cores, 0) if args.tensor_cores else (0, 2)
            for tc in (pair if forms else (args.tensor_cores,)):
                pc[FORM_NAMES[tc]] = to_tol(
                    solver, vd, clean, eps, alpha, beta, spec.k, P.STEP_PC_EXACT, tc)
            if len(pc) == 2:
                a_, b_ = pc.values()
                pc["mpsnr_diff_db"] = abs(a_["mpsnr_restored"] - b_["mpsnr_restored"])
            tol_run["pc_exact"] = pc
        solver.set_option(P.OPT_STEP_POLICY, policy)
        solver.set_option(P.OPT_TENSOR_CORES, args.tensor_cores)

    # ---- the precision form's comparison (304x304x191, k = 5): time to the stop
    # rule of both product forms at equal MPSNR (PC_EXACT step sizes) ----
    precision = None
    if (args.workload == DEFAULT_WORKLOAD and not args.no_tol_run and not args.no_precision_run
            and forms is not None):
        from synthetic import WORKLOADS
        spec3 = WORKLOADS["s3ttv_304x304x191_k5"]
        clean3, v3 = make_cube(spec3)
        e3, a3, b3 = P.radii(v3.size, spec3.sigma, spec3.p_s, spec3.p_t, 0.95)
        v3d = torch.from_numpy(v3).to(f"cuda:{dev}")
        s3 = P.Solver(dev, stream=stream)
        precision = {"workload": "s3ttv_304x304x191_k5", "policy": "pc_exact"}
        chosen = args.tensor_cores or 2
        for tc in (chosen, 0):
            precision[FORM_NAMES[tc]] = to_tol(s3, v3d, clean3, e3, a3, b3, spec3.k, P.STEP_PC_EXACT, tc)
        precision["mpsnr_diff_db"] = abs(precision[FORM_NAMES[chosen]]["mpsnr_restored"]
                                         - precision[FORM_NAMES[0]]["mpsnr_restored"])
        precision["mpsnr_observed"] = mpsnr(v3, clean3)
        s3.close()
        del v3d

    # ---- cost per pass against the block side (the paper's block-size study,
    # Fig. Param_Anal, runs k up to 16 on 100x100x198-sized cubes) ----
    sweep = None
    if args.workload == DEFAULT_WORKLOAD and not args.no_block_sweep:
        sweep = block_size_sweep(P, dev, stream)

    # ---- CPU baseline (oracle), rank 0 at N = 1 only: one full-cube pass timed
    # on all host cores, and a one-thread run on a crop ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        full_s, full_cores = oracle_full_pass(spec, args.policy)
        one = oracle_one_thread(args.workload, 32, args.cpu_seconds, args.policy)
        cpu = {"value": 1.0 / full_s, "unit": UNIT, "cores": round(full_cores, 2),
               "cores_available": os.cpu_count(), "cpu_model": cpu_model(), "kind": "oracle",
               "sample": f"one oracle pass (FP64, numpy/LAPACK SVD per block) over the whole "
                         f"{spec.N1}x{spec.N2}x{spec.N3} cube, k={spec.k}, timed, not scaled",
               "seconds": full_s,
               "one_thread": (None if one is None else
                              {"value": one["rate"], "unit": UNIT, "cores": round(one["cores"], 2),
                               "sample": one["sample"] + " (BLAS/OpenMP pools limited to one thread)",
                               "seconds": one["seconds"]})}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "N1": spec.N1, "N2": spec.N2, "N3": spec.N3, "k": spec.k,
                       "policy": args.policy, "layout": args.layout, "spectral": args.spectral, "reg": args.reg,
                       "autotuned_form": ({"tensor_cores": tuned[0], "ctas_per_sm": tuned[1]} if tuned else None),
                       "parallelism": f"replicas{world}",
                       "block_dual_products": FORM_TEXT[args.tensor_cores],
                       "l2": "inputs larger than L2 (block duals Y: %.2f GB, read and written every pass)"
                             % (8 * k2 * N / 1e9)},
            "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
            "cpu_baseline": cpu,
            "pass_roofline": {"bound": "hbm", "algorithmic_bytes": pass_bytes,
                              "achieved": pass_bytes / (ms_max / args.steps / 1000.0) / 1e9, "peak": peak,
                              "unit": "GB/s"},
            "kernel_avg_ms": kernel_ms, "jacobi_nonconverged": info["jacobi_nonconverged"],
            "jacobi_sweeps_mean": info["jacobi_sweeps"],
            "to_tol": tol_run, "forms": forms, "precision_form": precision, "block_size_sweep": sweep,
        }
        out["pass_roofline"]["frac"] = out["pass_roofline"]["achieved"] / peak
        print(json.dumps(out), flush=True)
    solver.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def block_size_sweep(P, dev, stream, ks=(5, 6, 8, 10, 12, 13, 14, 16), warm=3, timed=4):
    """ms per pass at block side k on the 100x100x198 cube of the paper's
    simulated experiments (its noise recipe, seeded), k = 5..16: warm passes,
    then `timed` passes between CUDA events on the solver's stream, with the
    block-dual kernel's own average from the solver's profile."""
    import torch
    from synthetic import WORKLOADS, CubeSpec, make_cube
    base = WORKLOADS["paper_100x100x198_k10"]
    rows = []
    for k in ks:
        spec = CubeSpec(base.N1, base.N2, base.N3, regions=base.regions, endmembers=base.endmembers,
                        sigma=base.sigma, p_s=base.p_s, p_t=base.p_t, k=k, seed=base.seed)
        _, v = make_cube(spec)
        e, a, b = P.radii(v.size, spec.sigma, spec.p_s, spec.p_t, 0.95)
        s = P.Solver(dev, stream=stream)
        s.setup(torch.from_numpy(v).to(f"cuda:{dev}"), e, a, b, k)
        s.set_option(P.OPT_CHECK_EVERY, 1000)
        s.iterate(warm)
        s.set_option(P.OPT_PROFILE, 1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = s.iterate(timed)
        e1.record(stream)
        torch.cuda.synchronize()
        bd_ms, bd_n = s.kernel_stats()["block_dual"]
        rows.append({"k": k, "ms_per_pass": e0.elapsed_time(e1) / timed, "block_dual_ms": bd_ms / max(bd_n, 1),
                     "jacobi_sweeps_mean": info["jacobi_sweeps"],
                     "jacobi_nonconverged": info["jacobi_nonconverged"]})
        s.close()
    return {"workload": "100x100x198 (paper_100x100x198 recipe), block side k", "warm_passes": warm,
            "timed_passes": timed, "rows": rows}


BATCH_WORKLOAD = "batch_64_uneven"
BATCH_METRIC = "S3TTV batched P-PDS passes/s over 64 uneven cubes (one pass = every cube advanced once)"
BATCH_UNIT = "batch passes/s"


def run_batch(args):
    """The uneven batch: 64 seeded cubes (synthetic.batch_specs) solved together
    through s3ttv_solve_batched; value = batch passes/s from CUDA events on the
    solver's stream around K passes (inputs device-resident; setup included,
    one call); the same K passes with each cube alone, back to back, for the
    batching gain; per-cube agreement of the two."""
    import numpy as np
    import torch
    import paper_2404_03313_gb300 as P
    from synthetic import batch_specs, make_cube

    rank, local_rank, world = dist_env()
    if world > 1:
        dist_init("nccl")
    dev = local_rank if world > 1 else 0
    torch.cuda.set_device(dev)
    P.library()
    specs = batch_specs(64, seed=0)
    probs, voxels, pass_bytes = [], 0, 0
    for sp in specs:
        _, v = make_cube(sp)
        eps, alpha, beta = P.radii(v.size, sp.sigma, sp.p_s, sp.p_t, 0.95)
        probs.append({"v": torch.from_numpy(v).to(f"cuda:{dev}"), "eps": eps, "alpha": alpha, "beta": beta,
                      "k": sp.k})
        voxels += v.size
        pass_bytes += (16 * sp.k * sp.k + 120) * v.size
    stream = torch.cuda.Stream(device=dev)
    solver = P.Solver(dev, stream=stream)
    solver.set_option(P.OPT_TENSOR_CORES, args.tensor_cores)
    solver.set_option(P.OPT_CHECK_EVERY, 16)
    solver.solve_batched(probs, max_iter=args.warmup, tol=0.0)
    torch.cuda.synchronize()
    sampler = ClockSampler(nvsmi_id(dev)).start()
    time.sleep(0.3)
    dist_barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = solver.solve_batched(probs, max_iter=args.steps, tol=0.0)
    e1.record(stream)
    torch.cuda.synchronize()
    dist_barrier(world)
    clocks = sampler.stop()
    ms = dist_max(e0.elapsed_time(e1), world, device=f"cuda:{dev}")
    launches = solver.launch_count()
    # the same passes with the block duals of all cubes in one work-list launch
    # per block side (S3TTV_OPT_BATCH_WORKLIST)
    worklist = None
    if args.tensor_cores == 2:
        solver.set_option(P.OPT_BATCH_WORKLIST, 1)
        solver.solve_batched(probs, max_iter=args.warmup, tol=0.0)
        w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0.record(stream)
        outw = solver.solve_batched(probs, max_iter=args.steps, tol=0.0)
        w1.record(stream)
        torch.cuda.synchronize()
        wms = w0.elapsed_time(w1)
        worklist = {"value": args.steps / (wms / 1000.0), "unit": BATCH_UNIT, "ms_per_step": wms / args.steps,
                    "max_rel_diff_vs_default": max(float((a[0] - b_[0]).norm() / b_[0].norm())
                                                   for a, b_ in zip(outw, out))}
        solver.set_option(P.OPT_BATCH_WORKLIST, 0)
    # each cube alone, the same passes, back to back
    alone_u, t_alone = [], 0.0
    for p in probs:
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        u, _, _, _ = solver.solve(p["v"], p["eps"], p["alpha"], p["beta"], p["k"], max_iter=args.steps, tol=0.0)
        a1.record(stream)
        torch.cuda.synchronize()
        t_alone += a0.elapsed_time(a1)
        alone_u.append(u)
    agree = max(float((o[0] - a).norm() / a.norm()) for o, a in zip(out, alone_u))
    # to the stop rule: every cube with its own stop rule (PC_EXACT step sizes,
    # with which it fires; bounded so the run stays short), per-cube times
    tol_run = None
    if not args.no_tol_run:
        solver.set_option(P.OPT_STEP_POLICY, P.STEP_PC_EXACT)
        t0 = time.perf_counter()
        res = solver.solve_batched(probs, max_iter=args.batch_max_iter, tol=args.batch_tol)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        secs = sorted(r[3]["seconds"] for r in res)
        q = lambda f: secs[min(len(secs) - 1, int(round(f * (len(secs) - 1))))]
        tol_run = {"policy": "pc_exact", "tol": args.batch_tol, "max_iter": args.batch_max_iter,
                   "seconds": wall, "cubes_per_s": len(probs) / wall,
                   "converged": sum(1 for r in res if r[3]["converged"]),
                   "p50_s": q(0.5), "p99_s": q(0.99),
                   "iters_p50": sorted(r[3]["iters"] for r in res)[len(res) // 2]}
    solver.close()
    value = world * args.steps / (ms / 1000.0)
    peak, peak_src = measured_peaks()
    achieved = pass_bytes * args.steps / (ms / 1000.0) / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": BATCH_METRIC, "value": value, "unit": BATCH_UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "cubes": len(specs), "voxels": voxels,
                       "k": sorted({sp.k for sp in specs}), "N3": sorted({sp.N3 for sp in specs}),
                       "parallelism": f"replicas{world}", "graph": "one CUDA graph launch per 16 passes",
                       "l2": "inputs larger than L2 (block duals of all cubes: %.1f GB)"
                             % (sum(8 * sp.k * sp.k * sp.N1 * sp.N2 * sp.N3 for sp in specs) / 1e9)},
            "clocks": clocks, "gpu_launches": launches,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "whole pass, all cubes",
                         "peak_source": peak_src, "algorithmic_bytes_per_step": pass_bytes},
            "cubes_alone_ms_per_step": t_alone / args.steps, "batching_gain": t_alone / ms,
            "block_dual_worklist": worklist,
            "max_rel_diff_batched_vs_alone": agree,
            "to_tol": tol_run,
        }), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


WARM_WORKLOAD = "warm_start_256x256x128"
WARM_METRIC = "S3TTV seconds-to-tol at 256×256×128 from the learned warm start (inference included)"


def unet_forward_flops(V0):
    """Multiply-adds x 2 of one network forward over V0 voxels: per voxel of each
    level, 27 c_in c_out for each 3x3x3 convolution, plus the 1x1x1 head."""
    lvl0 = 27 * (1 * 32 + 32 * 32 + 96 * 32 + 32 * 32) + 3 * 32
    lvl1 = 27 * (32 * 64 + 64 * 64 + 192 * 64 + 64 * 64)
    lvl2 = 27 * (64 * 128 + 128 * 128)
    return 2.0 * V0 * (lvl0 + lvl1 / 8.0 + lvl2 / 64.0)


def run_warm_start(args):
    """The learned warm start (no counterpart in the paper): train the network on
    12 solver-solved 128x128x64 cubes (seeds 10000..), then solve held-out
    256x256x128 cubes (seeds 20000.., one per timed step) from the cold start and
    from the network's prediction, both to the stop rule (1e-5, cap 5000) with
    the PC_EXACT step sizes (with the PAPER ones the stop rule does not fire
    within the cap at this size).  value = mean seconds to the stop rule from
    the warm start, inference included (lower is better); the cold figures sit
    beside it.  roofline = the network forward at 256x256x128 on the tensor
    pipe (convolution FLOPs / CUDA-event time, warm)."""
    import numpy as np
    import torch
    import paper_2404_03313_gb300 as P
    from paper_2404_03313_gb300 import warmstart as WS
    from synthetic import make_cube, network_params, warm_start_specs

    rank, local_rank, world = dist_env()
    if world > 1:
        dist_init("nccl")
    dev = local_rank if world > 1 else 0
    torch.cuda.set_device(dev)
    P.library()
    policy = P.STEP_PC_EXACT
    train_specs = warm_start_specs(12, 10000, (128, 128, 64))
    cubes, radii = [], []
    for sp in train_specs:
        _, v = make_cube(sp)
        cubes.append(torch.from_numpy(v).to(f"cuda:{dev}"))
        radii.append(P.radii(v.size, sp.sigma, sp.p_s, sp.p_t))
    t0 = time.perf_counter()
    targets = WS.solver_targets(cubes, radii, 5, 5000, 1e-5, policy, device=dev)
    t_targets = time.perf_counter() - t0
    stream = torch.cuda.Stream(device=dev)
    net = P.WarmStartNet(dev, stream=stream)
    shapes = [(co, 27, ci) for ci, co in ((1, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128),
                                          (192, 64), (64, 64), (96, 32), (32, 32))]
    flat_shapes = []
    for w in shapes:
        flat_shapes += [w, (w[0],)]
    flat_shapes += [(3, 32), (3,)]
    net.set_params(network_params(flat_shapes, seed=0, head_scale=0.1))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = WS.train(net, cubes, [x[:3] for x in targets], 800, crop=(32, 32, 32), batch=4, lr=1e-3,
                      lr_final=1e-4, seed=0)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0

    # network forward at full size: CUDA events on the network's stream
    x = torch.rand(256, 256, 128, device=f"cuda:{dev}")
    for _ in range(args.warmup):
        net.forward(x)
    sampler = ClockSampler(nvsmi_id(dev)).start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nf = 5
    f0.record(stream)
    for _ in range(nf):
        net.forward(x)
    f1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = f0.elapsed_time(f1) / nf

    evals = []

    def first_within(trace, target):
        return next((n for n, m in trace if m >= target), None)

    for sp in warm_start_specs(args.steps, 20000, (256, 256, 128)):
        clean, v = make_cube(sp)
        vd = torch.from_numpy(v).to(f"cuda:{dev}")
        cref = torch.from_numpy(clean).to(f"cuda:{dev}")
        e, a, b = P.radii(v.size, sp.sigma, sp.p_s, sp.p_t)
        cold = WS.solve(vd, e, a, b, 5, None, 5000, 1e-5, policy, device=dev)
        warm = WS.solve(vd, e, a, b, 5, net, 5000, 1e-5, policy, device=dev)
        # the same runs with MPSNR traced every 16 passes, and a warm start whose
        # block duals also start from the prediction (singular values of
        # 16 X(u_pred) clipped at 1)
        cold_t = WS.solve(vd, e, a, b, 5, None, 5000, 1e-5, policy, device=dev, trace_ref=cref)
        warm_t = WS.solve(vd, e, a, b, 5, net, 5000, 1e-5, policy, device=dev, trace_ref=cref)
        warm_y = WS.solve(vd, e, a, b, 5, net, 5000, 1e-5, policy, device=dev, dual_scale=16.0)
        target = cold_t["trace"][-1][1] - 0.01
        # the paper's printed step sizes: the stop rule does not fire, so compare
        # the restored cube after a fixed budget of passes
        cold_p = WS.solve(vd, e, a, b, 5, None, args.ws_paper_passes, 0.0, P.STEP_PAPER, device=dev)
        warm_p = WS.solve(vd, e, a, b, 5, net, args.ws_paper_passes, 0.0, P.STEP_PAPER, device=dev)
        pred = net.forward(vd)[0]
        evals.append({"cold_s": cold["seconds"], "cold_iters": cold["info"]["iters"],
                      "warm_s": warm["seconds"], "warm_iters": warm["info"]["iters"],
                      "net_s": warm["net_seconds"],
                      "warm_dual_init": {"dual_scale": 16.0, "s": warm_y["seconds"],
                                         "iters": warm_y["info"]["iters"],
                                         "mpsnr": mpsnr(warm_y["u"].cpu().numpy(), clean)},
                      "passes_to_cold_final_mpsnr_minus_0p01": {"cold": first_within(cold_t["trace"], target),
                                                               "warm": first_within(warm_t["trace"], target)},
                      "mpsnr_observed": mpsnr(v, clean), "mpsnr_network": mpsnr(pred.cpu().numpy(), clean),
                      "mpsnr_cold": mpsnr(cold["u"].cpu().numpy(), clean),
                      "mpsnr_warm": mpsnr(warm["u"].cpu().numpy(), clean),
                      "paper_steps": {"passes": args.ws_paper_passes,
                                      "cold_s": cold_p["seconds"], "warm_s": warm_p["seconds"],
                                      "mpsnr_cold": mpsnr(cold_p["u"].cpu().numpy(), clean),
                                      "mpsnr_warm": mpsnr(warm_p["u"].cpu().numpy(), clean)}})
    clocks = sampler.stop()
    net.close()
    warm_s = statistics.mean(ev["warm_s"] for ev in evals)
    cold_s = statistics.mean(ev["cold_s"] for ev in evals)
    flops = unet_forward_flops(256 * 256 * 128)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    peak = peaks.get("bf16_tflops") or 1900.0
    achieved = flops / (fwd_ms / 1000.0) / 1e12
    if rank == 0:
        print(json.dumps({
            "metric": WARM_METRIC, "value": warm_s, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * warm_s, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": WARM_WORKLOAD, "N1": 256, "N2": 256, "N3": 128, "k": 5, "policy": "pc_exact",
                       "train": "12 cubes 128x128x64, 800 Adam steps on 4 crops of 32^3",
                       "parallelism": f"replicas{world}",
                       "l2": "solver inputs larger than L2 (block duals 1.68 GB)"},
            "clocks": clocks,
            "cold_seconds": cold_s, "evals": evals,
            "train_seconds": t_train, "targets_seconds": t_targets, "final_train_loss": losses[-1],
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "network forward (conv_fwd_kernel launches and the CUDA-core layers)",
                         "peak_source": "MEASURED_PEAKS.json bf16_tflops" if "bf16_tflops" in peaks
                         else "fallback 1900 TFLOP/s",
                         "flops_per_forward": flops, "forward_ms": fwd_ms},
        }), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


NET_FORWARD_PREFIX = "net_forward_"


def run_net_forward(args):
    """The warm-start network's forward alone on a random cube of the size the
    workload names (net_forward_<N1>x<N2>x<N3>), seeded He-normal parameters:
    value = voxels/s over `steps` forwards after `warmup`, CUDA events on the
    network's stream; roofline = convolution FLOPs / time on the tensor pipe."""
    import torch
    import paper_2404_03313_gb300 as P
    from synthetic import network_params

    N1, N2, N3 = (int(x) for x in args.workload[len(NET_FORWARD_PREFIX):].split("x"))
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream(device=0)
    net = P.WarmStartNet(0, stream=stream)
    shapes = []
    for ci, co in ((1, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128), (192, 64), (64, 64), (96, 32),
                   (32, 32)):
        shapes += [(co, 27, ci), (co,)]
    shapes += [(3, 32), (3,)]
    net.set_params(network_params(shapes, seed=0, head_scale=0.1))
    x = torch.rand(N1, N2, N3, device="cuda:0")
    for _ in range(args.warmup):
        net.forward(x)
    sampler = ClockSampler(nvsmi_id(0)).start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        net.forward(x)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    net.close()
    V = N1 * N2 * N3
    flops = unet_forward_flops(V)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    peak = peaks.get("bf16_tflops") or 1900.0
    achieved = flops / (ms / 1000.0) / 1e12
    print(json.dumps({
        "metric": "warm-start network forward, voxels/s", "value": V / (ms / 1000.0), "unit": "voxel/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": args.workload, "N1": N1, "N2": N2, "N3": N3,
                   "l2": "activations larger than L2 (%.2f GB per 32-channel full-size tensor)" % (64 * V / 1e9)},
        "clocks": clocks,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "network forward (all launches)",
                     "peak_source": "MEASURED_PEAKS.json bf16_tflops" if "bf16_tflops" in peaks
                     else "fallback 1900 TFLOP/s", "flops_per_forward": flops},
    }), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--policy", choices=("paper", "pc_exact"), default="paper")
    ap.add_argument("--tensor-cores", type=int, choices=(0, 1, 2), default=2,
                    help="block-dual form: tensor cores with a warp streaming each block (2), tensor "
                         "cores with four warps sharing each block (1), CUDA cores (0)")
    ap.add_argument("--layout", choices=("paper", "stacked"), default="paper",
                    help="block matrices: the paper's k^2 x 2N3 or the stacked 2k^2 x N3")
    ap.add_argument("--spectral", choices=("periodic", "open"), default="periodic",
                    help="spectral difference: periodic (the paper) or open (no wrap-around)")
    ap.add_argument("--reg", choices=("s3ttv", "stv", "sstv", "hsstv1", "hsstv2", "ssst"), default="s3ttv",
                    help="regularisation function: S3TTV (the paper) or a comparison one run by the same P-PDS")
    ap.add_argument("--autotune", action="store_true",
                    help="let the library time the block-dual forms on the warm-up passes and keep the fastest")
    ap.add_argument("--batch-tol", type=float, default=1e-4,
                    help="stop rule of the batched to-tolerance run (per cube)")
    ap.add_argument("--batch-max-iter", type=int, default=600)
    ap.add_argument("--ws-paper-passes", type=int, default=1000,
                    help="warm-start workload: fixed pass budget of the runs with the paper's step sizes")
    ap.add_argument("--no-tol-run", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-block-sweep", action="store_true",
                    help="skip the ms-per-pass sweep over block sides k = 5..16 (100x100x198)")
    ap.add_argument("--no-precision-run", action="store_true",
                    help="skip the 304x304x191 time-to-tolerance comparison of the two product forms")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.workload == BATCH_WORKLOAD:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times single cubes; "
                              "run it on their workloads"}), flush=True)
            return 0
        return run_batch(args)
    if args.workload.startswith(NET_FORWARD_PREFIX):
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the network forward has no solver "
                              "counterpart in the oracle arm"}), flush=True)
            return 0
        return run_net_forward(args)
    if args.workload == WARM_WORKLOAD:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the learned warm start has no oracle "
                              "counterpart to time; the oracle arm times the solver workloads"}), flush=True)
            return 0
        return run_warm_start(args)
    from synthetic import WORKLOADS
    spec = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, spec)
    return run_ours(args, spec)


if __name__ == "__main__":
    sys.exit(main())
