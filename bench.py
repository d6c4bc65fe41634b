#!/usr/bin/env python
"""Benchmark of the ParaDiag-II all-at-once solve on one GB300 (or N replicas).

Metric: space-time unknowns per second for a solve that reaches 1e-10
relative error against the FP64 oracle (mixed-precision path; the plain FP64
GPU path is timed beside it).  Workload: 2D advection-diffusion, 255 x 255
grid (x periodic, y Dirichlet), Crank-Nicolson, Nt = 256, alpha = 1e-3,
Gaussian initial value, zero source: 16,646,400 unknowns per solve.

One step = one stationary solve from a zero initial guess with b resident in
HBM, enqueued with pd_solve_async (the solves run back to back on the GPU; the
convergence outcome is read after the timed region).
The working set (iterate and right-hand side in double-float, 2 spectra) is
about 400 MB, larger than the 129 MB L2, so no flush is needed between steps.
With --impl reference the FP64 CPU oracle (sequential time stepping, the
exact solution of the all-at-once system) is timed instead, on the host.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "space-time unknowns/sec to 1e-10 rel err (mixed vs FP64 GPU path); % HBM roofline"
UNIT = "unknowns/s"
WORKLOAD = "ade2d_cn_255x255x256"
TOL = 1e-11          # relative residual; gives an error below 1e-10 vs the oracle (checked)
KERNELS = ["resid_gamma_fft", "xform_fwd", "tridiag", "xform_inv", "ifft_gamma_update"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-check", action="store_true", help="skip the oracle error check")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline leg")
    ap.add_argument("--small", action="store_true", help="a small case (profiling runs)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-workload leg")
    ap.add_argument("--batch-only", action="store_true",
                    help="only the batched-workload leg (the command ncu captures profile)")
    ap.add_argument("--no-pd1", action="store_true", help="skip the ParaDiag-I leg")
    ap.add_argument("--pd1-only", action="store_true",
                    help="only the ParaDiag-I leg (one JSON object; profiling runs)")
    ap.add_argument("--pd1-kernels", action="store_true",
                    help="only the ParaDiag-I mixed kernel profile (the command ncu captures profile)")
    ap.add_argument("--no-hybrid", action="store_true", help="skip the hybrid ParaDiag-I leg")
    ap.add_argument("--no-control", action="store_true", help="skip the optimal-control leg")
    ap.add_argument("--mode", default="replicas", choices=["replicas", "sharded"],
                    help="replicas: one whole problem per GPU (weak scaling, the default); "
                         "sharded: one problem split over the GPUs, grid-line slabs for the "
                         "time steps and frequency slabs for step (b), all-to-all between "
                         "(strong scaling)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 1D advection-diffusion, heat-source adjoint and 1D wave "
                         "GMRES legs")
    ap.add_argument("--no-wave", action="store_true",
                    help="skip the second-order (wave) hybrid ParaDiag-I leg")
    ap.add_argument("--clocks-dir", default=os.path.join(ROOT, "bench_out"),
                    help="folder for the nvidia-smi clock samples of the timed region")
    ap.add_argument("--no-nonlinear", action="store_true",
                    help="skip the nonlinear (simplified Newton) leg")
    ap.add_argument("--nonlinear-only", action="store_true",
                    help="only the nonlinear (simplified Newton) leg (one JSON object)")
    ap.add_argument("--wave-only", action="store_true",
                    help="only the second-order (wave) hybrid ParaDiag-I leg (one JSON object)")
    ap.add_argument("--control-only", action="store_true",
                    help="only the optimal-control leg (one JSON object)")
    ap.add_argument("--hybrid-only", action="store_true",
                    help="only the hybrid ParaDiag-I leg (one JSON object)")
    ap.add_argument("--hybrid-kernels", action="store_true",
                    help="only the hybrid ParaDiag-I mixed kernel profile (the command ncu captures profile)")
    ap.add_argument("--profile-iteration", action="store_true",
                    help="only time the kernels of one iteration (the command ncu captures profile)")
    ap.add_argument("--profile-precision", default="mixed", choices=["mixed", "fp64"],
                    help="--profile-iteration: the plan's precision")
    ap.add_argument("--profile-xform", default="auto", choices=["auto", "tensor", "fft"],
                    help="--profile-iteration: pin the x-transform engine of a mixed plan")
    ap.add_argument("--sweep", action="store_true",
                    help="roofline sweep of the iteration kernels over 1D sizes "
                         "nx in {255, 1023, 4095} x Nt in {256, 1024, 4096}")
    ap.add_argument("--sweep-size", default=None,
                    help="--sweep: one size only, given as NXxNT (e.g. 4095x4096)")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    return 6800.0, 1900.0, "fallback"


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, outdir):
        self.index = index
        self.proc = None
        self.path = os.path.join(outdir, f"clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("PD_BENCH_GLOO") is None else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v, device):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(small):
    import workloads as W
    if small:
        return W.ade2d(nx=127, ny=127, nt=128)
    return W.ade2d()


def bench_config(w, small, ws):
    """The workload description both arms print (the same keys and values)."""
    pb = w.problem
    sp = pb.space
    return {"workload": WORKLOAD if not small else "ade2d_cn_127x127x128",
            "nx": sp.nx, "ny": sp.ny, "nt": pb.nt, "scheme": "crank-nicolson",
            "alpha": pb.alpha, "nu": sp.nu, "velocity": [sp.ax, sp.ay],
            "bc": "x periodic, y Dirichlet", "unknowns": pb.unknowns, "residual_tol": TOL,
            "l2": "working set ~0.8 GB > 129 MB L2, no flush",
            "parallelism": f"{ws} independent replica(s)"}


def bytes_per_unknown(nt, fp64):
    """Algorithmic DRAM bytes per space-time unknown for each kernel of one
    iteration (half spectrum: (nt/2+1)/nt complex values per real unknown)."""
    h = (nt // 2 + 1) / nt
    c = 16.0 if fp64 else 8.0          # complex value bytes
    st = 8.0                            # iterate / rhs bytes (FP64 or double-float)
    return {"resid_gamma_fft": 2 * st + h * c, "xform_fwd": 2 * h * c, "tridiag": 2 * h * c,
            "xform_inv": 2 * h * c, "ifft_gamma_update": h * c + 2 * st}


def flops_per_launch_xform(rows, nx):
    """Algorithmic flops of one x-transform: a complex GEMM of rows x nx by nx x nx."""
    return 8.0 * rows * nx * nx


# DRAM bytes (read + write) per launch from one ncu capture of each kernel on
# the bench workload (the time kernels as recaptured after their last change);
# a kernel's entry goes back to None whenever that kernel changes.
NCU_TRAFFIC = {"resid_gamma_fft": 319.4e6, "xform_fwd": 78.3e6, "tridiag": 79.5e6,
               "xform_inv": 79.0e6, "ifft_gamma_update": 279.7e6}


def cpu_info():
    """(nproc, CPU model) of this host."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            k = line.split(":")[0].strip().lower()
            if k in ("model name", "cpu model", "hardware"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if model is None:
        # Arm hosts: /proc/cpuinfo names only the part number; lscpu names the core
        try:
            import subprocess
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            info = dict(l.split(":", 1) for l in out.splitlines() if ":" in l)
            name = info.get("Model name", "").strip()
            vendor = info.get("Vendor ID", "").strip()
            if name:
                model = f"{vendor} {name}".strip()
        except (OSError, ValueError, subprocess.SubprocessError):
            pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    return os.cpu_count() or 1, model


def oracle_pool(nproc):
    """A pool of ``nproc`` spawned processes for the oracle's independent
    x-modes.  The workers run single-threaded BLAS / LAPACK (the variables are
    set only while they start, so this process keeps its own threaded BLAS for
    the transforms along x)."""
    import multiprocessing as mp
    keys = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    try:
        return mp.get_context("spawn").Pool(nproc)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def oracle_sample_problem(w, nts):
    """The first ``nts`` time levels of the workload and their right-hand side."""
    import workloads as W
    from oracle import operators as O
    pb = w.problem
    sub = W.Problem(space=pb.space, nt=nts, dt=pb.dt, scheme=pb.scheme, alpha=pb.alpha)
    K = O.stencil(pb.space)
    b = O.build_rhs(sub, w.u0, w.u1, None if w.f is None else w.f[: nts + 1], K)
    return sub, K, b


def cpu_oracle_sample(w, seconds_hint=10.0):
    """Time the oracle's exact solve (O1) on the first time levels of the
    workload: on one core (sparse-LU stepping) and on all host cores (the
    mode-by-mode stepping of a periodic x direction, modes spread over a pool
    of spawned processes; time stays sequential).  Returns the cpu_baseline
    object."""
    from oracle import stepping as S
    nts = 32
    sub, K, b = oracle_sample_problem(w, nts)
    nproc, model = cpu_info()
    t0 = time.perf_counter()
    reps = 0
    while True:
        S.solve_sequential(sub, b, K)
        reps += 1
        el = time.perf_counter() - t0
        if el > seconds_hint or reps >= 50:
            break
    one = {"value": reps * sub.unknowns / el, "unit": UNIT, "cores": 1,
           "sample": f"oracle sequential time stepping (sparse LU per step) on the first {nts} "
                     f"of {w.problem.nt} time steps of the same grid, {reps} repetitions, "
                     f"{el:.1f} s"}
    with oracle_pool(nproc) as pool:
        S.solve_sequential_xmodes(sub, b, pool=pool, chunks=nproc)      # start-up
        t0 = time.perf_counter()
        reps_a = 0
        while True:
            S.solve_sequential_xmodes(sub, b, pool=pool, chunks=nproc)
            reps_a += 1
            el_a = time.perf_counter() - t0
            if el_a > seconds_hint or reps_a >= 200:
                break
    return {"value": reps_a * sub.unknowns / el_a, "unit": UNIT, "cores": nproc, "kind": "oracle",
            "sample": f"oracle sequential time stepping mode by mode (naive DFT along the "
                      f"periodic x, dense LU per mode and step) over the first {nts} of "
                      f"{w.problem.nt} time steps of the same grid, modes spread over {nproc} "
                      f"spawned processes, {reps_a} repetitions, {el_a:.1f} s",
            "nproc": nproc, "cpu_model": model, "single_core": one}


def cpu_oracle_entry(seconds, unknowns, what):
    """The oracle's wall time on this host (one core) for a configuration."""
    nproc, model = cpu_info()
    return {"s": seconds, "value": unknowns / seconds, "unit": UNIT, "cores": 1,
            "kind": "oracle", "sample": what, "nproc": nproc, "cpu_model": model}


def batched_leg(pd, torch, dev, args):
    """64 independent 1D advection-diffusion problems (nx uniform on 63..1023,
    Nt uniform on 32..1024, nu = 10^U[-3,-1], BE, alpha = 1e-2) solved together
    to a relative residual of 1e-10 per problem (mixed path)."""
    import numpy as np
    import workloads as W
    wls = W.batched(count=64, pow2=False)
    probs = [dict(space=dict(nx=w.problem.space.nx, nu=w.problem.space.nu,
                             ax=w.problem.space.ax),
                  nt=w.problem.nt, dt=w.problem.dt, alpha=w.problem.alpha, scheme=0, theta=1.0)
             for w in wls]
    batch = pd.Batch(probs, pd.PD_MIXED)
    u0 = torch.from_numpy(np.concatenate([w.u0 for w in wls])).to(dev)
    f = torch.from_numpy(np.concatenate([w.f.reshape(-1) for w in wls])).to(dev)
    b = batch.build_rhs(u0, f)
    u = torch.zeros_like(b)
    for _ in range(3):
        u.zero_()
        batch.solve(b, u, tol=1e-10, maxit=40)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    k = max(1, min(args.steps, 10))
    l0 = batch.launches()
    e0.record(stream)
    for _ in range(k):
        u.zero_()
        _, it, rel = batch.solve(b, u, tol=1e-10, maxit=40)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / k
    # algorithmic HBM bytes of one solve: entry split (read u, b; write the
    # double-float U, B: 32 B per unknown), per iteration K1 (read U, B; write
    # the half spectrum: 16 + 8h), K2 (16h), K3 (read the spectrum, update U:
    # 8h + 16), the final norm-only K1 (16) and the exit (read U, write u: 16);
    # h = (Nt/2 + 1)/Nt complex values per real unknown
    byts = 0.0
    for w in wls:
        n = w.problem.nt * w.problem.space.nx
        h = (w.problem.nt // 2 + 1) / w.problem.nt
        byts += n * (32.0 + it * (32.0 + 32.0 * h) + 16.0 + 16.0)
    hbm, _, src = peaks()
    gbs = byts / (ms / 1e3) / 1e9
    # per-kernel times of one sweep (persistent launches over all members) and
    # their algorithmic bytes: forward 16 + 8h, tridiagonal 16h, inverse 8h + 16
    kms = batch.profile_sweep(b, torch.zeros_like(b), reps=5)
    kb = [0.0, 0.0, 0.0]
    for w in wls:
        n = w.problem.nt * w.problem.space.nx
        h = (w.problem.nt // 2 + 1) / w.problem.nt
        kb[0] += n * (16.0 + 8.0 * h)
        kb[1] += n * 16.0 * h
        kb[2] += n * (8.0 * h + 16.0)
    kroof = {}
    for name, t, by in zip(("time_fwd", "tridiag", "time_inv"), kms, kb):
        g = by / (t / 1e3) / 1e9
        kroof[name] = {"ms": t, "bound": "hbm", "achieved": g, "peak": hbm, "unit": "GB/s",
                       "frac": g / hbm, "algorithmic_bytes": by}
    # the oracle (O1, sequential stepping) for every member: its time on this
    # host and the largest relative error of the batch's solution
    from oracle import operators as O
    from oracle import stepping as S
    uh = u.cpu().numpy()
    t_cpu, err_max, off = 0.0, 0.0, 0
    for w in wls:
        pbw = w.problem
        n = pbw.nt * pbw.space.nx
        bw = O.build_rhs(pbw, w.u0, None, w.f)
        t0 = time.perf_counter()
        uw = S.solve_sequential(pbw, bw)
        t_cpu += time.perf_counter() - t0
        err_max = max(err_max, float(np.linalg.norm(uh[off:off + n] - uw.reshape(-1))
                                     / np.linalg.norm(uw)))
        off += n
    out = {"workload": "64 x 1D advection-diffusion, nx ~ U{63..1023}, Nt ~ U{32..1024} "
                       "(Bluestein for non-powers of two), BE, alpha = 1e-2",
           "error_vs_oracle_max": err_max,
           "cpu_oracle": cpu_oracle_entry(t_cpu, int(batch.total),
                                          "O1 sequential stepping of all 64 members"),
           "unknowns": int(batch.total), "ms_per_step": ms,
           "value": batch.total / (ms / 1e3), "unit": UNIT, "iterations": it,
           "relres_max": rel, "residual_tol": 1e-10,
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                        "frac": gbs / hbm, "traffic": None, "algorithmic_bytes": byts,
                        "scope": "the whole solve (every kernel) over its CUDA-event time",
                        "peak_source": f"{src} (MEASURED_PEAKS.json)"},
           "kernel_roofline": kroof, "autotuned": batch.tuned(),
           "gpu_launches": (batch.launches() - l0) // k}
    batch.close()
    return out


# DRAM bytes (read + write) per launch of the ParaDiag-I mixed kernels from one ncu
# capture of each on the 255 x 1023 x 32 window; an entry goes back to absent
# whenever its kernel changes.
PD1_NCU_TRAFFIC = {("mixed", "pd1_resid_step_a"): 169.9e6, ("mixed", "pd1_step_c_update"): 155.0e6}


def pd1_bytes_per_unknown(fp64):
    """Algorithmic DRAM bytes per space-time unknown of the ParaDiag-I kernels
    of one refinement sweep: step (a) reads the iterate and b and writes one
    complex spectrum value; step (c) reads the spectrum and updates the iterate."""
    st = 8.0
    c = 16.0 if fp64 else 8.0
    return {"pd1_resid_step_a": 2 * st + c, "pd1_step_c_update": c + 2 * st}


def pd1_kernel_profile(pd, torch, dev, precisions):
    """Per-kernel times of a ParaDiag-I refinement sweep on a 255 x 1023 x 32
    window (8.3 M unknowns; the sweep's working set exceeds the 129 MB L2),
    as algorithmic HBM throughput against the measured copy peak."""
    import workloads as W
    wl = W.pd1_ade2d()
    pb = wl.problem
    sp = pb.space
    big = dict(dim=2, nx=sp.nx, ny=1023, nu=sp.nu, ax=sp.ax, ay=sp.ay, bc_x=sp.bc_x,
               bc_y=sp.bc_y)
    stream = torch.cuda.current_stream()
    hbm, _, src = peaks()
    nsb = sp.nx * 1023 * pb.nt
    kern = {}
    for prec in precisions:
        tag = "fp64" if prec == pd.PD_FP64 else "mixed"
        pl = pd.Plan1(big, pb.nt, pb.dt_last, pb.tau, pd.PD_BE, True, prec, stream)
        u0b = torch.exp(-torch.linspace(-3.0, 3.0, sp.nx * 1023, dtype=torch.float64,
                                        device=dev) ** 2)
        bb = pl.build_rhs(u0b)
        ub = torch.empty_like(bb)
        pl.profile_sweep(bb, ub, reps=2)
        kms = pl.profile_sweep(bb, ub, reps=5)
        bpu = pd1_bytes_per_unknown(prec == pd.PD_FP64)
        ent = {}
        for name, t in (("pd1_resid_step_a", kms[0]), ("pd1_step_c_update", kms[2])):
            gbs = bpu[name] * nsb / (t / 1e3) / 1e9
            ent[name] = {"ms": t, "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                         "frac": gbs / hbm, "algorithmic_bytes": bpu[name] * nsb,
                         "traffic": PD1_NCU_TRAFFIC.get((tag, name)),
                         "peak_source": f"{src} (MEASURED_PEAKS.json)"}
        ent["step_b_ms"] = kms[1]
        kern[tag] = ent
        pl.close()
    return kern


def pd1_leg(pd, torch, dev, args):
    """ParaDiag-I (geometric steps, Section 2.1.1): one window of the 2D grid,
    255 x 255, Nt = 32, tau = 1.16, dt_Nt = 0.05, backward Euler.  Timed: the
    mixed solve (FP32 steps, double-float residual sweeps) to a relative
    residual of 1e-12, L2 flushed before every solve (the window's working set,
    ~0.1 GB, fits in L2); beside it the FP64 direct solve (the paper's
    method) and the FP64 solve refined to the same residual.  The per-kernel
    rooflines come from a 255 x 1023 x 32 window (working set above L2)."""
    import workloads as W
    wl = W.pd1_ade2d()
    pb = wl.problem
    sp = pb.space
    space = dict(dim=2, nx=sp.nx, ny=sp.ny, nu=sp.nu, ax=sp.ax, ay=sp.ay, bc_x=sp.bc_x,
                 bc_y=sp.bc_y)
    stream = torch.cuda.current_stream()
    NS = pb.unknowns
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)   # 256 MB > L2
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(plan, b, u, k, **kw):
        tot = 0.0
        res = None
        for i in range(k):
            flush.fill_(float(i))
            e0.record(stream)
            res = plan.solve(b, u, **kw)
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / k, res

    plan = pd.Plan1(space, pb.nt, pb.dt_last, pb.tau, pd.PD_BE, True, pd.PD_MIXED, stream)
    b = plan.build_rhs(torch.from_numpy(wl.u0).to(dev))
    u = torch.empty_like(b)
    for _ in range(3):
        plan.solve(b, u, tol=1e-12, max_refine=20)
    k = max(1, min(args.steps, 20))
    l0 = plan.launches()
    ms, (_, sweeps, rel) = timed(plan, b, u, k, tol=1e-12, max_refine=20)
    launches = (plan.launches() - l0) // k
    r64 = float(torch.linalg.norm(b - plan.apply_A(u)) / torch.linalg.norm(b))

    plan64 = pd.Plan1(space, pb.nt, pb.dt_last, pb.tau, pd.PD_BE, True, pd.PD_FP64, stream)
    u64 = torch.empty_like(b)
    plan64.solve(b, u64)
    k64 = max(1, min(args.steps, 3))
    ms_direct, (_, _, rel_direct) = timed(plan64, b, u64, k64)
    ms64, (_, sweeps64, rel64) = timed(plan64, b, u64, k64, tol=1e-12, max_refine=20)
    plan.close()
    plan64.close()

    kern = pd1_kernel_profile(pd, torch, dev, (pd.PD_MIXED, pd.PD_FP64))
    del flush
    return {"workload": "pd1_ade2d_be_255x255x32: 2D advection-diffusion (x periodic, "
                        "y Dirichlet, nu = 1e-3, velocity (1, 0.5)), backward Euler, "
                        "geometric steps dt_n = 0.05 * 1.16^(n-32), column-scaled V",
            "unknowns": NS, "ms_per_solve": ms, "value": NS / (ms / 1e3), "unit": UNIT,
            "refinement_sweeps": sweeps, "relres": rel, "relres_fp64_apply_A": r64,
            "gpu_launches": launches, "l2": "flushed (256 MB write) before every solve",
            "fp64_direct": {"ms_per_solve": ms_direct, "value": NS / (ms_direct / 1e3),
                            "relres": rel_direct},
            "fp64_refined": {"ms_per_solve": ms64, "value": NS / (ms64 / 1e3),
                             "refinement_sweeps": sweeps64, "relres": rel64},
            "kernel_roofline_255x1023x32": kern}


FP32_ALU_PEAK = 152 * 128 * 2 * 2.07e9 / 1e12   # TFLOP/s: SMs x FP32 lanes x FMA x max SM clock


def hybrid_kernel_profile(pd, torch, dev, precisions):
    """Per-stage times of a hybrid ParaDiag-I refinement sweep on the bench
    workload (255 x 255 x 256): the residual (HBM: 20 bytes per unknown on the
    mixed path, 24 on the FP64 path), the two dense time contractions and step
    (b).  Mixed plans run the contractions on the tensor cores (tcgen05); they
    are then HBM-bound (step (a): 4 B of r in + 4 B of spectrum out per
    unknown; step (c): 4 B of spectrum in + 16 B of double-float iterate in and
    out per unknown; the spectrum transpose of step (c) is extra traffic, not
    algorithmic).  The CUDA-core engine of the same plan is timed beside it
    ("mixed_cuda_cores"), and the FP64 plan (CUDA cores), against the FP32 /
    FP64 ALU rate: 2 Nt flops per unknown each."""
    import workloads as W
    wl = W.hybrid_ade2d()
    pb = wl.problem
    sp = pb.space
    space = dict(dim=2, nx=sp.nx, ny=sp.ny, nu=sp.nu, ax=sp.ax, ay=sp.ay, bc_x=sp.bc_x,
                 bc_y=sp.bc_y)
    stream = torch.cuda.current_stream()
    hbm, _, src = peaks()
    ns = pb.unknowns
    out = {}
    runs = []
    for prec in precisions:
        runs.append((prec, None))
        if prec == pd.PD_MIXED:
            runs.append((prec, False))
    for prec, tc in runs:
        fp64 = prec == pd.PD_FP64
        pl = pd.PlanHybrid(space, pb.nt, pb.dt, prec, stream)
        if tc is not None:
            pl.set_tensor_cores(tc)
        on_tc = pl.tensor_cores
        b = pl.build_rhs(torch.from_numpy(wl.u0).to(dev))
        u = torch.empty_like(b)
        pl.profile_sweep(b, u, reps=1)
        kms = pl.profile_sweep(b, u, reps=3 if fp64 else 5)
        nh = (pb.nt + 1) // 2
        flops = 2.0 * (2 * nh) * pb.nt * sp.nx * sp.ny
        rb = (24.0 if fp64 else 20.0) * ns
        gbs = rb / (kms[0] / 1e3) / 1e9
        ent = {"engine": "tcgen05" if on_tc else "cuda_cores",
               "resid": {"ms": kms[0], "bound": "hbm", "achieved": gbs, "peak": hbm,
                         "unit": "GB/s", "frac": gbs / hbm, "algorithmic_bytes": rb,
                         "peak_source": f"{src} (MEASURED_PEAKS.json)"},
               "step_b_ms": kms[2]}
        for name, t, bpu in (("gemm_step_a", kms[1], 8.0), ("gemm_step_c_update", kms[3], 20.0)):
            tf = flops / (t / 1e3) / 1e12
            if on_tc:
                ab = bpu * ns
                ach = ab / (t / 1e3) / 1e9
                ent[name] = {"ms": t, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                             "frac": ach / hbm, "algorithmic_bytes": ab,
                             "peak_source": f"{src} (MEASURED_PEAKS.json)",
                             "tensor_tflops_algorithmic": tf}
                continue
            pk = FP32_ALU_PEAK / 64.0 if fp64 else FP32_ALU_PEAK
            ent[name] = {"ms": t, "bound": "alu", "achieved": tf, "peak": pk, "unit": "TFLOP/s",
                         "frac": tf / pk, "algorithmic_flops": flops,
                         "peak_source": ("FP64 CUDA-core rate taken as 1/64 of " if fp64 else "")
                         + "152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz (derived, nominal)"}
        key = "fp64" if fp64 else ("mixed" if tc is None else "mixed_cuda_cores")
        out[key] = ent
        pl.close()
    return out


def hybrid_leg(pd, torch, dev, args):
    """ParaDiag-I with the hybrid midpoint + backward-Euler discretisation
    (Section 2.1.2) on the bench grid: 255 x 255, Nt = 256, T = 1 (16.6 M
    unknowns).  Timed: the mixed solve (direct + refinement sweeps) to a
    relative residual of 1e-11 (the tolerance of the main metric); beside it
    the FP64 direct solve and the FP64 solve refined to the same residual."""
    import workloads as W
    wl = W.hybrid_ade2d()
    pb = wl.problem
    sp = pb.space
    space = dict(dim=2, nx=sp.nx, ny=sp.ny, nu=sp.nu, ax=sp.ax, ay=sp.ay, bc_x=sp.bc_x,
                 bc_y=sp.bc_y)
    stream = torch.cuda.current_stream()
    NS = pb.unknowns
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(plan, b, u, k, **kw):
        res = None
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(k):
            res = plan.solve(b, u, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k, res

    plan = pd.PlanHybrid(space, pb.nt, pb.dt, pd.PD_MIXED, stream)
    b = plan.build_rhs(torch.from_numpy(wl.u0).to(dev))
    u = torch.empty_like(b)
    for _ in range(3):
        plan.solve(b, u, tol=TOL, max_refine=20)
    k = max(1, min(args.steps, 20))
    l0 = plan.launches()
    ms, (_, sweeps, rel) = timed(plan, b, u, k, tol=TOL, max_refine=20)
    launches = (plan.launches() - l0) // k
    r64 = float(torch.linalg.norm(b - plan.apply_A(u)) / torch.linalg.norm(b))
    cond = plan.condition()
    plan.close()
    plan64 = pd.PlanHybrid(space, pb.nt, pb.dt, pd.PD_FP64, stream)
    u64 = torch.empty_like(b)
    plan64.solve(b, u64)
    k64 = max(1, min(args.steps, 2))
    ms_direct, (_, _, rel_direct) = timed(plan64, b, u64, k64)
    ms64, (_, sweeps64, rel64) = timed(plan64, b, u64, k64, tol=TOL, max_refine=20)
    plan64.close()
    return {"workload": "hybrid_ade2d_255x255x256: 2D advection-diffusion (x periodic, "
                        "y Dirichlet, nu = 1e-3, velocity (1, 0.5)), midpoint steps + one "
                        "backward-Euler step, dt = 1/256",
            "unknowns": NS, "ms_per_solve": ms, "value": NS / (ms / 1e3), "unit": UNIT,
            "refinement_sweeps": sweeps, "relres": rel, "relres_fp64_apply_A": r64,
            "residual_tol": TOL, "cond_V_frobenius": cond, "gpu_launches": launches,
            "l2": "working set ~0.6 GB > 129 MB L2, no flush",
            "fp64_direct": {"ms_per_solve": ms_direct, "value": NS / (ms_direct / 1e3),
                            "relres": rel_direct},
            "fp64_refined": {"ms_per_solve": ms64, "value": NS / (ms64 / 1e3),
                             "refinement_sweeps": sweeps64, "relres": rel64},
            "kernels": hybrid_kernel_profile(pd, torch, dev, (pd.PD_MIXED, pd.PD_FP64))}


def wave_leg(pd, torch, dev, args):
    """Second-order hybrid ParaDiag-I (B_2nd = B^2, Section 2.1.2) on the wave
    problem of Table Ex2Tab1 at its strong-scaling setting: dx = dy = 1/512
    (511 x 511 interior points), Nt = 512, T = 2 (133.7 M unknowns).  Timed: the
    mixed solve (direct + refinement sweeps) to a relative residual of 1e-10,
    far below the 7.88e-5 discretisation error; beside it the FP64 direct solve.
    The table's CPU seconds (1 and 256 cores) are quoted as context."""
    import numpy as np
    import workloads as W
    wl = W.hybrid_wave2d()
    pb = wl.problem
    sp = pb.space
    space = dict(dim=2, nx=sp.nx, ny=sp.ny, nu=sp.nu, bc_x=sp.bc_x, bc_y=sp.bc_y)
    stream = torch.cuda.current_stream()
    NS = pb.unknowns
    tol = 1e-10
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t = torch.from_numpy(np.sin(2.0 * np.pi * pb.dt * np.arange(1, pb.nt + 1))).to(dev)
    phi = torch.from_numpy(wl.extra["phi"]).to(dev)

    def max_err(u):
        return float((u - torch.outer(t, phi)).abs().max())

    def timed(plan, b, u, k, **kw):
        res = None
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(k):
            res = plan.solve(b, u, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k, res

    plan = pd.PlanHybrid(space, pb.nt, pb.dt, pd.PD_MIXED, stream, order=2)
    b = plan.build_rhs_wave(torch.from_numpy(wl.u0).to(dev), torch.from_numpy(wl.u1).to(dev),
                            torch.from_numpy(wl.f).to(dev))
    u = torch.empty_like(b)
    for _ in range(3):
        plan.solve(b, u, tol=tol, max_refine=20)
    k = max(1, min(args.steps, 10))
    l0 = plan.launches()
    ms, (_, sweeps, rel) = timed(plan, b, u, k, tol=tol, max_refine=20)
    launches = (plan.launches() - l0) // k
    err = max_err(u)
    r64 = float(torch.linalg.norm(b - plan.apply_A(u)) / torch.linalg.norm(b))
    cond = plan.condition()
    plan.close()
    plan64 = pd.PlanHybrid(space, pb.nt, pb.dt, pd.PD_FP64, stream, order=2)
    u64 = torch.empty_like(b)
    plan64.solve(b, u64)
    ms_direct, (_, _, rel_direct) = timed(plan64, b, u64, 1)
    err64 = max_err(u64)
    plan64.close()
    return {"workload": "hybrid_wave2d_511x511x512: u_tt - Lap u = f on (0,1)^2 x (0,2), "
                        "Dirichlet, dx = 1/512, midpoint steps + one backward-Euler step on "
                        "the first-order form, B_2nd = B^2 (Table Ex2Tab1, strong scaling)",
            "unknowns": NS, "ms_per_solve": ms, "value": NS / (ms / 1e3), "unit": UNIT,
            "refinement_sweeps": sweeps, "relres": rel, "relres_fp64_apply_A": r64,
            "residual_tol": tol, "max_error_vs_exact": err, "paper_error": 7.88e-5,
            "cond_V_frobenius": cond, "gpu_launches": launches,
            "l2": "working set ~4 GB > 129 MB L2, no flush",
            "fp64_direct": {"ms_per_solve": ms_direct, "value": NS / (ms_direct / 1e3),
                            "relres": rel_direct, "max_error_vs_exact": err64},
            "paper_cpu_seconds_context": {"1_core": 1328.6, "256_cores": 20.3}}


def nonlinear_leg(pd, torch, dev, args):
    """Nonlinear problems by simplified Newton with the averaged Jacobian (eq.
    1.4, eq. 1.5) on the bench grid: the ade2d problem (255 x 255, Nt = 256,
    CN, alpha = 1e-3, Gaussian bump) with the reaction phi(u) = u^3.  Timed: a
    mixed-plan solve (FP64 residual, FP32 preconditioner with the averaged
    shift) from a zero guess to ||r|| <= 1e-10 ||b||, the zero fill of the
    iterate included; beside it one FP64-plan solve, and the residual kernels
    on their own (double-float on mixed plans: 24 bytes per unknown; FP64 on
    FP64 plans: 29 flops per unknown)."""
    import workloads as W
    wl = W.nl_ade2d()
    pb = wl.problem
    sp = pb.space
    a = wl.extra["reaction"]
    space = dict(dim=2, nx=sp.nx, ny=sp.ny, nu=sp.nu, ax=sp.ax, ay=sp.ay, bc_x=sp.bc_x,
                 bc_y=sp.bc_y)
    stream = torch.cuda.current_stream()
    NS = pb.unknowns
    tol = 1e-10
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    plan = pd.Plan(space, pb.nt, pb.dt, pb.alpha, pd.PD_CN, 0.5, pd.PD_MIXED, stream)
    b = plan.nl_build_rhs(a, torch.from_numpy(wl.u0).to(dev))
    u = torch.zeros_like(b)
    plan.nl_solve(a, b, u, tol=tol, maxit=80)
    k = max(1, min(args.steps, 3))
    l0 = plan.launches()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(k):
        u.zero_()
        _, it, rel = plan.nl_solve(a, b, u, tol=tol, maxit=80)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / k
    launches = (plan.launches() - l0) // k
    _, sigma, _ = plan.nl_residual(a, b, u)
    def time_resid(pl, reps=5):
        r = torch.empty_like(b)
        pl.nl_residual(a, b, u, r)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            pd.pd_nl_residual(pl._h, a, b.data_ptr(), u.data_ptr(), r.data_ptr(), scalars=False)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    # the residual kernel alone: double-float on the mixed plan
    ms_r = time_resid(plan)
    plan.close()
    hbm, _, src = peaks()
    rbytes = 24.0 * NS
    gbs = rbytes / (ms_r / 1e3) / 1e9
    plan64 = pd.Plan(space, pb.nt, pb.dt, pb.alpha, pd.PD_CN, 0.5, pd.PD_FP64, stream)
    ms_r64 = time_resid(plan64, reps=3)
    flops = 29.0 * NS
    fp64_peak = FP32_ALU_PEAK / 64.0
    tf = flops / (ms_r64 / 1e3) / 1e12
    u64 = torch.zeros_like(b)
    torch.cuda.synchronize()
    e0.record(stream)
    _, it64, rel64 = plan64.nl_solve(a, b, u64, tol=tol, maxit=80)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    diff = float((u - u64).abs().max() / u64.abs().max())
    plan64.close()
    return {"workload": "nl_ade2d_255x255x256: u_t - nu Lap u + a.grad u + u^3 = 0 on the "
                        "ade2d grid (x periodic, y Dirichlet, nu = 1e-3, velocity (1, 0.5)), "
                        "Crank-Nicolson, alpha = 1e-3, Gaussian bump",
            "unknowns": NS, "ms_per_solve": ms, "value": NS / (ms / 1e3), "unit": UNIT,
            "newton_corrections": it, "relres": rel, "residual_tol": tol,
            "sigma_at_solution": sigma, "gpu_launches": launches,
            "residual_kernel": {"kernel": "k_nl_resid_df (double-float on the FP32 pipes)",
                                "ms": ms_r, "algorithmic_bytes": rbytes, "achieved_GBps": gbs,
                                "frac_of_measured_hbm": gbs / hbm, "peak_source": src,
                                "limiter": "instruction issue (double-float arithmetic and the "
                                           "integer splits of the FP64 inputs)"},
            "residual_kernel_fp64_plan": {"kernel": "k_nl_resid (FP64)", "ms": ms_r64,
                                          "bound": "alu", "achieved": tf, "peak": fp64_peak,
                                          "unit": "TFLOP/s (FP64)", "frac": tf / fp64_peak,
                                          "algorithmic_flops": flops, "traffic": 374.4e6,
                                          "peak_source": "FP64 CUDA-core rate taken as 1/64 of "
                                                         "152 SMs x 128 FP32 lanes x 2 flops x "
                                                         "2070 MHz (derived)"},
            "fp64_plan": {"ms_per_solve": ms64, "value": NS / (ms64 / 1e3),
                          "newton_corrections": it64, "relres": rel64,
                          "max_rel_diff_vs_mixed": diff}}


def control_leg(pd, torch, dev, args):
    """Optimal control of the 2D wave equation (Section 4) on the largest mesh of
    Table T2A, (256, 256, 257): 255 x 255 interior points, Nt = 257, T = 2,
    gamma in {1e-2, 1e-4, 1e-8}; FGMRES(40) on the balanced saddle-point system
    with the Theorem 4 preconditioner (FP64; FP32 as well at gamma = 1e-8),
    tol 1e-7, zero initial guess.
    The right-hand side is the saddle-point operator applied to the exact
    optimal pair on the grid.  The table's CPU seconds are quoted as context."""
    import numpy as np
    import workloads as W
    n, nt, T = 256, 257, 2.0
    sp = W.Space(dim=2, nx=n - 1, ny=n - 1, nu=1.0, bc_x=W.DIRICHLET, bc_y=W.DIRICHLET)
    space = dict(dim=2, nx=n - 1, ny=n - 1, nu=1.0, bc_x=0, bc_y=0)
    X, Y = sp.mesh()
    s = (np.sin(np.pi * X) * np.sin(np.pi * Y)).reshape(-1)
    t = (T / nt) * np.arange(1, nt + 1)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    table = [(1e-2, pd.PD_FP64, 17, 226.6), (1e-4, pd.PD_FP64, 5, 59.6),
             (1e-8, pd.PD_FP64, 5, 61.0), (1e-8, pd.PD_MIXED, 5, 61.0)]
    rows = []
    for g, prec, it_paper, cpu_paper in table:
        pl = pd.PlanControl(space, nt, T, g, prec, stream)
        sg = np.sqrt(g)
        xb = torch.from_numpy(np.concatenate([sg * np.outer(np.exp(t), s).reshape(-1),
                                              np.outer((t - T) ** 2, s).reshape(-1)])).to(dev)
        b = pl.apply_A(xb)
        m = nt * sp.size
        b[:m] /= sg
        x = torch.empty_like(b)
        pl.solve(b, x, tol=1e-7, maxit=100, restart=40)
        k = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(k):
            _, it, rel = pl.solve(b, x, tol=1e-7, maxit=100, restart=40)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k
        x[:m] *= sg
        err = float(torch.linalg.norm(x - xb) / torch.linalg.norm(xb))
        left = None
        if prec == pd.PD_FP64:
            # left preconditioning, stopping on the preconditioned residual
            xl = torch.empty_like(b)
            torch.cuda.synchronize()
            e0.record(stream)
            _, itl, rell = pl.solve(b, xl, tol=1e-7, maxit=100, restart=50, left=True)
            e1.record(stream)
            torch.cuda.synchronize()
            left = {"ms_per_solve": e0.elapsed_time(e1), "gmres_iterations": itl,
                    "preconditioned_relres": rell}
        rows.append({"gamma": g, "preconditioner": "fp64" if prec == pd.PD_FP64 else "fp32",
                     "ms_per_solve": ms, "gmres_iterations": it, "relres": rel,
                     "rel_error_vs_exact_pair": err, "unknowns": 2 * m,
                     "value": 2 * m / (ms / 1e3), "unit": UNIT,
                     "left_preconditioned": left,
                     "paper_iterations": it_paper, "paper_cpu_seconds_context": cpu_paper})
        pl.close()
    return {"workload": "control_wave2d_256x256x257: optimal control of u_tt - Lap u = f + "
                        "control on (0,1)^2 x (0,2), leap-frog saddle point (Table T2A's "
                        "largest mesh)",
            "solves": rows}


def timed_solves(torch, stream, fn, k):
    """Average CUDA-event milliseconds of k calls of fn() on the stream (each
    call returns its own result; the last result is returned)."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    res = None
    for _ in range(k):
        res = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / k, res


def ade1d_leg(pd, torch, dev, args):
    """The 1D advection-diffusion configuration: nx = 127 (Dirichlet), Nt = 64,
    backward Euler, nu = 1e-2, a = 1, alpha = 1e-2, u0 = sin(pi x), source on 8
    seeded sine modes; the stationary iteration from a zero guess to a relative
    residual of 1e-12 (FP64 plan, the configuration's solver; the mixed plan
    beside it).  8128 unknowns: a latency-bound size, no roofline claim."""
    import numpy as np
    import workloads as W
    from oracle import operators as O
    from oracle import stepping as S
    w = W.ade1d()
    pb = w.problem
    sp = pb.space
    from oracle import paradiag as PDO
    bref = O.build_rhs(pb, w.u0, None, w.f)
    t0 = time.perf_counter()
    for _ in range(20):
        uref = S.solve_sequential(pb, bref)
    t_cpu = (time.perf_counter() - t0) / 20
    # the naive-DFT ParaDiag (O2, the stationary iteration with a dense Fourier
    # matrix and a sparse LU per frequency) on the host: a CPU ParaDiag reference
    t0 = time.perf_counter()
    for _ in range(5):
        _, it_o2, _ = PDO.stationary(pb, bref, tol=1e-12, maxit=30)
    t_o2 = (time.perf_counter() - t0) / 5
    stream = torch.cuda.current_stream()
    out = {"workload": "ade1d_be_127x64: 1D advection-diffusion, Dirichlet, nu = 1e-2, a = 1, "
                       "backward Euler, alpha = 1e-2", "unknowns": pb.unknowns,
           "residual_tol": 1e-12, "roofline": "none (latency-bound size)",
           "cpu_oracle": cpu_oracle_entry(t_cpu, pb.unknowns, "O1 sequential stepping, 20 repetitions"),
           "cpu_paradiag_o2": dict(cpu_oracle_entry(t_o2, pb.unknowns,
                                                    "O2 naive-DFT ParaDiag, stationary to 1e-12, "
                                                    "5 repetitions"), iterations=it_o2)}
    for prec, tag in ((pd.PD_FP64, "fp64"), (pd.PD_MIXED, "mixed")):
        plan = pd.Plan(dict(dim=1, nx=sp.nx, nu=sp.nu, ax=sp.ax), pb.nt, pb.dt, pb.alpha,
                       pd.PD_BE, 1.0, prec, stream)
        b = plan.build_rhs(torch.from_numpy(w.u0).to(dev), None, torch.from_numpy(w.f).to(dev))
        u = torch.zeros_like(b)
        for _ in range(3):
            plan.solve(b, u.zero_(), tol=1e-12, maxit=30)
        k = max(1, min(args.steps, 50))
        ms, (_, it, rel) = timed_solves(torch, stream,
                                        lambda: plan.solve(b, u.zero_(), tol=1e-12, maxit=30), k)
        err = float(np.linalg.norm(u.cpu().numpy() - uref) / np.linalg.norm(uref))
        out[tag] = {"ms_per_solve": ms, "value": pb.unknowns / (ms / 1e3), "unit": UNIT,
                    "iterations": it, "relres": rel, "error_vs_oracle": err}
        plan.close()
    return out


def adjoint_leg(pd, torch, dev, args):
    """The heat-source inversion: 127 x 127 grid (Dirichlet, nu = 1), backward
    Euler, Nt = 128, J(f) = 1/2 ||U_Nt - u_target||^2 + 1/2 1e-4 ||f||^2 with
    u_target a seeded sum of 4 Gaussians.  One forward solve and one transposed
    solve (backward in time) through PDSolve (torch.autograd.Function), mixed
    plan, to a relative residual of 1e-11; timed as a pair.  Checked: J and
    dJ/df against the oracle (sequential forward and backward stepping), and
    16 central differences of J at h = 1e-6 (and at h = 1e-2: J is quadratic in
    f, so central differences are exact at any h up to the solves' error)."""
    import numpy as np
    import workloads as W
    from oracle import control as C
    w = W.heat2d_control()
    pb = w.problem
    sp = pb.space
    tgt = torch.from_numpy(w.extra["u_target"]).to(dev)
    reg = w.extra["reg"]
    f0 = w.extra["f_probe"]
    stream = torch.cuda.current_stream()
    space = dict(dim=2, nx=sp.nx, ny=sp.ny, nu=sp.nu, bc_x=sp.bc_x, bc_y=sp.bc_y)
    t0 = time.perf_counter()
    J_ref, g_ref, _, _ = C.gradient(pb, f0, w.extra["u_target"], reg)
    t_cpu = time.perf_counter() - t0
    out = {"workload": "heat2d_adjoint_127x127x128: 2D heat equation source inversion, "
                       "backward Euler, Dirichlet", "unknowns_per_solve": pb.unknowns,
           "residual_tol": 1e-11,
           "cpu_oracle": cpu_oracle_entry(t_cpu, 2 * pb.unknowns,
                                          "O5 gradient: forward and backward sequential stepping")}
    for prec, tag in ((pd.PD_MIXED, "mixed"), (pd.PD_FP64, "fp64")):
        plan = pd.Plan(space, pb.nt, pb.dt, pb.alpha, pd.PD_BE, 1.0, prec, stream)

        def J_of(fd):
            b = fd.unsqueeze(0).expand(pb.nt, -1).contiguous()      # b_n = f (BE, u0 = 0)
            u = pd.PDSolve.apply(plan, b, pd.PD_STATIONARY, 1e-11, 60)
            e = u[-1] - tgt
            return 0.5 * (e * e).sum() + 0.5 * reg * (fd * fd).sum()

        def pair():
            fd = torch.from_numpy(f0).to(dev).requires_grad_(True)
            J = J_of(fd)
            J.backward()
            return J.detach(), fd.grad

        for _ in range(2):
            pair()
        k = max(1, min(args.steps, 10 if prec == pd.PD_MIXED else 2))
        ms, (J, grad) = timed_solves(torch, stream, pair, k)
        gh = grad.cpu().numpy()
        ent = {"ms_per_pair": ms, "value": 2 * pb.unknowns / (ms / 1e3), "unit": UNIT,
               "J": float(J), "J_rel_error_vs_oracle": abs(float(J) - J_ref) / abs(J_ref),
               "grad_norm": float(np.linalg.norm(gh)),
               "grad_rel_error_vs_oracle": float(np.linalg.norm(gh - g_ref) / np.linalg.norm(g_ref))}
        if prec == pd.PD_MIXED:
            fd = torch.from_numpy(f0).to(dev)
            for h in (1e-6, 1e-2):
                errs = []
                with torch.no_grad():
                    for i in range(16):
                        d = torch.from_numpy(W.uniform(W.SEED_BASE + 200 + i, sp.size, -1.0,
                                                       1.0)).to(dev)
                        fdiff = (float(J_of(fd + h * d)) - float(J_of(fd - h * d))) / (2 * h)
                        dot = float((grad * d).sum())
                        errs.append(abs(fdiff - dot) / abs(dot))
                ent[f"fd_rel_error_max_h{h:g}"] = max(errs)
        out[tag] = ent
        plan.close()
    return out


def wave_gmres_leg(pd, torch, dev, args):
    """The 1D wave equation: u_tt = u_xx on (0, 1), Dirichlet, nx = 1023,
    leap-frog (eq. 3.2b), Nt = 1024, T = 2, u0 = exp(-100 (x - 1/2)^2), u_t(0) = 0;
    FGMRES(30) right-preconditioned by P_alpha, alpha = 0.1, FP64 Krylov
    vectors, to a relative residual of 1e-10 from a zero guess (Section 3; Table
    T4A reports 3 iterations at alpha = 0.1), and to 1e-12, which brings the
    error below 1e-10.  Both plans (FP32 or FP64 preconditioner); error against
    the oracle's sequential stepping."""
    import numpy as np
    import workloads as W
    from oracle import operators as O
    from oracle import stepping as S
    w = W.wave1d()
    pb = w.problem
    sp = pb.space
    t0 = time.perf_counter()
    uref = S.solve_sequential(pb, O.build_rhs(pb, w.u0, w.u1, None))
    t_cpu = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    out = {"workload": "wave1d_leapfrog_1023x1024: 1D wave, Dirichlet, leap-frog, T = 2, "
                       "alpha = 0.1, FGMRES(30)", "unknowns": pb.unknowns, "residual_tol": 1e-10,
           "paper_iterations_T4A": 3, "l2": "working set ~0.3 GB (30 Krylov vectors) > L2",
           "cpu_oracle": cpu_oracle_entry(t_cpu, pb.unknowns, "O1 sequential leap-frog stepping")}
    for prec, tag in ((pd.PD_MIXED, "mixed"), (pd.PD_FP64, "fp64")):
        plan = pd.Plan(dict(dim=1, nx=sp.nx, nu=sp.nu), pb.nt, pb.dt, pb.alpha, pd.PD_LEAPFROG,
                       1.0, prec, stream)
        b = plan.build_rhs(torch.from_numpy(w.u0).to(dev), torch.from_numpy(w.u1).to(dev))
        u = torch.zeros_like(b)
        plan.solve(b, u.zero_(), mode=pd.PD_GMRES, tol=1e-10, maxit=60, restart=30)
        k = max(1, min(args.steps, 10))
        ms, (_, it, rel) = timed_solves(
            torch, stream,
            lambda: plan.solve(b, u.zero_(), mode=pd.PD_GMRES, tol=1e-10, maxit=60, restart=30), k)
        err = float(np.linalg.norm(u.cpu().numpy() - uref) / np.linalg.norm(uref))
        # the same solve to 1e-12: the leap-frog system amplifies the residual
        # about tenfold into the error, so this is the solve that meets 1e-10
        ms12, (_, it12, rel12) = timed_solves(
            torch, stream,
            lambda: plan.solve(b, u.zero_(), mode=pd.PD_GMRES, tol=1e-12, maxit=60, restart=30), k)
        err12 = float(np.linalg.norm(u.cpu().numpy() - uref) / np.linalg.norm(uref))
        out[tag] = {"ms_per_solve": ms, "value": pb.unknowns / (ms / 1e3), "unit": UNIT,
                    "gmres_iterations": it, "relres": rel, "error_vs_oracle": err,
                    "tol_1e-12": {"ms_per_solve": ms12, "value": pb.unknowns / (ms12 / 1e3),
                                  "gmres_iterations": it12, "relres": rel12,
                                  "error_vs_oracle": err12}}
        plan.close()
    return out


def run_sweep(pd, torch, dev, only=None):
    """Per-kernel time and algorithmic HBM throughput of one mixed iteration on
    1D advection-diffusion problems (nu = 1e-2, a = 1, BE, alpha = 1e-2) of
    growing size, so that the working set passes the 129 MB L2."""
    import workloads as W
    hbm, _, src = peaks()
    rows = []
    sizes = [(nx, nt) for nx in (255, 1023, 4095) for nt in (256, 1024, 4096)]
    if only:
        sizes = [tuple(int(v) for v in only.lower().split("x"))]
    for nx, nt in sizes:
        w = W.ade1d(nx=nx, nt=nt, nu=1e-2, a=1.0, scheme=W.BE, alpha=1e-2)
        pb = w.problem
        sp = pb.space
        plan = pd.Plan(dict(dim=1, nx=sp.nx, nu=sp.nu, ax=sp.ax), pb.nt, pb.dt, pb.alpha,
                       pd.PD_BE, 1.0, pd.PD_MIXED, torch.cuda.current_stream())
        b = plan.build_rhs(torch.from_numpy(w.u0).to(dev), None,
                           torch.from_numpy(w.f).to(dev))
        u = torch.zeros_like(b)
        plan.profile_iteration(b, u, reps=2)
        kms = plan.profile_iteration(b, u, reps=5)
        bpu = bytes_per_unknown(nt, False)
        ns = nx * nt
        ker = {}
        for name, t in zip(KERNELS, kms):
            if t > 0:
                gbs = bpu[name] * ns / (t / 1e3) / 1e9
                ker[name] = {"ms": t, "GB/s": gbs, "frac": gbs / hbm}
        row = {"nx": nx, "nt": nt, "unknowns": ns, "time_cluster": plan.time_cluster,
               "tile_columns": plan.tuning()[0], "kernels": ker}
        # the time kernels with each tile split the plan allows (one block,
        # or a cluster of 2, 4 or 8 blocks)
        if nt >= 1024:
            chosen = plan.time_cluster
            by = {}
            for cr in (1, 2, 4, 8):
                try:
                    plan.set_time_cluster(cr)
                except pd.PDError:
                    continue
                plan.profile_iteration(b, u, reps=1)
                km = plan.profile_iteration(b, u, reps=5)
                by[str(cr)] = {"tile_columns": plan.tuning()[0],
                               "resid_gamma_fft_ms": km[0], "ifft_gamma_update_ms": km[-1]}
            row["time_kernels_by_cluster"] = by
            plan.set_time_cluster(chosen)
        rows.append(row)
        plan.close()
    return {"sweep": rows, "peak_GBps": hbm, "peak_source": src}


def run_reference(args):
    """The reference arm: the FP64 CPU oracle (the exact solution of the
    all-at-once system by sequential time stepping) on this host's cores, each
    step a bounded sample of the workload: its first 32 time levels, solved
    mode by mode along the periodic x with the modes spread over one spawned
    process per core (time stays sequential).  Rank 0 only."""
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    from oracle import stepping as S
    w = workload(args.small)
    pb = w.problem
    nts = 32
    sub, _, b = oracle_sample_problem(w, nts)
    nproc, model = cpu_info()
    with oracle_pool(nproc) as pool:
        for _ in range(args.warmup):
            S.solve_sequential_xmodes(sub, b, pool=pool, chunks=nproc)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            S.solve_sequential_xmodes(sub, b, pool=pool, chunks=nproc)
        el = time.perf_counter() - t0
    ms = el / args.steps * 1e3
    value = sub.unknowns / (ms / 1e3)
    desc = (f"each step: oracle sequential time stepping mode by mode (naive DFT along the "
            f"periodic x, dense LU per mode and step) over the first {nts} of {pb.nt} time "
            f"steps of the {WORKLOAD} grid, modes spread over {nproc} spawned processes")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded Gaussian initial value, zero source)",
           "config": bench_config(w, args.small, ws),
           "sample": {"time_levels": nts, "of": pb.nt, "unknowns_per_step": sub.unknowns},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": nproc, "kind": "oracle",
                            "sample": desc, "nproc": nproc, "cpu_model": model},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_sharded(args, ws, rank, local):
    """The headline workload as one problem split over the ranks
    (paradiag_gb300.shard): rank r owns a slab of grid lines (y) for the
    residual, the time transforms and the x-transforms, and a slab of time
    frequencies for the shifted solves; an all-to-all of the spectrum (NCCL)
    sits on either side of step (b) and an all-reduce of ||r||^2 decides the
    stopping test.  Timed like the main leg: W warm-up solves, K timed solves
    between barriers, the slowest rank's time."""
    import numpy as np
    import torch
    import paradiag_gb300 as pd
    from paradiag_gb300 import shard
    pd.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload(args.small)
    pb = w.problem
    sp = pb.space
    space = dict(dim=2, nx=sp.nx, ny=sp.ny, nu=sp.nu, ax=sp.ax, ay=sp.ay, bc_x=sp.bc_x,
                 bc_y=sp.bc_y)
    layout = shard.SlabLayout(sp.ny, sp.nx, pb.nt // 2 + 1, ws)
    rk = shard.RankState(pd, torch, space, pb.nt, pb.dt, pb.alpha, pd.PD_CN, 0.5, pd.PD_MIXED,
                         layout, rank, dev)
    if ws > 1:
        ex = shard.DistExchange(torch)
    else:
        ex = shard.LocalExchange(torch)
    solver = shard.ShardedSolver(pd, torch, [rk], ex)
    bw = rk.whole.build_rhs(torch.from_numpy(w.u0).to(dev))
    solver.set_rhs([bw.view(pb.nt, sp.ny, sp.nx)[:, rk.l0:rk.l1, :].reshape(pb.nt, -1)])
    for _ in range(max(args.warmup, 3)):
        solver.solve(tol=TOL, maxit=40)
    stream = torch.cuda.current_stream()
    barrier(ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        it, rel = solver.solve(tol=TOL, maxit=40)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    ms = max_over_ranks(ws, e0.elapsed_time(e1) / args.steps, dev)
    NS = pb.unknowns
    err = None
    if ws == 1 and not args.no_check:
        from oracle import operators as O
        from oracle import stepping as S
        uref = S.solve_sequential(pb, O.build_rhs(pb, w.u0, None, None))
        un = solver.owned(rk, rk.u).cpu().numpy()
        err = float(np.linalg.norm(un - uref) / np.linalg.norm(uref))
    if rank == 0:
        cfg = bench_config(w, args.small, ws)
        cfg["parallelism"] = (f"one problem over {ws} GPU(s): y slabs for the residual and the "
                              f"time transforms, frequency slabs for step (b), all-to-all of the "
                              f"FP32 spectrum between them")
        out = {"metric": METRIC, "value": NS / (ms / 1e3), "unit": UNIT, "n_gpus": ws,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
               "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
               "dtype": "f32 preconditioner + f64 residual", "data": "synthetic",
               "config": cfg, "mode": "sharded", "iterations": it, "relres": rel,
               "error_vs_oracle": err,
               "exchange_bytes_per_iteration": 2 * 8 * (pb.nt // 2 + 1) * sp.ny * (sp.nx + sp.nx % 2)}
        print(json.dumps(out), flush=True)
    rk.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.mode == "sharded":
        ws, rank, local = dist_setup()
        run_sharded(args, ws, rank, local)
        return
    ws, rank, local = dist_setup()
    import numpy as np
    import torch
    import paradiag_gb300 as pd

    pd.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload(args.small)
    pb = w.problem
    sp = pb.space
    space = dict(dim=2, nx=sp.nx, ny=sp.ny, nu=sp.nu, ax=sp.ax, ay=sp.ay, bc_x=sp.bc_x,
                 bc_y=sp.bc_y)
    NS = pb.unknowns
    stream = torch.cuda.current_stream()
    plan = pd.Plan(space, pb.nt, pb.dt, pb.alpha, pd.PD_CN, 0.5, pd.PD_MIXED, stream)
    u0 = torch.from_numpy(w.u0).to(dev)
    b = plan.build_rhs(u0)
    u = torch.zeros_like(b)
    torch.cuda.synchronize()
    if args.batch_only:
        out = batched_leg(pd, torch, dev, args)
        if rank == 0:
            print(json.dumps(out), flush=True)
        plan.close()
        return
    if args.control_only:
        out = control_leg(pd, torch, dev, args)
        if rank == 0:
            print(json.dumps(out), flush=True)
        plan.close()
        return
    if args.nonlinear_only:
        out = nonlinear_leg(pd, torch, dev, args)
        if rank == 0:
            print(json.dumps(out), flush=True)
        plan.close()
        return
    if args.wave_only:
        out = wave_leg(pd, torch, dev, args)
        if rank == 0:
            print(json.dumps(out), flush=True)
        plan.close()
        return
    if args.hybrid_kernels or args.hybrid_only:
        out = (hybrid_kernel_profile(pd, torch, dev, (pd.PD_MIXED,)) if args.hybrid_kernels
               else hybrid_leg(pd, torch, dev, args))
        if rank == 0:
            print(json.dumps(out), flush=True)
        plan.close()
        return
    if args.pd1_kernels:
        out = pd1_kernel_profile(pd, torch, dev, (pd.PD_MIXED,))
        if rank == 0:
            print(json.dumps(out), flush=True)
        plan.close()
        return
    if args.pd1_only:
        out = pd1_leg(pd, torch, dev, args)
        if rank == 0:
            print(json.dumps(out), flush=True)
        plan.close()
        return
    if args.sweep:
        out = run_sweep(pd, torch, dev, args.sweep_size)
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    if args.profile_iteration:
        # the residual-mode iteration of the solver, kernel by kernel (the command ncu captures profile)
        if args.profile_precision == "fp64":
            plan.close()
            plan = pd.Plan(space, pb.nt, pb.dt, pb.alpha, pd.PD_CN, 0.5, pd.PD_FP64, stream)
        elif args.profile_xform != "auto":
            plan.set_xform_engine(pd.PD_XFORM_TENSOR if args.profile_xform == "tensor"
                                  else pd.PD_XFORM_FFT)
        for _ in range(2):
            kms = plan.profile_iteration(b, u, reps=5)
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"workload": WORKLOAD, "kernel_ms": dict(zip(KERNELS, kms))}),
                  flush=True)
        plan.close()
        return

    clk = ClockSampler(local, args.clocks_dir)
    clk.start()
    for _ in range(max(args.warmup, 3)):
        u.zero_()
        _, iters, rel = plan.solve(b, u, tol=TOL, maxit=40)

    l0 = plan.launches()
    barrier(ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    # solves are enqueued back to back (pd_solve_async: the whole solve is one
    # CUDA graph plus entry/exit kernels), the outcome read once at the end
    for _ in range(args.steps):
        u.zero_()
        plan.solve_async(b, u, tol=TOL, maxit=40)
    e1.record(stream)
    iters, rel = plan.result()
    iters_all = [iters]
    torch.cuda.synchronize()
    barrier(ws)
    clocks = clk.stop()
    launches = (plan.launches() - l0) // args.steps
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ws, ms, dev)
    value = ws * NS / (ms / 1e3)

    # per-kernel times of one iteration (CUDA events on the plan's stream)
    kms = plan.profile_iteration(b, torch.zeros_like(b), reps=5)
    bpu = bytes_per_unknown(pb.nt, False)
    hbm, bf16, src = peaks()
    per_kernel = {}
    for name, t in zip(KERNELS, kms):
        if t <= 0:
            continue
        by = bpu[name] * NS
        per_kernel[name] = {"ms": t, "GB/s": by / (t / 1e3) / 1e9}
    rows = (pb.nt // 2 + 1) * sp.ny
    roofs = {}
    for name, pk in per_kernel.items():
        if name.startswith("xform") and plan.xform_engine != pd.PD_XFORM_TENSOR:
            # the FFT along x: HBM-bound, 8 B in + 8 B out per complex spectrum value
            roofs[name] = {"bound": "hbm", "achieved": pk["GB/s"], "peak": hbm, "unit": "GB/s",
                           "frac": pk["GB/s"] / hbm, "traffic": None, "engine": "fft",
                           "algorithmic_bytes": bpu[name] * NS,
                           "peak_source": f"{src} (MEASURED_PEAKS.json)"}
        elif name.startswith("xform"):
            # FP16 tensor-core GEMM (three products per k-step); FP16 runs at the bf16 rate
            ach = flops_per_launch_xform(rows, sp.nx) / (pk["ms"] / 1e3) / 1e12
            executed = 3 * 2.0 * rows * (2 * sp.nx) ** 2 / (pk["ms"] / 1e3) / 1e12
            roofs[name] = {"bound": "tensor", "achieved": ach, "peak": bf16, "unit": "TFLOP/s",
                           "frac": ach / bf16, "executed_tflops": executed,
                           "traffic": NCU_TRAFFIC.get(name),
                           "peak_source": f"{src} dense bf16 burst (MEASURED_PEAKS.json)"}
        else:
            roofs[name] = {"bound": "hbm", "achieved": pk["GB/s"], "peak": hbm, "unit": "GB/s",
                           "frac": pk["GB/s"] / hbm, "traffic": NCU_TRAFFIC.get(name),
                           "algorithmic_bytes": bpu[name] * NS,
                           "peak_source": f"{src} (MEASURED_PEAKS.json)"}
    dom = max(per_kernel, key=lambda k: per_kernel[k]["ms"])
    roof = dict(roofs[dom], kernel=dom)

    # the same kernels in a stand-alone preconditioner application
    # (pd_apply_precond: FP64 r in, FP64 z out, no residual): the FFT kernels
    # without the double-float residual of the solver
    zb = torch.empty_like(b)
    plan.profile_precond(b, zb, reps=2)
    pms = plan.profile_precond(b, zb, reps=5)
    hh = (pb.nt // 2 + 1) / pb.nt
    pbpu = {"fft_gamma_standalone": 8.0 + 8.0 * hh, "xform_fwd": 16.0 * hh, "tridiag": 16.0 * hh,
            "xform_inv": 16.0 * hh, "ifft_gamma_out64": 8.0 * hh + 8.0}
    precond_kernels = {}
    for name, t in zip(["fft_gamma_standalone", "xform_fwd", "tridiag", "xform_inv",
                        "ifft_gamma_out64"], pms):
        if t <= 0:
            continue
        gbs = pbpu[name] * NS / (t / 1e3) / 1e9
        precond_kernels[name] = {"ms": t, "GB/s": gbs, "frac_of_measured_hbm": gbs / hbm,
                                 "algorithmic_bytes": pbpu[name] * NS}

    # e2e through the C ABI with host buffers (copies inside the timed region)
    bh = b.cpu().pin_memory()
    uh = torch.zeros_like(bh).pin_memory()
    plan.solve_host(bh, uh, tol=TOL, maxit=40)
    ke = max(1, min(args.steps, 5))
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(ke):
        uh.zero_()
        plan.solve_host(bh, uh, tol=TOL, maxit=40)
    e2e_ms = (time.perf_counter() - t0) / ke * 1e3
    e2e_ms = max_over_ranks(ws, e2e_ms, dev)
    e2e = {"value": ws * NS / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": 2 * NS * 8,
           "d2h_bytes_per_step": NS * 8, "ms_per_step": e2e_ms}

    # plain FP64 GPU path at the same tolerance
    plan64 = pd.Plan(space, pb.nt, pb.dt, pb.alpha, pd.PD_CN, 0.5, pd.PD_FP64, stream)
    u64 = torch.zeros_like(b)
    plan64.solve(b, u64, tol=TOL, maxit=40)
    k64 = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(k64):
        u64.zero_()
        _, it64, rel64 = plan64.solve(b, u64, tol=TOL, maxit=40)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = max_over_ranks(ws, e0.elapsed_time(e1) / k64, dev)
    kms64 = plan64.profile_iteration(b, torch.zeros_like(b), reps=1)

    batched = None
    if not args.no_batch:
        batched = batched_leg(pd, torch, dev, args)
    pd1 = None
    if not args.no_pd1:
        pd1 = pd1_leg(pd, torch, dev, args)
    hybrid = None
    if not args.no_hybrid:
        hybrid = hybrid_leg(pd, torch, dev, args)
    nonlinear = None
    if not args.no_nonlinear:
        nonlinear = nonlinear_leg(pd, torch, dev, args)
    wave = None
    if not args.no_wave:
        wave = wave_leg(pd, torch, dev, args)
    control = None
    if not args.no_control:
        control = control_leg(pd, torch, dev, args)
    ade1d = adjoint = wave_gmres = None
    if not args.no_configs:
        ade1d = ade1d_leg(pd, torch, dev, args)
        adjoint = adjoint_leg(pd, torch, dev, args)
        wave_gmres = wave_gmres_leg(pd, torch, dev, args)

    err = err64 = None
    if rank == 0 and not args.no_check:
        from oracle import operators as O
        from oracle import stepping as S
        bref = O.build_rhs(pb, w.u0, None, None)
        uref = S.solve_sequential(pb, bref)
        un = u.cpu().numpy()
        err = float(np.linalg.norm(un - uref) / np.linalg.norm(uref))
        err64 = float(np.linalg.norm(u64.cpu().numpy() - uref) / np.linalg.norm(uref))

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_oracle_sample(w)

    if rank == 0:
        # the other configurations and legs first, the headline keys last (the
        # end of the line is what a truncated log keeps)
        out = {"batched": batched,
               "ade1d_be_127x64": ade1d,
               "heat2d_adjoint_127x127x128": adjoint,
               "wave1d_gmres_1023x1024": wave_gmres,
               "paradiag1": pd1,
               "paradiag1_hybrid": hybrid,
               "paradiag1_hybrid_wave": wave,
               "nonlinear_simplified_newton": nonlinear,
               "optimal_control_wave": control,
               "precond_kernel_roofline": precond_kernels,
               "kernel_roofline": roofs,
               "kernel_ms": {k: v["ms"] for k, v in per_kernel.items()},
               "solver": {"iterations": iters_all[-1], "relres": rel,
                          "cuda_graph": plan.uses_graph(),
                          "autotuned": dict(zip(("tile_columns", "tri_lanes", "tri_rows"),
                                                plan.get_tuning()),
                                            xform_engine={0: "tensor", 1: "fft", 2: "dense"}.get(
                                                plan.xform_engine, "none"))},
               "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32 preconditioner + df64 residual",
               "data": "synthetic (seeded Gaussian initial value, zero source)",
               "config": bench_config(w, args.small, ws),
               "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
               "fp64_path": {"value": ws * NS / (ms64 / 1e3), "ms_per_step": ms64,
                             "iterations": it64, "error_vs_oracle": err64,
                             "mixed_speedup": ms64 / ms,
                             "kernel_ms": dict(zip(KERNELS, kms64))},
               "roofline": roof,
               "gpu_launches": launches,
               "error_vs_oracle": err}
        print(json.dumps(out), flush=True)
    plan.close()
    plan64.close()


if __name__ == "__main__":
    main()
