#!/usr/bin/env python
"""Throughput of the swift left inverse x~ = Zh^- x on B300 (one JSON line).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

A step is one application of the left inverse to one batch of R right-hand
sides of the named workload (default: 256 x 256 periodic grid x 32 levels,
K = 64 members, L = 949 kept modes, R = 64 per batch, mixed precision), with
the inputs already resident in HBM.  The metric is right-hand-side vectors per
second (setup excluded; it is reported separately).  Under torchrun every rank
runs an independent replica on its own batch (the right-hand sides are
independent problems): weak scaling, no collective on the data path; the time
is the max over ranks.

--impl reference times the FP64 CPU oracle (the only other implementation of
this method) on the host cores, one right-hand side per step.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2609_13327_b300 import synth  # noqa: E402

DEFAULT_WORKLOAD = "c3_256x256x32"
BATCHED = "c4_batched"        # 200 uneven instances in one batch (synth.batched_instances)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(synth.WORKLOADS) + [BATCHED])
    ap.add_argument("--prec", default=None, choices=["fp64", "fp32", "mixed"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--op", choices=["left_inverse", "gradient"], default="left_inverse",
                    help="gradient: a step is the gradient of J = 1/2 ||Zh^- x||^2, i.e. the left inverse followed "
                         "by the adjoint (the 512x512x16 differentiation workload)")
    ap.add_argument("--partition", choices=["replicas", "slabs"], default="replicas",
                    help="replicas: every rank an independent batch (weak scaling); slabs: the ranks split the "
                         "grid rows of one batch and all-reduce the K L partial sums (strong scaling)")
    ap.add_argument("--fp64-steps", type=int, default=5,
                    help="timed steps of the plain FP64 GPU form of the same workload (0: skip)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(value, device):
    """Max of a per-rank float over the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def slab_rows(ny, world, rank):
    """Rows [y0, y1) of rank `rank` when `world` ranks split ny grid rows as evenly as possible."""
    base, extra = divmod(ny, world)
    y0 = rank * base + min(rank, extra)
    return y0, y0 + base + (1 if rank < extra else 0)


def aggregate_value(world, steps, R, seconds):
    """Whole-job vectors/s: every rank processed steps x R right-hand sides in at most `seconds`."""
    return world * steps * R / seconds


# ----------------------------------------------------------------------------- bytes and peaks

def element_sizes(prec):
    """(s_x, s_z): bytes per state/coefficient element and per ensemble element.

    The mixed-precision workload fixes the ensemble operand at 2 bytes (BF16 class)."""
    if prec == "fp64":
        return 8, 8
    if prec == "mixed":
        return 4, 2
    return 4, 4


def algorithmic_bytes_per_rhs(w, L, prec, R):
    """Read x once, write x~ once, read the ensemble once per batch of R."""
    sx, sz = element_sizes(prec)
    return sx * (w.n + w.K * L) + sz * w.n * w.K / R


# FP32 FMA peak from the unit counts: 148 SMs x 128 FP32 lanes x 2 flops per FMA x the
# 2032 MHz maximum SM clock (nominal; the CUDA-core kernels are bound by FMA issue)
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12


def column_flops_per_rhs(w, plan):
    """FMA-pipe flops of the FP32 column kernel per rhs: V1 (K x n_w per column) + x-pass (K x P_x per grid point)."""
    import numpy as np
    Px = len(np.unique(plan.modes() % w.Nx))
    return 2.0 * w.K * (w.nw * w.Nx * w.Ny + w.Ny * w.Nx * Px)


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def kernel_sources_sha(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, workload, prec):
    """DRAM bytes per launch from a committed ncu summary, if the kernel has not changed since."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            table = json.load(f)
    except Exception:
        return None
    for e in table:
        if e.get("kernel") == kernel and e.get("workload") == workload and e.get("prec") == prec:
            if e.get("sources_sha") == kernel_sources_sha(e.get("sources", [])):
                return e.get("dram_bytes_per_launch")
    return None


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.file = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "20"]
        if uuid:
            cmd.insert(1, f"--id={uuid}")
        try:
            self.proc = subprocess.Popen(cmd, stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.count(",") >= 8]
        self.file.close()
        os.unlink(self.file.name)
        return rows

    @staticmethod
    def summarize(rows, t_start, t_stop):
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- CPU oracle timing

def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info() if i.get("user_api") == "blas"]
        return max(n) if n else 1
    except Exception:
        return os.cpu_count() or 1


def oracle_plan(w, prec):
    from oracle import basis, swift
    Z = synth.ensemble(w).astype(synth.storage_dtype(prec)).astype(np.float64)
    lam = basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc)
    t0 = time.perf_counter()
    plan = swift.Plan(Z, w.Nx, w.Ny, lam, w.tau)
    return plan, time.perf_counter() - t0


def cpu_baseline(w, prec, x):
    """The oracle as it stands, on the host cores: setup untimed, then the right-hand sides x
    (a sample of the GPU's batch).  Returns the timing record and the oracle's output."""
    from oracle import swift
    plan, t_setup = oracle_plan(w, prec)
    nrhs = len(x)
    swift.apply_left_inverse(plan, x[:1])
    t0 = time.perf_counter()
    ref = swift.apply_left_inverse(plan, x)
    dt = time.perf_counter() - t0
    return {"value": nrhs / dt, "unit": "vectors/s", "cores": blas_threads(), "kind": "oracle",
            "sample": f"the first {nrhs} right-hand sides of the GPU batch of the full {w.name} workload through "
                      f"the FP64 NumPy oracle (setup {t_setup:.1f} s, excluded like the GPU setup)"}, ref


def run_reference(args, w, prec):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import swift
    plan, t_setup = oracle_plan(w, prec)
    L = plan.L
    x = synth.rhs(w, R=1, dtype=synth.storage_dtype(prec)).astype(np.float64)
    for _ in range(args.warmup):
        swift.apply_left_inverse(plan, x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        swift.apply_left_inverse(plan, x)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    cores = blas_threads()
    line = {
        "impl": "reference", "metric": "left-inverse applications/s", "value": value, "unit": "vectors/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(w, L, prec, 1),
        "cpu_baseline": {"value": value, "unit": "vectors/s", "cores": cores, "kind": "oracle",
                         "sample": f"one right-hand side of {w.name} per step (FP64 NumPy oracle, "
                                   f"setup {t_setup:.1f} s excluded)"},
        "e2e": {"value": value, "unit": "vectors/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm

def workload_config(w, L, prec, R):
    return {"workload": f"{w.name}: {w.Nx}x{w.Ny} periodic grid x {w.nw} levels, K={w.K} members, "
                        f"L={L} kept modes, {R} right-hand sides per step, {prec}",
            "nx": w.Nx, "ny": w.Ny, "nw": w.nw, "K": w.K, "L": L, "rhs_per_step": R, "prec": prec,
            "tau": w.tau, "ell_loc": w.ell_loc,
            "l2": "no flush: every step reads a different-order stream of x larger than the 126 MB L2"}


def run_ours(args, w, prec):
    import torch
    world, rank, local = dist_env()
    from paper_2609_13327_b300 import zl
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    R = w.R
    sdt = synth.storage_dtype(prec)

    Z = torch.from_numpy(synth.ensemble(w).astype(sdt)).to(dev)
    lam = zl.zl_gaussian_spectrum(w.Nx, w.Ny, w.ell_loc)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = zl.zl_setup(Z, lam, tau=w.tau, prec=prec, max_rhs=R, nx=w.Nx, ny=w.Ny)
    setup_s = time.perf_counter() - t0
    del Z
    x = torch.from_numpy(synth.rhs(w, R=R, seed=w.seed + 1000 * rank, dtype=sdt)).to(dev)
    out = torch.empty((R, w.K, plan.L), dtype=x.dtype, device=dev)
    stream = torch.cuda.current_stream()

    for _ in range(max(args.warmup, 3)):
        zl.zl_apply_left_inverse(plan, x, out, stream)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    time.sleep(0.3)
    barrier()
    plan.set_stage_timing(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_wall0 = time.time()
    ev0.record(stream)
    for _ in range(args.steps):
        zl.zl_apply_left_inverse(plan, x, out, stream)
    ev1.record(stream)
    barrier()
    t_wall1 = time.time()
    plan.set_stage_timing(False)
    rows = sampler.stop()
    ms = reduce_max(ev0.elapsed_time(ev1), dev)
    stages = plan.stage_times()
    launches = sum(n for n, _ in stages.values())
    value = aggregate_value(world, args.steps, R, ms / 1e3)

    # dominant kernel: the column/x-pass stage
    n_col, ms_col = stages["fwd_column"]
    avg_col_s = ms_col / max(n_col, 1) / 1e3
    bpr = algorithmic_bytes_per_rhs(w, plan.L, prec, R)
    peak, peak_kind = measured_peak_hbm()
    achieved = bpr * R / avg_col_s / 1e9
    if prec == "mixed" and plan_uses_tc(plan):
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": recorded_traffic("fwd_column_tc_kernel", w.name, prec), "kernel": "fwd_column_tc_kernel",
                    "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback"}
    elif prec in ("fp32", "mixed"):
        # the CUDA-core FP32 column kernel is bound by FMA issue: flops against the FP32 peak
        tflops = column_flops_per_rhs(w, plan) * R / avg_col_s / 1e12
        roofline = {"bound": "alu", "achieved": tflops, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": tflops / FP32_PEAK_TFLOPS, "traffic": recorded_traffic("fwd_column_f32_kernel", w.name, prec),
                    "kernel": "fwd_column_f32_kernel (or fwd_column_xpass where its tile does not apply)",
                    "peak_source": "148 SMs x 128 FP32 FMA lanes x 2 x 2032 MHz (nominal)",
                    "hbm_frac": achieved / peak}
    else:
        roofline = {"bound": "alu", "achieved": None, "peak": None, "unit": "TFLOP/s", "frac": None, "traffic": None,
                    "kernel": "fwd_column_xpass", "peak_source": "FP64 path: FP64 FMA bound, not measured against a peak",
                    "hbm_frac": achieved / peak}
    roofline.update({"kernel_ms_per_launch": avg_col_s * 1e3,
                     "step_frac": bpr * R / (ms / args.steps / 1e3) / 1e9 / peak,
                     "stages_ms_per_launch": {k: (v[1] / v[0] if v[0] else None) for k, v in stages.items()}})

    # end to end through the host-buffer entry point: H2D of x and D2H of x~ inside every step
    xh = x.cpu().pin_memory()
    oh = torch.empty((R, w.K, plan.L), dtype=x.dtype).pin_memory()
    zl.zl_apply_left_inverse_host(plan, xh, oh, stream)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        zl.zl_apply_left_inverse_host(plan, xh, oh, stream)
    barrier()
    e2e_s = reduce_max(time.perf_counter() - t0, dev)
    e2e = {"value": aggregate_value(world, args.e2e_steps, R, e2e_s), "unit": "vectors/s",
           "h2d_bytes_per_step": xh.numel() * xh.element_size(), "d2h_bytes_per_step": oh.numel() * oh.element_size(),
           "steps": args.e2e_steps, "api": "zl_apply_left_inverse_host (pinned host buffers)"}

    # the host link alone: one pinned host -> device copy of a step's x (cudaMemcpyAsync), events
    xd = torch.empty_like(x)
    link_s = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        xd.copy_(xh, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        link_s.append(e0.elapsed_time(e1) / 1e3)
    del xd
    link_gbs = e2e["h2d_bytes_per_step"] / min(link_s) / 1e9
    e2e["link_h2d_gbs"] = link_gbs
    e2e["h2d_gbs_achieved"] = e2e["h2d_bytes_per_step"] * e2e["value"] / R / 1e9
    e2e["frac_of_link"] = e2e["h2d_gbs_achieved"] / link_gbs

    clocks = ClockSampler.summarize(rows, t_wall0, t_wall1)
    vs_fp64 = None
    if prec != "fp64" and args.fp64_steps > 0:
        vs_fp64 = fp64_gpu_form(w, R, rank, dev, args.fp64_steps, stream)
        vs_fp64["ratio"] = value / world / vs_fp64["value"]
    line = {
        "metric": "left-inverse applications/s", "value": value, "unit": "vectors/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "vs_fp64_gpu": vs_fp64,
        "dtype": "f16x3 split, f32 accumulate" if (prec == "mixed" and plan_uses_tc(plan)) else
                 ("f64" if prec == "fp64" else "f32"),
        "data": "synthetic (seeded Gaussian-correlated ensemble, N(0,1) right-hand sides)",
        "config": workload_config(w, plan.L, prec, R), "setup_s": setup_s,
        "roofline": roofline, "clocks": clocks, "e2e": e2e, "gpu_launches": launches,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on the first right-hand sides of this batch: a CPU timing and the GPU's accuracy
        nchk = min(8, R)
        xs = x[:nchk].cpu().numpy().astype(np.float64)
        got = out[:nchk].cpu().numpy().astype(np.float64).reshape(nchk, -1)
        line["cpu_baseline"], ref = cpu_baseline(w, prec, xs)
        ref = ref.reshape(nchk, -1)
        err = float(np.max(np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)))
        line["accuracy"] = {"max_rel_err_vs_fp64_oracle": err, "rhs_checked": nchk,
                            "norm": "per right-hand side ||out - ref||_2 / ||ref||_2",
                            "tolerance": {"mixed": 1e-5, "fp32": 1e-6, "fp64": 1e-10}[prec]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.destroy()
    if world > 1:
        torch.distributed.destroy_process_group()


def fp64_gpu_form(w, R, rank, dev, steps, stream):
    """The plain FP64 GPU form of the same algorithm (ZL_FP64 plan, CUDA-core kernels) on the
    same workload and right-hand sides, timed with CUDA events: the speedup denominator."""
    import torch
    from paper_2609_13327_b300 import zl
    Z = torch.from_numpy(synth.ensemble(w)).to(dev)
    lam = zl.zl_gaussian_spectrum(w.Nx, w.Ny, w.ell_loc)
    plan = zl.zl_setup(Z, lam, tau=w.tau, prec="fp64", max_rhs=R, nx=w.Nx, ny=w.Ny)
    del Z
    x = torch.from_numpy(synth.rhs(w, R=R, seed=w.seed + 1000 * rank, dtype=np.float64)).to(dev)
    out = torch.empty((R, w.K, plan.L), dtype=torch.float64, device=dev)
    for _ in range(2):
        zl.zl_apply_left_inverse(plan, x, out, stream)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        zl.zl_apply_left_inverse(plan, x, out, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    plan.destroy()
    del x, out
    torch.cuda.empty_cache()
    return {"value": R / (ms / 1e3), "unit": "vectors/s", "ms_per_step": ms, "steps": steps,
            "what": "ZL_FP64 plan (FP64 CUDA-core kernels) on the same workload, this GPU; ratio = value / this"}


def run_slabs(args, w, prec):
    """The y-slab partition of the paper's parallel decomposition: rank r holds grid rows
    slab_rows(ny, N, r) of the ensemble's and the right-hand sides' segments, computes its
    unscaled partial sums (zl_apply_left_inverse_rows), the ranks add them with one NCCL
    all-reduce of K L values per right-hand side, and every rank scales the sum
    (zl_scale_modes).  A step is one batch of R right-hand sides through all of it."""
    import torch
    world, rank, local = dist_env()
    from paper_2609_13327_b300 import zl
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    R = w.R
    sdt = synth.storage_dtype(prec)
    y0, y1 = slab_rows(w.Ny, world, rank)
    Z = torch.from_numpy(synth.ensemble(w).astype(sdt)).to(dev)
    lam = zl.zl_gaussian_spectrum(w.Nx, w.Ny, w.ell_loc)
    t0 = time.perf_counter()
    plan = zl.zl_setup(Z, lam, tau=w.tau, prec=prec, max_rhs=R, nx=w.Nx, ny=w.Ny)
    setup_s = time.perf_counter() - t0
    del Z
    x = synth.rhs(w, R=R, dtype=sdt)
    xs = torch.from_numpy(np.ascontiguousarray(x[:, :, y0 * w.Nx:y1 * w.Nx])).to(dev)
    part = torch.empty((R, w.K, plan.L), dtype=xs.dtype, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        if y1 > y0:
            zl.zl_apply_left_inverse_rows(plan, y0, y1, xs, part, stream)
        else:                                   # more ranks than grid rows: this one adds nothing
            part.zero_()
        if dist is not None:
            dist.all_reduce(part)
        zl.zl_scale_modes(plan, part, part, stream)

    for _ in range(max(args.warmup, 3)):
        step()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ms = reduce_max(ev0.elapsed_time(ev1), dev)
    value = args.steps * R / (ms / 1e3)
    line = {"metric": "left-inverse applications/s", "value": value, "unit": "vectors/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None,
            "dtype": "f16x3 split, f32 accumulate" if prec == "mixed" else ("f64" if prec == "fp64" else "f32"),
            "data": "synthetic (seeded Gaussian-correlated ensemble, N(0,1) right-hand sides)",
            "config": dict(workload_config(w, plan.L, prec, R), partition=f"{world} y-slabs, one all-reduce of "
                                                                        f"K L values per right-hand side"),
            "setup_s": setup_s, "gpu_launches": None}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import compare
        _, ref = cpu_baseline(w, prec, x[:2].astype(np.float64))
        line["accuracy"] = {"max_rel_err_vs_fp64_oracle": compare.measures(part[:2].cpu().numpy(), ref, 2)[0],
                            "rhs_checked": 2}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.destroy()
    if dist is not None:
        dist.destroy_process_group()


def run_gradient(args, w, prec):
    """Gradient of J(x) = 1/2 ||Zh^- x||^2 for a batch of R right-hand sides: x~ = Zh^- x
    (left inverse) then g = (Zh^-)^T x~ (adjoint kernels); replicas under torchrun."""
    import torch
    world, rank, local = dist_env()
    from paper_2609_13327_b300 import zl
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    R = w.R
    sdt = synth.storage_dtype(prec)
    Z = torch.from_numpy(synth.ensemble(w).astype(sdt)).to(dev)
    lam = zl.zl_gaussian_spectrum(w.Nx, w.Ny, w.ell_loc)
    t0 = time.perf_counter()
    plan = zl.zl_setup(Z, lam, tau=w.tau, prec=prec, max_rhs=R, nx=w.Nx, ny=w.Ny)
    setup_s = time.perf_counter() - t0
    del Z
    x = torch.from_numpy(synth.rhs(w, R=R, seed=w.seed + 1000 * rank, dtype=sdt)).to(dev)
    xt = torch.empty((R, w.K, plan.L), dtype=x.dtype, device=dev)
    g = torch.empty_like(x)
    stream = torch.cuda.current_stream()

    def step():
        zl.zl_apply_left_inverse(plan, x, xt, stream)
        zl.zl_apply_adjoint(plan, xt, g, stream)

    for _ in range(max(args.warmup, 3)):
        step()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    plan.set_stage_timing(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    plan.set_stage_timing(False)
    ms = reduce_max(ev0.elapsed_time(ev1), dev)
    stages = plan.stage_times()
    value = aggregate_value(world, args.steps, R, ms / 1e3)
    sx, sz = element_sizes(prec)
    # read x, write x~, read x~, write g; the ensemble operand once per batch in each direction
    bpr = sx * (2 * w.n + 2 * w.K * plan.L) + 2 * sz * w.n * w.K / R
    peak, peak_kind = measured_peak_hbm()
    line = {"metric": "gradient applications/s", "value": value, "unit": "vectors/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "fp64" else ("f16x3 split, f32 accumulate (left inverse)" if plan_uses_tc(plan) else "f32"),
            "data": "synthetic (seeded Gaussian-correlated ensemble, N(0,1) right-hand sides)",
            "config": dict(workload_config(w, plan.L, prec, R), op="gradient of 1/2 ||Zh^- x||^2 (left inverse + adjoint)"),
            "setup_s": setup_s,
            "roofline": {"bound": "hbm", "step_frac": bpr * R / (ms / args.steps / 1e3) / 1e9 / peak, "peak": peak,
                         "unit": "GB/s", "peak_source": peak_kind,
                         "stages_ms_per_launch": {k: (v[1] / v[0] if v[0] else None) for k, v in stages.items()}},
            "gpu_launches": sum(n for n, _ in stages.values())}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import compare, swift
        plan_o, _ = oracle_plan(w, prec)
        xs = x[:2].cpu().numpy().astype(np.float64)
        ref = swift.apply_adjoint(plan_o, swift.apply_left_inverse(plan_o, xs))
        line["accuracy"] = {"max_rel_err_vs_fp64_oracle": compare.measures(g[:2].cpu().numpy(), ref, 1)[0],
                            "rhs_checked": 2}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.destroy()
    if world > 1:
        torch.distributed.destroy_process_group()


def plan_uses_tc(plan):
    return getattr(plan, "uses_tc", lambda: False)()


def batched_config(ws, prec):
    return {"workload": f"{BATCHED}: {len(ws)} independent instances, square periodic grids of side 32-192, "
                        f"4-24 levels, K 16-64, 1-32 right-hand sides each ({sum(w.R for w in ws)} per step), {prec}",
            "instances": len(ws), "rhs_per_step": sum(w.R for w in ws), "prec": prec,
            "l2": "no flush: one step streams every instance's x and ensemble operand (several GB) through L2"}


def run_batched(args, prec):
    """The batched workload: one apply of all instances per step (one CUDA graph launch)."""
    import torch
    world, rank, local = dist_env()
    from paper_2609_13327_b300 import zl
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    ws = synth.batched_instances()
    sdt = synth.storage_dtype(prec)
    # an instance whose draw has a rank-deficient column (the library reports ZL_ERR_RANK and
    # which instance) gets a new ensemble draw; the redraws are counted in the JSON line.
    # setup_s times the library's setup only (not the host's synthetic draws).
    redrawn = {}
    ens = {}
    while True:
        for i, w in enumerate(ws):
            key = (i, redrawn.get(i, 0))
            if key not in ens:
                ens[key] = synth.ensemble(w, seed=w.seed + 1000003 * redrawn.get(i, 0)).astype(sdt)
        insts = [{"Z": torch.from_numpy(ens[(i, redrawn.get(i, 0))]).to(dev),
                  "spectrum": zl.zl_gaussian_spectrum(w.Nx, w.Ny, w.ell_loc), "nx": w.Nx, "ny": w.Ny, "prec": prec,
                  "tau": w.tau, "max_rhs": w.R} for i, w in enumerate(ws)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            batch = zl.zl_setup_batch(insts)
            torch.cuda.synchronize()
            setup_s = time.perf_counter() - t0
            break
        except zl.ZLError as err:
            if err.code != zl.ZL_ERR_RANK or err.failed_instance < 0 or redrawn.get(err.failed_instance, 0) >= 3:
                raise
            redrawn[err.failed_instance] = redrawn.get(err.failed_instance, 0) + 1
    del insts
    xs = [torch.from_numpy(synth.rhs(w, seed=w.seed + 1000 * rank, dtype=sdt)).to(dev) for w in ws]
    outs = [torch.empty((x.shape[0], p.K, p.L), dtype=x.dtype, device=dev) for x, p in zip(xs, batch.plans)]
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        batch.apply_left_inverse(xs, outs, stream)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    time.sleep(0.3)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_wall0 = time.time()
    ev0.record(stream)
    for _ in range(args.steps):
        batch.apply_left_inverse(xs, outs, stream)
    ev1.record(stream)
    barrier()
    t_wall1 = time.time()
    rows = sampler.stop()
    ms = reduce_max(ev0.elapsed_time(ev1), dev)
    rhs = sum(w.R for w in ws)
    value = aggregate_value(world, args.steps, rhs, ms / 1e3)
    peak, peak_kind = measured_peak_hbm()
    step_bytes = sum(algorithmic_bytes_per_rhs(w, p.L, prec, w.R) * w.R for w, p in zip(ws, batch.plans))
    achieved = step_bytes / (ms / args.steps / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": "one graph launch of all instances (per-kernel timing is not available "
                                             "inside a graph)",
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
                "variants": {str(v): batch.variants.count(v) for v in sorted(set(batch.variants))},
                "tensor_core_instances": sum(1 for p in batch.plans if p.uses_tc())}
    # end to end: H2D of every instance's x and D2H of every x~ inside the timed loop
    xh = [x.cpu().pin_memory() for x in xs]
    oh = [torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in outs]
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        for a, b in zip(xs, xh):
            a.copy_(b, non_blocking=True)
        batch.apply_left_inverse(xs, outs, stream)
        for a, b in zip(oh, outs):
            a.copy_(b, non_blocking=True)
    barrier()
    e2e_s = reduce_max(time.perf_counter() - t0, dev)
    e2e = {"value": aggregate_value(world, args.e2e_steps, rhs, e2e_s), "unit": "vectors/s",
           "h2d_bytes_per_step": sum(x.numel() * x.element_size() for x in xh),
           "d2h_bytes_per_step": sum(o.numel() * o.element_size() for o in oh), "steps": args.e2e_steps,
           "api": "zl_apply_left_inverse_batch with pinned host copies of every instance"}
    clocks = ClockSampler.summarize(rows, t_wall0, t_wall1)
    line = {
        "metric": "left-inverse applications/s", "value": value, "unit": "vectors/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16x3 split, f32 accumulate (per-instance autotuned)",
        "data": "synthetic (seeded Gaussian-correlated ensembles, N(0,1) right-hand sides)",
        "config": dict(batched_config(ws, prec), redrawn_rank_deficient=sorted(redrawn)), "setup_s": setup_s,
        "roofline": roofline, "clocks": clocks, "e2e": e2e,
        # every instance's apply is two kernels (column pass, y-pass) per pass of max_rhs right-hand sides
        "gpu_launches": args.steps * sum(2 * ((w.R + w.R - 1) // w.R) for w in ws),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on three instances of the batch (all their right-hand sides)
        from oracle import basis, swift
        errs, t_or, n_or = [], 0.0, 0
        for i in (0, 1, 2):
            w = ws[i]
            Zo = synth.ensemble(w, seed=w.seed + 1000003 * redrawn.get(i, 0)).astype(sdt).astype(np.float64)
            op = swift.Plan(Zo, w.Nx, w.Ny, basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc), w.tau)
            xo = xs[i].cpu().numpy().astype(np.float64)
            ta = time.perf_counter()
            ref = swift.apply_left_inverse(op, xo)
            t_or += time.perf_counter() - ta
            n_or += len(xo)
            got = outs[i].cpu().numpy().astype(np.float64)
            errs.append(float(np.max(np.linalg.norm((got - ref).reshape(len(xo), -1), axis=1) /
                                     np.linalg.norm(ref.reshape(len(xo), -1), axis=1))))
        line["cpu_baseline"] = {"value": n_or / t_or, "unit": "vectors/s", "cores": blas_threads(), "kind": "oracle",
                                "sample": f"all right-hand sides of instances 0-2 of the batch ({n_or} vectors) "
                                          f"through the FP64 NumPy oracle, setup excluded"}
        line["accuracy"] = {"max_rel_err_vs_fp64_oracle": max(errs), "rhs_checked": n_or,
                            "norm": "per right-hand side ||out - ref||_2 / ||ref||_2, instances 0-2",
                            "tolerance": {"mixed": 1e-5, "fp32": 1e-6, "fp64": 1e-10}[prec]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    batch.destroy()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_reference_batched(args, prec):
    """The oracle on the batched workload: each step applies one right-hand side to each of
    the first three instances (a bounded sample of one batch step)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import basis, swift
    ws = synth.batched_instances()[:3]
    plans = [swift.Plan(synth.ensemble(w).astype(synth.storage_dtype(prec)).astype(np.float64), w.Nx, w.Ny,
                        basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc), w.tau) for w in ws]
    xs = [synth.rhs(w, R=1, dtype=synth.storage_dtype(prec)).astype(np.float64) for w in ws]
    for _ in range(args.warmup):
        for p, x in zip(plans, xs):
            swift.apply_left_inverse(p, x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for p, x in zip(plans, xs):
            swift.apply_left_inverse(p, x)
    dt = time.perf_counter() - t0
    value = len(ws) * args.steps / dt
    line = {
        "impl": "reference", "metric": "left-inverse applications/s", "value": value, "unit": "vectors/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": batched_config(synth.batched_instances(), prec),
        "cpu_baseline": {"value": value, "unit": "vectors/s", "cores": blas_threads(), "kind": "oracle",
                         "sample": "one right-hand side of each of instances 0-2 per step (FP64 NumPy oracle)"},
        "e2e": {"value": value, "unit": "vectors/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.workload == BATCHED:
        prec = args.prec or "mixed"
        if args.impl == "reference":
            run_reference_batched(args, prec)
        else:
            run_batched(args, prec)
        return
    w = synth.WORKLOADS[args.workload]
    prec = args.prec or w.prec
    if args.impl == "reference":
        run_reference(args, w, prec)
    elif args.partition == "slabs":
        run_slabs(args, w, prec)
    elif args.op == "gradient":
        run_gradient(args, w, prec)
    else:
        run_ours(args, w, prec)


if __name__ == "__main__":
    main()
