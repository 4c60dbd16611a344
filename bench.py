"""Benchmark of the 3-D FFT hot path on GB300: one JSON line on rank 0.

Workload (one "step"): the r2c forward transform and the c2r backward
transform of one 512^3 float32 random-mode field (64 Fourier modes with
|k| <= n/4 plus 1e-3 Gaussian noise), i.e. every stage of the pencil
algorithm in both directions.  Inputs are larger than L2 (537 MB vs 129 MB),
so no explicit flush is needed between steps.

value = whole-job algorithmic bytes per second as a percentage of one GB300's
measured HBM bandwidth (MEASURED_PEAKS.json), the algorithmic bytes being
the 3-pass minimum: one full-array read and write per axis stage.  At N > 1
GPUs the one 512^3 transform is distributed in slabs of 512/N planes (the
paper's slab decomposition, Algorithm 3: N2 and N1 stages per rank, one NCCL
all-to-all, the N0 stage), so the total work is fixed (strong scaling);
`--decomp replicas` instead runs an independent transform per GPU (weak
scaling), and `--decomp slab` runs the slab path even on one GPU.

The default line also carries, under "also", the metric's other
configurations measured in the same run: r2c 512^3 FP64, c2c 512^3 FP32/FP64,
c2c 1024^3 FP32/FP64/split precision, the fused Poisson solve, the 200-field
batched uneven workload (solves/s) and the serving workload (solves/s, p50/p99
at 200 and 700 requests/s and at saturation), plus cuFFT on the same shapes as
a reference baseline.  `--no-extra` leaves them out.

`cpu_baseline` times the CPU oracle on the host cores on the same 512^3 field:
the FP32 build of its source for this FP32 workload (the FP64 build and
single-threaded numpy.fft beside it).  `--impl reference` times that FP32
oracle build alone, one whole 512^3 r2c + c2r per step (the only other place
this script runs oracle code), reported in the same unit.
"""
from __future__ import annotations

import argparse
import math
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3-D FFT %HBM roofline at 512^3/1024^3 FP32/FP64; batched solves/s & p99"
UNIT = "% of one GB300's measured HBM bandwidth (3-pass algorithmic bytes), summed over GPUs"
FALLBACK_HBM_GBS = 6800.0
SHAPE = (512, 512, 512)
WORKLOAD = ("r2c forward + c2r backward, 512x512x512 %s random-mode field (64 modes, |k|<=n/4, "
            "+1e-3 noise)")
STAGE_NAMES_FWD = ["r2c z-stage (N2)", "strided y-stage (N1)", "strided x-stage (N0)"]
STAGE_NAMES_BWD = ["strided x-stage (N0)", "strided y-stage (N1)", "c2r z-stage (N2)"]


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def workload_bytes(shape, real_bytes, cplx_bytes):
    """3-pass algorithmic bytes of r2c forward (and, mirrored, c2r backward), per stage."""
    n0, n1, n2 = shape
    N = n0 * n1 * n2
    Nh = n0 * n1 * (n2 // 2 + 1)
    z = N * real_bytes + Nh * cplx_bytes
    y = 2 * Nh * cplx_bytes
    x = 2 * Nh * cplx_bytes
    return z, y, x


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1506_07933_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")) and f != "noalloc.cu":
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on these sources."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    src = source_hash()
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        kv = dict(tok.split("=", 1) for tok in line.split() if "=" in tok)
        if kv.get("kernel") == kernel and kv.get("workload") == workload and kv.get("src") == src:
            return int(kv["dram_bytes_per_launch"])
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms; summary() keeps the samples
    taken inside [t0, t1] (host wall-clock seconds), the timed region."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.5)   # let nvidia-smi start before the timed region
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self, t0=None, t1=None):
        import datetime
        sm, mx, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = None
            if t0 is not None and ts is not None and not (t0 - 0.05 <= ts <= t1 + 0.05):
                continue
            try:
                sm.append(float(f[2]))
                mx = float(f[3])
                power.append(float(f[4]))
            except ValueError:
                continue
            for name, v in zip(names, f[6:10]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# ------------------------------------------------------------------ CPU leg --

def cpu_field(shape=SHAPE):
    """The benchmark's FP32 random-mode field (mode seed 5121), as the GPU arm's rank 0 uses."""
    import numpy as np
    from paper_1506_07933_gb300 import synth
    return synth.random_mode_field(shape, 5121, n_modes=64, noise=1e-3).astype(np.float32)


def cpu_step_seconds(field, engine, threads=None):
    """Seconds of one r2c + c2r of `field` on the CPU: engine "oracle_f32" (the oracle's source
    built with FP32 arithmetic, all threads), "oracle_f64" (the FP64 oracle) or "numpy"
    (numpy.fft.rfftn / irfftn, pocketfft, one thread)."""
    import numpy as np
    import oracle
    n2 = field.shape[2]
    t0 = time.perf_counter()
    if engine == "oracle_f32":
        oracle.c2r_f32(oracle.r2c_f32(field, threads), n2, threads)
    elif engine == "oracle_f64":
        oracle.c2r(oracle.r2c(field, "fft", threads), n2, "fft", threads)
    else:
        np.fft.irfftn(np.fft.rfftn(field, axes=(0, 1, 2)), s=field.shape, axes=(0, 1, 2))
    return time.perf_counter() - t0


def cpu_baseline_block(step_bytes, peak):
    """The CPU baseline of the GPU arm: the oracle timed on the host cores on the same 512^3
    field (the FP32 build: one untimed and one timed step), with the FP64 oracle and
    single-threaded numpy.fft timed once each beside it."""
    import oracle
    field = cpu_field()
    threads = oracle.max_threads()
    cpu_step_seconds(field, "oracle_f32", threads)
    t32 = cpu_step_seconds(field, "oracle_f32", threads)
    t64 = cpu_step_seconds(field, "oracle_f64", threads)
    tnp = cpu_step_seconds(field, "numpy")
    pct = lambda t: 100.0 * step_bytes / t / 1e9 / peak
    return {"value": pct(t32), "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "one whole r2c + c2r of the same 512^3 float32 field per step, the oracle's "
                      "recursive mixed-radix source built with FP32 arithmetic, %d threads (1 untimed + "
                      "1 timed step)" % threads,
            "ms_per_step": t32 * 1e3,
            "oracle_fp64": {"value": pct(t64), "ms_per_step": t64 * 1e3, "cores": threads},
            "numpy_fft_single_thread": {"value": pct(tnp), "ms_per_step": tnp * 1e3, "cores": 1}}


def run_reference(args):
    """The reference arm: the oracle (FP32 build of its source) on the host cores, one whole
    r2c + c2r of the 512^3 float32 field per step; rank 0 alone under torchrun."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    peak, _ = peaks()
    field = cpu_field()
    threads = oracle.max_threads()
    for _ in range(args.warmup):
        cpu_step_seconds(field, "oracle_f32", threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cpu_step_seconds(field, "oracle_f32", threads)
    t = (time.perf_counter() - t0) / args.steps
    step_bytes = 2 * sum(workload_bytes(SHAPE, 4, 8))
    value = 100.0 * step_bytes / t / 1e9 / peak
    sample = ("one whole r2c + c2r of the 512^3 float32 field per step, the oracle's recursive "
              "mixed-radix source built with FP32 arithmetic, %d threads" % threads)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": gpu_config(step_bytes, 1, (SHAPE[0] * SHAPE[1] * SHAPE[2] * 4) >> 20),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def gpu_config(step_bytes, world, input_mb):
    """The line's `config`, the same for both arms."""
    return {"workload": WORKLOAD % "float32",
            "l2": "inputs larger than L2 (%d MB > 129 MB), no flush" % input_mb,
            "bytes_per_step": step_bytes, "parallelism": "replicas x%d" % world}


# ------------------------------------------------------------- replicas -----
# With `--decomp replicas` every rank transforms its own field, so the step time is the
# slowest rank's and the value adds up over ranks (the default at N > 1 is the slab
# decomposition, one transform over all ranks: see run_slab).

def max_over_ranks(value, world, dist, device):
    """The largest of every rank's `value` (world == 1: the value itself)."""
    if world <= 1:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_percent(step_bytes_per_rank, world, ms, peak):
    """The metric: every rank's algorithmic bytes per step over the slowest rank's step time,
    as a percentage of one GPU's measured HBM bandwidth."""
    return 100.0 * world * step_bytes_per_rank / (ms * 1e-3) / 1e9 / peak


# ------------------------------------------------------------------ GPU leg --

def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1506_07933_gb300 import afft, synth
    from paper_1506_07933_gb300 import build as libbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    decomp = args.decomp or ("slab" if world > 1 else "plan")
    if world > 1 or decomp == "slab":
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29517")
        os.environ.setdefault("RANK", str(rank))
        os.environ.setdefault("WORLD_SIZE", str(world))
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    if rank == 0:
        libbuild.build()
    if dist.is_initialized():
        dist.barrier()
    afft.load()
    if decomp == "slab":
        return run_slab(args, world, rank, local)

    def barrier():
        if dist.is_initialized():
            dist.barrier()
        torch.cuda.synchronize()

    peak, peak_kind = peaks()
    prec = args.precision
    real_b, cplx_b = (4, 8) if prec == "f32" else (8, 16)
    rdt = np.float32 if prec == "f32" else np.float64
    plan = afft.Plan(SHAPE, "r2c", prec)
    field = synth.random_mode_field(SHAPE, 5121 + rank, n_modes=64, noise=1e-3).astype(rdt)
    x = torch.from_numpy(field).cuda()
    X = torch.empty(plan.spectral_shape, dtype=plan.spectral_dtype, device="cuda")
    y = torch.empty(plan.spatial_shape, dtype=plan.spatial_dtype, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        plan.forward(x, X)
        plan.backward(X, y)

    for _ in range(args.warmup):
        step()
    barrier()
    plan.timing_begin(2 * args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        t_begin = time.time()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        barrier()
        t_end = time.time()
    ms = e0.elapsed_time(e1) / args.steps
    stage = plan.timing_end()
    # accuracy of the last timed step (outside the timed region): backward(forward(x)) against x
    xd = x.double()
    round_trip = float(torch.linalg.vector_norm(y.double() - xd) / torch.linalg.vector_norm(xd))
    ms = max_over_ranks(ms, world, dist, "cuda")
    z, yb, xb = workload_bytes(SHAPE, real_b, cplx_b)
    step_bytes = 2 * (z + yb + xb)
    value = whole_job_percent(step_bytes, world, ms, peak)

    # dominant kernel from the per-stage events of the timed region
    fwd = [r for i, r in enumerate(stage) if i % 2 == 0]
    bwd = [r for i, r in enumerate(stage) if i % 2 == 1]
    desc = plan.describe()
    kernels = []
    for rows, names, knames, sbytes in ((fwd, STAGE_NAMES_FWD, desc["stage_kernels_forward"], (z, yb, xb)),
                                        (bwd, STAGE_NAMES_BWD, desc["stage_kernels_backward"], (xb, yb, z))):
        for s in range(3):
            ts = [r[s] for r in rows]
            kernels.append({"stage": names[s] + (" fwd" if rows is fwd else " bwd"), "kernel": knames[s],
                            "mean_ms": sum(ts) / len(ts), "bytes": sbytes[s],
                            "gbs": sbytes[s] / (sum(ts) / len(ts) * 1e-3) / 1e9})
    total_stage_ms = sum(k["mean_ms"] for k in kernels)
    dom = max(kernels, key=lambda k: k["mean_ms"])
    workload_tag = "512c_r2c_%s" % prec
    traffic = profiled_traffic(dom["stage"].replace(" ", "_"), workload_tag)
    roofline = {"bound": "hbm", "achieved": dom["gbs"], "peak": peak, "unit": "GB/s",
                "frac": dom["gbs"] / peak, "traffic": traffic, "kernel": dom["kernel"],
                "stage": dom["stage"], "peak_source": peak_kind,
                "bytes_per_launch": dom["bytes"], "mean_launch_ms": dom["mean_ms"]}

    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(args, plan, field, x, X, y, stream, barrier, world, step_bytes, peak, torch, dist)
    launches = args.steps * (plan.launches(False) + plan.launches(True))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": prec, "data": "synthetic",
        "config": gpu_config(step_bytes, world, plan.input_bytes >> 20),
        "roofline": roofline,
        "stages": [{k: (round(v, 5) if isinstance(v, float) else v) for k, v in kk.items()} for kk in kernels],
        "stage_ms_total": total_stage_ms,
        "round_trip_rel_l2": round_trip,
        # r2c + c2r of the field counted as 2 x 2.5 N log2 N flops, all GPUs
        "gflops": world * 5.0 * math.prod(SHAPE) * math.log2(math.prod(SHAPE)) / (ms * 1e-3) / 1e9,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk.summary(t_begin, t_end),
    }
    del x, X, y
    plan.close()
    torch.cuda.empty_cache()

    if not args.no_extra and rank == 0:
        t_extra = time.time()
        line["also"] = {"roofline_configs": extra_configs(afft, torch, peak),
                        "batched": batched_workload(afft, torch),
                        "serving": serving_workload(torch),
                        "cufft_reference": cufft_reference(torch, peak)}
        line["also"]["seconds"] = round(time.time() - t_extra, 1)
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline_block(step_bytes, peak)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist.is_initialized():
        dist.barrier()
        dist.destroy_process_group()


def run_slab(args, world, rank, local):
    """The 512^3 r2c + c2r step distributed in slabs over the ranks (Algorithm 3): rank r holds
    planes r 512/N ...; forward = N2 and N1 stages, NCCL all-to-all, N0 stage (its output block
    is all k0, rows r 512/N ..., all k2); backward the reverse.  Strong scaling: the whole job is
    one transform."""
    import torch
    import torch.distributed as dist
    from paper_1506_07933_gb300 import slab

    peak, peak_kind = peaks()
    prec = args.precision
    real_b, cplx_b = (4, 8) if prec == "f32" else (8, 16)
    f = slab.SlabFFT(SHAPE, "r2c", prec)
    field = cpu_field() if prec == "f32" else cpu_field().astype("float64")
    mine = field[rank * f.n0p:(rank + 1) * f.n0p]
    x = torch.from_numpy(mine.copy()).cuda()
    stream = torch.cuda.current_stream()

    def step():
        return f.backward(f.forward(x))

    def barrier():
        dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    zy, xp = f.engine.zy, f.engine.x
    zy.timing_begin(2 * args.steps)
    xp.timing_begin(2 * args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        t_begin = time.time()
        e0.record(stream)
        for _ in range(args.steps):
            y = step()
        e1.record(stream)
        barrier()
        t_end = time.time()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dist, "cuda")
    # this rank's stage kernels: records alternate forward / backward; zy slots (N2, N1, -) forward
    # and (-, N1, N2) backward, x slots (-, -, N0) forward and (N0, -, -) backward
    tz, tx = zy.timing_end(), xp.timing_end()
    nh = SHAPE[2] // 2 + 1
    local_planes = f.n0p * SHAPE[1]
    b_z = local_planes * (SHAPE[2] * real_b + nh * cplx_b)
    b_y = 2 * local_planes * nh * cplx_b
    b_x = 2 * SHAPE[0] * f.n1p * nh * cplx_b
    dz, dx = zy.describe(), xp.describe()
    cand = []
    for i, r in enumerate(tz):
        fw = i % 2 == 0
        cand.append(("N2 " + ("fwd" if fw else "bwd"), dz["stage_kernels_forward" if fw else "stage_kernels_backward"][0 if fw else 2],
                     r[0] if fw else r[2], b_z))
        cand.append(("N1 " + ("fwd" if fw else "bwd"), dz["stage_kernels_forward"][1], r[1], b_y))
    for i, r in enumerate(tx):
        fw = i % 2 == 0
        cand.append(("N0 " + ("fwd" if fw else "bwd"), dx["stage_kernels_forward"][2], r[2] if fw else r[0], b_x))
    stages = {}
    for name, kern, t, b in cand:
        stages.setdefault((name, kern, b), []).append(t)
    means = [(sum(v) / len(v), name, kern, b) for (name, kern, b), v in stages.items()]
    t_dom, name_dom, kern_dom, b_dom = max(means)
    roofline = {"bound": "hbm", "achieved": b_dom / (t_dom * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                "frac": b_dom / (t_dom * 1e-3) / 1e9 / peak, "traffic": None, "kernel": kern_dom,
                "stage": name_dom + " (rank 0's slab)", "peak_source": peak_kind, "bytes_per_launch": b_dom,
                "mean_launch_ms": t_dom}
    xd = x.double()
    round_trip = float(torch.linalg.vector_norm(y.double() - xd) / torch.linalg.vector_norm(xd))
    step_bytes = 2 * sum(workload_bytes(SHAPE, real_b, cplx_b))
    value = whole_job_percent(step_bytes, 1, ms, peak)
    # end to end: each rank uploads its slab from pinned memory and reads its result back
    hx = torch.from_numpy(mine.copy()).pin_memory()
    hy = torch.empty_like(hx).pin_memory()
    for _ in range(2):
        x.copy_(hx, non_blocking=True)
        hy.copy_(step(), non_blocking=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        x.copy_(hx, non_blocking=True)
        hy.copy_(step(), non_blocking=True)
    e1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dist, "cuda")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": prec, "data": "synthetic",
        "config": {"workload": WORKLOAD % {"f32": "float32", "f64": "float64"}[prec],
                   "l2": "inputs larger than L2 in total, no flush", "bytes_per_step": step_bytes,
                   "parallelism": "slab decomposition x%d (NCCL all-to-all)" % world},
        "round_trip_rel_l2": round_trip,
        "e2e": {"value": whole_job_percent(step_bytes, 1, e2e_ms, peak), "unit": UNIT,
                "h2d_bytes_per_step": hx.numel() * hx.element_size() * world,
                "d2h_bytes_per_step": hy.numel() * hy.element_size() * world, "ms_per_step": e2e_ms,
                "call": "SlabFFT.forward + backward with the slab copied in and out (torch copies)"},
        "gpu_launches": args.steps * (f.engine.zy.launches(False) + f.engine.zy.launches(True)
                                      + f.engine.x.launches(False) + f.engine.x.launches(True)),
        "clocks": clk.summary(t_begin, t_end),
        "roofline": roofline,
        "stages": [{"stage": n, "kernel": k, "mean_ms": round(t, 5), "bytes": b} for t, n, k, b in sorted(means)],
    }
    f.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist.barrier()
    dist.destroy_process_group()


def measure_e2e(args, plan, field, x, X, y, stream, barrier, world, step_bytes, peak, torch, dist):
    """The step end to end through the host-buffer C-ABI entry points (pinned host memory): every
    step uploads its field, runs forward + backward and reads both results back.  Two steps are in
    flight: step k runs on stream k % 2 with its own plan and device buffers, so one step's copies
    back to the host overlap the next step's uploads (the host link carries ~200 GB/s each way and
    ~340 GB/s both ways at once, measured)."""
    from paper_1506_07933_gb300 import afft
    hx = torch.from_numpy(field).pin_memory()
    plans = [plan, afft.Plan(plan.shape, "r2c", {torch.float32: "f32", torch.float64: "f64"}[plan.spatial_dtype])]
    lanes = []
    for i, p in enumerate(plans):
        lanes.append({
            "plan": p, "stream": torch.cuda.Stream(),
            "x": x if i == 0 else torch.empty_like(x), "X": X if i == 0 else torch.empty_like(X),
            "y": y if i == 0 else torch.empty_like(y), "dspec": torch.empty_like(X),
            "hX": torch.empty(p.spectral_shape, dtype=p.spectral_dtype).pin_memory(),
            "hy": torch.empty(p.spatial_shape, dtype=p.spatial_dtype).pin_memory()})

    def e2e_step(k):
        L = lanes[k % 2]
        L["plan"].forward_host(hx, L["hX"], L["x"], L["X"], stream=L["stream"])
        L["plan"].backward_host(L["hX"], L["hy"], L["dspec"], L["y"], stream=L["stream"])

    for k in range(max(2, args.warmup)):
        e2e_step(k)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for L in lanes:
        L["stream"].wait_event(e0)
    for k in range(args.steps):
        e2e_step(k)
    for L in lanes:
        ev = torch.cuda.Event()
        ev.record(L["stream"])
        stream.wait_event(ev)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dist, "cuda")
    h2d = plan.input_bytes + plan.output_bytes
    d2h = plan.output_bytes + plan.input_bytes
    plans[1].close()
    return {"value": whole_job_percent(step_bytes, world, e2e_ms, peak), "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
            "call": "afft_execute_forward_host + afft_execute_backward_host, two steps in flight on two streams"}


def mode_field_gpu(torch, n, seed, n_modes=64, noise=1e-3):
    """The random-mode field (synth.random_mode_field_torch: same modes and recipe) of an n^3 grid,
    evaluated on the GPU and rounded to float32.  Input generation only."""
    from paper_1506_07933_gb300 import synth
    return synth.random_mode_field_torch((n, n, n), seed, n_modes, noise).to(torch.float32)


def batched_workload(afft, torch, steps=10, warmup=3, count=200, seed=200):
    """200 float32 r2c fields of cubic sizes drawn from {48, 64, 96, 120, 128, 160, 256}: one
    forward + backward of every field per step.  Three ways: one execute per field (a plan per
    size, reused), batched plans per size run as one captured CUDA graph, and the same after
    autotuning.  Returns solves/s (field round trips per second) for each."""
    import collections
    from paper_1506_07933_gb300 import synth
    sizes = synth.batched_sizes(count, seed)
    groups = sorted(collections.Counter(sizes).items())
    fields = {n: torch.stack([mode_field_gpu(torch, n, seed * 1000 + 7 * n + i) for i in range(c)])
              for n, c in groups}
    single = {n: afft.Plan((n, n, n), "r2c", "f32") for n, _ in groups}
    spec1 = {n: torch.empty(single[n].spectral_shape, dtype=torch.complex64, device="cuda") for n, _ in groups}
    back1 = {n: torch.empty((n, n, n), dtype=torch.float32, device="cuda") for n, _ in groups}
    order = [(n, i) for n, c in groups for i in range(c)]

    def per_field():
        for n, i in order:
            single[n].forward(fields[n][i], spec1[n])
            single[n].backward(spec1[n], back1[n])

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    ms_single = timed(per_field)
    results = {}
    # one persistent launch per direction over every field (afft_queue)
    plans = [afft.Plan((n, n, n), "r2c", "f32", batch=c) for n, c in groups]
    specs = [torch.empty(p.spectral_shape, dtype=torch.complex64, device="cuda") for p in plans]
    backs = [torch.empty(p.spatial_shape, dtype=torch.float32, device="cuda") for p in plans]
    ins = [fields[n] for n, _ in groups]
    q = afft.Queue(plans)

    def queued():
        q.forward(ins, specs)
        q.backward(specs, backs)

    ms_q = timed(queued)
    err_q = max(float(torch.linalg.vector_norm(b - x) / torch.linalg.vector_norm(x)) for b, x in zip(backs, ins))
    status_q = q.status()
    items_q = (q.items(False), q.items(True))
    q.close()
    for p in plans:
        p.close()
    for tuned in (False, True):
        plans = [afft.Plan((n, n, n), "r2c", "f32", batch=c) for n, c in groups]
        if tuned:
            for p in plans:
                p.tune()
        specs = [torch.empty(p.spectral_shape, dtype=torch.complex64, device="cuda") for p in plans]
        backs = [torch.empty(p.spatial_shape, dtype=torch.float32, device="cuda") for p in plans]
        ins = [fields[n] for n, _ in groups]
        m = afft.Multi(plans)

        def batched():
            m.forward(ins, specs)
            m.backward(specs, backs)

        ms = timed(batched)
        err = max(float(torch.linalg.vector_norm(b - x) / torch.linalg.vector_norm(x)) for b, x in zip(backs, ins))
        results["tuned" if tuned else "batched"] = (ms, err, [p.describe() for p in plans] if tuned else None)
        m.close()
        for p in plans:
            p.close()
    for p in single.values():
        p.close()
    step_bytes = sum(c * 2 * sum(workload_bytes((n, n, n), 4, 8)) for n, c in groups)
    out = {"workload": "%d float32 r2c+c2r fields, sizes %s (counts %s)" % (
               count, [n for n, _ in groups], [c for _, c in groups]),
           "algorithmic_bytes_per_step": step_bytes,
           "frac_of_hbm_roofline_batched_graph": step_bytes / (results["batched"][0] * 1e-3) / 1e9 / peaks()[0],
           "solves_per_s_one_execute_per_field": count / (ms_single * 1e-3),
           "solves_per_s_batched_graph": count / (results["batched"][0] * 1e-3),
           "solves_per_s_batched_graph_tuned": count / (results["tuned"][0] * 1e-3),
           "solves_per_s_persistent_queue": count / (ms_q * 1e-3),
           "frac_of_hbm_roofline_persistent_queue": step_bytes / (ms_q * 1e-3) / 1e9 / peaks()[0],
           "persistent_queue": {"launches_per_step": 2, "work_items": list(items_q), "status": status_q,
                                "round_trip_rel_l2_max": err_q},
           "ms_per_step": {"one_execute_per_field": ms_single, "batched_graph": results["batched"][0],
                           "batched_graph_tuned": results["tuned"][0], "persistent_queue": ms_q},
           "round_trip_rel_l2_max": max(results["batched"][1], results["tuned"][1])}
    out["speedup_batched_tuned_vs_per_field"] = ms_single / results["tuned"][0]
    return out


def serving_workload(torch, count=1200, rate=200.0, saturation=200, loaded=700.0):
    """Spectral Poisson requests (sizes uniform over 64..512 cubed, 30% FP64, Poisson arrivals at
    `rate` per second): the continuous-batching server against one request at a time, in real time,
    then both again at `loaded` requests per second (near the GPU's capacity) and with every request
    arriving at once (saturation).  Every solution is checked
    against its closed form after the timed run."""
    from paper_1506_07933_gb300 import serve
    sizes = serve.SIZES
    pool = serve.RhsPool(sizes)
    out = {"workload": "Poisson solves -Lap u = f on [0,2pi)^3, n uniform over %s, 30%% float64, "
                       "f from 16 random modes, resident in HBM before the clock starts" % (sizes,)}
    for tag, n_req, r in (("at_%g_per_s" % rate, count, rate), ("at_%g_per_s" % loaded, count, loaded),
                          ("saturation", saturation, 0.0)):
        srv = serve.PoissonServer(pool, slots=4)
        srv.warm(sizes)
        reqs = serve.poisson_requests(n_req, rate=r, sizes=sizes, seed=5)
        got, wall = srv.run(reqs)
        srv.close()
        torch.cuda.empty_cache()
        served = serve.summarize(got, wall)
        reqs = serve.poisson_requests(n_req, rate=r, sizes=sizes, seed=5)
        got, wall = serve.run_plain(pool, reqs, warm_sizes=sizes)
        torch.cuda.empty_cache()
        plain = serve.summarize(got, wall)
        out[tag] = {"batched_server": {k: (float("%.4g" % v) if isinstance(v, float) else v) for k, v in served.items()},
                    "one_at_a_time": {k: (float("%.4g" % v) if isinstance(v, float) else v) for k, v in plain.items()}}
    return out


# FP64 FMA rate of one GB300 measured with 8 independent DFMA chains per thread (TFLOP/s): the
# native FP64 roofline that the float-float FP64 transforms are set against
NATIVE_FP64_TFLOPS = 1.26


def extra_configs(afft, torch, peak):
    """The other roofline configurations of the metric, fewer repetitions, same method.  Each
    entry also gives GFLOP/s by the usual count, 5 N log2 N per c2c transform and 2.5 N log2 N per
    r2c or c2r, and FP64 entries their ratio to the native FP64 FMA rate."""
    out = []
    for shape, kind, prec in (((512,) * 3, "r2c", "f32"), ((512,) * 3, "r2c", "f64"), ((512,) * 3, "c2c", "f32"),
                              ((512,) * 3, "c2c", "f64"), ((1024,) * 3, "c2c", "f32"),
                              ((1024,) * 3, "c2c", "f64"), ((1024,) * 3, "c2c", "f32_split")):
        p = afft.Plan(shape, kind, prec)
        x = torch.empty(p.spatial_shape, dtype=p.spatial_dtype, device="cuda")
        if kind == "c2c":
            afft.fill_uniform(x, 10240)
        else:
            x.uniform_(-1, 1)
        X = torch.empty(p.spectral_shape, dtype=p.spectral_dtype, device="cuda")
        y = torch.empty(p.spatial_shape, dtype=p.spatial_dtype, device="cuda")
        cb = 16 if prec == "f64" else 8
        rb = cb // 2
        if kind == "c2c":
            b = 3 * 2 * shape[0] * shape[1] * shape[2] * cb
        else:
            b = sum(workload_bytes(shape, rb, cb))
        for _ in range(3):
            p.forward(x, X)
            p.backward(X, y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record()
        for _ in range(reps):
            p.forward(x, X)
            p.backward(X, y)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        N = shape[0] * shape[1] * shape[2]
        flops = 2 * (5.0 if kind == "c2c" else 2.5) * N * math.log2(N)   # forward + backward
        entry = {"workload": "%s %dx%dx%d %s fwd+bwd" % ((kind,) + shape + (prec,)), "ms_per_step": ms,
                 "frac_of_hbm_roofline": 2 * b / (ms * 1e-3) / 1e9 / peak,
                 "gflops": flops / (ms * 1e-3) / 1e9}
        if prec == "f64":
            entry["vs_native_fp64_fma_peak"] = entry["gflops"] / (NATIVE_FP64_TFLOPS * 1e3)
        out.append(entry)
        if kind == "r2c":
            # the fused spectral Poisson solve on the same field: 5 array passes (r2c N2, N1; fused
            # N0 forward / 1/|k|^2 / inverse; c2r N1, N2) against the 6 of forward + backward
            e0.record()
            for _ in range(reps):
                p.poisson(x, y)
            e1.record()
            torch.cuda.synchronize()
            pms = e0.elapsed_time(e1) / reps
            out.append({"workload": "poisson %dx%dx%d %s (fused N0 stage)" % (shape + (prec,)), "ms_per_step": pms,
                        "frac_of_hbm_roofline_6pass": 2 * b / (pms * 1e-3) / 1e9 / peak,
                        "ms_fwd_plus_bwd": ms})
        del x, X, y
        p.close()
        torch.cuda.empty_cache()
    return out


def cufft_reference(torch, peak):
    """cuFFT (through torch.fft) on the same configurations, a reference baseline only: forward
    unscaled and backward scaled by 1/N as in afft (rfftn / irfftn, fftn / ifftn).  Same timing
    method and bytes as extra_configs."""
    out = []
    for shape, kind, dt in (((512,) * 3, "r2c", torch.float32), ((512,) * 3, "r2c", torch.float64),
                            ((512,) * 3, "c2c", torch.complex64), ((512,) * 3, "c2c", torch.complex128),
                            ((1024,) * 3, "c2c", torch.complex64), ((1024,) * 3, "c2c", torch.complex128)):
        x = torch.empty(shape, dtype=dt, device="cuda")
        if kind == "c2c":
            x.real.uniform_(-1, 1)
            x.imag.uniform_(-1, 1)
            fwd = lambda: torch.fft.fftn(x)
            bwd = lambda X: torch.fft.ifftn(X)
            cb = 16 if dt == torch.complex128 else 8
            b = 3 * 2 * math.prod(shape) * cb
        else:
            x.uniform_(-1, 1)
            fwd = lambda: torch.fft.rfftn(x)
            bwd = lambda X: torch.fft.irfftn(X, s=shape)
            cb = 16 if dt == torch.float64 else 8
            b = sum(workload_bytes(shape, cb // 2, cb))
        for _ in range(3):
            bwd(fwd())
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record()
        for _ in range(reps):
            bwd(fwd())
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        prec = {torch.float32: "f32", torch.float64: "f64", torch.complex64: "f32", torch.complex128: "f64"}[dt]
        out.append({"workload": "cuFFT %s %dx%dx%d %s fwd+bwd" % ((kind,) + shape + (prec,)), "ms_per_step": ms,
                    "frac_of_hbm_roofline": 2 * b / (ms * 1e-3) / 1e9 / peak})
        del x
        torch.cuda.empty_cache()
    return out


def run_case(args):
    """One configuration, `kind:n0xn1xn2:precision` (e.g. c2c:256x256x256:f64): W warm-up and K
    timed forward + backward transforms of a seeded uniform input on one GPU, one JSON line with
    the per-stage times.  For profiling single stage kernels; not the benchmark's metric line."""
    import torch
    from paper_1506_07933_gb300 import afft
    from paper_1506_07933_gb300 import build as libbuild
    kind, dims, prec = args.case.split(":")
    shape = tuple(int(v) for v in dims.split("x"))
    torch.cuda.set_device(0)
    libbuild.build()
    afft.load()
    p = afft.Plan(shape, kind, prec)
    x = torch.empty(p.spatial_shape, dtype=p.spatial_dtype, device="cuda")
    if kind == "c2c":
        afft.fill_uniform(x, 10240)
    else:
        x.uniform_(-1, 1)
    X = torch.empty(p.spectral_shape, dtype=p.spectral_dtype, device="cuda")
    y = torch.empty(p.spatial_shape, dtype=p.spatial_dtype, device="cuda")
    for _ in range(args.warmup):
        p.forward(x, X)
        p.backward(X, y)
    torch.cuda.synchronize()
    p.timing_begin(2 * args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        p.forward(x, X)
        p.backward(X, y)
    e1.record()
    torch.cuda.synchronize()
    st = p.timing_end()
    fwd = [sum(r[i] for r in st[0::2]) / args.steps for i in range(3)]
    bwd = [sum(r[i] for r in st[1::2]) / args.steps for i in range(3)]
    print(json.dumps({"case": args.case, "ms_per_step": e0.elapsed_time(e1) / args.steps, "stage_ms_forward": fwd,
                      "stage_ms_backward": bwd, "plan": p.describe()}), flush=True)
    p.close()


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["afft", "reference"], default="afft")
    ap.add_argument("--precision", choices=["f32", "f64"], default="f32")
    ap.add_argument("--no-extra", action="store_true",
                    help="leave out the metric's other configurations (the 'also' block)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end timing")
    ap.add_argument("--case", default=None,
                    help="time one configuration kind:n0xn1xn2:precision instead (for profiling)")
    ap.add_argument("--decomp", choices=["plan", "slab", "replicas"], default=None,
                    help="one plan per GPU at N = 1 (default), slab decomposition (default at N > 1) "
                         "or independent replicas per GPU")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.case:
        run_case(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
