#!/usr/bin/env python
"""Benchmark of the batched pentadiagonal solve on the hyperdiffusion parametric batch.

Workload: 65,536 independent systems A_s = I + sigma_s D4 of N = 1024 rows
(sigma_s log-uniform in [1e-3, 10], initial fields uniform in [-1, 1]),
factored once (untimed, as in the paper's benchmark, Sec. 3), then implicit
time steps x <- A^{-1} x captured in one CUDA graph.  A bench step is one
implicit step over the whole batch: forward and back substitution (and, for
FP32+refine, the refinement residuals and corrections) for every row.

Metric: row-solves/s = sum(N) * steps / time.  The headline precision is
FP32 + float-float refinement; the FP64 solve is measured beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl own|reference]
  python bench.py --workload NAME[,NAME...]   (other workloads, one JSON line each)

One JSON line is printed by rank 0.  Under torchrun each rank runs its own
copy of the batch (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "row-solves/s and % of HBM peak; FP32+refine vs FP64 solve at rel err 1e-12"
UNIT = "row-solves/s"
BATCH, N = 65536, 1024
WORKLOAD = ("hyperdiffusion parametric batch: 65,536 systems x N=1024, sigma_i log-uniform [1e-3,10], "
            "C0 uniform [-1,1], implicit steps x <- (I + sigma D4)^-1 x in one CUDA graph, factors resident")
# Algorithmic bytes per row and step (the paper's six-vector method, Sec. 2.4: read the
# row's factors and f, write x).  FP64: 5 x 8 B factors + 8 B f + 8 B x.  FP32+refine:
# 5 x 4 B factors + 8 B f + 8 B x (the refinement residual's band comes from sigma).
# The FP32 kernel itself needs only 24 B/row (it stores 1/alpha and beta and rebuilds the
# other three factors of the symmetric band from sigma), so its fraction of the HBM
# roofline on the 36 B/row basis can exceed what its DRAM traffic alone would allow.
ALG_BYTES = {"f64": 56, "f32_refine": 36, "f32_refine_general": 36, "f32_refine_res64": 36}
# the headline variants: FP64; FP32 + one refinement step on the interior-constant kernel (the
# default), on the general kernel that loads every row's factors, and with the residual in native FP64
KERNEL = {"f64": "k_solve64_pair", "f32_refine": "k_solve32u", "f32_refine_general": "k_solve32r",
          "f32_refine_res64": "k_solve32r (FP64 residual)"}
_CS = "paper_1807_07382_gb300/csrc/"
# the sources a kernel is compiled from (its file and the headers it includes): the ncu table's gate
KERNEL_SRC = {"f64": [_CS + "core64.cu", _CS + "internal.cuh"],
              "f32_refine": [_CS + "f32u.cu", _CS + "ff.cuh", _CS + "internal.cuh"],
              "f32_refine_general": [_CS + "f32r.cu", _CS + "ff.cuh", _CS + "internal.cuh"],
              "f32_refine_res64": [_CS + "f32r.cu", _CS + "ff.cuh", _CS + "internal.cuh"],
              "adi": [_CS + "adi.cu", _CS + "internal.cuh"]}


# ----------------------------------------------------------------------------- helpers

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def source_sha(paths):
    """sha256 prefix of a source file, or of several concatenated in order."""
    h = hashlib.sha256()
    for path in ([paths] if isinstance(paths, str) else paths):
        with open(os.path.join(ROOT, path), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_entry(variant):
    """The ncu figures of profiles/traffic.json for this variant's kernel, or None once the
    kernel source has changed since they were taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        e = json.load(fh).get(variant)
    if not e or e.get("source_sha") != source_sha(KERNEL_SRC[variant]):
        return None
    return e


# Each SM has 4 schedulers, each issuing at most one warp instruction per clock.  The FP64
# solve does 4 FMA + 1 MUL per row (9 flops, 5 operations of the FP64 pipe, which takes a
# multiply as long as an FMA): g = (1/alpha)(f - beta g1 - sigma g2), x = g - gamma x1 - delta x2.
# The pipe's rate is measured on the GPU at hand (pent_probe_fp64_fma, see measure_fp64_peak).
SCHEDULERS, F64_FLOPS_PER_ROW, F64_OPS_PER_ROW = 4, 9, 5


def compute_roofline(variant, rows, ms_step, sm_mhz, sms, fp64=None):
    """The compute side of the solve: the FP64 pipe for the FP64 solve (against the measured
    FMA rate), warp-instruction issue for FP32+refine (instructions per row from the ncu
    capture, against sms x 4 schedulers x the sampled SM clock)."""
    if variant == "f64":
        if not fp64:
            return None
        return fp64_roofline(F64_OPS_PER_ROW, F64_FLOPS_PER_ROW, rows, ms_step, fp64, "row")
    e = profile_entry(variant)
    if not e or "warp_inst_per_row" not in e or not sm_mhz:
        return None
    achieved = e["warp_inst_per_row"] * rows / (ms_step / 1e3)
    peak = sms * SCHEDULERS * sm_mhz * 1e6
    return {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "warp instructions/s",
            "frac": achieved / peak,
            "peak_kind": f"{sms} SMs (device query) x 4 schedulers x 1 per clock at the sampled SM clock",
            "warp_inst_per_row": e["warp_inst_per_row"]}


def fp64_roofline(ops_per_unit, flops_per_unit, units, ms_step, fp64, unit_name):
    """FP64-pipe roofline: pipe operations (FMA, add, multiply: one each) per second against the
    measured FMA rate; the flop rate beside it."""
    t = ms_step / 1e3
    peak_ops = fp64["tflops"] * 1e12 / 2  # FMA per second
    achieved = ops_per_unit * units / t
    return {"bound": "fp64", "achieved": achieved, "peak": peak_ops, "unit": "FP64 pipe operations/s",
            "frac": achieved / peak_ops, "peak_kind": "measured (pent_probe_fp64_fma, this run)",
            f"ops_per_{unit_name}": ops_per_unit, "tflops": flops_per_unit * units / t / 1e12,
            f"flops_per_{unit_name}": flops_per_unit}


def measure_fp64_peak(pb, dev, stream, sms):
    """FP64 FMA rate of this GPU: pent_probe_fp64_fma over 8 CTAs of 256 threads per SM (eight
    independent FMA chains a thread), CUDA events on the launching stream, best of 5 launches
    of ~0.1 s after one warm-up launch, SM clocks sampled meanwhile."""
    import ctypes
    import torch
    L = pb._lib.load()
    sink = torch.zeros(1, dtype=torch.float64, device=dev)
    flops = ctypes.c_double()
    blocks, iters = 8 * sms, 1500
    st = ctypes.c_void_p(stream.cuda_stream)

    def launch():
        r = L.pent_probe_fp64_fma(blocks, iters, ctypes.c_void_p(sink.data_ptr()), st, ctypes.byref(flops))
        if r != 0:
            raise RuntimeError(f"pent_probe_fp64_fma: status {r}")
    launch()
    torch.cuda.synchronize(dev)
    times = []
    with ClockSampler(dev.index or 0) as cs:
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            launch()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            times.append(e0.elapsed_time(e1))
    ms = min(times)
    return {"tflops": flops.value / (ms / 1e3) / 1e12, "ms": ms, "flops_per_launch": flops.value,
            "launch": f"{blocks} CTAs x 256 threads, 8 FMA chains x {16 * iters} steps a thread",
            "clocks": cs.summary()}


def traffic_per_row(variant):
    """DRAM bytes per row from a committed ncu summary, if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    e = d.get(variant)
    if not e or e.get("source_sha") != source_sha(KERNEL_SRC[variant]):
        return None
    return float(e["dram_bytes_per_row"])


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(self.idx).uuid)
            sel = uuid if uuid.startswith("GPU-") else f"GPU-{uuid}"
        except Exception:  # noqa: BLE001
            sel = str(self.idx)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", sel, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(ms: float, world: int, device=None) -> float:
    """The slowest rank's time: every rank runs its own replica of the batch, and the
    whole job's throughput is all ranks' rows over this time (weak scaling)."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(rows_per_rank: int, steps: int, world: int, ms: float) -> float:
    """Row-solves per second of the whole job: every rank's rows over the slowest rank's time."""
    return world * rows_per_rank * steps / (ms / 1e3)


# ----------------------------------------------------------------------------- CPU baseline (oracle)

def cpu_baseline(w, budget_s=15.0, gpu_results=None):
    """Time the oracle (plain serial FP64 per system, OpenMP over systems as in the paper's
    Sec. 3.3) on a bounded sample of the same workload, and check the GPU's one-step results
    for the sampled systems against it."""
    import oracle
    cores = oracle.max_threads()
    n = N
    sample = min(4096, w.batch)
    idx = np.arange(sample) * (w.batch // sample)
    band = oracle.band_hyperdiff_batch(np.full(sample, n), w.sigma[idx])
    fac, bad, _ = oracle.factor_batch(np.full(sample, n), band)
    f = np.concatenate([w.field0[s * n:(s + 1) * n] for s in idx])
    t0 = time.perf_counter()
    x1 = oracle.solve_batch(np.full(sample, n), fac, f)
    t1 = time.perf_counter() - t0
    steps = max(1, int(budget_s / max(t1, 1e-6)))
    x = x1
    t0 = time.perf_counter()
    for _ in range(steps):
        x = oracle.solve_batch(np.full(sample, n), fac, x)
    dt = time.perf_counter() - t0
    out = {"value": sample * n * steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{sample} of {w.batch} systems (every {w.batch // sample}th) x N={n}, {steps} implicit steps, "
                     f"factored untimed; OpenMP over systems"}
    # the paper's serial C arm (Sec. 3.3): one thread, the first 512 sampled systems, about 3 s
    ns = min(512, sample)
    fs = x1[:ns * n].copy()
    facs = [v[:ns * n] for v in fac]
    t0 = time.perf_counter()
    oracle.solve_batch(np.full(ns, n), facs, fs, nthreads=1)
    t1 = time.perf_counter() - t0
    reps = max(1, int(min(3.0, budget_s / 5) / max(t1, 1e-6)))
    t0 = time.perf_counter()
    for _ in range(reps):
        fs = oracle.solve_batch(np.full(ns, n), facs, fs, nthreads=1)
    out["serial_1_core"] = {"value": ns * n * reps / (time.perf_counter() - t0), "unit": UNIT,
                            "sample": f"{ns} sampled systems x N={n}, {reps} implicit steps, one thread"}
    errs = {}
    if gpu_results:
        ref = x1.reshape(sample, n)
        for k, g in gpu_results.items():
            got = g[idx]
            errs[k] = float(np.max(np.max(np.abs(got - ref), axis=1) / np.max(np.abs(ref), axis=1)))
    return out, errs


# ----------------------------------------------------------------------------- own arm

def _variant_options(pb, name):
    return {"f64": {}, "f32_refine": {}, "f32_refine_general": {pb.PENT_OPT_FP32_KERNEL: 1},
            "f32_refine_res64": {pb.PENT_OPT_RESIDUAL: pb.PENT_RESIDUAL_F64}}[name]


def run_own(args):
    import torch
    import paper_1807_07382_gb300 as pb
    from paper_1807_07382_gb300 import build as pbuild

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    pbuild.build()
    dev = torch.device("cuda", local)
    # a stream of its own: step graphs are captured on it (the legacy stream cannot be captured)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count

    BATCH = args.batch
    w = synth.hyperdiff_parametric(batch=BATCH, n=N, steps=args.steps)
    f0 = torch.from_numpy(w.field0).to(dev)
    sigma = torch.from_numpy(w.sigma).to(dev)
    rows = BATCH * N
    peak, peak_kind = measured_peaks()
    fp64 = measure_fp64_peak(pb, dev, stream, sms)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    variants = {}
    one_step = {}
    order = ["f64", "f32_refine", "f32_refine_general", "f32_refine_res64"] if args.precision == "both" \
        else [args.precision]
    clocks = None
    for name in order:
        prec = pb.PENT_F64 if name == "f64" else pb.PENT_F32_REFINE
        plan = pb.Plan(N, batch=BATCH, precision=prec, device=dev, stream=stream,
                       options=_variant_options(pb, name))
        plan.factor_hyperdiff(sigma)
        x = f0.clone()
        # one step from C0 for the accuracy check against the oracle
        one_step[name] = plan.solve(f0, max_refine=args.max_refine).view(BATCH, N).cpu().numpy()
        # warm-up: W steps, then the K-step graph once (capture + instantiate + run)
        plan.solve_steps(x, args.warmup, max_refine=args.max_refine)
        plan.solve_steps(x, args.steps, max_refine=args.max_refine)
        torch.cuda.synchronize(dev)
        st = plan.info()[0]
        if st != pb.PENT_OK:
            raise RuntimeError(f"{name}: device status {st}")
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize(dev)
        with ClockSampler(local) as cs:
            ev0.record(stream)
            plan.solve_steps(x, args.steps, max_refine=args.max_refine)
            ev1.record(stream)
            torch.cuda.synchronize(dev)
        barrier()
        ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
        ms_step = ms / args.steps
        value = job_throughput(rows, args.steps, world, ms)
        achieved = ALG_BYTES[name] * rows / (ms_step / 1e3) / 1e9
        tr = traffic_per_row(name)
        variants[name] = {
            "value": value, "ms_per_step": ms_step, "dtype": "f64" if name == "f64" else "f32",
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": (tr * rows) if tr is not None else None,
                         "kernel": KERNEL[name], "alg_bytes_per_row": ALG_BYTES[name],
                         "peak_kind": peak_kind},
            "clocks": cs.summary(),
        }
        variants[name]["compute_roofline"] = compute_roofline(name, rows, ms_step,
                                                              variants[name]["clocks"].get("sm_mhz"), sms, fp64)
        if name != "f64":
            variants[name]["max_refine"] = args.max_refine
            variants[name]["refine_steps_used"] = plan.info()[3]
        if name == "f32_refine":
            variants[name]["note"] = ("interior-constant kernel: factors loaded only near the walls; the field "
                                      "stays as scaled float pairs between graph steps")
        clocks = variants[name]["clocks"]
        del plan
        torch.cuda.empty_cache()

    head = "f32_refine" if "f32_refine" in variants else order[0]
    hv = variants[head]

    # end to end through the public API: per step, H2D of the step's RHS from pinned
    # host memory, the solve, D2H of the solution
    e2e = None
    if not args.no_e2e:
        prec = pb.PENT_F64 if head == "f64" else pb.PENT_F32_REFINE
        plan = pb.Plan(N, batch=BATCH, precision=prec, device=dev, stream=stream)
        plan.factor_hyperdiff(sigma)
        fh = torch.from_numpy(w.field0).pin_memory()
        xh = torch.empty_like(fh).pin_memory()
        fd = torch.empty_like(f0)
        xd = torch.empty_like(f0)
        e2e_steps = 10

        runs_ms = {}

        def timed(call, key=None):
            # three runs of e2e_steps steps; the median run is reported (the host link and host
            # memory are shared with other work on the node, which now and then slows one run)
            for _ in range(2):
                call()
            out = []
            for _ in range(3):
                torch.cuda.synchronize(dev)
                barrier()
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                for _ in range(e2e_steps):
                    call()
                ev1.record(stream)
                torch.cuda.synchronize(dev)
                barrier()
                out.append(max_over_ranks(ev0.elapsed_time(ev1), world, dev))
            if key:
                runs_ms[key] = [v / e2e_steps for v in out]
            return statistics.median(out)

        # staged: copies in, solve, copies out, 16 overlapping slices
        modes = {"staged": timed(lambda: plan.solve_host(fh, xh, fd, xd, max_refine=args.max_refine), "staged")}
        match = None
        if prec == pb.PENT_F32_REFINE:
            # direct: the solve kernels read f from and write x to the pinned host buffers
            staged_x = xh.clone()
            xh.zero_()
            modes["direct"] = timed(lambda: plan.solve_host(fh, xh, max_refine=args.max_refine, direct=True), "direct")
            match = bool(torch.equal(staged_x, xh))
        # the host link's floor: the step's two copies alone, both directions at once
        side = torch.cuda.Stream(dev)

        def copies():
            side.wait_stream(stream)
            fd.copy_(fh, non_blocking=True)
            with torch.cuda.stream(side):
                xh.copy_(xd, non_blocking=True)
            stream.wait_stream(side)

        link_ms = timed(copies)
        best = min(modes, key=modes.get)
        e2e = {"value": job_throughput(rows, e2e_steps, world, modes[best]), "unit": UNIT,
               "h2d_bytes_per_step": int(fh.numel() * 8), "d2h_bytes_per_step": int(xh.numel() * 8),
               "steps": e2e_steps, "precision": head, "mode": best,
               "ms_per_step": {k: v / e2e_steps for k, v in modes.items()}, "ms_per_step_runs": runs_ms,
               "timing": f"median of 3 runs of {e2e_steps} steps",
               "link_floor_ms_per_step": link_ms / e2e_steps, "frac_of_link_floor": link_ms / modes[best]}
        if match is not None:
            e2e["direct_equals_staged"] = match
        del plan
        torch.cuda.empty_cache()

    # the other workloads of the method (uneven batch, 2D ADI), each timed on its own graph after the
    # headline's timed region; one GPU only
    if world == 1 and not args.no_workloads:
        for k, v in measure_uneven(pb, dev, stream, fp64, sms, steps=args.workload_steps or 200).items():
            variants[k] = v
        variants["adi"] = measure_adi(pb, dev, stream, fp64)

    base, errs = (None, {})
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base, errs = cpu_baseline(w, budget_s=args.cpu_budget, gpu_results=one_step)
    for k, v in errs.items():
        variants[k]["max_rel_err_vs_oracle"] = v

    if rank == 0:
        line = {
            "metric": METRIC, "value": hv["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": hv["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": hv["dtype"], "data": "synthetic",
            "config": {"workload": WORKLOAD if BATCH == 65536 else WORKLOAD.replace("65,536", f"{BATCH:,}"),
                       "batch": BATCH, "n": N, "precision": head,
                       "max_refine": args.max_refine if head != "f64" else 0,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "working set (factors + field) >= 1.9 GB, larger than L2; no flush"},
            "roofline": hv["roofline"], "compute_roofline": hv["compute_roofline"], "cpu_baseline": base,
            "e2e": e2e, "gpu_launches": args.steps,
            "clocks": clocks, "fp64_peak": fp64, "sms": sms, "variants": variants,
        }
        if errs:
            line["max_rel_err_vs_oracle"] = errs.get(head)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def measure_uneven(pb, dev, stream, fp64, sms, steps=200):
    """The uneven batch (20,000 systems, N log-uniform in [64, 16384], sum N = 59.1 M) with the GB300
    tune cache, both precisions, one refinement step: ms per graph step, error of one solve against
    the oracle on every 97th system, HBM roofline on the algorithmic bytes."""
    import torch
    import oracle
    w = synth.uneven(steps=steps)
    f0 = torch.from_numpy(w.field0).to(dev)
    sig = torch.from_numpy(w.sigma).to(dev)
    off = w.offsets
    pick = np.arange(0, w.batch, 97)
    ref = oracle.hyperdiff_steps(w.n[pick], w.sigma[pick], np.concatenate([w.field0[off[s]:off[s + 1]] for s in pick]),
                                 1)
    roff = oracle.offsets(w.n[pick])
    tune = os.path.join(ROOT, "paper_1807_07382_gb300", "tune_gb300.txt")
    peak, peak_kind = measured_peaks()
    out = {}
    for prec, pname, alg, kern in ((pb.PENT_F64, "f64", 56, "k_swin64_fwd + k_swin64_bwd (system windows of 1024 rows) + k_solve64_pair"),
                                   (pb.PENT_F32_REFINE, "f32_refine", 36,
                                    "k_solve32u (windows of 1024 rows, single CTAs)")):
        plan = pb.Plan(list(w.n), precision=prec, stream=stream, device=dev, tune_cache=tune)
        plan.factor_hyperdiff(sig)
        one = plan.solve(f0, max_refine=1).cpu().numpy()
        got = np.concatenate([one[off[s]:off[s + 1]] for s in pick])
        err = max(float(np.max(np.abs(got[roff[k]:roff[k + 1]] - ref[roff[k]:roff[k + 1]])) /
                        np.max(np.abs(ref[roff[k]:roff[k + 1]]))) for k in range(len(pick)))
        x = f0.clone()
        plan.solve_steps(x, steps, max_refine=1)
        ms, ck = _time_device(stream, lambda: plan.solve_steps(x, steps, max_refine=1), steps, dev)
        ms_step = ms / steps
        achieved = alg * w.rows / (ms_step / 1e3) / 1e9
        out[f"uneven_{pname}"] = {
            "value": w.rows * steps / (ms / 1e3), "ms_per_step": ms_step, "dtype": pname.split("_")[0],
            "workload": "20,000 systems, N log-U[64,16384] (sum 59.1 M rows), sigma log-U[1e-2,10], "
                        f"{steps} implicit steps (1 graph), tuned launch settings",
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "kernel": kern, "alg_bytes_per_row": alg, "peak_kind": peak_kind},
            "max_rel_err_vs_oracle": err, "err_sample": f"{len(pick)} systems, one solve",
            "windows": plan.get_option(pb.PENT_OPT_WINDOWS),
            "max_refine": 1 if prec == pb.PENT_F32_REFINE else 0, "clocks": ck}
        del plan
        torch.cuda.empty_cache()
    return out


def adi_fp64_counts():
    """FP64 pipe operations and flops per cell of one ADI step from a committed ncu count
    (profiles/traffic.json), or None once the ADI kernels' sources have changed since."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        e = json.load(fh).get("adi")
    if not e or e.get("source_sha") != source_sha(KERNEL_SRC["adi"]):
        return None
    return float(e["fp64_ops_per_cell"]), float(e["fp64_flops_per_cell"])


def measure_adi(pb, dev, stream, fp64, steps=500):
    """The 2D Cahn-Hilliard ADI step on 2048^2 (gamma = 0.01, dt = 1e-6, dx = 1/2048): ms per step in a
    500-step graph, the step's change against the oracle's, mass drift, and the FP64-pipe roofline
    (the step is bound by FP64 arithmetic, its 33.5 MB field staying in L2)."""
    import torch
    import oracle
    w = synth.ch_adi(steps=steps)
    adi = pb.ADI2D(w.nx, w.ny, w.gamma, w.dt, w.dx, device=dev, stream=stream)
    C = torch.from_numpy(w.field0).to(dev)
    one = adi.step(C.clone()).cpu().numpy()
    ref = oracle.adi_step(w.field0, w.gamma, w.dt, w.dx)
    # the exact dC is O(sigma) times the field's rounding: compare the step's change, normwise
    err = float(np.max(np.abs(one - ref)) / np.max(np.abs(ref - w.field0)))
    m0 = float(C.sum())
    adi.step(C.clone(), nsteps=steps)
    ms, ck = _time_device(stream, lambda: adi.step(C, nsteps=steps), steps, dev)
    drift = abs(float(C.sum()) - m0) / float(np.abs(w.field0).sum())
    ms_step = ms / steps
    cells = w.nx * w.ny
    counts = adi_fp64_counts()
    comp = fp64_roofline(counts[0], counts[1], cells, ms_step, fp64, "cell") if counts and fp64 else None
    return {"value": 2 * cells * steps / (ms / 1e3), "ms_per_step": ms_step, "dtype": "f64",
            "workload": "2048 x 2048 Cahn-Hilliard ADI (Douglas), gamma=0.01, dt=1e-6, dx=1/2048, "
                        f"{steps} steps (1 graph); rows = both sweeps",
            "compute_roofline": comp,
            "memory": "about 40 B per cell and step of algorithmic traffic (C read with its halo, the "
                      "intermediates, C written); the 33.5 MB field and the sweeps' scratch stay in the 129 MB L2",
            "max_rel_err_vs_oracle": err, "err_metric": "max|dC - dC_ref| / max|dC_ref| after one step",
            "mass_drift_rel": drift, "clocks": ck}


# ----------------------------------------------------------------------------- other workloads

def _sys_err(got, ref):
    """Per-system max|x - x_ref| / max|x_ref|, maximised over the rows of 2D arrays."""
    return float(np.max(np.max(np.abs(got - ref), axis=1) / np.max(np.abs(ref), axis=1)))


def _time_device(stream, run, steps, dev):
    """CUDA-event time of run() on `stream` (after a warm call), with clocks sampled meanwhile."""
    import torch
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index or 0) as cs:
        ev0.record(stream)
        run()
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    return ev0.elapsed_time(ev1), cs.summary()


def _line(name, workload, rows_per_step, steps, ms, alg_bytes, kernel, err, extra=None, dtype="f64", clocks=None):
    peak, peak_kind = measured_peaks()
    ms_step = ms / steps
    achieved = alg_bytes * rows_per_step / (ms_step / 1e3) / 1e9
    line = {"workload_name": name, "metric": METRIC, "value": rows_per_step * steps / (ms / 1e3), "unit": UNIT,
            "n_gpus": 1, "steps": steps, "ms_per_step": ms_step, "higher_is_better": True, "dtype": dtype,
            "data": "synthetic", "config": {"workload": workload},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "kernel": kernel, "alg_bytes_per_row": alg_bytes, "peak_kind": peak_kind},
            "max_rel_err_vs_oracle": err, "clocks": clocks}
    line.update(extra or {})
    print(json.dumps(line), flush=True)


def run_workloads(names, args):
    import torch
    import oracle
    import paper_1807_07382_gb300 as pb
    from paper_1807_07382_gb300 import build as pbuild
    from paper_1807_07382_gb300 import autograd as pag

    pbuild.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)  # a stream of its own: step graphs are captured on it
    torch.cuda.set_stream(stream)
    tune = os.path.join(ROOT, "paper_1807_07382_gb300", "tune_gb300.txt")
    for name in names:
        if name == "cosines":
            w = synth.hyperdiff_cosines()
            n = int(w.n[0])
            plan = pb.Plan(n, batch=w.batch, shared=True, stream=stream)
            plan.factor_hyperdiff(torch.from_numpy(w.sigma).to(dev))
            x = torch.from_numpy(w.field0).to(dev)
            plan.solve_steps(x.clone(), w.steps)
            ref = oracle.hyperdiff_steps(w.n, w.sigma, w.field0, w.steps, shared=True)
            ms, ck = _time_device(stream, lambda: plan.solve_steps(x, w.steps), w.steps, dev)
            err = _sys_err(x.cpu().numpy().reshape(w.batch, n), ref.reshape(w.batch, n))
            _line(name, "64 systems x N=256, shared sigma=0.5, 4 cosine modes + noise, 100 implicit steps (1 graph)",
                  w.rows, w.steps, ms, 16, "k_solve64_pair<shared>", err, clocks=ck,
                  extra={"note": "shared factors broadcast; latency bound (16,384 rows per step)"})
        elif name == "uneven":
            for k, v in measure_uneven(pb, dev, stream, None, 0, steps=args.workload_steps or 200).items():
                print(json.dumps({"workload_name": k, "metric": METRIC, "unit": UNIT, "n_gpus": 1,
                                  "higher_is_better": True, "data": "synthetic", **v}), flush=True)
        elif name == "adi":
            v = measure_adi(pb, dev, stream, None)
            print(json.dumps({"workload_name": name, "metric": METRIC, "unit": UNIT, "n_gpus": 1,
                              "higher_is_better": True, "data": "synthetic", **v}), flush=True)
        elif name == "adjoint":
            w = synth.adjoint_batch()
            n = int(w.n[0])
            c0 = torch.from_numpy(w.field0.reshape(w.batch, n)).to(dev).requires_grad_(True)
            sig = torch.from_numpy(w.sigma).to(dev).requires_grad_(True)
            target = pag.hyperdiff_steps(c0.detach(), sig.detach() * (1 + w.extra["perturb"]), w.steps)

            pick = np.arange(0, w.batch, 128)
            _, rgc, rgs = oracle.hyperdiff_loss_grad(w.sigma[pick], w.steps, w.field0.reshape(w.batch, n)[pick],
                                                     target.detach().cpu().numpy()[pick])
            for prec, pname, mr, kern in ((pb.PENT_F64, "", 0, "k_solve64_pair + k_adjoint64 + k_sigma_grad"),
                                          (pb.PENT_F32_REFINE, "_f32_refine", 2, "k_solve32r + k_sigma_grad")):
                def grad():
                    xT = pag.hyperdiff_steps(c0, sig, w.steps, 10, precision=prec, max_refine=mr)
                    loss = ((xT - target) ** 2).sum()
                    return torch.autograd.grad(loss, (c0, sig))
                gc, gs = grad()
                err_s = float(np.max(np.abs(gs.cpu().numpy()[pick] - rgs) / np.abs(rgs)))
                err_c = float(np.max(np.abs(gc.cpu().numpy()[pick] - rgc)) / np.max(np.abs(rgc)))
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                reps = 3
                for _ in range(reps):
                    grad()
                torch.cuda.synchronize(dev)
                ms = (time.perf_counter() - t0) * 1e3 / reps
                solves = 3 * w.steps  # forward, recompute from checkpoints, adjoint
                _line(name + pname, "4,096 systems x N=1024, loss over T=50 implicit steps, gradient w.r.t. C0 and "
                      "sigma (checkpoints every 10 steps)", w.batch * n * solves, 1, ms, 56 if not pname else 36,
                      kern, err_s, dtype="f64" if not pname else "f32",
                      extra={"ms_per_gradient": ms, "max_refine": mr,
                             "err_metric": "relative error of dL/dsigma vs the oracle adjoint "
                                           f"({len(pick)} systems)",
                             "err_dC0": err_c, "timing": "host wall clock around torch.autograd (3 gradients)"})
        elif name == "periodic_cn":
            w = synth.periodic_cn(batch=args.batch or 65536)
            n = int(w.n[0])
            s = torch.from_numpy(w.sigma).to(dev)
            pick = np.arange(0, w.batch, max(1, w.batch // 128))
            ref = oracle.periodic_steps(n, w.sigma, w.field0.reshape(w.batch, n)[pick].reshape(-1), 1, cn=True,
                                        shared=True)
            for prec, pname, alg, kern in ((pb.PENT_F64, "f64", 16, "k_solve_periodic<shared, rhs>"),
                                           (pb.PENT_F32_REFINE, "f32_refine", 16, "k_solve32r<step, periodic>")):
                plan = pb.Plan(n, batch=w.batch, shared=True, periodic=True, stream=stream, precision=prec)
                plan.factor_hyperdiff(s)
                C = torch.from_numpy(w.field0).to(dev)
                c1 = C.clone()
                plan.step(c1, nu=s, max_refine=3)
                err = _sys_err(c1.cpu().numpy().reshape(w.batch, n)[pick], ref.reshape(len(pick), n))
                used = plan.info()[3]
                plan.step(C.clone(), nu=s, nsteps=w.steps, max_refine=3)
                ms, ck = _time_device(stream, lambda: plan.step(C, nu=s, nsteps=w.steps, max_refine=3), w.steps, dev)
                _line(f"{name}_{pname}", f"periodic Crank-Nicolson hyperdiffusion (Navon reduction), {w.batch:,} systems "
                      f"x N={n}, shared sigma_x = dt/(2 dx^4) = 343.6 (dt=1e-8, dx=1/512), C0 U[-1,1], 250 steps "
                      "(1 graph)", w.rows, w.steps, ms, alg, kern, err, clocks=ck,
                      dtype="f64" if prec == pb.PENT_F64 else "f32",
                      extra={"note": "reduction shared by the batch; f assembled in the forward sweep"
                                     + ("" if prec == pb.PENT_F64 else "; FP32 solve of E + 2x2 tail, refined "
                                        "against the float-float residual (max_refine 3; kappa ~ 5.5e3)"),
                             "refine_steps_used": used if prec != pb.PENT_F64 else 0,
                             "err_sample": f"{len(pick)} systems, one step"})
                del plan
        elif name == "ch1d":
            w = synth.ch_batch(batch=args.batch or 65536)
            n = int(w.n[0])
            mu = torch.from_numpy(w.extra["mu"]).to(dev)
            sig = torch.from_numpy(w.sigma).to(dev)
            pick = np.arange(0, w.batch, max(1, w.batch // 128))
            ref = oracle.explicit_steps(np.full(len(pick), n), w.sigma[pick], w.extra["mu"][pick], None,
                                        w.field0.reshape(w.batch, n)[pick].reshape(-1), 1)
            for prec, pname, alg, kern in ((pb.PENT_F64, "f64", 48, "k_step64_pair"),
                                           (pb.PENT_F32_REFINE, "f32_refine", 24, "k_solve32r<step>")):
                plan = pb.Plan(n, batch=w.batch, stream=stream, precision=prec)
                plan.factor_hyperdiff(sig)
                C = torch.from_numpy(w.field0).to(dev)
                c1 = C.clone()
                plan.step(c1, mu=mu, max_refine=1)
                err = _sys_err(c1.cpu().numpy().reshape(w.batch, n)[pick], ref.reshape(len(pick), n))
                plan.step(C.clone(), mu=mu, nsteps=w.steps, max_refine=1)
                ms, ck = _time_device(stream, lambda: plan.step(C, mu=mu, nsteps=w.steps, max_refine=1), w.steps, dev)
                note = ("48 B/row: 4 FP64 record planes + C read + C written" if prec == pb.PENT_F64 else
                        "24 B/row: FP32 1/alpha and beta + C read + C written; one refinement step")
                _line(f"{name}_{pname}", f"1D Cahn-Hilliard parameter batch (semi-implicit, no-flux), {w.batch:,} systems "
                      f"x N={n}, sigma log-U[1e-3,10], mu log-U[1e-4,1e-1], 200 steps (1 graph)", w.rows, w.steps, ms,
                      alg, kern, err, clocks=ck, dtype="f64" if prec == pb.PENT_F64 else "f32",
                      extra={"note": note + "; the right-hand side C + mu D2(C^3 - C) is assembled in the kernel",
                             "err_sample": f"{len(pick)} systems, one step"})
                del plan
        elif name == "shared":
            # the paper's benchmark configuration (Sec. 3): every system has the same matrix
            w = synth.hyperdiff_parametric(batch=args.batch or 65536, steps=200)
            n = int(w.n[0])
            sig1 = np.array([1.0])
            f0 = torch.from_numpy(w.field0).to(dev)
            pick = np.arange(0, w.batch, max(1, w.batch // 128))
            ref = oracle.hyperdiff_steps(np.full(len(pick), n), np.full(len(pick), 1.0),
                                         w.field0.reshape(w.batch, n)[pick].reshape(-1), 1)
            for prec, pname, alg, kern in ((pb.PENT_F64, "f64", 16, "k_solve64_pair<shared>"),
                                           (pb.PENT_F32_REFINE, "f32_refine", 16, "k_solve32r (shared block)")):
                plan = pb.Plan(n, batch=w.batch, shared=True, stream=stream, precision=prec)
                plan.factor_hyperdiff(torch.from_numpy(sig1).to(dev))
                one = plan.solve(f0, max_refine=1).cpu().numpy().reshape(w.batch, n)
                err = _sys_err(one[pick], ref.reshape(len(pick), n))
                x = f0.clone()
                plan.solve_steps(x, w.steps, max_refine=1)
                ms, ck = _time_device(stream, lambda: plan.solve_steps(x, w.steps, max_refine=1), w.steps, dev)
                _line(f"{name}_{pname}", f"one matrix for the batch (the paper's identical systems, Sec. 3): {w.batch:,} "
                      f"systems x N={n}, sigma = 1, C0 U[-1,1], {w.steps} implicit steps (1 graph)", w.rows, w.steps, ms,
                      alg, kern, err, clocks=ck, dtype="f64" if prec == pb.PENT_F64 else "f32",
                      extra={"note": "16 B/row: f read, x written; the factors are one broadcast block",
                             "err_sample": f"{len(pick)} systems, one step"})
                del plan
        elif name == "rewrite":
            w = synth.hyperdiff_parametric(batch=args.batch or 65536, steps=200)
            n = int(w.n[0])
            K = 20
            plan = pb.Plan(n, batch=w.batch, stream=stream)
            sigs = [torch.from_numpy(w.sigma * (1.0 + 1e-3 * k)).to(dev) for k in range(K)]
            f = torch.from_numpy(w.field0).to(dev)
            x1 = plan.refactor_solve(sigs[0], f)
            pick = np.arange(0, w.batch, max(1, w.batch // 128))
            ref = oracle.hyperdiff_steps(np.full(len(pick), n), w.sigma[pick],
                                         w.field0.reshape(w.batch, n)[pick].reshape(-1), 1)
            err = _sys_err(x1.cpu().numpy().reshape(w.batch, n)[pick], ref.reshape(len(pick), n))
            x = f.clone()

            def run():
                for k in range(K):
                    plan.refactor_solve(sigs[k], x, x)
            run()
            ms, ck = _time_device(stream, run, K, dev)
            _line(name, f"refactor + solve every step (the paper's Rewrite), {w.batch:,} systems x N={n}, a new sigma per "
                  "system and step, 20 steps", w.rows, K, ms, 48, "k_refactor_solve64", err, clocks=ck,
                  extra={"note": "48 B/row: f read, x written, 4 record planes written (the plan stays factored)",
                         "err_sample": f"{len(pick)} systems, one step"})
        else:
            raise SystemExit(f"unknown workload {name}")


# ----------------------------------------------------------------------------- reference arm

def run_reference(args):
    """The oracle as it stands on the host cores, same workload, metric and unit; each
    step solves a bounded sample of the batch so the run ends in a few minutes."""
    world, rank, local = dist_setup()
    if rank != 0:
        return
    import oracle
    w = synth.hyperdiff_parametric(batch=BATCH, n=N, steps=1)
    cores = oracle.max_threads()
    n = N
    budget = 120.0
    probe = 256
    idx = np.arange(probe)
    band = oracle.band_hyperdiff_batch(np.full(probe, n), w.sigma[idx])
    fac, _, _ = oracle.factor_batch(np.full(probe, n), band)
    f = w.field0[:probe * n].copy()
    t0 = time.perf_counter()
    oracle.solve_batch(np.full(probe, n), fac, f)
    per_row = (time.perf_counter() - t0) / (probe * n)
    per_step_budget = budget / max(1, args.steps + args.warmup)
    sample = int(min(BATCH, max(32, per_step_budget / max(per_row, 1e-12) / n)))
    idx = np.arange(sample) * (BATCH // sample)
    band = oracle.band_hyperdiff_batch(np.full(sample, n), w.sigma[idx])
    fac, _, _ = oracle.factor_batch(np.full(sample, n), band)
    x = np.concatenate([w.field0[s * n:(s + 1) * n] for s in idx])
    ns = np.full(sample, n)
    for _ in range(args.warmup):
        x = oracle.solve_batch(ns, fac, x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        x = oracle.solve_batch(ns, fac, x)
    dt = time.perf_counter() - t0
    value = sample * n * args.steps / dt
    desc = (f"{sample} of {BATCH} systems (every {BATCH // sample}th) x N={n} per step, FP64 serial per system, "
            f"OpenMP over systems, factored untimed")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "batch": BATCH, "n": N, "precision": "f64"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


PROFILE_CASES = ("fp32_steps", "fp64_solve", "fp32_windows", "fp64_windows", "fp64_group_windows", "uneven_fp32",
                 "uneven_fp64", "uneven_fp64_group_windows",
                 "adi_step")


def run_profile_case(name):
    """One small run of a kernel for an ncu capture (never a bench value): the launch to capture
    is the second of its kind.  fp32_steps: 16,384 x 1024 parametric FP32+refine, a 4-step graph
    (k_solve32u with float pairs in and out in the middle steps); fp64_solve: 32,768 x 1024 FP64,
    two solves (k_solve64_pair); fp32_windows: 2,000 x 8,192 FP32+refine, two out-of-place
    solves (k_solve32u windows); fp64_windows: 4,096 x 8,192 FP64, two in-place solves
    (k_srec64 once, then k_swin64_fwd, k_swin64_bwd; fp64_group_windows: the same with group
    windows, k_win64_halo, k_solve64w); uneven_fp32 / uneven_fp64 (/ uneven_fp64_group_windows): the
    uneven batch (20,000 systems),
    factor and two 2-step graphs (the launch list of its steps); adi_step: the 2048^2 ADI workload,
    factor and one step (every kernel of the step once)."""
    import torch
    import paper_1807_07382_gb300 as pb
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    if name == "adi_step":
        w = synth.ch_adi(steps=1)
        adi = pb.ADI2D(w.nx, w.ny, w.gamma, w.dt, w.dx, device=dev, stream=stream)
        adi.step(torch.from_numpy(w.field0).to(dev))
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": name, "cells": w.nx * w.ny}))
        return
    tune = os.path.join(ROOT, "paper_1807_07382_gb300", "tune_gb300.txt")
    prec = pb.PENT_F64 if "fp64" in name else pb.PENT_F32_REFINE
    if name.startswith("uneven"):
        w = synth.uneven(steps=2)
    elif name.endswith("windows"):
        w = synth.hyperdiff_parametric(batch=2000 if prec == pb.PENT_F32_REFINE else 4096, n=8192, steps=1,
                                       seed_index=3, sigma_range=(1e-2, 10.0))
    else:
        w = synth.hyperdiff_parametric(batch=16384 if prec == pb.PENT_F32_REFINE else 32768, n=1024, steps=1)
    opts = {pb.PENT_OPT_WINDOW_FORM: 0} if name.endswith("group_windows") else {}
    plan = pb.Plan(list(w.n), precision=prec, stream=stream, device=dev, tune_cache=tune, options=opts)
    plan.factor_hyperdiff(torch.from_numpy(w.sigma).to(dev))
    x = torch.from_numpy(w.field0).to(dev)
    if name == "fp32_steps":
        plan.solve_steps(x, 4, max_refine=1)
    elif name.startswith("uneven"):
        for _ in range(2):
            plan.solve_steps(x, 2, max_refine=1)
    elif name == "fp32_windows":
        y = torch.empty_like(x)
        for _ in range(2):
            plan.solve(x, y, max_refine=1)
    else:
        for _ in range(2):
            plan.solve(x, x, max_refine=1)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": name, "rows": int(w.n.sum()), "windows": plan.get_option(pb.PENT_OPT_WINDOWS)}))


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["own", "reference"], default="own")
    ap.add_argument("--precision", choices=["both", "f64", "f32_refine", "f32_refine_general", "f32_refine_res64"],
                    default="both", help="headline variants to time (both: all four)")
    ap.add_argument("--max-refine", type=int, default=1,
                    help="FP32 refinement steps (one reaches the 1e-12 bar on this workload; the error is measured)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--batch", type=int, default=None,
                    help="systems (default: the full workload; smaller for profiling, also for --workload "
                         "periodic_cn, ch1d and rewrite)")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the uneven and ADI workloads that the default line carries under variants")
    ap.add_argument("--workload-steps", type=int, default=None,
                    help="steps of the uneven workload's timed graph (default 200; fewer for profiling)")
    ap.add_argument("--workload", default=None,
                    help="comma-separated other workloads: cosines, uneven, adi, adjoint, periodic_cn, ch1d, rewrite, shared, "
                         "or all (one JSON line each; the default run is the parametric headline line)")
    ap.add_argument("--profile-case", choices=PROFILE_CASES, default=None,
                    help="run one small case of a kernel for an ncu capture and exit (no timing)")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args.profile_case)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.workload:
        names = ["cosines", "uneven", "adi", "adjoint", "periodic_cn", "ch1d", "rewrite", "shared"] \
            if args.workload == "all" else args.workload.split(",")
        run_workloads(names, args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        if args.batch is None:
            args.batch = BATCH
        run_own(args)


if __name__ == "__main__":
    main()
