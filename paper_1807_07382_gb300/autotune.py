"""Autotuner for the batched solves: times candidate launch settings per row-count
bucket on the GPU at hand and writes a tune cache (format in include/pentbatch.h).

Knobs, per bucket of row counts (n_lo, n_hi]:
  FP32+refine  rows per thread (the chunk a thread owns: 4 or 8, which also sets
               the chunked factor layout) and threads per system (the fewest
               that cover n, or twice that);
  FP64         rows loaded ahead of the arithmetic (unroll 2, 4, 8) and warps
               per CTA (1, 2, 4) of the thread-per-system substitution.
Each candidate is timed on a batch of systems of the bucket's largest n,
hyperdiffusion matrices with sigma log-uniform in [1e-2, 10] and right-hand
sides uniform in [-1, 1] (seeded), as implicit steps captured in a CUDA graph,
with CUDA events on the plan's stream.  The fastest candidate wins.  Windows of long systems
(PENT_OPT_WINDOW_WARPS, PENT_OPT_WINDOW_ROWS) are off while tuning: the knobs tune the
per-system solves, which windows replace where they apply.

    python -m paper_1807_07382_gb300.autotune --out tune.txt [--buckets 64,128,...]
    plan = Plan(ns, precision=..., tune_cache="tune.txt")
"""
from __future__ import annotations

import argparse
import math
from typing import Iterable, Optional

from . import PENT_F32_REFINE, PENT_F64, PENT_OPT_BLOCK_WARPS, PENT_OPT_PARTITION_ROWS, PENT_OPT_ROWS_PER_THREAD, \
    PENT_OPT_THREADS_PER_SYSTEM, PENT_OPT_UNROLL, PENT_OPT_WINDOW_ROWS, PENT_OPT_WINDOW_WARPS, Plan

DEFAULT_BUCKETS = (64, 128, 256, 512, 1024, 2048, 4096, 8192, 16384)


def _valid_tps(t: int) -> Optional[int]:
    """Smallest launchable threads-per-system count >= t (32 W, W <= 16, or 512 C, C <= 8)."""
    if t <= 512:
        return max(32, 32 * math.ceil(t / 32))
    c = math.ceil(t / 512)
    return 512 * c if c <= 8 else None


def f32_candidates(n: int) -> list:
    """(rows per thread, threads per system) pairs that can hold n rows."""
    out = []
    for rpt in (4, 8):
        t = _valid_tps(math.ceil(n / rpt))
        if t is None:
            continue
        out.append((rpt, t))
        t2 = _valid_tps(2 * t)
        if t2 is not None and t2 != t and t2 <= 1024:
            out.append((rpt, t2))
    return out


def f64_candidates(n: int) -> list:
    return [(u, bw) for u in (2, 4, 8) for bw in (1, 2, 4)]


def _inputs(n: int, batch: int, device, seed: int):
    import torch
    g = torch.Generator(device=device).manual_seed(seed)
    u = torch.rand(batch, generator=g, device=device, dtype=torch.float64)
    sigma = torch.exp(math.log(1e-2) + (math.log(10.0) - math.log(1e-2)) * u)
    f = 2.0 * torch.rand(batch * n, generator=g, device=device, dtype=torch.float64) - 1.0
    return sigma, f


def time_candidate(n: int, batch: int, precision: int, options: dict, sigma, f, steps: int = 10,
                   max_refine: int = 1) -> float:
    """Milliseconds per implicit step (graph of `steps` solves) for one setting."""
    import torch
    plan = Plan(n, batch=batch, precision=precision, device=f.device, options=options)
    plan.factor_hyperdiff(sigma)
    x = f.clone()
    mr = max_refine if precision == PENT_F32_REFINE else 0
    plan.solve_steps(x, steps, max_refine=mr)  # capture + first run
    plan.solve_steps(x, steps, max_refine=mr)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(f.device)
    e0.record(plan.stream)
    plan.solve_steps(x, steps, max_refine=mr)
    e1.record(plan.stream)
    torch.cuda.synchronize(f.device)
    ms = e0.elapsed_time(e1) / steps
    plan.close()
    return ms


def tune(buckets: Iterable[int] = DEFAULT_BUCKETS, rows: int = 1 << 26, steps: int = 10,
         precisions: Iterable[str] = ("f64", "f32"), max_refine: int = 1, device=None, seed: int = 1807,
         log=print) -> list:
    """Rules [(kind, n_lo, n_hi, a, b, ms)] with the fastest setting of every bucket."""
    import torch
    device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    rules = []
    lo = 1
    for n in sorted(int(b) for b in buckets):
        batch = max(64, rows // n)
        sigma, f = _inputs(n, batch, device, seed + n)
        for kind in precisions:
            if kind == "f32":
                cands = [((rpt, tps), {PENT_OPT_ROWS_PER_THREAD: rpt, PENT_OPT_THREADS_PER_SYSTEM: tps,
                                       PENT_OPT_WINDOW_WARPS: 0})
                         for rpt, tps in f32_candidates(n)]
                prec = PENT_F32_REFINE
            else:
                # partitioning off: the knobs tune the thread-per-system walk, which partitioned groups
                # (long systems, or small batches) do not use
                cands = [((u, bw), {PENT_OPT_UNROLL: u, PENT_OPT_BLOCK_WARPS: bw, PENT_OPT_PARTITION_ROWS: 0,
                                    PENT_OPT_WINDOW_ROWS: 0})
                         for u, bw in f64_candidates(n)]
                prec = PENT_F64
            best = None
            for knobs, opts in cands:
                ms = time_candidate(n, batch, prec, opts, sigma, f, steps, max_refine)
                if log:
                    log(f"{kind} n={n:6d} batch={batch:6d} {knobs}: {ms:.4f} ms/step")
                if best is None or ms < best[1]:
                    best = (knobs, ms)
            a, b = best[0]
            if kind == "f32" and b == (_valid_tps(math.ceil(n / a)) or -1):
                b = 0  # the fewest threads that cover each n of the bucket
            rules.append((kind, lo, n, a, b, best[1]))
        del sigma, f
        torch.cuda.empty_cache()
        lo = n + 1
    return rules


def format_cache(rules: list, header: str = "") -> str:
    lines = ["# pentbatch tune cache v1" + (f" -- {header}" if header else ""),
             "# kind n_lo n_hi a b   (f32: rows/thread threads/system; f64: unroll warps/CTA)   ms/step"]
    for kind, lo, hi, a, b, ms in rules:
        lines.append(f"{kind} {lo} {hi} {a} {b}  # {ms:.4f}")
    # the last bucket's rule also covers longer systems
    if rules:
        last = {}
        for r in rules:
            last[r[0]] = r
        for kind, r in last.items():
            lines.append(f"{kind} {r[2] + 1} 2147483647 {r[3]} {r[4]}")
    return "\n".join(lines) + "\n"


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--buckets", default=",".join(str(b) for b in DEFAULT_BUCKETS))
    ap.add_argument("--rows", type=int, default=1 << 26, help="rows per timed batch (the scale of the workload)")
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--precisions", default="f64,f32")
    args = ap.parse_args(argv)
    import torch
    rules = tune([int(b) for b in args.buckets.split(",")], rows=args.rows, steps=args.steps,
                 precisions=args.precisions.split(","))
    text = format_cache(rules, header=torch.cuda.get_device_name())
    with open(args.out, "w") as fh:
        fh.write(text)
    print(text, end="")


if __name__ == "__main__":
    main()
