"""Benchmark of the nonlocal-operator hot path on one GB300.

Workload (one step): on the 2-D heterogeneous 1024^2 grid (variable horizon
delta = h (4 + 12 s), lognormal coefficient a(x) a(y), Gaussian random field u):
  * one direct apply  (nl_apply, FP32, gamma = C_delta |xi|^{-1.5}), and
  * one fast apply    (nl_apply_fast, Sec. 3 algorithm, p^0 = 1, same fields).
value = grid points processed per second over both applies (2 N per step), Gpts/s.

Timing: W untimed warm-up steps, then K steps timed with CUDA events on the
launching stream; the L2 is flushed (a 256 MiB write) before every timed step,
outside the events.  Rank 0 prints one JSON line.  Under torchrun every rank
runs an independent replica of the workload (the operator needs no exchange
on one GPU: replicas only); value sums the replicas over max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
FP64_NOMINAL_TFLOPS = 1.25


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        d["_source"] = "measured"
        return d
    d = dict(PEAKS_FALLBACK)
    d["_source"] = "fallback"
    return d


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0:   # first sample before timing
                time.sleep(0.02)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def build_workload(n=1024, seed=0):
    from paper_1905_08375_gb300 import synth
    return synth.heterogeneous_2d(n=n, seed=seed)


def algorithmic_counts(f, n):
    """Neighbour count of the direct sum (sum over nodes of |ball|) from the horizon field."""
    rho = f["delta"] * n
    R2 = rho * rho
    thr = np.ceil(R2) - 1.0
    rmax = int(np.ceil(rho.max()))
    o = np.arange(-rmax, rmax + 1)
    o2 = np.sort((o[:, None] ** 2 + o[None, :] ** 2).reshape(-1))
    o2 = o2[o2 > 0]
    cnt = np.searchsorted(o2, thr, side="right")
    return int(cnt.sum())


def run_gpu(args, peaks):
    import torch
    import torch.distributed as dist

    from paper_1905_08375_gb300 import binding as nl

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    n = args.n
    N = n * n
    f = build_workload(n, seed=args.seed + rank)
    direct = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_POWER, alpha=1.5,
                               coef=nl.NL_COEF_XY, a=f["a"])
    fast = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_POLY, alpha=1.5, K=0,
                             coef=nl.NL_COEF_XY, a=f["a"])
    u = torch.tensor(f["u"][0], dtype=torch.float32, device=dev)
    out_d = torch.empty_like(u)
    out_f = torch.empty_like(u)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        nl.nl_apply(direct, u, out_d)
        nl.nl_apply_fast(fast, u, out_f)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed steps (events on the launching stream, L2 flushed before each) ----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    ms_step = float(np.mean(ms))
    if ws > 1:
        t = torch.tensor([ms_step], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    value = ws * 2 * N / (ms_step * 1e-3) / 1e9

    # ---- per-kernel timing for the roofline (same stream, flushed) ----
    def time_fn(fn, reps):
        ts = []
        for r in range(reps):
            flush.fill_(float(r))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.mean(ts))

    reps = max(3, min(args.steps, 50))
    t_direct = time_fn(lambda: nl.nl_apply(direct, u, out_d), reps)
    t_fast = time_fn(lambda: nl.nl_apply_fast(fast, u, out_f), reps)
    fast_pan = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_POLY, alpha=1.5, K=0,
                                 coef=nl.NL_COEF_XY, a=f["a"], fast_variant=nl.NL_FAST_PANELS)
    fast_f64 = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_POLY, alpha=1.5, K=0,
                                 coef=nl.NL_COEF_XY, a=f["a"],
                                 fast_variant=nl.NL_FAST_FP64_PANELS)
    t_fast_pan = time_fn(lambda: nl.nl_apply_fast(fast_pan, u, out_f), reps)
    t_fast_f64 = time_fn(lambda: nl.nl_apply_fast(fast_f64, u, out_f), reps)
    nl.nl_apply_fast(fast, u, out_f)
    u64 = u.double()
    o64 = torch.empty_like(u64)
    t_direct64 = time_fn(lambda: nl.nl_apply(direct, u64, o64), max(3, reps // 2))
    nb = algorithmic_counts(f, n)
    flops_direct = 4.0 * nb                    # per neighbour: b_j g, u_j - u_i, fma
    fp32_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    achieved = flops_direct / (t_direct * 1e-3) / 1e12
    roofline = {"kernel": "k_direct_scalar<2,float,POWER,staged>", "bound": "alu",
                "achieved": round(achieved, 3), "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                "frac": round(achieved / fp32_peak, 4), "traffic": None,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                "algorithmic_flops_per_launch": flops_direct}

    # ---- end to end through the public API with host buffers ----
    uh = torch.tensor(f["u"][0], dtype=torch.float32).pin_memory()
    res_d = torch.empty(N, dtype=torch.float32).pin_memory()
    res_f = torch.empty(N, dtype=torch.float32).pin_memory()
    ud = torch.empty_like(u)
    e_ts = []
    for k in range(args.steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ud.copy_(uh, non_blocking=True)
        nl.nl_apply(direct, ud, out_d)
        nl.nl_apply_fast(fast, ud, out_f)
        res_d.copy_(out_d, non_blocking=True)
        res_f.copy_(out_f, non_blocking=True)
        b.record(stream)
        b.synchronize()
        e_ts.append(a.elapsed_time(b))
    e2e_ms = float(np.mean(e_ts))
    e2e = {"value": round(ws * 2 * N / (e2e_ms * 1e-3) / 1e9, 4), "unit": "Gpts/s",
           "h2d_bytes_per_step": N * 4, "d2h_bytes_per_step": 2 * N * 4, "ms_per_step": e2e_ms}

    result = dict(
        metric="L_delta u applies (direct + fast) in Gpts/s on the 2-D heterogeneous 1024^2 grid",
        value=round(value, 4), unit="Gpts/s", n_gpus=ws, steps=args.steps,
        warmup=args.warmup, ms_per_step=round(ms_step, 4), higher_is_better=True,
        scaling="weak", vs_baseline=None, dtype="f32 (direct) / f64 sums (fast)",
        data="synthetic",
        config={"workload": "2D heterogeneous nonlocal diffusion 1024x1024, delta=h(4+12s), "
                            "a lognormal sigma 0.5 smoothed 8h, gamma=a(x)a(y)C_delta|xi|^-1.5; "
                            "direct FP32 apply + fast (Sec. 3, K=0) apply per step",
                "n": n, "points": N, "l2": "flushed (256 MiB write) before every timed step",
                "parallelism": f"replicas x{ws}"},
        per_path_gpts={"direct_fp32": round(N / (t_direct * 1e-3) / 1e9, 4),
                       "fast_k0_rowprefix": round(N / (t_fast * 1e-3) / 1e9, 4),
                       "fast_k0_panels_int": round(N / (t_fast_pan * 1e-3) / 1e9, 4),
                       "fast_k0_panels_fp64": round(N / (t_fast_f64 * 1e-3) / 1e9, 4),
                       "direct_fp64": round(N / (t_direct64 * 1e-3) / 1e9, 4)},
        per_path_ms={"direct_fp32": round(t_direct, 4), "fast_k0_rowprefix": round(t_fast, 4),
                     "fast_k0_panels_int": round(t_fast_pan, 4),
                     "fast_k0_panels_fp64": round(t_fast_f64, 4),
                     "direct_fp64": round(t_direct64, 4)},
        roofline=roofline, e2e=e2e,
        gpu_launches=args.steps * (1 + 2 + fast.info()["levels"]),
        peaks_source=peaks["_source"],
    )
    clocks = clk.summary()
    result["clocks"] = clocks
    outs = dict(direct=out_d.double().cpu().numpy(), fast=out_f.double().cpu().numpy())
    return result, f, outs, rank, ws


def cpu_baseline(f, n, outs, budget_s=20.0):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload."""
    import oracle
    rng = np.random.default_rng(123)
    N = n * n
    t0 = time.perf_counter()
    idx = rng.choice(N, size=256, replace=False)
    ref_d = oracle.direct_scalar(f["u"][0], 2, n, f["delta"], alpha=1.5, coef=oracle.COEF_XY,
                                 a=f["a"], idx=idx)
    t1 = time.perf_counter()
    ref_f = oracle.fast_leafset(f["u"][0], 2, 10, f["delta"], K=0, alpha=1.5,
                                coef=oracle.COEF_XY, a=f["a"], idx=idx)
    t2 = time.perf_counter()
    # grow the sample to fill the budget
    per_pt = (t2 - t0) / len(idx)
    m = int(min(N, max(len(idx), budget_s / max(per_pt, 1e-9))))
    idx2 = rng.choice(N, size=m, replace=False)
    t0 = time.perf_counter()
    ref_d2 = oracle.direct_scalar(f["u"][0], 2, n, f["delta"], alpha=1.5, coef=oracle.COEF_XY,
                                  a=f["a"], idx=idx2)
    t1 = time.perf_counter()
    ref_f2 = oracle.fast_leafset(f["u"][0], 2, 10, f["delta"], K=0, alpha=1.5,
                                 coef=oracle.COEF_XY, a=f["a"], idx=idx2)
    t2 = time.perf_counter()
    pts_per_s = 2 * m / (t2 - t0)
    parity = None
    if outs is not None:
        def rel(x, r):
            return float(np.linalg.norm(x - r) / np.linalg.norm(r))
        parity = {"direct_fp32_rel_l2": rel(outs["direct"][idx2], ref_d2),
                  "fast_rel_l2": rel(outs["fast"][idx2], ref_f2), "sampled_points": m}
    return {"value": round(pts_per_s / 1e9, 9), "unit": "Gpts/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{m} random nodes of the 1024^2 workload, direct + fast leaf-set sums "
                      f"({t2 - t0:.1f} s)"}, parity


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores, bounded sample per step."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    n = args.n
    f = build_workload(n, seed=args.seed)
    rng = np.random.default_rng(7)
    m = 512
    N = n * n

    def step():
        idx = rng.choice(N, size=m, replace=False)
        oracle.direct_scalar(f["u"][0], 2, n, f["delta"], alpha=1.5, coef=oracle.COEF_XY,
                             a=f["a"], idx=idx)
        oracle.fast_leafset(f["u"][0], 2, 10, f["delta"], K=0, alpha=1.5,
                            coef=oracle.COEF_XY, a=f["a"], idx=idx)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    value = 2 * m / dt / 1e9
    line = dict(impl="reference",
                metric="L_delta u applies (direct + fast) in Gpts/s on the 2-D heterogeneous "
                       "1024^2 grid",
                value=value, unit="Gpts/s", n_gpus=ws, steps=args.steps, warmup=args.warmup,
                ms_per_step=dt * 1e3, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic",
                config={"workload": "2D heterogeneous nonlocal diffusion 1024x1024 (oracle on "
                                    f"{m} sampled nodes per step)", "n": n},
                cpu_baseline={"value": value, "unit": "Gpts/s", "cores": oracle.num_threads(),
                              "kind": "oracle",
                              "sample": f"{m} random nodes per step, direct + fast leaf-set"},
                e2e={"value": value, "unit": "Gpts/s", "h2d_bytes_per_step": 0,
                     "d2h_bytes_per_step": 0})
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return
    peaks = load_peaks()
    result, f, outs, rank, ws = run_gpu(args, peaks)
    if rank == 0:
        if ws == 1 and not args.no_cpu_baseline:
            cb, parity = cpu_baseline(f, args.n, outs)
            result["cpu_baseline"] = cb
            result["parity"] = parity
        print(json.dumps(result))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
