"""Benchmark of the nonlocal-operator hot path on one GB300.

Default workload (c2, one step): on the 2-D heterogeneous 1024^2 grid (variable horizon
delta = h (4 + 12 s), lognormal coefficient a(x) a(y), Gaussian random field u)
  * one direct apply  (nl_apply, FP32, gamma = C_delta |xi|^{-1.5}), and
  * one fast apply    (nl_apply_fast, the Sec. 3 algorithm with p^0 = 1, same fields);
value = grid points processed per second over both applies (2 N per step), Gpts/s.

Other workloads (--workload): c1 1-D FP64 direct (4096 nodes); c2k the kappa part of the
Sec. 3 splitting (kappa = s^-1.5 - p^2, direct FP32) on the c2 fields; c3 2-D peridynamics 512^2
FP32; c3b batched Jacobi-CG to 1e-8 over 64 uneven peridynamic instances 128^2..512^2 (the
operator one persistent launch over all instances; time per solve); c4 (c4_512) CG to
relative residual 1e-8 on 256^2 (512^2), 8 right-hand sides, with the learned two-level
preconditioner trained at set-up (Jacobi-CG timed beside it; time per solve); c5 3-D 256^3
with 8 right-hand sides, direct + fast FP32; ex1 / ex2 the paper's Example 1 (2-D,
delta = 1/2, 128^2) and Example 2 (1-D, K = 3, 4096 nodes), fast vs direct in FP64.

Timing: W untimed warm-up steps, then K steps timed with CUDA events on the launching stream;
the L2 is flushed (a 256 MiB write) before every timed step, outside the events.  Rank 0
prints one JSON line.  Under torchrun every rank runs an independent replica (the operator
needs no exchange on one GPU: replicas only); value sums the replicas over max-over-ranks time.
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
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12   # 80.5
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
                 "--format=csv,noheader,nounits", "-lms", "25"],
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


def ball_counts(delta, n, d):
    """Per-node number of lattice offsets 0 < |o|^2 < (delta n)^2 (the direct sum's terms)."""
    rho = np.asarray(delta) * n
    thr = np.ceil(rho * rho) - 1.0
    rmax = int(np.ceil(rho.max()))
    o = np.arange(-rmax, rmax + 1)
    grids = np.meshgrid(*([o] * d), indexing="ij")
    o2 = np.sort(sum(g.astype(np.int64) ** 2 for g in grids).reshape(-1))
    o2 = o2[o2 > 0]
    return np.searchsorted(o2, thr, side="right")


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
class Workload:
    name = ""
    metric = ""
    unit = "Gpts/s"
    higher_is_better = True
    dtype = "f32"
    launches = None

    def __init__(self, dev, seed):
        import torch
        from paper_1905_08375_gb300 import binding as nl
        self.torch, self.nl, self.dev, self.seed = torch, nl, dev, seed

    def time_fn(self, fn, reps, flush):
        torch = self.torch
        stream = torch.cuda.current_stream()
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

    def value(self, ms):
        return self.units / (ms * 1e-3) / 1e9


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the roofline
# kernel, from one ncu --set full capture of that kernel on the workload; None where no capture
# of the current kernel exists
PROFILED_TRAFFIC = {
    "k_direct2d_x2": 21.03e6,          # c2, variant <16, 2, 3>
    "k_direct2d_x2_kappa": 29.42e6,    # c2k, variant <16, 2, 3, kappa>: 29.42 MB read, 256 B written
    "k_direct_pd_x2": 9.48e6,          # c3, <8, 2>
    "k_fast_gather_slots": 178.53e6,   # c2, 174.85 MB read + 3.68 MB written (32 x 8 node tiles)
}


def _alu_roof(kernel, flops, ms, peak, src, traffic_key=None):
    ach = flops / (ms * 1e-3) / 1e12
    base = kernel.split("<")[0].split(" ")[0]           # the kernel's name without arguments
    traffic = PROFILED_TRAFFIC.get(traffic_key or base)
    return {"kernel": kernel, "bound": "alu", "achieved": round(ach, 4), "peak": round(peak, 3),
            "unit": "TFLOP/s", "frac": round(ach / peak, 4), "traffic": traffic,
            "peak_source": src}


FP32_SRC = "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (no measurement)"
FP64_SRC = "nominal FP64 1.25 TFLOP/s (profiling recipe; no measurement)"

# FMA peaks measured on the device by nl_measure_peaks before the timed region (run_gpu)
MEASURED_ALU = {}


def fp32_peak():
    """The FP32 roofline denominator: the measured FMA peak (the larger of the scalar and the
    paired f32x2 chains, as the kernels use both) or, without a measurement, the derived one."""
    if MEASURED_ALU:
        a, b = MEASURED_ALU["fp32_tflops"], MEASURED_ALU["fp32x2_tflops"]
        return max(a, b), (f"measured FMA-chain microbenchmark (nl_measure_peaks): max of scalar "
                           f"{a:.2f} and paired f32x2 {b:.2f} TFLOP/s")
    return FP32_PEAK_TFLOPS, FP32_SRC


def fp64_peak():
    if MEASURED_ALU:
        v = MEASURED_ALU["fp64_tflops"]
        return v, f"measured FMA-chain microbenchmark (nl_measure_peaks): FP64 {v:.3f} TFLOP/s"
    return FP64_NOMINAL_TFLOPS, FP64_SRC


class C2(Workload):
    """2-D heterogeneous 1024^2: direct FP32 + fast (K = 0) per step; beside the timed step the
    FP64 applies, every route of the fast algorithm and CG to 1e-8 (learned vs Jacobi) at
    256^2 are timed and checked against the oracle."""
    name = "c2"
    metric = "L_delta u applies (direct + fast) in Gpts/s on the 2-D heterogeneous 1024^2 grid"
    dtype = "f32 data; exact 64-bit integer partial sums (fast)"
    # the route of the fast algorithm the timed step uses, and the others timed beside it
    STEP_ROUTE = "panels"
    ROUTES = (("panels", "NL_FAST_PANELS", "Sec. 3 as written: Step 2 panel sums level by level, "
               "Step 3 adds the panels of Algorithm 1 one by one"),
              ("rowprefix", "NL_FAST_ROWPREFIX", "deviation (f1): per-level row prefix sums, "
               "each run of Algorithm 1's panels added as one difference"),
              ("leafrows", "NL_FAST_LEAFROWS", "deviation: the panels of Algorithm 1 tile the "
               "leaf cells meeting the ball, so each leaf row of the ball is one difference of "
               "leaf-row prefix sums; the coarse levels are not formed"))
    FAST_BYTES_PER_NODE = 27        # u 4 + b 4 + out 4 + plan 4 + the pyramid written and read

    def setup(self, n=1024):
        nl, torch = self.nl, self.torch
        from paper_1905_08375_gb300 import synth
        self.n = n
        self.f = synth.heterogeneous_2d(n=n, seed=self.seed)
        f = self.f
        self.direct = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_POWER, alpha=1.5,
                                        coef=nl.NL_COEF_XY, a=f["a"])
        # every route of the Sec. 3 sums (bitwise equal outputs)
        self.fast_routes = {
            name: nl.nl_plan_create(2, n, f["delta"], family=nl.NL_POLY, alpha=1.5, K=0,
                                    coef=nl.NL_COEF_XY, a=f["a"],
                                    fast_variant=getattr(nl, const))
            for name, const, _ in self.ROUTES}
        self.fast = self.fast_routes[self.STEP_ROUTE]
        # the symmetrised (divergence-type) fast operator on the same fields (f4)
        self.fast_sym = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_POLY, alpha=1.5, K=0,
                                          coef=nl.NL_COEF_XY, a=f["a"], symmetric=True)
        # and with the polynomial p^4 (K = 2): two-limb integer coefficients of the target column
        self.fast_sym_k2 = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_POLY, alpha=1.5,
                                             K=2, coef=nl.NL_COEF_XY, a=f["a"], symmetric=True)
        self.u = torch.tensor(f["u"][0], dtype=torch.float32, device=self.dev)
        self.out_d = torch.empty_like(self.u)
        self.out_f = torch.empty_like(self.u)
        self.u64 = torch.tensor(f["u"][0], dtype=torch.float64, device=self.dev)
        self.out_d64 = torch.empty_like(self.u64)
        self.out_f64 = torch.empty_like(self.u64)
        self.units = 2 * n * n
        self.launches = 1 + 3             # direct; fast: bounds, fused Step 2, gather
        self.config = {"workload": "2D heterogeneous nonlocal diffusion 1024x1024, "
                                   "delta=h(4+12s), a lognormal sigma 0.5 smoothed 8h, "
                                   "gamma=a(x)a(y)C_delta|xi|^-1.5; direct FP32 apply + fast "
                                   "(Sec. 3, K=0, p=1, Algorithm 1 panel by panel) apply per "
                                   "step", "n": n, "points": n * n,
                       "fast_route": self.STEP_ROUTE}
        # CG on the symmetrised operator at 256^2 (the second half of the metric): the learned
        # preconditioner is trained here, before any timing
        self.cg = C4(self.dev, self.seed)
        self.cg.peaks = getattr(self, "peaks", None)
        self.cg.setup()
        # the two applies of a step are independent: the fast one runs on a second stream
        self.side = torch.cuda.Stream(device=self.dev)
        self.fork = torch.cuda.Event()
        self.join = torch.cuda.Event()
        self.config["streams"] = "direct and fast applies on two streams, joined per step"

    def _both(self, u, out_d, out_f, after_direct=None):
        torch, nl = self.torch, self.nl
        main = torch.cuda.current_stream()
        self.fork.record(main)
        self.side.wait_event(self.fork)
        nl.nl_apply(self.direct, u, out_d)
        if after_direct is not None:
            after_direct()
        nl.nl_apply_fast(self.fast, u, out_f, stream=self.side)
        self.join.record(self.side)
        main.wait_event(self.join)

    def step(self):
        self._both(self.u, self.out_d, self.out_f)

    def step_sequential(self):
        self.nl.nl_apply(self.direct, self.u, self.out_d)
        self.nl.nl_apply_fast(self.fast, self.u, self.out_f)

    def kernels(self, flush, reps):
        nl = self.nl
        n = self.n
        N = n * n
        pk = self.peaks["hbm_gbs"]
        t_direct = self.time_fn(lambda: nl.nl_apply(self.direct, self.u, self.out_d), reps, flush)
        t_seq = self.time_fn(self.step_sequential, reps, flush)
        per = {"direct_fp32_ms": round(t_direct, 4),
               "direct_gpts": round(N / (t_direct * 1e-3) / 1e9, 4),
               "step_one_stream_ms": round(t_seq, 4)}
        routes = {}
        for name, const, what in self.ROUTES:
            plan = self.fast_routes[name]
            nl.nl_plan_profile(plan, True)
            t = self.time_fn(lambda: nl.nl_apply_fast(plan, self.u, self.out_f), min(reps, 40),
                             flush)
            prof = nl.nl_plan_profile_read(plan)
            nl.nl_plan_profile(plan, False)
            k = max(prof["applies"], 1)
            # bytes: inputs, outputs, plan data and the pyramid (27 B per node), plus the
            # stored decomposition where the route reads one (the panel route)
            ach = (self.FAST_BYTES_PER_NODE * N + plan.info()["step1_bytes"]) / (t * 1e-3) / 1e9
            routes[name] = {"variant": const, "what": what, "ms": round(t, 4),
                            "step2_ms": round(prof["step2_ms"] / k, 4),
                            "step3_ms": round(prof["step3_ms"] / k, 4),
                            "gpts": round(N / (t * 1e-3) / 1e9, 4),
                            "hbm_frac": round(ach / pk, 4),
                            "paper_algorithm": name == "panels"}
        per["fast_routes"] = routes
        per["fast_route_timed_in_step"] = self.STEP_ROUTE
        per["fast_ms"] = routes[self.STEP_ROUTE]["ms"]
        per["fast_gpts"] = routes[self.STEP_ROUTE]["gpts"]
        per["fast_hbm_bytes_per_node"] = (f"{self.FAST_BYTES_PER_NODE} (u 4, b 4, out 4, plan "
                                          "4, pyramid 8 written + 8 read, coarse levels 1/3)")
        o_sym = self.torch.empty_like(self.u)
        t_sym = self.time_fn(lambda: nl.nl_apply_fast(self.fast_sym, self.u, o_sym),
                             min(reps, 20), flush)
        per["fast_sym_fp32_ms"] = round(t_sym, 4)
        t_sym2 = self.time_fn(lambda: nl.nl_apply_fast(self.fast_sym_k2, self.u, o_sym),
                              min(reps, 10), flush)
        per["fast_sym_K2_fp32_ms"] = round(t_sym2, 4)
        per["fast_sym_note"] = ("symmetrised leaf-set operator (K = 0): one-sided fast apply "
                                "(leaf rows) + transpose scatter into per-row difference "
                                "arrays with 64-bit integer atomics + row prefix sums")
        # FP64 data: the direct sum in FP64 and the fast apply with FP64 panel sums
        t_d64 = self.time_fn(lambda: nl.nl_apply(self.direct, self.u64, self.out_d64),
                             min(reps, 10), flush)
        t_f64 = self.time_fn(lambda: nl.nl_apply_fast(self.fast, self.u64, self.out_f64),
                             min(reps, 10), flush)
        per.update({"direct_fp64_ms": round(t_d64, 4), "fast_fp64_ms": round(t_f64, 4),
                    "direct_fp64_gpts": round(N / (t_d64 * 1e-3) / 1e9, 4),
                    "fast_fp64_gpts": round(N / (t_f64 * 1e-3) / 1e9, 4)})
        nl.nl_apply(self.direct, self.u64, self.out_d64)
        nl.nl_apply_fast(self.fast, self.u64, self.out_f64)
        nl.nl_apply(self.direct, self.u, self.out_d)
        nl.nl_apply_fast(self.fast, self.u, self.out_f)
        # CG to relative residual 1e-8, learned two-level preconditioner vs Jacobi
        _, cgp = self.cg.kernels(flush, 3)
        per["cg_256_8rhs"] = dict(cgp)
        nb = float(ball_counts(self.f["delta"], n, 2).sum())
        flops = 4.0 * nb
        t_fast = routes[self.STEP_ROUTE]["ms"]
        step1 = self.fast.info()["step1_bytes"]
        per["fast_panels_step1_bytes"] = step1
        if t_direct >= t_fast:
            roof = _alu_roof("k_direct2d_x2<16,TY> (direct FP32)", flops, t_direct, *fp32_peak())
            roof["algorithmic_per_launch"] = f"{flops:.4g} flop (4 per neighbour term)"
        else:
            # the dominant kernel is the panel route's Step 3 gather: it reads the stored
            # decomposition (Step 1 output, step1 bytes), the pyramid (8 B x 4/3 per node) and
            # u 4 + selfQ 8 + Fh 4 per node, and writes Lu 4 per node
            t_s3 = routes[self.STEP_ROUTE]["step3_ms"]
            byts = step1 + (8.0 * 4.0 / 3.0 + 20.0) * N
            ach = byts / (t_s3 * 1e-3) / 1e9
            roof = {"kernel": "k_fast_gather_slots (Step 3 of the panel route)",
                    "bound": "hbm", "achieved": round(ach, 2), "peak": pk, "unit": "GB/s",
                    "frac": round(ach / pk, 4),
                    "traffic": PROFILED_TRAFFIC.get("k_fast_gather_slots"),
                    "peak_source": f"{self.peaks['_source']} hbm_gbs",
                    "algorithmic_per_launch": f"{byts:.4g} B ({step1:.4g} B of stored "
                                              "decomposition + 30.7 B per node)"}
        return roof, per

    def e2e(self, flush, steps):
        torch, nl = self.torch, self.nl
        N = self.n * self.n
        uh = torch.tensor(self.f["u"][0], dtype=torch.float32).pin_memory()
        rd = torch.empty(N, dtype=torch.float32).pin_memory()
        rf = torch.empty(N, dtype=torch.float32).pin_memory()
        ud = torch.empty_like(self.u)

        def one():
            ud.copy_(uh, non_blocking=True)
            # the direct result's copy back overlaps the fast apply
            self._both(ud, self.out_d, self.out_f,
                       after_direct=lambda: rd.copy_(self.out_d, non_blocking=True))
            rf.copy_(self.out_f, non_blocking=True)
        ms = self.time_fn(one, steps, flush)
        return {"value": round(self.value(ms), 4), "unit": self.unit, "h2d_bytes_per_step": N * 4,
                "d2h_bytes_per_step": 2 * N * 4, "ms_per_step": round(ms, 4)}

    def outputs(self):
        return {"direct": self.out_d.double().cpu().numpy(),
                "fast": self.out_f.double().cpu().numpy(),
                "direct_fp64": self.out_d64.cpu().numpy(),
                "fast_fp64": self.out_f64.cpu().numpy(),
                "cg": self.cg.outputs()}

    @staticmethod
    def oracle_step(f, n, idx):
        import oracle
        d = oracle.direct_scalar(f["u"][0], 2, n, f["delta"], alpha=1.5, coef=oracle.COEF_XY,
                                 a=f["a"], idx=idx)
        fs = oracle.fast_leafset(f["u"][0], 2, int(np.log2(n)), f["delta"], K=0, alpha=1.5,
                                 coef=oracle.COEF_XY, a=f["a"], idx=idx)
        return {"direct": d, "fast": fs}, 2 * len(idx)


class C2K(Workload):
    """The kappa part of the splitting of Sec. 3 on the 2-D heterogeneous 1024^2 fields: one
    direct FP32 apply with kappa(s) = s^-1.5 - p^2(s) (K = 1) per step."""
    name = "c2k"
    metric = ("L_delta u kappa-part direct apply (Sec. 3 splitting, K=1) in Gpts/s on the 2-D "
              "heterogeneous 1024^2 grid")

    def setup(self, n=1024):
        nl, torch = self.nl, self.torch
        from paper_1905_08375_gb300 import synth
        self.n = n
        self.f = synth.heterogeneous_2d(n=n, seed=self.seed)
        f = self.f
        self.plan = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_KAPPA, alpha=1.5, K=1,
                                      coef=nl.NL_COEF_XY, a=f["a"])
        self.u = torch.tensor(f["u"][0], dtype=torch.float32, device=self.dev)
        self.out = torch.empty_like(self.u)
        self.units = n * n
        self.launches = 1
        self.config = {"workload": "2D heterogeneous nonlocal diffusion 1024x1024, "
                                   "delta=h(4+12s), a lognormal sigma 0.5 smoothed 8h, "
                                   "kappa(s)=s^-1.5-(7/4-3/4 s^2) inside the ball (the Sec. 3 "
                                   "splitting remainder, K=1), C=a(x)a(y); direct FP32 apply",
                       "n": n, "points": n * n}

    def step(self):
        self.nl.nl_apply(self.plan, self.u, self.out)

    def kernels(self, flush, reps):
        t = self.time_fn(self.step, reps, flush)
        nb = float(ball_counts(self.f["delta"], self.n, 2).sum())
        # per term: t = o2/R2, p = p0 + p1 t, ra g - p, times b_j, u_j - u_i, times, add
        roof = _alu_roof("k_direct2d_x2<16,TY,MB,kappa> (paired columns, per-output weights)",
                         9.0 * nb, t, *fp32_peak(), traffic_key="k_direct2d_x2_kappa")
        roof["algorithmic_per_launch"] = f"{9 * nb:.4g} flop (9 per neighbour term)"
        return roof, {"kappa_direct_fp32_ms": round(t, 4)}

    def e2e(self, flush, steps):
        torch = self.torch
        N = self.n * self.n
        uh = torch.tensor(self.f["u"][0], dtype=torch.float32).pin_memory()
        rh = torch.empty(N, dtype=torch.float32).pin_memory()
        ud = torch.empty_like(self.u)

        def one():
            ud.copy_(uh, non_blocking=True)
            self.nl.nl_apply(self.plan, ud, self.out)
            rh.copy_(self.out, non_blocking=True)
        ms = self.time_fn(one, steps, flush)
        return {"value": round(self.value(ms), 4), "unit": self.unit, "h2d_bytes_per_step": N * 4,
                "d2h_bytes_per_step": N * 4, "ms_per_step": round(ms, 4)}

    def outputs(self):
        return {"kappa": self.out.double().cpu().numpy()}

    @staticmethod
    def oracle_step(f, n, idx):
        import oracle
        return {"kappa": oracle.direct_scalar(f["u"][0], 2, n, f["delta"], family=oracle.KAPPA,
                                              alpha=1.5, K=1, coef=oracle.COEF_XY, a=f["a"],
                                              idx=idx)}, len(idx)


class C1(Workload):
    name = "c1"
    metric = "1-D nonlocal diffusion direct apply (FP64) in Gpts/s, N=4096, delta=0.05"
    dtype = "f64"

    def setup(self):
        nl, torch = self.nl, self.torch
        from paper_1905_08375_gb300 import synth
        self.n = 4096
        self.f = synth.diffusion_1d(n=4096, delta=0.05, seed=self.seed)
        self.plan = nl.nl_plan_create(1, 4096, 0.05, family=nl.NL_POWER, alpha=0.0)
        self.u = torch.tensor(self.f["u"], dtype=torch.float64, device=self.dev)
        self.out = torch.empty_like(self.u)
        self.units = 4096
        self.launches = 1
        self.config = {"workload": "1D nonlocal diffusion, N=4096, delta=0.05, gamma=3/delta^3, "
                                   "u=sin(2 pi x)+0.01 N(0,1), FP64 direct apply", "n": 4096}

    def step(self):
        self.nl.nl_apply(self.plan, self.u, self.out)

    def kernels(self, flush, reps):
        t = self.time_fn(self.step, reps, flush)
        nb = float(ball_counts(self.f["delta"], self.n, 1).sum())
        roof = _alu_roof("k_direct_split<1,double,POWER>", 4.0 * nb, t, *fp64_peak())
        roof["algorithmic_per_launch"] = f"{4 * nb:.4g} flop (4 per term)"
        return roof, {"direct_fp64_ms": round(t, 4)}

    def e2e(self, flush, steps):
        torch = self.torch
        uh = torch.tensor(self.f["u"], dtype=torch.float64).pin_memory()
        rh = torch.empty(self.n, dtype=torch.float64).pin_memory()
        ud = torch.empty_like(self.u)

        def one():
            ud.copy_(uh, non_blocking=True)
            self.nl.nl_apply(self.plan, ud, self.out)
            rh.copy_(self.out, non_blocking=True)
        ms = self.time_fn(one, steps, flush)
        return {"value": round(self.value(ms), 6), "unit": self.unit,
                "h2d_bytes_per_step": self.n * 8, "d2h_bytes_per_step": self.n * 8,
                "ms_per_step": round(ms, 4)}

    def outputs(self):
        return {"direct": self.out.cpu().numpy()}

    @staticmethod
    def oracle_step(f, n, idx):
        import oracle
        return {"direct": oracle.direct_scalar(f["u"], 1, n, 0.05, alpha=0.0, idx=idx)}, len(idx)


class C3(Workload):
    name = "c3"
    metric = "2-D linear bond-based peridynamics direct apply (FP32) in Gpts/s, 512^2, delta=8h"

    def setup(self):
        nl, torch = self.nl, self.torch
        from paper_1905_08375_gb300 import synth
        self.n = 512
        self.f = synth.pd_2d(n=512, seed=self.seed)
        f = self.f
        self.plan = nl.nl_plan_create(2, 512, f["delta"], family=nl.NL_PD_BOND,
                                      coef=nl.NL_COEF_MEAN, a=f["c"])
        self.u = torch.tensor(f["u"], dtype=torch.float32, device=self.dev)
        self.out = torch.empty_like(self.u)
        self.out_f = torch.empty_like(self.u)
        # the same fields with a four times larger horizon (32h): the fast path's cost grows
        # like the horizon, the direct sum's like its square
        self.plan32 = nl.nl_plan_create(2, 512, 4.0 * f["delta"], family=nl.NL_PD_BOND,
                                        coef=nl.NL_COEF_MEAN, a=f["c"])
        # the fast path with the polynomial micromodulus p^4 (K = 2) matched to s^-3
        self.plan_k2 = nl.nl_plan_create(2, 512, f["delta"], family=nl.NL_PD_BOND,
                                         coef=nl.NL_COEF_MEAN, a=f["c"], K=2)
        self.out_k2 = torch.empty_like(self.u)
        # the 3-D fast path (K = 0) on a 128^3 two-phase grid with delta = 4h
        rng = np.random.default_rng(self.seed + 7)
        n3 = 128
        c3 = synth.voronoi_phase(rng, 3, n3)
        u3 = np.stack([synth.gaussian_field(rng, 3, n3).reshape(-1) for _ in range(3)])
        self.plan3 = nl.nl_plan_create(3, n3, 4.0 / n3, family=nl.NL_PD_BOND,
                                       coef=nl.NL_COEF_MEAN, a=c3)
        self.u3 = torch.tensor(u3, dtype=torch.float32, device=self.dev)
        self.out3 = torch.empty_like(self.u3)
        self.units = 512 * 512
        self.launches = 1
        self.config = {"workload": "2D linear bond-based PD, 512x512, delta=8h, micromodulus "
                                   "c(x,y) xi xi^T/|xi|^3, two-phase Voronoi (64 cells, c in "
                                   "{1,10}), FP32 apply with FP64 accumulation", "n": 512}

    def step(self):
        self.nl.nl_apply(self.plan, self.u, self.out)

    def kernels(self, flush, reps):
        t = self.time_fn(self.step, reps, flush)
        t_f = self.time_fn(lambda: self.nl.nl_apply_fast(self.plan, self.u, self.out_f), reps,
                           flush)
        o32 = self.torch.empty_like(self.u)
        t_d32 = self.time_fn(lambda: self.nl.nl_apply(self.plan32, self.u, o32), reps, flush)
        t_f32 = self.time_fn(lambda: self.nl.nl_apply_fast(self.plan32, self.u, o32), reps, flush)
        t_k2 = self.time_fn(lambda: self.nl.nl_apply_fast(self.plan_k2, self.u, self.out_k2),
                            reps, flush)
        t_3 = self.time_fn(lambda: self.nl.nl_apply_fast(self.plan3, self.u3, self.out3), reps,
                           flush)
        nb = float(ball_counts(self.f["delta"], self.n, 2).sum())
        roof = _alu_roof("k_direct_pd_x2<8,2> (paired columns)", 14.0 * nb, t, *fp32_peak())
        roof["algorithmic_per_launch"] = f"{14 * nb:.4g} flop (14 per bond)"
        return roof, {"pd_fp32_ms": round(t, 4), "pd_fast_deg0_fp32_ms": round(t_f, 4),
                      "pd_delta32h_direct_fp32_ms": round(t_d32, 4),
                      "pd_delta32h_fast_deg0_fp32_ms": round(t_f32, 4),
                      "pd_fast_poly_K2_fp32_ms": round(t_k2, 4),
                      "pd3d_128_delta4h_fast_deg0_fp32_ms": round(t_3, 4),
                      "pd3d_128_delta4h_fast_gpts": round(128 ** 3 / t_3 / 1e6, 4),
                      "pd_fast_note": "nl_apply_fast on the PD plan: degree-0 bond tensor "
                                      "xi xi^T / delta^3 over the leaf set (a different "
                                      "operator), exact 64-bit leaf-row moment sums"}

    def e2e(self, flush, steps):
        torch = self.torch
        uh = torch.tensor(self.f["u"], dtype=torch.float32).pin_memory()
        rh = torch.empty_like(uh).pin_memory()
        ud = torch.empty_like(self.u)

        def one():
            ud.copy_(uh, non_blocking=True)
            self.nl.nl_apply(self.plan, ud, self.out)
            rh.copy_(self.out, non_blocking=True)
        ms = self.time_fn(one, steps, flush)
        b = int(uh.numel()) * 4
        return {"value": round(self.value(ms), 4), "unit": self.unit, "h2d_bytes_per_step": b,
                "d2h_bytes_per_step": b, "ms_per_step": round(ms, 4)}

    def outputs(self):
        return {"pd": self.out.double().cpu().numpy().reshape(2, -1),
                "pd_fast": self.out_f.double().cpu().numpy().reshape(2, -1),
                "pd_fast_k2": self.out_k2.double().cpu().numpy().reshape(2, -1)}

    @staticmethod
    def oracle_step(f, n, idx):
        import oracle
        return {"pd": oracle.pd_direct(f["u"], 2, n, f["delta"], f["c"], idx=idx)[0],
                "pd_fast": oracle.fast_pd_leafset(f["u"][0], 2, 9, f["delta"], f["c"],
                                                  idx=idx),
                "pd_fast_k2": oracle.fast_pd_leafset(f["u"][0], 2, 9, f["delta"], f["c"], K=2,
                                                     idx=idx)}, 2 * len(idx)


class C3B(Workload):
    """64 uneven peridynamic instances, 128^2 .. 512^2: batched Jacobi-CG to 1e-8 per step."""
    name = "c3b"
    metric = ("batched CG time to relative residual 1e-8 (FP64 true residual, worst instance) "
              "over 64 uneven 2-D peridynamic instances 128^2..512^2, ms")
    unit = "ms"
    higher_is_better = False
    dtype = "f32 operator, f64 vectors and reductions"

    def setup(self, count=64):
        nl, torch = self.nl, self.torch
        from paper_1905_08375_gb300 import synth
        self.sizes = synth.pd_batch_sizes(count, 128, 512)
        self.inst = []
        for k, n in enumerate(self.sizes):
            f = synth.pd_2d(n=n, seed=self.seed * 1000 + k, radius_cells=8)
            self.inst.append((n, f["delta"], f["c"], f["u"][0].reshape(-1)))
        self.batch = nl.nl_batch_create([(n, d, c) for n, d, c, _ in self.inst],
                                        family=nl.NL_PD_BOND, coef=nl.NL_COEF_MEAN,
                                        tile_shape=nl.NL_TILE_AUTO)
        self.rhs = np.concatenate([u for *_, u in self.inst])
        self.fr = torch.tensor(self.rhs, dtype=torch.float64, device=self.dev)
        self.x = torch.empty_like(self.fr)
        self.units = 1
        self.points = int(sum(n * n for n in self.sizes))
        self.config = {"workload": "64 uneven 2D linear bond-based PD instances, n_k = 128 + "
                                   "round(384 k/63), delta=8h, two-phase Voronoi c in {1,10}; "
                                   "one batched Jacobi-CG to rtol 1e-8 (FP64 true residual) per "
                                   "step, operator = one persistent launch over all instances",
                       "instances": count, "points": self.points,
                       "tile_shape": ["32x4", "32x8", "32x16"][self.batch.tile_shape]}
        self.last = None

    def step(self):
        self.last = self.nl.nl_batch_cg_solve(self.batch, self.fr, self.x, rtol=1e-8,
                                              maxit=100000)

    def value(self, ms):
        return ms

    def kernels(self, flush, reps):
        torch, nl = self.torch, self.nl
        u = torch.randn(self.batch.total, device=self.dev)
        o = torch.empty_like(u)
        t = self.time_fn(lambda: nl.nl_batch_apply(self.batch, u, o), reps, flush)
        nb = float(sum(ball_counts(d, n, 2).sum() for n, d, _, _ in self.inst))
        if self.last:
            self.launches = 5 * self.last["iterations"] + 8
        roof = _alu_roof("k_batch_pdx2<8,TY> (all 64 instances, one launch)",
                         14.0 * nb, t, *fp32_peak())
        roof["algorithmic_per_launch"] = f"{14 * nb:.4g} flop (14 per bond, all instances)"
        return roof, {"batch_apply_fp32_ms": round(t, 4),
                      "batch_apply_gpts_s": round(self.points / (t * 1e-3) / 1e9, 3),
                      "cg": self.last}

    def e2e(self, flush, steps):
        torch = self.torch
        fh = torch.tensor(self.rhs, dtype=torch.float64).pin_memory()
        xh = torch.empty_like(fh).pin_memory()
        fd = torch.empty_like(self.fr)

        def one():
            fd.copy_(fh, non_blocking=True)
            self.nl.nl_batch_cg_solve(self.batch, fd, self.x, rtol=1e-8, maxit=100000)
            xh.copy_(self.x, non_blocking=True)
        ms = self.time_fn(one, max(1, steps), flush)
        b = int(fh.numel()) * 8
        return {"value": round(ms, 4), "unit": "ms", "h2d_bytes_per_step": b,
                "d2h_bytes_per_step": b, "ms_per_step": round(ms, 4)}

    def outputs(self):
        return {"x": self.x.cpu().numpy()}


class C4(Workload):
    """Batched CG on -L u = f with the learned two-level preconditioner (trained at set-up on
    pairs from the method's own Jacobi-CG runs), Jacobi-CG timed beside it."""
    name = "c4"
    unit = "ms"
    higher_is_better = False
    dtype = "f32 operator, f64 vectors and reductions, bf16 network weights"
    N_DEFAULT = 256

    def setup(self, nrhs=8):
        nl, torch = self.nl, self.torch
        from paper_1905_08375_gb300 import precond, synth
        n = self.n = self.N_DEFAULT
        self.nrhs = nrhs
        self.metric = (f"batched CG time to relative residual 1e-8 (FP64 true residual) on "
                       f"-L u = f, {nrhs} right-hand sides, {n}^2, learned two-level "
                       f"preconditioner, ms")
        self.f = synth.heterogeneous_2d(n=n, seed=self.seed)
        f = self.f
        self.plan = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_POWER, alpha=1.5,
                                      coef=nl.NL_COEF_XY, a=f["a"], symmetric=True)
        self.rhs = synth.cg_rhs(n, seed=self.seed + 1, count=nrhs)
        self.fr = torch.tensor(self.rhs, dtype=torch.float64, device=self.dev)
        self.x = torch.empty_like(self.fr)
        # training (set-up, not timed): (r, e) pairs from Jacobi-CG runs of 64 other
        # right-hand sides, 20k field samples of the energy-norm loss
        t0 = time.perf_counter()
        xp, ep = precond.collect_pairs(self.plan, n, seeds=range(1000, 1064), cap=64)
        t1 = time.perf_counter()
        self.net = nl.nl_net_create(precond.init_weights(0, two_level=True))
        block = precond.coarse_block(n)
        nl.nl_net_set_coarse(self.net, block)
        hist = precond.train_energy(self.net, self.plan, xp, ep, pairs=20000, batch=8, lr=3e-3,
                                    log_every=500)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        nl.nl_plan_set_net(self.plan, self.net)
        self.train_info = {"pair_fields": int(xp.shape[0]), "samples": 20000, "block": block,
                           "coarse_cells": (-(-n // block)) ** 2,
                           "collect_s": round(t1 - t0, 2), "train_s": round(t2 - t1, 2),
                           "loss_first_last": [round(hist[0][2], 4), round(hist[-1][2], 4)]}
        del xp, ep
        self.units = 1
        self.config = {"workload": f"CG on -L u = f, {n}x{n}, kernel and horizon of the 2-D "
                                   "heterogeneous workload symmetrised (divergence form), "
                                   f"{nrhs} Gaussian random field right-hand sides solved "
                                   "together, rtol 1e-8 (FP64 true residual); preconditioner "
                                   "M = D^-1 + gamma P K^T K R with K the 3-layer 32-channel "
                                   "conv net (bf16 weights) on a coarse grid", "n": n,
                       "rhs": nrhs}
        self.last = None

    def solve(self, pc):
        return self.nl.nl_cg_solve(self.plan, self.fr, self.x, rtol=1e-8, maxit=100000,
                                   precond=pc)

    def step(self):
        self.last = self.solve(self.nl.NL_PRECOND_LEARNED)

    def value(self, ms):
        return ms

    def kernels(self, flush, reps):
        nl = self.nl
        reps = max(3, min(reps, 10))
        sj = self.solve(nl.NL_PRECOND_JACOBI)
        self.jacobi_its = sj["iterations"]
        self.x_jacobi = self.x.clone()
        t_j = self.time_fn(lambda: self.solve(nl.NL_PRECOND_JACOBI), reps, flush)
        t_l = self.time_fn(lambda: self.solve(nl.NL_PRECOND_LEARNED), reps, flush)
        u = self.torch.randn(self.n * self.n, device=self.dev)
        o = self.torch.empty_like(u)
        t = self.time_fn(lambda: nl.nl_apply(self.plan, u, o), reps, flush)
        # the pieces of one iteration for all right-hand sides: operator and preconditioner
        r8 = self.torch.randn(self.nrhs, self.n * self.n, device=self.dev, dtype=self.torch.float64)
        z8 = self.torch.empty_like(r8)
        u8 = r8.float()
        o8 = self.torch.empty_like(u8)
        t_op8 = self.time_fn(lambda: nl.nl_apply(self.plan, u8, o8), reps, flush)
        t_net8 = self.time_fn(lambda: nl.nl_net_apply(self.net, self.plan, r8, z8), reps, flush)
        # the FP64 operator of the true-residual checks (all right-hand sides in one launch)
        t_op64 = self.time_fn(lambda: nl.nl_apply(self.plan, r8, z8), reps, flush)
        t_opp = self.time_fn(lambda: nl.nl_apply(self.plan, r8, z8, pairs=True), reps, flush)
        nb = float(ball_counts(self.f["delta"], self.n, 2).sum())
        self.launches = None
        # the operator as CG applies it: all right-hand sides in one launch
        kname = "k_direct2d_x2r" if self.nrhs >= 2 else "k_direct2d_x2s"
        roof = _alu_roof(f"{kname} (symmetric CG operator, {self.nrhs} RHS)",
                         6.0 * nb * self.nrhs, t_op8, *fp32_peak())
        roof["algorithmic_per_launch"] = (f"{6 * nb * self.nrhs:.4g} flop (6 per one-sided ball "
                                          f"term, {self.nrhs} RHS)")
        sl = self.solve(nl.NL_PRECOND_LEARNED)     # leave the learned solution in x
        return roof, {"learned_ms": round(t_l, 3), "learned": sl,
                      "jacobi_ms": round(t_j, 3), "jacobi": sj,
                      "learned_speedup_over_jacobi": round(t_j / t_l, 3),
                      "sym_apply_fp32_ms": round(t, 4),
                      f"sym_apply_fp32_{self.nrhs}rhs_ms": round(t_op8, 4),
                      f"learned_precond_apply_{self.nrhs}rhs_ms": round(t_net8, 4),
                      f"sym_apply_fp64_{self.nrhs}rhs_ms": round(t_op64, 4),
                      f"sym_apply_fp64_pairs_{self.nrhs}rhs_ms": round(t_opp, 4),
                      "training": self.train_info}

    def e2e(self, flush, steps):
        torch = self.torch
        fh = torch.tensor(self.rhs, dtype=torch.float64).pin_memory()
        xh = torch.empty_like(fh).pin_memory()
        fd = torch.empty_like(self.fr)

        def one():
            fd.copy_(fh, non_blocking=True)
            self.nl.nl_cg_solve(self.plan, fd, self.x, rtol=1e-8, maxit=100000,
                                precond=self.nl.NL_PRECOND_LEARNED)
            xh.copy_(self.x, non_blocking=True)
        ms = self.time_fn(one, max(1, min(steps, 10)), flush)
        b = int(fh.numel()) * 8
        return {"value": round(ms, 4), "unit": "ms", "h2d_bytes_per_step": b,
                "d2h_bytes_per_step": b, "ms_per_step": round(ms, 4)}

    def outputs(self):
        out = {"x": self.x.cpu().numpy()}
        if getattr(self, "x_jacobi", None) is not None:
            out["x_jacobi"] = self.x_jacobi.cpu().numpy()
        return out


class C4L(C4):
    """The same at 512^2."""
    name = "c4_512"
    N_DEFAULT = 512


class C5(Workload):
    name = "c5"
    metric = ("3-D nonlocal diffusion 256^3 x 8 right-hand sides, direct + fast applies (FP32) "
              "in Gpts/s")

    def setup(self):
        nl, torch = self.nl, self.torch
        from paper_1905_08375_gb300 import synth
        n = self.n = getattr(self, "size", None) or 256
        self.f = synth.diffusion_3d(n=n, seed=self.seed, nrhs=8, radius_cells=4)
        f = self.f
        self.direct = nl.nl_plan_create(3, n, f["delta"], family=nl.NL_POWER, alpha=1.0,
                                        coef=nl.NL_COEF_XY, a=f["a"])
        self.fast = nl.nl_plan_create(3, n, f["delta"], family=nl.NL_POLY, alpha=1.0, K=0,
                                      coef=nl.NL_COEF_XY, a=f["a"])
        self.u = torch.tensor(f["u"], dtype=torch.float32, device=self.dev)
        self.out_d = torch.empty_like(self.u)
        self.out_f = torch.empty_like(self.u)
        self.units = 2 * 8 * n ** 3
        self.launches = 1 + 8 * 3
        self.config = {"workload": f"3D nonlocal diffusion {n}^3, delta=4h, a lognormal sigma "
                                   "0.3, gamma=a(x)a(y)C_delta/|xi|, 8 RHS; direct + fast (K=0) "
                                   "FP32 applies per step", "n": n, "rhs": 8}

    def step(self):
        self.nl.nl_apply(self.direct, self.u, self.out_d)
        self.nl.nl_apply_fast(self.fast, self.u, self.out_f)

    def kernels(self, flush, reps):
        nl = self.nl
        t_d = self.time_fn(lambda: nl.nl_apply(self.direct, self.u, self.out_d), reps, flush)
        nl.nl_plan_profile(self.fast, True)
        t_f = self.time_fn(lambda: nl.nl_apply_fast(self.fast, self.u, self.out_f), reps, flush)
        prof = nl.nl_plan_profile_read(self.fast)
        nl.nl_plan_profile(self.fast, False)
        n = self.n
        N = n ** 3
        k = max(prof["applies"], 1)
        s2 = prof["step2_ms"] / k
        # Step 2 of the 8 right-hand sides: per right-hand side u (4) read and the 64-bit
        # leaf-row prefix (8) written, and the coefficient b (4) read once: 100 B per node
        s2_bytes = (8 * 12.0 + 4.0) * N
        s2_ach = s2_bytes / (s2 * 1e-3) / 1e9
        nb = 8.0 * float(ball_counts(np.full(1, 4.0 / n), n, 3)[0]) * n ** 3
        roof = _alu_roof("k_direct3d_x2<4,4> (slab sweep)", 4.0 * nb, t_d,
                         *fp32_peak())
        roof["algorithmic_per_launch"] = f"{4 * nb:.4g} flop (4 per term, 8 RHS)"
        return roof, {"direct_fp32_8rhs_ms": round(t_d, 4), "fast_fp32_8rhs_ms": round(t_f, 4),
                      "fast_step2_8rhs_ms": round(s2, 4),
                      "fast_step3_8rhs_ms": round(prof["step3_ms"] / k, 4),
                      "fast_step2_hbm_gbs": round(s2_ach, 1),
                      "fast_step2_hbm_frac": round(s2_ach / self.peaks["hbm_gbs"], 4),
                      "fast_step2_bytes": f"{s2_bytes:.4g} (per node: 12 B per right-hand side + 4 B "
                                          "of b)"}

    def e2e(self, flush, steps):
        torch = self.torch
        uh = torch.tensor(self.f["u"], dtype=torch.float32).pin_memory()
        rd = torch.empty_like(uh).pin_memory()
        rf = torch.empty_like(uh).pin_memory()
        ud = torch.empty_like(self.u)

        def one():
            ud.copy_(uh, non_blocking=True)
            self.nl.nl_apply(self.direct, ud, self.out_d)
            self.nl.nl_apply_fast(self.fast, ud, self.out_f)
            rd.copy_(self.out_d, non_blocking=True)
            rf.copy_(self.out_f, non_blocking=True)
        ms = self.time_fn(one, max(1, steps), flush)
        b = int(uh.numel()) * 4
        return {"value": round(self.value(ms), 4), "unit": self.unit, "h2d_bytes_per_step": b,
                "d2h_bytes_per_step": 2 * b, "ms_per_step": round(ms, 4)}

    def outputs(self):
        return {"direct": self.out_d.double().cpu().numpy().reshape(8, -1),
                "fast": self.out_f.double().cpu().numpy().reshape(8, -1)}


class EX(Workload):
    """The paper's examples (Sec. 4): fast vs direct in FP64."""
    dtype = "f64"

    def __init__(self, dev, seed, which):
        super().__init__(dev, seed)
        self.which = which
        self.name = which
        self.metric = ("Example 1 (2-D, delta=1/2, 128^2, K=0): fast + direct FP64 applies, "
                       "Gpts/s" if which == "ex1" else
                       "Example 2 (1-D, K=3, delta0=1/4 variable, 4096): fast + direct FP64 "
                       "applies, Gpts/s")

    def setup(self):
        nl, torch = self.nl, self.torch
        from paper_1905_08375_gb300 import synth
        if self.which == "ex1":
            self.d, self.n = 2, 128
            self.delta = 0.5
            kw = dict(family=nl.NL_POLY, K=0, normalize=False, self_term=nl.NL_SELF_PAPER)
            u = np.random.default_rng(self.seed).standard_normal(128 * 128)
        else:
            self.d, self.n = 1, 4096
            f = synth.example2_1d(n=4096, seed=self.seed)
            self.delta = f["delta"]
            kw = dict(family=nl.NL_POLY, K=3, alpha=1.0, normalize=False)
            u = f["u"]
        self.uh = u
        self.plan = nl.nl_plan_create(self.d, self.n, self.delta, **kw)
        self.u = torch.tensor(u, dtype=torch.float64, device=self.dev)
        self.out_d = torch.empty_like(self.u)
        self.out_f = torch.empty_like(self.u)
        N = self.n ** self.d
        self.units = 2 * N
        self.launches = 2 + self.plan.info()["levels"] + 1
        self.config = {"workload": self.metric, "n": self.n, "dim": self.d}

    def step(self):
        self.nl.nl_apply(self.plan, self.u, self.out_d)
        self.nl.nl_apply_fast(self.plan, self.u, self.out_f)

    def kernels(self, flush, reps):
        nl = self.nl
        t_d = self.time_fn(lambda: nl.nl_apply(self.plan, self.u, self.out_d), reps, flush)
        t_f = self.time_fn(lambda: nl.nl_apply_fast(self.plan, self.u, self.out_f), reps, flush)
        dl = self.delta if not np.isscalar(self.delta) else np.full(self.n ** self.d, self.delta)
        nb = float(ball_counts(dl, self.n, self.d).sum())
        roof = _alu_roof("k_direct_split (direct FP64)", 4.0 * nb, t_d, *fp64_peak())
        roof["algorithmic_per_launch"] = f"{4 * nb:.4g} flop (4 per term)"
        return roof, {"direct_fp64_ms": round(t_d, 4), "fast_fp64_ms": round(t_f, 4),
                      "fast_over_direct_speedup": round(t_d / t_f, 2)}

    def e2e(self, flush, steps):
        torch = self.torch
        uh = torch.tensor(self.uh, dtype=torch.float64).pin_memory()
        rd = torch.empty_like(uh).pin_memory()
        rf = torch.empty_like(uh).pin_memory()
        ud = torch.empty_like(self.u)

        def one():
            ud.copy_(uh, non_blocking=True)
            self.nl.nl_apply(self.plan, ud, self.out_d)
            self.nl.nl_apply_fast(self.plan, ud, self.out_f)
            rd.copy_(self.out_d, non_blocking=True)
            rf.copy_(self.out_f, non_blocking=True)
        ms = self.time_fn(one, steps, flush)
        b = int(uh.numel()) * 8
        return {"value": round(self.value(ms), 6), "unit": self.unit, "h2d_bytes_per_step": b,
                "d2h_bytes_per_step": 2 * b, "ms_per_step": round(ms, 4)}

    def outputs(self):
        return {"direct": self.out_d.cpu().numpy(), "fast": self.out_f.cpu().numpy()}


def make_workload(name, dev, seed):
    if name in ("ex1", "ex2"):
        return EX(dev, seed, name)
    return {"c1": C1, "c2": C2, "c2k": C2K, "c3": C3, "c3b": C3B, "c4": C4, "c4_512": C4L,
            "c5": C5}[name](dev, seed)


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle, as it stands, on a bounded sample
# ---------------------------------------------------------------------------
def _rel(x, r):
    return float(np.linalg.norm(x - r) / np.linalg.norm(r))


def oracle_sample(w, outs, budget_s=20.0):
    import oracle
    rng = np.random.default_rng(123)
    name = w.name
    if name in ("c4", "c4_512"):
        Lx = oracle.direct_scalar(outs["x"], 2, w.n, w.f["delta"], alpha=1.5,
                                  coef=oracle.COEF_XY, a=w.f["a"], symmetric=True)
        res = np.linalg.norm(w.rhs + Lx, axis=1) / np.linalg.norm(w.rhs, axis=1)
        par = {"gpu_learned_solution_fp64_oracle_residual_max": float(res.max())}
        if w.n <= 256:
            t0 = time.perf_counter()
            _, it, _ = oracle.cg(w.rhs[0], 2, w.n, w.f["delta"], alpha=1.5, coef=oracle.COEF_XY,
                                 a=w.f["a"], rtol=1e-8)
            dt = time.perf_counter() - t0
            return ({"value": round(dt * 1e3 * w.nrhs, 1), "unit": "ms",
                     "cores": oracle.num_threads(), "kind": "oracle",
                     "sample": f"one full FP64 Jacobi-CG solve at {w.n}^2 ({it} iterations, "
                               f"{dt:.1f} s) times {w.nrhs} right-hand sides"}, par)
        t0 = time.perf_counter()
        oracle.direct_scalar(w.rhs[0], 2, w.n, w.f["delta"], alpha=1.5, coef=oracle.COEF_XY,
                             a=w.f["a"], symmetric=True)
        dt = time.perf_counter() - t0
        its = w.last["iterations"] if w.last else 0
        jits = getattr(w, "jacobi_its", None) or its
        return ({"value": round(dt * 1e3 * jits * w.nrhs, 1), "unit": "ms",
                 "cores": oracle.num_threads(), "kind": "oracle",
                 "sample": f"one FP64 oracle operator apply at {w.n}^2 ({dt:.2f} s) times "
                           f"{jits} Jacobi-CG iterations times {w.nrhs} right-hand sides "
                           "(operator time only; a lower bound)"}, par)
    if name == "c3b":
        n, d, c, f0 = w.inst[0]
        t0 = time.perf_counter()
        _, it, _ = oracle.cg(f0, 2, n, d, kind="pd", c=c, rtol=1e-8)
        dt = time.perf_counter() - t0
        scale = w.points / float(n * n)
        par = {}
        for k in (0, len(w.inst) // 2, len(w.inst) - 1):
            nk, dk, ck, fk = w.inst[k]
            sl = slice(int(w.batch.offsets[k]), int(w.batch.offsets[k + 1]))
            Lx = oracle.pd_direct(outs["x"][sl].reshape(1, 2, -1), 2, nk, dk, ck).reshape(-1)
            par[f"instance{k}_n{nk}_fp64_oracle_residual"] = float(
                np.linalg.norm(fk + Lx) / np.linalg.norm(fk))
        return ({"value": round(dt * 1e3 * scale, 1), "unit": "ms", "cores": oracle.num_threads(),
                 "kind": "oracle",
                 "sample": f"one FP64 Jacobi-CG solve of the 128^2 instance ({it} iterations, "
                           f"{dt * 1e3:.0f} ms), scaled by total points / 128^2 = {scale:.1f} "
                           "(a lower bound: larger instances need more iterations)"}, par)
    if name == "c5":
        n = w.n
        N = n ** 3
        f = w.f
        t0 = time.perf_counter()
        idx = rng.choice(N, size=2000, replace=False)
        ref_d = oracle.direct_scalar(f["u"], 3, n, f["delta"], alpha=1.0, coef=oracle.COEF_XY,
                                     a=f["a"], idx=idx)
        ref_f = oracle.fast_leafset(f["u"], 3, int(np.log2(n)), f["delta"], K=0, alpha=1.0,
                                    coef=oracle.COEF_XY, a=f["a"], idx=idx)
        dt = time.perf_counter() - t0
        pts = 2 * 8 * len(idx)
        par = {"direct_rel_l2": _rel(outs["direct"][:, idx], ref_d),
               "fast_rel_l2": _rel(outs["fast"][:, idx], ref_f), "sampled_points": len(idx)}
        return ({"value": round(pts / dt / 1e9, 9), "unit": "Gpts/s",
                 "cores": oracle.num_threads(), "kind": "oracle",
                 "sample": f"{len(idx)} random nodes x 8 RHS, direct + fast leaf-set sums "
                           f"({dt:.1f} s)"}, par)
    if name in ("ex1", "ex2"):
        N = w.n ** w.d
        m = min(N, 4096 if name == "ex2" else 2048)
        idx = rng.choice(N, size=m, replace=False)
        L = int(np.log2(w.n))
        t0 = time.perf_counter()
        if name == "ex1":
            rd = oracle.direct_scalar(w.uh, 2, w.n, 0.5, family=oracle.POLY, K=0, normalize=False,
                                      idx=idx)
            rf = oracle.fast_tree(w.uh, 2, L, 0.5, K=0, normalize=False,
                                  self_mode=oracle.SELF_PAPER, idx=idx)
        else:
            rd = oracle.direct_scalar(w.uh, 1, w.n, w.delta, family=oracle.POLY, K=3, alpha=1.0,
                                      normalize=False, idx=idx)
            rf = oracle.fast_tree(w.uh, 1, L, w.delta, K=3, alpha=1.0, normalize=False, idx=idx)
        dt = time.perf_counter() - t0
        par = {"direct_rel_l2": _rel(outs["direct"][idx], rd),
               "fast_rel_l2": _rel(outs["fast"][idx], rf), "sampled_points": m}
        return ({"value": round(2 * m / dt / 1e9, 9), "unit": "Gpts/s",
                 "cores": oracle.num_threads(), "kind": "oracle",
                 "sample": f"{m} nodes, direct + literal tree algorithm ({dt:.1f} s)"}, par)
    # c1, c2, c2k, c3: grow a random node sample to fill the budget
    cls = type(w)
    f, n = w.f, w.n
    d = 1 if name == "c1" else 2
    N = n ** d
    cores = oracle.num_threads()
    t0 = time.perf_counter()
    idx = rng.choice(N, size=min(N, 256), replace=False)
    cls.oracle_step(f, n, idx)
    per_pt = (time.perf_counter() - t0) / len(idx)
    m = int(min(N, max(len(idx), budget_s / max(per_pt, 1e-9))))
    idx2 = rng.choice(N, size=m, replace=False)
    t0 = time.perf_counter()
    refs, units = cls.oracle_step(f, n, idx2)
    dt = time.perf_counter() - t0
    par = {"sampled_points": m}
    for k, got_all in outs.items():
        base = k[:-5] if k.endswith("_fp64") else k
        if base not in refs:
            continue
        got = got_all[..., idx2] if got_all.ndim > 1 else got_all[idx2]
        par[f"{k}_rel_l2"] = _rel(got, refs[base])
    if "cg" in outs:
        par.update(cg_residuals(w.cg, outs["cg"]))
    # the same oracle on one thread, on a sample a tenth of the budget
    m1 = int(min(N, max(64, 0.1 * budget_s / max(per_pt * cores, 1e-9))))
    idx1 = rng.choice(N, size=m1, replace=False)
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        _, units1 = cls.oracle_step(f, n, idx1)
        dt1 = time.perf_counter() - t0
    finally:
        oracle.set_threads(cores)
    return ({"value": round(units / dt / 1e9, 9), "unit": "Gpts/s", "cores": cores,
             "kind": "oracle", "sample": f"{m} random nodes of the workload ({dt:.1f} s)",
             "single_thread": {"value": round(units1 / dt1 / 1e9, 9), "unit": "Gpts/s",
                               "cores": 1, "sample": f"{m1} random nodes ({dt1:.1f} s)"}}, par)


def cg_residuals(cgw, outs):
    """FP64 oracle residuals ||f + L x|| / ||f|| of the GPU CG solutions of the CG workload."""
    import oracle
    Lx = oracle.direct_scalar(outs["x"], 2, cgw.n, cgw.f["delta"], alpha=1.5,
                              coef=oracle.COEF_XY, a=cgw.f["a"], symmetric=True)
    res = np.linalg.norm(cgw.rhs + Lx, axis=1) / np.linalg.norm(cgw.rhs, axis=1)
    out = {"cg_learned_fp64_oracle_residual_max": float(res.max())}
    if "x_jacobi" in outs:
        Lj = oracle.direct_scalar(outs["x_jacobi"], 2, cgw.n, cgw.f["delta"], alpha=1.5,
                                  coef=oracle.COEF_XY, a=cgw.f["a"], symmetric=True)
        rj = np.linalg.norm(cgw.rhs + Lj, axis=1) / np.linalg.norm(cgw.rhs, axis=1)
        out["cg_jacobi_fp64_oracle_residual_max"] = float(rj.max())
    return out


# ---------------------------------------------------------------------------
# rank aggregation and the timed run
# ---------------------------------------------------------------------------
def max_over_ranks(x, device):
    """The largest of the ranks' values of x, returned on every rank (all-reduce MAX)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(per_replica_value, ws, higher_is_better):
    """Replicas only: with every rank timed at the slowest rank's step time, a throughput is the
    sum over the ws replicas; a time-like metric is the slowest rank's time."""
    return per_replica_value * (ws if higher_is_better else 1)


def run_gpu(args, peaks):
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    w = make_workload(args.workload, dev, args.seed + rank)
    if args.size:
        w.size = args.size
    w.peaks = peaks
    from paper_1905_08375_gb300 import binding as nlb
    MEASURED_ALU.update(nlb.nl_measure_peaks())       # FMA peaks, before any timing
    w.setup()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    steps = args.steps
    if w.name in ("c4", "c4_512", "c3b"):
        steps = max(3, min(steps, 20 if w.name == "c4" else 5))   # one step is a whole solve
    if w.name == "c5":
        steps = max(3, min(steps, 30))
    for _ in range(args.warmup):
        w.step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed_steps")      # lets a profiler select the timed region
        for k in range(steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            w.step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    if ws > 1:
        dist.barrier()
    ms_step = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    if ws > 1:
        ms_step = max_over_ranks(ms_step, dev)
    value = whole_job_value(w.value(ms_step), ws, w.higher_is_better)
    reps = max(3, min(steps, 50))
    with ClockSampler(local) as clk2:
        roof, per = w.kernels(flush, reps)
        e2e = w.e2e(flush, min(steps, 20))
    result = dict(metric=w.metric, value=round(value, 6), unit=w.unit, n_gpus=ws, steps=steps,
                  warmup=args.warmup, ms_per_step=round(ms_step, 4),
                  higher_is_better=w.higher_is_better,
                  scaling="weak", vs_baseline=None, dtype=w.dtype, data="synthetic",
                  config=dict(w.config, l2="flushed (256 MiB write) before every timed step",
                              parallelism=f"replicas x{ws}"),
                  per_path=per, roofline=roof, e2e=e2e,
                  gpu_launches=(w.launches * steps) if w.launches else None,
                  peaks_source=peaks["_source"])
    result["clocks"] = clk.summary()
    result["clocks_per_path"] = clk2.summary()      # the per-path and end-to-end timings
    result["alu_peaks_measured"] = {k: round(v, 3) for k, v in MEASURED_ALU.items()}
    return result, w, rank, ws


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores, a bounded sample per step."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1905_08375_gb300 import synth
    n = 1024
    f = synth.heterogeneous_2d(n=n, seed=args.seed)
    rng = np.random.default_rng(7)
    m = 512
    N = n * n

    def step():
        idx = rng.choice(N, size=m, replace=False)
        C2.oracle_step(f, n, idx)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    value = 2 * m / dt / 1e9
    line = dict(impl="reference", metric=C2.metric, value=value, unit="Gpts/s", n_gpus=ws,
                steps=args.steps, warmup=args.warmup, ms_per_step=dt * 1e3,
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic",
                config={"workload": "2D heterogeneous nonlocal diffusion 1024x1024 (FP64 oracle "
                                    f"on {m} sampled nodes per step, direct + fast leaf-set)",
                        "n": n},
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
    ap.add_argument("--workload", default="c2",
                    choices=["c1", "c2", "c2k", "c3", "c3b", "c4", "c4_512", "c5", "ex1",
                             "ex2"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--size", type=int, default=0,
                    help="grid size override for c5 (a smaller case for profiling captures)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return
    peaks = load_peaks()
    result, w, rank, ws = run_gpu(args, peaks)
    if rank == 0:
        if ws == 1 and not args.no_cpu_baseline:
            cb, parity = oracle_sample(w, w.outputs())
            result["cpu_baseline"] = cb
            result["parity"] = parity
        print(json.dumps(result))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
