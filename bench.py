"""Benchmark of the QMC American-option hot path on GB300.

Workload (N=1): one American put, S0=100, K=100, r=0.05, sigma=0.3, T=1,
252 exercise dates, 2^20 Sobol' paths, LSM basis {1,x,x^2,x^3}, shift seed 2
(synthetic; the paper has no dataset).  One step = one full pricing: path
generation (Sobol' -> inverse normal -> bridge -> GBM store) and the LSM
backward sweep with its final sums, in the mixed precision (FP32 paths and
compensated FP32 sums, FP64 solve and price).  Metric: path-steps/s =
n_paths * n_steps / time per step.  The path array (1.06 GB) is larger than
L2, so every step streams it from HBM.

Keys beyond the base contract: fp64 (the same step in all-FP64 on the GPU),
err_vs_oracle (|price - FP64 oracle price| on identical points, in units of
K, from the CPU baseline leg), roofline (dominant kernel) and roofline_sweep, cpu_baseline (the oracle
on a bounded sample, host cores), clocks, oos (the second, out-of-sample
pass: the boundary valuation kernel and its HBM roofline), serving (a Poisson request replay),
batch and greeks (the 4096-option batch and 1024-option Greeks workloads
through their host calls).

Multi-GPU (torchrun, N>1): independent replicas, one option per rank (shift
seed 2 + rank), no collective on the data path; value sums all ranks.

--impl reference: the FP64 CPU oracle as it stands, on the host cores, on a
bounded sample of the same workload per step (rank 0 only).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "path-steps/s"
CONFIG_NAME = "american_put_lsm_2^20paths_252dates_p4"


def _config(opt, extra=None):
    c = {"workload": CONFIG_NAME, "n_paths": opt.n_paths, "n_steps": opt.n_steps, "basis": opt.basis,
         "type": "put", "S0": opt.S0, "K": opt.K, "r": opt.r, "sigma": opt.sigma, "T": opt.T,
         "l2": "path array 1.06 GB > 129 MB L2 (streamed every step)"}
    if extra:
        c.update(extra)
    return c


def replica_option(opt, rank):
    """The option rank `rank` prices in a multi-GPU run: the same contract with
    its own digital shift (seed + rank), so replicas do independent work."""
    return workloads.Option(**{**opt.as_dict(), "seed": opt.seed + rank})


def max_over_ranks(dist, value, device="cpu"):
    """Largest `value` over all ranks (identity without a process group)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", "amc_clocks_%d_%d.csv" % (os.getpid(), index))

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            out = parse_clocks(f)
        os.unlink(self.path)
        return out


def parse_clocks(lines):
    """Median SM clock, the maximum SM clock and every throttle reason seen
    Active in `nvidia-smi --query-gpu=<Clocks.FIELDS> --format=csv,noheader,
    nounits` lines; None without a usable sample."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        p = [x.strip() for x in line.split(",")]
        if len(p) < 9:
            continue
        try:
            sm.append(float(p[1]))
            mx.append(float(p[2]))
        except ValueError:
            continue
        for n, v in zip(names, p[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
            "reasons": sorted(reasons)}


def profile_traffic(kernel_src, summary, key="traffic_bytes_per_launch", conv=int):
    """DRAM bytes per launch (or another `key: value` field) recorded in a
    committed ncu summary, or None when the kernel source has changed since
    that capture (hash mismatch)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, kernel_src), "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()[:16]
        vals = {}
        with open(os.path.join(ROOT, summary)) as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    vals[k.strip()] = v.strip().split()[0] if v.strip() else ""
        if vals.get("source_sha256_16") != h:
            return None
        return conv(vals[key])
    except Exception:
        return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


def cpu_baseline(opt, n_sample=None):
    """The FP64 oracle as it stands on a bounded sample (first n_sample paths; default all of them,
    about 5 s on 16 host cores). A 64-path call first loads the library and its tables.  With the
    whole workload as the sample, the oracle price on the bench's own points comes back too."""
    import oracle
    n_sample = opt.n_paths if n_sample is None else n_sample
    oracle.lsm(oracle.paths(opt.S0, opt.r, opt.sigma, opt.T, opt.n_steps, 64, opt.seed),
               opt.type, opt.K, opt.r, opt.T, opt.basis)
    t = time.perf_counter()
    S = oracle.paths(opt.S0, opt.r, opt.sigma, opt.T, opt.n_steps, n_sample, opt.seed)
    res = oracle.lsm(S, opt.type, opt.K, opt.r, opt.T, opt.basis)
    dt = time.perf_counter() - t
    out = {"value": n_sample * opt.n_steps / dt, "unit": METRIC, "cores": oracle.threads(), "kind": "oracle",
           "sample": "first %d of %d paths, all %d dates, paths + LSM sweep, %.1f s" % (
               n_sample, opt.n_paths, opt.n_steps, dt)}
    # the same on one core, on the first 2^12 paths
    cores = oracle.threads()
    n1 = min(n_sample, 1 << 12)
    oracle.set_threads(1)
    try:
        t = time.perf_counter()
        S = oracle.paths(opt.S0, opt.r, opt.sigma, opt.T, opt.n_steps, n1, opt.seed)
        oracle.lsm(S, opt.type, opt.K, opt.r, opt.T, opt.basis)
        dt1 = time.perf_counter() - t
    finally:
        oracle.set_threads(cores)
    out["value_1core"] = n1 * opt.n_steps / dt1
    out["sample_1core"] = "first %d paths, all %d dates, one thread, %.2f s" % (n1, opt.n_steps, dt1)
    out["table2"] = table2_oracle()
    return out, (res["price"] if n_sample == opt.n_paths else None)


def batch_and_greeks(amc, device, hbm, peak_kind, reps=2):
    """The 4096-option batch and the 1024-option Greeks workloads through their host calls
    (host buffers in and out, so wall time), each after one warm-up call.  The batch's
    path-generation and sweep launches are also timed on the device (the context's
    opt-in profiling: CUDA events around every launch on its stream): the sweep's
    roofline is its algorithmic bytes (4 B per path-step, S read once) over the summed
    sweep-launch time, path generation's its 4 B per path-step written (with profiling
    on, the waves run one after another, so the launch times are not shared)."""
    bctx = amc.Context(device, arena_bytes=32 << 30)
    out = {}
    opts = workloads.batch_options()
    steps = sum(o.path_steps for o in opts)
    amc.amc_price_batch(bctx, opts, amc.AMC_MIXED)
    t = time.perf_counter()
    for _ in range(reps):
        res = amc.amc_price_batch(bctx, opts, amc.AMC_MIXED)
    dt = (time.perf_counter() - t) / reps
    failed = sum(r["status"] != 0 for r in res)
    bctx.profile()
    bctx.set_profiling(True)
    t = time.perf_counter()
    amc.amc_price_batch(bctx, opts, amc.AMC_MIXED)
    dt_prof = time.perf_counter() - t
    prof = bctx.profile()
    bctx.set_profiling(False)
    sweep_gbs = 4.0 * prof["sweep_path_steps"] / (prof["sweep_ms"] * 1e-3) / 1e9
    gen_gbs = 4.0 * prof["gen_path_steps"] / (prof["gen_ms"] * 1e-3) / 1e9
    out["batch"] = {"options": len(opts), "path_steps": steps, "s": dt, "value": steps / dt, "unit": METRIC,
                    "failed": failed, "workload": "4096 options, seed 3, 2^14..2^18 paths, 12..365 dates, p = 3",
                    "roofline": {"bound": "hbm", "achieved": sweep_gbs, "peak": hbm, "unit": "GB/s",
                                 "frac": sweep_gbs / hbm, "traffic": None, "peak_kind": peak_kind,
                                 "kernel": "sweep_cl_kernel (one cluster per option, on-chip exchange)",
                                 "sweep_launches": prof["sweep_launches"], "sweep_ms": prof["sweep_ms"],
                                 "algorithmic_bytes": 4.0 * prof["sweep_path_steps"]},
                    "roofline_pathgen": {"bound": "hbm", "achieved": gen_gbs, "peak": hbm, "unit": "GB/s",
                                         "frac": gen_gbs / hbm, "peak_kind": peak_kind, "kernel": "pathgen_kernel",
                                         "launches": prof["gen_launches"], "ms": prof["gen_ms"]},
                    "s_with_profiling": dt_prof}
    # the same batch with binary16 moneyness paths (AMC_MIXED16)
    amc.amc_price_batch(bctx, opts, amc.AMC_MIXED16)
    t = time.perf_counter()
    for _ in range(reps):
        res16 = amc.amc_price_batch(bctx, opts, amc.AMC_MIXED16)
    dt16 = (time.perf_counter() - t) / reps
    bctx.profile()
    bctx.set_profiling(True)
    amc.amc_price_batch(bctx, opts, amc.AMC_MIXED16)
    prof16 = bctx.profile()
    bctx.set_profiling(False)
    sweep16_gbs = 2.0 * prof16["sweep_path_steps"] / (prof16["sweep_ms"] * 1e-3) / 1e9
    out["batch"]["mixed16"] = {"s": dt16, "value": steps / dt16, "unit": METRIC,
                               "failed": sum(r["status"] != 0 for r in res16),
                               "sweep_ms": prof16["sweep_ms"], "gen_ms": prof16["gen_ms"],
                               "roofline": {"bound": "hbm", "achieved": sweep16_gbs, "peak": hbm, "unit": "GB/s",
                                            "frac": sweep16_gbs / hbm, "traffic": None, "peak_kind": peak_kind,
                                            "algorithmic_bytes": 2.0 * prof16["sweep_path_steps"]}}
    gopts = workloads.greeks_options()
    gsteps = sum(o.path_steps for o in gopts)
    amc.amc_greeks(bctx, gopts, amc.AMC_MIXED)
    t = time.perf_counter()
    for _ in range(reps):
        amc.amc_greeks(bctx, gopts, amc.AMC_MIXED)
    dt = (time.perf_counter() - t) / reps
    out["greeks"] = {"options": len(gopts), "path_steps": gsteps, "s": dt, "value": gsteps / dt, "unit": METRIC,
                     "workload": "1024 puts, seed 5, 2^18 paths, 100 dates, price + delta + vega"}
    bctx.close()
    return out


def oos_setup(amc, ctx, torch, stream, opt, value_seed):
    """Fit the boundary on the points of opt.seed, then write the paths of
    value_seed into S (mixed precision); returns (S, coef, res, vopt)."""
    ld = amc.amc_path_ld(opt.n_paths)
    S = torch.empty((opt.n_steps, ld), dtype=torch.float32, device="cuda")
    coef = torch.zeros((opt.n_steps, amc.AMC_COEF_STRIDE), dtype=torch.float64, device="cuda")
    res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    vopt = workloads.Option(**{**opt.as_dict(), "seed": value_seed})
    with torch.cuda.stream(stream):
        amc.amc_generate_paths(ctx, opt, amc.AMC_MIXED, S, stream=stream)
        amc.amc_fit_boundary(ctx, opt, amc.AMC_MIXED, S, coef, res, stream=stream)
        amc.amc_generate_paths(ctx, vopt, amc.AMC_MIXED, S, stream=stream)
    stream.synchronize()
    return S, coef, res, vopt


def oos_bench(amc, ctx, torch, stream, opt, hbm, peak_kind, reps=20, warmup=3):
    """Second pass on the bench workload: the boundary valuation kernel timed
    with CUDA events on its stream (device-resident paths, 1.06 GB > L2, so
    every launch streams them from HBM), and the whole out-of-sample pricing
    (two path generations, fit, valuation) through amc_price_oos."""
    S, coef, res, vopt = oos_setup(amc, ctx, torch, stream, opt, opt.seed + 5)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            amc.amc_value_boundary(ctx, vopt, amc.AMC_MIXED, S, coef, res, stream=stream)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            amc.amc_value_boundary(ctx, vopt, amc.AMC_MIXED, S, coef, res, stream=stream)
        e1.record(stream)
        stream.synchronize()
    ms = e0.elapsed_time(e1) / reps
    units = opt.n_paths * opt.n_steps
    nbytes = 4.0 * units
    gbs = nbytes / (ms * 1e-3) / 1e9
    val = amc.res_to_dict(res.cpu().numpy())
    # the same valuation with no path array: generation and valuation in one kernel
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            amc.amc_price_fused(ctx, vopt, amc.AMC_MIXED, res, coef, stream=stream)
        stream.synchronize()
        e0.record(stream)
        for _ in range(reps):
            amc.amc_price_fused(ctx, vopt, amc.AMC_MIXED, res, coef, stream=stream)
        e1.record(stream)
        stream.synchronize()
    fused_ms = e0.elapsed_time(e1) / reps
    amc.amc_price_oos(ctx, opt, opt.seed + 5, amc.AMC_MIXED)
    t = time.perf_counter()
    fit, val2 = amc.amc_price_oos(ctx, opt, opt.seed + 5, amc.AMC_MIXED)
    host_ms = (time.perf_counter() - t) * 1e3
    return {"kernel": "value_boundary_kernel", "ms": ms, "value": units / (ms * 1e-3), "unit": METRIC,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                         "traffic": profile_traffic("paper_1205_0106_gb300/csrc/value.cu",
                                                    "profiles/value_boundary_2p20x252_mixed.md"),
                         "peak_kind": peak_kind, "algorithmic_bytes": nbytes},
            "price_out_of_sample": val2["price"], "std_err": val2["std_err"], "price_in_sample": fit["price"],
            "oos_pricing_ms": host_ms, "fused_generate_and_value_ms": fused_ms,
            "workload": "boundary fitted on shift seed 2, applied to the 2^20 x 252 paths of shift seed 7"}


def paper_rule_bench(amc, ctx, torch, stream, opt, hbm, peak_kind, reps=20, warmup=3):
    """The paper's own exercise rule (Eqs. 10-11) on the bench workload's
    paths: its sweep alone, timed with CUDA events on its stream (paths
    resident, 1.06 GB > L2).  The rule reads the dates 1..m-1 once."""
    popt = workloads.Option(**{**opt.as_dict(), "rule": workloads.RULE_PAPER_UB})
    ld = amc.amc_path_ld(opt.n_paths)
    S = torch.empty((opt.n_steps, ld), dtype=torch.float32, device="cuda")
    res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        amc.amc_generate_paths(ctx, popt, amc.AMC_MIXED, S, stream=stream)
        for _ in range(warmup):
            amc.amc_sweep(ctx, popt, amc.AMC_MIXED, S, res, stream=stream)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            amc.amc_sweep(ctx, popt, amc.AMC_MIXED, S, res, stream=stream)
        e1.record(stream)
        stream.synchronize()
    ms = e0.elapsed_time(e1) / reps
    nbytes = 4.0 * opt.n_paths * (opt.n_steps - 1)
    gbs = nbytes / (ms * 1e-3) / 1e9
    got = amc.res_to_dict(res.cpu().numpy())
    fused = fused_bench(amc, ctx, torch, stream, popt, reps, warmup)
    return {"fused": fused, "kernel": "sweep_pathwise_kernel (paper rule)", "ms": ms,
            "value": opt.n_paths * opt.n_steps / (ms * 1e-3), "unit": METRIC,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                         "traffic": profile_traffic("paper_1205_0106_gb300/csrc/sweep.cu",
                                                    "profiles/sweep_pathwise_paper_2p20x252_mixed.md"),
                         "peak_kind": peak_kind, "algorithmic_bytes": nbytes},
            "price": got["price"], "workload": "Eqs. 10-11 on the 2^20 x 252 paths of shift seed 2"}


DUAL_OUTER, DUAL_INNER = 4096, 128
# SM count and maximum SM clock for the issue-slot peak: set from the device
# properties and the nvidia-smi samples of the run (GB300 nominal until then)
DEVICE = {"sms": 152, "sm_max_mhz": 2070.0, "source": "nominal GB300"}


def _pipes(v):
    return {k: float(x) for k, x in (kv.split("=") for kv in v.split(","))}


def issue_roofline(kernel_src, summary, units_per_s):
    """Issue-slot roofline of a kernel: warp instructions per unit of work
    from its committed ncu capture (hash-checked) x the units per second
    timed by CUDA events, against SMs x 4 schedulers x 1 warp instruction
    per clock at the maximum SM clock; with the capture's pipe utilisation
    (instructions executed, % of each pipe's peak)."""
    per_unit = profile_traffic(kernel_src, summary, "warp_instr_per_unit", float)
    peak = DEVICE["sms"] * 4 * DEVICE["sm_max_mhz"] * 1e6
    achieved = None if per_unit is None else per_unit * units_per_s
    return {"bound": "alu", "unit": "warp-instr/s", "achieved": achieved, "peak": peak,
            "frac": None if achieved is None else achieved / peak, "warp_instr_per_unit": per_unit,
            "pipes_pct_of_peak": profile_traffic(kernel_src, summary, "pipes_pct", _pipes),
            "peak_kind": "issue slots: %d SMs x 4 schedulers x 1 warp instruction per clock at %.0f MHz (%s)" % (
                DEVICE["sms"], DEVICE["sm_max_mhz"], DEVICE["source"])}


def dual_setup(amc, ctx, torch, stream, opt):
    """Boundary fitted on the bench workload's points; 4096 outer paths of
    shift seed opt.seed + 11 (mixed precision).  Returns (S, coef, outer)."""
    S, coef, _, _ = oos_setup(amc, ctx, torch, stream, opt, opt.seed + 5)
    del S
    outer = workloads.Option(**{**opt.as_dict(), "n_paths": DUAL_OUTER, "seed": opt.seed + 11})
    So = torch.empty((opt.n_steps, amc.amc_path_ld(DUAL_OUTER)), dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        amc.amc_generate_paths(ctx, outer, amc.AMC_MIXED, So, stream=stream)
    stream.synchronize()
    return So, coef, outer


def dual_bench(amc, ctx, torch, stream, opt, reps=5, warmup=2):
    """Dual upper bound of the bench workload's fitted boundary on 4096 outer
    paths with 128 inner paths per outer path and date: the inner-simulation
    kernel and its reduction timed with CUDA events on their stream; the
    lower bound (the boundary applied to the same outer paths) beside it."""
    So, coef, outer = dual_setup(amc, ctx, torch, stream, opt)
    res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    low = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        amc.amc_value_boundary(ctx, outer, amc.AMC_MIXED, So, coef, low, stream=stream)
        for _ in range(warmup):
            amc.amc_dual_upper(ctx, outer, amc.AMC_MIXED, So, coef, DUAL_INNER, 13, res, stream=stream)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            amc.amc_dual_upper(ctx, outer, amc.AMC_MIXED, So, coef, DUAL_INNER, 13, res, stream=stream)
        e1.record(stream)
        stream.synchronize()
    ms = e0.elapsed_time(e1) / reps
    r, lo = res.cpu().numpy(), amc.res_to_dict(low.cpu().numpy())
    steps = float(r[7])
    # issue-slot roofline: warp instructions per inner step from the committed
    # ncu capture x steps/s, against 152 SMs x 4 schedulers x 1 issue/clock
    summary = "profiles/dual_inner_2p20x252_4096x128_mixed.md"
    rl = issue_roofline("paper_1205_0106_gb300/csrc/dual.cu", summary, steps / (ms * 1e-3))
    rl["traffic"] = profile_traffic("paper_1205_0106_gb300/csrc/dual.cu", summary)
    return {"kernel": "dual_inner_kernel + dual_final_kernel", "ms": ms, "inner_steps": steps,
            "value": steps / (ms * 1e-3), "unit": "inner path-steps/s", "roofline": rl,
            "upper": float(r[0]), "upper_std_err": float(r[1]), "L0": float(r[6]),
            "lower": lo["price"], "lower_std_err": lo["std_err"], "gap": float(r[0]) - lo["price"],
            "workload": "boundary fitted on the 2^20 x 252 paths of shift seed 2; 4096 outer paths of shift "
                        "seed 13, 128 inner paths per outer path and date, inner seed 13"}


def fused_bench(amc, ctx, torch, stream, popt, reps, warmup):
    """The paper's rule priced with no path array (amc_price_fused: one
    path-generation kernel that values every path as it is formed, then
    finalize), timed with CUDA events on its stream; the stored-path
    pricing (path generation + the rule's sweep) beside it."""
    res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    ld = amc.amc_path_ld(popt.n_paths)
    S = torch.empty((popt.n_steps, ld), dtype=torch.float32, device="cuda")

    def timed(fn):
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                fn()
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            stream.synchronize()
        return e0.elapsed_time(e1) / reps

    ms = timed(lambda: amc.amc_price_fused(ctx, popt, amc.AMC_MIXED, res, stream=stream))
    fused_price = amc.res_to_dict(res.cpu().numpy())["price"]
    ms_stored = timed(lambda: amc.amc_price_device(ctx, popt, amc.AMC_MIXED, S, res, stream=stream))
    units = popt.n_paths * popt.n_steps
    summary = "profiles/pathgen_fused_paper_2p20x252_mixed.md"
    rl = issue_roofline("paper_1205_0106_gb300/csrc/pathgen.cu", summary, units / (ms * 1e-3))
    rl["traffic"] = profile_traffic("paper_1205_0106_gb300/csrc/pathgen.cu", summary)
    return {"ms": ms, "value": units / (ms * 1e-3), "unit": METRIC, "price": fused_price, "roofline": rl,
            "stored_ms": ms_stored, "stored_over_fused": ms_stored / ms,
            "workload": "Eqs. 10-11 on the 2^20 x 252 points of shift seed 2, no path array"}


def large_bench(amc, ctx, torch, stream, hbm, peak_kind, reps=3, warmup=1):
    """An option too large for the register-resident LSM sweep: 2^22 paths x
    252 dates (4.2 GB of FP32 paths), priced by path generation and the
    streaming sweep (cash flows in device memory, one pass and one solve per
    date), timed with CUDA events on their stream; the streaming sweep alone
    against its algorithmic traffic (S_j and S_{j+1} read, the cash flows
    read and written: 16 bytes per path and date)."""
    opt = workloads.Option(100.0, 100.0, 0.05, 0.3, 1.0, 252, 2 ** 22, basis=4, type=workloads.PUT, seed=2)
    ld = amc.amc_path_ld(opt.n_paths)
    S = torch.empty((opt.n_steps, ld), dtype=torch.float32, device="cuda")
    res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")

    def timed(fn):
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                fn()
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            stream.synchronize()
        return e0.elapsed_time(e1) / reps

    ms = timed(lambda: amc.amc_price_device(ctx, opt, amc.AMC_MIXED, S, res, stream=stream))
    price = amc.res_to_dict(res.cpu().numpy())
    ms_sweep = timed(lambda: amc.amc_sweep(ctx, opt, amc.AMC_MIXED, S, res, stream=stream))
    units = opt.n_paths * opt.n_steps
    nbytes = 16.0 * opt.n_paths * (opt.n_steps - 1)
    gbs = nbytes / (ms_sweep * 1e-3) / 1e9
    del S
    # the same with the path array as binary16 moneyness: 12 B per path and date
    Y = torch.empty((opt.n_steps, ld), dtype=torch.float16, device="cuda")
    ms16 = timed(lambda: amc.amc_price_device(ctx, opt, amc.AMC_MIXED16, Y, res, stream=stream))
    price16 = amc.res_to_dict(res.cpu().numpy())
    ms16_sweep = timed(lambda: amc.amc_sweep(ctx, opt, amc.AMC_MIXED16, Y, res, stream=stream))
    nbytes16 = 12.0 * opt.n_paths * (opt.n_steps - 1)
    gbs16 = nbytes16 / (ms16_sweep * 1e-3) / 1e9
    del Y
    return {"ms": ms, "value": units / (ms * 1e-3), "unit": METRIC, "price": price["price"],
            "std_err": price["std_err"], "sweep_ms": ms_sweep,
            "roofline_sweep": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                               "traffic": None, "peak_kind": peak_kind, "algorithmic_bytes": nbytes},
            "mixed16": {"ms": ms16, "value": units / (ms16 * 1e-3), "unit": METRIC, "price": price16["price"],
                        "sweep_ms": ms16_sweep,
                        "roofline_sweep": {"bound": "hbm", "achieved": gbs16, "peak": hbm, "unit": "GB/s",
                                           "frac": gbs16 / hbm, "traffic": None, "peak_kind": peak_kind,
                                           "algorithmic_bytes": nbytes16}},
            "workload": "put S0 100 K 100 r 0.05 sigma 0.3 T 1, 2^22 paths x 252 dates, basis 4, shift seed 2, "
                        "mixed: above the register-resident sweep's 1.17 M paths"}


TABLE2_PATHS = (10, 100, 1000, 10000, 100000, 200000, 300000, 500000, 1000000)
TABLE2_OPTION = dict(S0=36.0, K=40.0, r=0.06, sigma=0.2, T=1.0, n_steps=10, basis=3, type=0, seed=1)


def table2_bench(amc, ctx, reps=20):
    """The paper's Table 2 experiment (one pricing vs the number of paths, ten
    exercise dates) on one GB300: host wall time of one blocking
    amc_price_american call (median of reps, after two warm-up calls), for
    the paper's rule (Eqs. 10-11) and for LSM.  The paper prints no option
    parameters; this uses the Longstaff-Schwartz Table 1 put."""
    o = TABLE2_OPTION
    rows = []
    for n in TABLE2_PATHS:
        row = {"paths": n}
        for name, rule in (("paper_rule_ms", amc.AMC_RULE_PAPER_UB), ("lsm_ms", amc.AMC_RULE_LSM)):
            call = lambda: amc.amc_price_american(ctx, o["S0"], o["K"], o["r"], o["sigma"], o["T"], o["n_steps"], n,
                                                  o["basis"], o["type"], o["seed"], rule, amc.AMC_MIXED)
            call()
            call()
            ts = []
            for _ in range(reps):
                t = time.perf_counter()
                call()
                ts.append((time.perf_counter() - t) * 1e3)
            row[name] = statistics.median(ts)
        rows.append(row)
    return {"rows": rows, "workload": "put S0 36 K 40 r 0.06 sigma 0.2 T 1, 10 dates, basis 3, mixed; host wall "
                                      "time of one blocking call, median of %d" % reps}


def table2_oracle():
    """The oracle (paths + the paper's rule, all host cores) on the Table 2
    path counts: seconds per pricing."""
    import oracle
    o = TABLE2_OPTION
    oracle.price(o["S0"], o["K"], o["r"], o["sigma"], o["T"], o["n_steps"], 10, basis=o["basis"], type=o["type"],
                 seed=o["seed"], rule=oracle.RULE_PAPER_UB)            # loads the library and its tables
    out = []
    for n in TABLE2_PATHS:
        t = time.perf_counter()
        oracle.price(o["S0"], o["K"], o["r"], o["sigma"], o["T"], o["n_steps"], n, basis=o["basis"], type=o["type"],
                     seed=o["seed"], rule=oracle.RULE_PAPER_UB)
        out.append({"paths": n, "paper_rule_ms": (time.perf_counter() - t) * 1e3})
    return out


def fig1_bench(amc, device):
    """The paper's Fig. 1 data: value vs number of exercise dates for LSM and
    the paper's rule (the Longstaff-Schwartz Table 1 put, 2^16 paths), all
    points in one batch call, mixed precision."""
    bctx = amc.Context(device, arena_bytes=4 << 30)
    opts = workloads.fig1_options()
    amc.amc_price_batch(bctx, opts, amc.AMC_MIXED)
    t = time.perf_counter()
    res = amc.amc_price_batch(bctx, opts, amc.AMC_MIXED)
    dt = time.perf_counter() - t
    bctx.close()
    n = len(workloads.FIG1_DATES)
    return {"dates": list(workloads.FIG1_DATES),
            "lsm": [round(r["price"], 5) for r in res[:n]], "lsm_std_err": [round(r["std_err"], 5) for r in res[:n]],
            "paper_rule": [round(r["price"], 5) for r in res[n:]], "s": dt,
            "workload": "put S0 36 K 40 r 0.06 sigma 0.2 T 1, basis 3, 2^16 paths, shift seed 21"}


def randomization_bench(amc, ctx, torch, stream, opt, R=32):
    """The paper's randomisation (LCG permutation of each dimension's points)
    vs the digital shift: the spread of the LSM price over R independent
    seeds (LS Table 1 put, 50 dates, 2^16 paths, mixed), and the permuted
    path generation timed on the bench workload."""
    base = workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 50, 2 ** 16, basis=3, seed=0)
    seeds = [1000 + s for s in range(R)]
    shifted = [r["price"] for r in amc.amc_price_batch(ctx, [workloads.Option(**{**base.as_dict(), "seed": s})
                                                             for s in seeds], amc.AMC_MIXED)]
    ld = amc.amc_path_ld(base.n_paths)
    S = torch.empty((base.n_steps, ld), dtype=torch.float32, device="cuda")
    res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    permuted = []
    with torch.cuda.stream(stream):
        for s in seeds:
            o = workloads.Option(**{**base.as_dict(), "seed": s})
            amc.amc_generate_paths_permuted(ctx, o, amc.AMC_MIXED, S, stream=stream)
            amc.amc_sweep(ctx, o, amc.AMC_MIXED, S, res, stream=stream)
            stream.synchronize()
            permuted.append(float(res[0].item()))
        # permuted path generation on the bench workload
        Sb = torch.empty((opt.n_steps, amc.amc_path_ld(opt.n_paths)), dtype=torch.float32, device="cuda")
        for _ in range(2):
            amc.amc_generate_paths_permuted(ctx, opt, amc.AMC_MIXED, Sb, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            amc.amc_generate_paths_permuted(ctx, opt, amc.AMC_MIXED, Sb, stream=stream)
        e1.record(stream)
        stream.synchronize()
    sd_s, sd_p = statistics.stdev(shifted), statistics.stdev(permuted)
    return {"seeds": R, "digital_shift_mean": statistics.fmean(shifted), "digital_shift_sd": sd_s,
            "lcg_permutation_mean": statistics.fmean(permuted), "lcg_permutation_sd": sd_p,
            "variance_ratio_perm_over_shift": (sd_p / sd_s) ** 2 if sd_s > 0 else None,
            "permuted_pathgen_ms_bench_workload": e0.elapsed_time(e1) / 5,
            "workload": "LSM price over %d seeds: put S0 36 K 40 r 0.06 sigma 0.2 T 1, 50 dates, 2^16 paths" % R}


def serve_replay(amc, ctx, times, opts, slots=3, max_batch=128, prec=1):
    """Replay arrivals (seconds from start) through the serving loop.
    Returns latency percentiles, throughput and counts."""
    amc.amc_serve_start(ctx, slots=slots, max_batch=max_batch, prec=prec)
    lat, steps, bad = [], 0, 0
    outstanding = 0
    t0 = time.perf_counter()
    last_drain = 0.0

    def drain():
        nonlocal outstanding, steps, bad
        for _, r, l in amc.amc_serve_drain(ctx):
            outstanding -= 1
            lat.append(l)
            bad += r["status"] != 0
    for t, o in zip(times, opts):
        while True:
            now = time.perf_counter() - t0
            if now >= t:
                break
            if now - last_drain > 0.001:
                drain()
                last_drain = now
            time.sleep(min(0.0002, t - now))
        amc.amc_serve_submit(ctx, o)
        outstanding += 1
        steps += o.n_paths * o.n_steps
    while outstanding > 0:
        drain()
        time.sleep(0.0005)
    wall = time.perf_counter() - t0
    stats = amc.amc_serve_stats_get(ctx)
    amc.amc_serve_stop(ctx)
    lat.sort()
    q = lambda f: lat[min(len(lat) - 1, int(f * len(lat)))] * 1e3
    return {"requests": len(lat), "offered_per_s": len(times) / max(times[-1], 1e-9), "wall_s": wall,
            "p50_ms": q(0.50), "p99_ms": q(0.99), "max_ms": lat[-1] * 1e3, "failed": bad,
            "path_steps_per_s": steps / wall, "batches": stats["batches"], "slots": slots}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    opt = workloads.single_large()
    n_sample = 2 ** 14
    times = []
    for k in range(args.warmup + args.steps):
        t = time.perf_counter()
        S = oracle.paths(opt.S0, opt.r, opt.sigma, opt.T, opt.n_steps, n_sample, opt.seed)
        oracle.lsm(S, opt.type, opt.K, opt.r, opt.T, opt.basis)
        if k >= args.warmup:
            times.append(time.perf_counter() - t)
    per = sum(times) / len(times)
    value = n_sample * opt.n_steps / per
    sample = "first %d of %d paths, all %d dates per step (paths + LSM sweep)" % (n_sample, opt.n_paths,
                                                                                   opt.n_steps)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(opt, {"sample_paths": n_sample}),
            "cpu_baseline": {"kind": "oracle", "cores": oracle.threads(), "sample": sample, "value": value,
                             "unit": METRIC},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_amc(args):
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    if rank == 0 or ws == 1:
        __graft_entry__.build()
    if dist is not None:
        dist.barrier()
        __graft_entry__.build()
    import paper_1205_0106_gb300 as amc

    opt = workloads.single_large()
    if ws > 1:
        opt = replica_option(opt, rank)
    ctx = amc.Context(local, arena_bytes=4 << 30)
    stream = torch.cuda.Stream()
    ld = amc.amc_path_ld(opt.n_paths)
    units = opt.n_paths * opt.n_steps

    def time_steps(prec, steps, warmup, split=False, streaming=False):
        # streaming: every sweep through the streaming design (context injection kind 3)
        dt = {amc.AMC_FP64: torch.float64, amc.AMC_MIXED16: torch.float16}.get(prec, torch.float32)
        S = torch.empty((opt.n_steps, ld), dtype=dt, device="cuda")
        res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")

        def price():
            if streaming:
                ctx.inject(3)
            amc.amc_price_device(ctx, opt, prec, S, res, stream=stream)
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                price()
            stream.synchronize()
            if dist is not None:
                dist.barrier()
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * steps + 1 if split else 2)]
            if split:
                ev[0].record(stream)
                for k in range(steps):
                    amc.amc_generate_paths(ctx, opt, prec, S, stream=stream)
                    ev[2 * k + 1].record(stream)
                    amc.amc_sweep(ctx, opt, prec, S, res, stream=stream)
                    ev[2 * k + 2].record(stream)
            else:
                ev[0].record(stream)
                for _ in range(steps):
                    price()
                ev[1].record(stream)
            stream.synchronize()
            torch.cuda.synchronize()
        if split:
            gen = [ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(steps)]
            swp = [ev[2 * k + 1].elapsed_time(ev[2 * k + 2]) for k in range(steps)]
            total = ev[0].elapsed_time(ev[2 * steps])
            return total, sum(gen) / steps, sum(swp) / steps, res
        return ev[0].elapsed_time(ev[1]), None, None, res

    if args.profile_cluster:
        # profiling mode: one batch-class option (2^18 paths, 252 dates, p = 4), its paths once,
        # then only its cluster-sweep launches (for ncu)
        copt = workloads.scaled(opt, n_paths=2 ** 18)
        S = torch.empty((copt.n_steps, amc.amc_path_ld(copt.n_paths)), dtype=torch.float32, device="cuda")
        res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            amc.amc_generate_paths(ctx, copt, amc.AMC_MIXED, S, stream=stream)
            for _ in range(args.warmup + args.steps):
                amc.amc_sweep(ctx, copt, amc.AMC_MIXED, S, res, stream=stream)
            stream.synchronize()
        if rank == 0:
            print(json.dumps({"profile": "cluster", "price": float(res[0].item()), "status": float(res[5].item())}),
                  flush=True)
        ctx.close()
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.profile_batch:
        bctx = amc.Context(local, arena_bytes=32 << 30)
        opts = workloads.batch_options()
        for _ in range(2):
            amc.amc_price_batch(bctx, opts, amc.AMC_MIXED)
        if rank == 0:
            print(json.dumps({"profile": "batch", "options": len(opts)}), flush=True)
        bctx.close()
        ctx.close()
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.profile_paper:
        # profiling mode: the paper-rule sweep on resident paths (for ncu)
        popt = workloads.Option(**{**opt.as_dict(), "rule": workloads.RULE_PAPER_UB})
        S = torch.empty((opt.n_steps, ld), dtype=torch.float32, device="cuda")
        res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            amc.amc_generate_paths(ctx, popt, amc.AMC_MIXED, S, stream=stream)
            for _ in range(args.warmup + args.steps):
                amc.amc_sweep(ctx, popt, amc.AMC_MIXED, S, res, stream=stream)
            stream.synchronize()
        if rank == 0:
            print(json.dumps({"profile": "paper", "steps": args.steps, "warmup": args.warmup}), flush=True)
        ctx.close()
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.profile_value:
        # profiling mode: fit once, then only the valuation launches (for ncu)
        S, coef, res, vopt = oos_setup(amc, ctx, torch, stream, opt, opt.seed + 5)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup + args.steps):
                amc.amc_value_boundary(ctx, vopt, amc.AMC_MIXED, S, coef, res, stream=stream)
            stream.synchronize()
        if rank == 0:
            print(json.dumps({"profile": "value", "steps": args.steps, "warmup": args.warmup}), flush=True)
        ctx.close()
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.profile_large:
        # profiling mode: the streaming LSM sweep of a 2^21-path, 50-date put (for ncu launch lists)
        lopt = workloads.Option(100.0, 100.0, 0.05, 0.3, 1.0, 50, 2 ** 21, basis=4, type=workloads.PUT, seed=2)
        S = torch.empty((lopt.n_steps, amc.amc_path_ld(lopt.n_paths)), dtype=torch.float32, device="cuda")
        res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            amc.amc_generate_paths(ctx, lopt, amc.AMC_MIXED, S, stream=stream)
            for _ in range(args.warmup + args.steps):
                amc.amc_sweep(ctx, lopt, amc.AMC_MIXED, S, res, stream=stream)
            stream.synchronize()
        if rank == 0:
            print(json.dumps({"profile": "large", "steps": args.steps, "warmup": args.warmup}), flush=True)
        ctx.close()
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.profile_fused:
        # profiling mode: only the paper rule priced with no path array (for ncu)
        popt = workloads.Option(**{**opt.as_dict(), "rule": workloads.RULE_PAPER_UB})
        res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            for _ in range(args.warmup + args.steps):
                amc.amc_price_fused(ctx, popt, amc.AMC_MIXED, res, stream=stream)
            stream.synchronize()
        if rank == 0:
            print(json.dumps({"profile": "fused", "steps": args.steps, "warmup": args.warmup}), flush=True)
        ctx.close()
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.profile_dual:
        # profiling mode: fit once, outer paths, then only the dual launches (for ncu)
        So, coef, outer = dual_setup(amc, ctx, torch, stream, opt)
        res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            for _ in range(args.warmup + args.steps):
                amc.amc_dual_upper(ctx, outer, amc.AMC_MIXED, So, coef, DUAL_INNER, 13, res, stream=stream)
            stream.synchronize()
        if rank == 0:
            print(json.dumps({"profile": "dual", "steps": args.steps, "warmup": args.warmup,
                              "inner_steps": float(res[7].item())}), flush=True)
        ctx.close()
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.profile:
        # profiling mode: only the timed mixed-precision steps (for ncu)
        t_ms, _, _, res = time_steps(amc.AMC_MIXED, args.steps, args.warmup)
        if rank == 0:
            print(json.dumps({"profile": True, "steps": args.steps, "ms_per_step": t_ms / args.steps}), flush=True)
        ctx.close()
        if dist is not None:
            dist.destroy_process_group()
        return
    clocks = Clocks(torch.cuda.current_device())
    # headline: mixed precision, device-resident
    clocks.start()
    t_ms, _, _, res = time_steps(amc.AMC_MIXED, args.steps, args.warmup)
    ck = clocks.stop()
    DEVICE.update(sms=torch.cuda.get_device_properties(local).multi_processor_count,
                  sm_max_mhz=float(ck["sm_max_mhz"]) if ck else DEVICE["sm_max_mhz"],
                  source="device properties, nvidia-smi maximum SM clock" if ck else "device properties")
    t_ms = max_over_ranks(dist, t_ms, "cuda")
    ms_per_step = t_ms / args.steps
    value = units * ws / (ms_per_step * 1e-3)
    price = amc.res_to_dict(res.cpu().numpy())

    # per-kernel times (same steps, generate and sweep timed apart)
    _, gen_ms, sweep_ms, _ = time_steps(amc.AMC_MIXED, max(3, args.steps // 2), 2, split=True)
    # FP64 GPU baseline on identical points: the first sweep design (FP64
    # everywhere, counter-based exchange) and the streaming sweep in FP64
    # (the fastest FP64 design: one pass and one solve per date, its cash
    # flows in device memory), each after FP64 path generation
    f_ms, _, _, fres = time_steps(amc.AMC_FP64, max(3, args.steps // 4), 2)
    fp64_ms = f_ms / max(3, args.steps // 4)
    fp64_price = amc.res_to_dict(fres.cpu().numpy())["price"]
    fs_ms, _, _, fsres = time_steps(amc.AMC_FP64, max(3, args.steps // 4), 2, streaming=True)
    fp64s_ms = fs_ms / max(3, args.steps // 4)
    fp64s_price = amc.res_to_dict(fsres.cpu().numpy())["price"]
    # the path array as binary16 moneyness (AMC_MIXED16): whole pricings, then generate and sweep apart
    h16_steps = max(3, args.steps // 2)
    h16_ms, _, _, h16res = time_steps(amc.AMC_MIXED16, h16_steps, 2)
    h16_ms /= h16_steps
    _, h16_gen_ms, h16_sweep_ms, _ = time_steps(amc.AMC_MIXED16, h16_steps, 2, split=True)
    h16_price = amc.res_to_dict(h16res.cpu().numpy())

    # end to end through the host API: option in, price out (host buffers)
    for _ in range(2):
        amc.amc_price_american(ctx, opt.S0, opt.K, opt.r, opt.sigma, opt.T, opt.n_steps, opt.n_paths, opt.basis,
                               opt.type, opt.seed, opt.rule, amc.AMC_MIXED)
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        amc.amc_price_american(ctx, opt.S0, opt.K, opt.r, opt.sigma, opt.T, opt.n_steps, opt.n_paths, opt.basis,
                               opt.type, opt.seed, opt.rule, amc.AMC_MIXED)
    e2e_s = time.perf_counter() - t0
    e2e_value = units * ws * args.steps / max_over_ranks(dist, e2e_s, "cuda")

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return
    hbm, peak_kind = _peaks()
    bytes_sweep = 4.0 * units                       # S read once: 4 B per path-step
    bytes_gen = 4.0 * units                         # S written once
    sweep_gbs = bytes_sweep / (sweep_ms * 1e-3) / 1e9
    gen_gbs = bytes_gen / (gen_ms * 1e-3) / 1e9
    rl_sweep = {"bound": "hbm", "achieved": sweep_gbs, "peak": hbm, "unit": "GB/s", "frac": sweep_gbs / hbm,
                "traffic": profile_traffic("paper_1205_0106_gb300/csrc/sweep_v2.cu",
                                           "profiles/sweep_lsm_v2_2p20x252_mixed.md"),
                "kernel": "sweep_lsm_v2_kernel", "ms": sweep_ms, "peak_kind": peak_kind,
                "algorithmic_bytes": bytes_sweep,
                "issue": issue_roofline("paper_1205_0106_gb300/csrc/sweep_v2.cu",
                                        "profiles/sweep_lsm_v2_2p20x252_mixed.md", units / (sweep_ms * 1e-3))}
    rl_gen = {"bound": "hbm", "achieved": gen_gbs, "peak": hbm, "unit": "GB/s", "frac": gen_gbs / hbm,
              "traffic": profile_traffic("paper_1205_0106_gb300/csrc/pathgen.cu", "profiles/pathgen_2p20x252_mixed.md"),
              "kernel": "pathgen_kernel", "ms": gen_ms, "peak_kind": peak_kind, "algorithmic_bytes": bytes_gen,
              "issue": issue_roofline("paper_1205_0106_gb300/csrc/pathgen.cu", "profiles/pathgen_2p20x252_mixed.md",
                                      units / (gen_ms * 1e-3)),
              "note": "issue-bound (ALU); the HBM write fraction is the secondary bound"}
    dominant = rl_gen if gen_ms >= sweep_ms else rl_sweep
    h16_gbs_sweep = 2.0 * units / (h16_sweep_ms * 1e-3) / 1e9
    h16_gbs_gen = 2.0 * units / (h16_gen_ms * 1e-3) / 1e9
    mixed16 = {"value": units * ws / (h16_ms * 1e-3), "unit": METRIC, "ms_per_step": h16_ms,
               "gen_ms": h16_gen_ms, "sweep_ms": h16_sweep_ms, "price": h16_price["price"],
               "std_err": h16_price["std_err"], "err_vs_oracle_over_K": None,
               "path_bytes": 2.0 * units, "path_bytes_mixed": 4.0 * units,
               "roofline_sweep": {"bound": "hbm", "achieved": h16_gbs_sweep, "peak": hbm, "unit": "GB/s",
                                  "frac": h16_gbs_sweep / hbm, "traffic": None, "peak_kind": peak_kind,
                                  "kernel": "sweep_lsm_v2_kernel (binary16 ring)", "algorithmic_bytes": 2.0 * units},
               "roofline_pathgen": {"bound": "hbm", "achieved": h16_gbs_gen, "peak": hbm, "unit": "GB/s",
                                    "frac": h16_gbs_gen / hbm, "traffic": None, "peak_kind": peak_kind,
                                    "kernel": "pathgen_kernel (binary16 store)", "algorithmic_bytes": 2.0 * units},
               "storage": "y = S/K - 1 in IEEE binary16, 2 B per path-step (AMC_MIXED16)"}
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": _config(opt, {"parallelism": "replicas" if ws > 1 else "single"}),
            "price": price["price"], "std_err": price["std_err"],
            "err_vs_oracle_over_K": None,
            "fp64": {"value": units * ws / (fp64_ms * 1e-3), "ms_per_step": fp64_ms, "price": fp64_price,
                     "mixed_over_fp64": fp64_ms / ms_per_step, "design": "first sweep design, FP64 throughout",
                     "streaming": {"value": units * ws / (fp64s_ms * 1e-3), "ms_per_step": fp64s_ms,
                                   "price": fp64s_price, "mixed_over_fp64": fp64s_ms / ms_per_step,
                                   "design": "streaming sweep in FP64 (one pass and one solve per date)"},
                     "mixed_over_fastest_fp64": min(fp64_ms, fp64s_ms) / ms_per_step},
            "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": 72, "d2h_bytes_per_step": 64},
            "gpu_launches": 3 * args.steps,
            "roofline": dominant, "roofline_sweep": rl_sweep, "roofline_pathgen": rl_gen,
            "mixed16": mixed16, "clocks": ck}
    if not args.no_oos:
        line["oos"] = oos_bench(amc, ctx, torch, stream, opt, hbm, peak_kind)
        line["paper_rule"] = paper_rule_bench(amc, ctx, torch, stream, opt, hbm, peak_kind)
        line["randomization"] = randomization_bench(amc, ctx, torch, stream, opt)
        line["dual"] = dual_bench(amc, ctx, torch, stream, opt)
        line["large"] = large_bench(amc, ctx, torch, stream, hbm, peak_kind)
    if args.serve_seconds > 0:
        times, sopts = workloads.serving_requests(rate=2000.0, duration=args.serve_seconds, seed=4)
        sctx = amc.Context(local, arena_bytes=24 << 30)
        # warm the tables and kernels for every date count the replay will see
        sv = serve_replay(amc, sctx, [0.0] * 8, sopts[:8])
        sv = serve_replay(amc, sctx, list(times), sopts)
        sv["workload"] = "Poisson 2000 req/s, %.0f s of the seed-4 request stream" % args.serve_seconds
        # saturated: the first 2 s of the stream offered at ten times the rate (capacity, not offered load)
        n2 = sum(1 for t in times if t < 2.0)
        sat = serve_replay(amc, sctx, [t / 10.0 for t in times[:n2]], sopts[:n2])
        sat["workload"] = "the first 2 s of the seed-4 stream offered at 10x the rate (20000 req/s)"
        sv["saturated"] = sat
        line["serving"] = sv
        sctx.close()
    if not args.no_batch:
        line.update(batch_and_greeks(amc, local, hbm, peak_kind))
        line["fig1"] = fig1_bench(amc, local)
        line["table2"] = table2_bench(amc, ctx)
    if not args.no_cpu_baseline:
        # the oracle on the whole workload: the CPU baseline, and its price on the same points
        line["cpu_baseline"], ref_price = cpu_baseline(opt)
        if ref_price is not None:
            line["err_vs_oracle_over_K"] = abs(price["price"] - ref_price) / opt.K
            line["mixed16"]["err_vs_oracle_over_K"] = abs(h16_price["price"] - ref_price) / opt.K
    print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # 300 steps of the 1.4 ms bench pricing: a 0.4 s timed region, several clock samples at 100 ms
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["amc", "reference"], default="amc")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batch and Greeks workloads")
    ap.add_argument("--no-oos", action="store_true", help="skip the out-of-sample second pass")
    ap.add_argument("--profile-value", action="store_true",
                    help="run only the boundary valuation launches (for ncu captures)")
    ap.add_argument("--profile-paper", action="store_true",
                    help="run only the paper-rule sweeps (for ncu captures)")
    ap.add_argument("--profile-cluster", action="store_true",
                    help="only the cluster-sweep launches of one 2^18-path option (for ncu)")
    ap.add_argument("--profile-batch", action="store_true",
                    help="run only the 4096-option batch, twice (for ncu launch lists)")
    ap.add_argument("--profile-large", action="store_true",
                    help="run only the streaming LSM sweep of a 2^21-path option (for ncu launch lists)")
    ap.add_argument("--profile-fused", action="store_true",
                    help="run only the paper rule priced with no path array (for ncu captures)")
    ap.add_argument("--profile-dual", action="store_true",
                    help="fit the boundary, then run only two dual upper-bound launches (for ncu captures)")
    ap.add_argument("--profile", action="store_true", help="run only the timed mixed steps (for ncu captures)")
    ap.add_argument("--serve-seconds", type=float, default=5.0,
                    help="length of the Poisson serving replay reported under 'serving' (0: skip)")
    args = ap.parse_args()
    if args.warmup < 3 and not (args.profile or args.profile_value or args.profile_paper or args.profile_batch
                                or args.profile_dual or args.profile_fused or args.profile_large):
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_amc(args)


if __name__ == "__main__":
    main()
