"""Benchmark: certified quantization-based W_2 bounds for many 128 x 128 pairs.

Workload (one step): 180 pairs = 45 pairs (all pairs of 10 seeded images) in
each of four synthetic value classes, 128 x 128 grids, p = 2, kappa = 4
(32 x 32 coarse grid), FP32 cost reductions / IPF (50 sweeps) / c-transforms
with FP64 bound sums (QWB_PREC_MIXED).

value  -- bound pairs/s of the device passes of the method (SumPool + C-bar,
          primal upscaling + IPF + upper bound, dual upscaling + two
          c-transforms + lower bound) in the batched form (persistent launches
          replayed from a CUDA graph), inputs resident in HBM; the exact coarse
          solves (host network simplex) are timed separately (host_solve).
e2e    -- the whole method per step through the public Batch API with host
          buffers: pinned host -> device copies of the measures, the device
          passes, the host exact solves, and the device -> host results.
plain  -- the same device passes launched one pair per kernel launch.
The CPU baseline / reference arm times the FP64 oracle on the same scope as
`value` (its passes, with the coarse solutions precomputed), on a bounded
sample of pairs, one pair per host core.

Multi-GPU: pairs are independent, so each rank processes its own 180 pairs
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N, KAPPA, P, SWEEPS = 128, 4, 2.0, 50
CLASSES = ("white", "gauss", "cauchy", "field")
METRIC = "bound pairs/s at 128×128 p=2 (batched vs plain); % of FP32/HBM roofline"
WORKLOAD = ("180 pairs (4 value classes x 45 pairs) of 128x128 measures, p=2, kappa=4 "
            "(32x32 coarse), FP32 cost/IPF(50 sweeps)/c-transform, FP64 bound sums")


def _workload_arrays(rank: int, per_class: int = 45):
    from paper_2506_00976_gb300 import synth
    mus, nus = [], []
    for ci, cls in enumerate(CLASSES):
        for mu, nu in synth.class_pairs(N, cls, workload=2 + 100 * rank, count=10)[:per_class]:
            mus.append(mu)
            nus.append(nu)
    return mus, nus


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as fh:
                for line in fh:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def _flush_l2(buf):
    buf.add_(1.0)   # a 256 MiB write: larger than the 129 MB L2


def _ct_traffic(digest):
    """DRAM bytes per c-transform launch from the committed ncu summary, or None
    when the kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "ctransform_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    if rec.get("kernel_source_sha256") != digest:
        return None
    return rec.get("dram_bytes_per_launch")


def _kernel_digest():
    """SHA-256 of the c-transform's source (csrc/ctransform.cu), which the
    traffic record names so that a changed kernel invalidates it."""
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_2506_00976_gb300", "csrc", "ctransform.cu"), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2506_00976_gb300 import api

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        raise SystemExit(f"bench.py: --gpus {args.gpus} but {world} rank(s) were started")
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    mus_h, nus_h = _workload_arrays(rank, args.pairs_per_class)
    n = len(mus_h)
    m = N * N
    host = torch.empty((n, 2, m), dtype=torch.float64).pin_memory()
    for t in range(n):
        host[t, 0] = torch.from_numpy(mus_h[t])
        host[t, 1] = torch.from_numpy(nus_h[t])
    dev_buf = host.to(dev)
    mus = [dev_buf[t, 0] for t in range(n)]
    nus = [dev_buf[t, 1] for t in range(n)]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    batch = api.Batch([(N, KAPPA, P)] * n, ipf_sweeps=SWEEPS, prec="mixed", device=dev)

    # exact coarse solves once (host), timed separately
    batch.coarse(mus, nus, batched=True)
    t0 = time.perf_counter()
    batch.solve(threads=args.threads)
    host_solve_s = time.perf_counter() - t0
    results = batch.results()
    assert all(r["status"] == 0 for r in results)
    # the C~ solves alone (the C-bar solves skipped), to split the host time
    with api.Batch([(N, KAPPA, P)] * n, ipf_sweeps=SWEEPS, prec="mixed", flags=api.QWB_FLAG_NO_WEIGHTED,
                   device=dev) as bt_ct:
        bt_ct.coarse(mus, nus, batched=True)
        t0 = time.perf_counter()
        bt_ct.solve(threads=args.threads)
        ctilde_solve_s = time.perf_counter() - t0

    stream = torch.cuda.current_stream(dev)

    def step(batched, bt=None):
        bt = bt or batch
        bt.coarse(mus, nus, batched=batched)
        bt.fine(mus, nus, batched=batched)

    def timed(batched, steps, warmup, per_kernel=False, bt=None):
        bt = bt or batch
        for _ in range(warmup):
            step(batched, bt)
        torch.cuda.synchronize()
        times, kern = [], {}
        launches0 = api.kernel_launch_count()
        for _ in range(steps):
            _flush_l2(flush)
            barrier()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(batched, bt)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            times.append(e0.elapsed_time(e1))
            if per_kernel:
                for k, v in bt.kernel_times().items():
                    kern.setdefault(k, []).append(v)
        launches = api.kernel_launch_count() - launches0
        return times, kern, launches

    with ClockSampler(local) as clk:
        times_b, kern, launches = timed(True, args.steps, args.warmup, per_kernel=True)
    clocks = clk.summary()
    times_p = timed(False, max(1, min(args.steps, 5)), 1)[0] if not args.skip_plain else [float("nan")]

    from paper_2506_00976_gb300 import shard
    ms_b = statistics.mean(times_b)
    ms_p = statistics.mean(times_p)
    ms_b_max = shard.max_over_ranks(ms_b, dev)
    ms_p_max = shard.max_over_ranks(ms_p, dev)
    value = n * world / (ms_b_max * 1e-3)
    plain_value = n * world / (ms_p_max * 1e-3)

    # e2e: whole method through the public API with host buffers
    e2e_steps = max(1, min(args.steps, args.e2e_steps)) if not args.skip_e2e else 0
    e2e_warmup = 1 if e2e_steps else 0
    res_h = results

    def e2e_step():
        dev_buf.copy_(host, non_blocking=True)
        batch.coarse(mus, nus, batched=True)
        batch.solve(threads=args.threads)
        batch.fine(mus, nus, batched=True)
        return batch.results()

    # one untimed step first: the host cores and the GPU leave their idle
    # states (a first step after an idle pause ran up to 5x slower)
    for _ in range(e2e_warmup):
        res_h = e2e_step()
    torch.cuda.synchronize()
    barrier()
    parts = {"h2d_and_coarse_enqueue": [], "solve_call": [], "host_exact_solves": [], "fine_and_results": []}
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ta = time.perf_counter()
        dev_buf.copy_(host, non_blocking=True)
        batch.coarse(mus, nus, batched=True)
        tb = time.perf_counter()
        batch.solve(threads=args.threads)
        tc = time.perf_counter()
        batch.fine(mus, nus, batched=True)
        res_h = batch.results()
        td = time.perf_counter()
        parts["h2d_and_coarse_enqueue"].append(tb - ta)
        parts["solve_call"].append(tc - tb)
        parts["host_exact_solves"].append(res_h[0]["t_solve_ms"] * 1e-3)
        parts["fine_and_results"].append(td - tc)
    torch.cuda.synchronize()
    barrier()
    e2e_s = (time.perf_counter() - t0) / max(1, e2e_steps) if e2e_steps else float("nan")
    e2e_parts = {k: round(1e3 * statistics.mean(v), 3) for k, v in parts.items() if v}
    e2e_s = shard.max_over_ranks(e2e_s, dev)
    assert all(r["status"] == 0 for r in res_h)
    # the same batch with the separable p = 2 c-transform (an exact O(N^3)
    # reformulation, not the paper's N^4 lazy transform): reported beside
    sep_times, sep_kern, sep_res = None, None, None
    lazy_res = batch.results()      # the lazy transform's bounds after the timed passes
    if not args.skip_separable:
        bsep = api.Batch([(N, KAPPA, P)] * n, ipf_sweeps=SWEEPS, prec="mixed",
                         flags=api.QWB_FLAG_SEPARABLE, device=dev)
        bsep.coarse(mus, nus, batched=True)
        bsep.solve(threads=args.threads)
        sep_times, sep_kern, _ = timed(True, args.steps, args.warmup, per_kernel=True, bt=bsep)
        sep_res = bsep.results()
        bsep.close()
    ms_sep_max = shard.max_over_ranks(statistics.mean(sep_times), dev) if sep_times else None

    h2d = int(host.numel() * host.element_size())
    M_C = (N // KAPPA) ** 2          # coarse cells: C-bar (M^2) and mu~, nu~ (M each) come back per pair
    d2h = n * 8 * 14   # the result records read back per step

    out = None
    if rank == 0:
        kmean = {k: statistics.mean(v) for k, v in kern.items() if all(x >= 0 for x in v)}
        pair_ops_ct = 2.0 * float(m) * float(m) * n          # 2 ops per (input, output) pair
        ct_ms = 0.5 * (kmean.get("ctransform_g", 0.0) + kmean.get("ctransform_f", 0.0))
        props = torch.cuda.get_device_properties(dev)
        sms = props.multi_processor_count
        peaks = {}
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
                peaks = json.load(fh)
        except (OSError, ValueError):
            pass
        sm_max = float(peaks.get("sm_max_mhz") or 2070.0)
        fp32_nominal = sms * 128 * 2 * sm_max * 1e6 / 1e12    # TFLOP/s from unit counts and clock
        alu = alu_rates(api)
        fp32_peak = alu["fp32_peak_tflops"]                    # measured FFMA rate x 2 flops
        hbm = float(peaks.get("hbm_gbs") or 6800.0)
        achieved = pair_ops_ct / (ct_ms * 1e-3) / 1e12 if ct_ms > 0 else None
        traffic = _ct_traffic(_kernel_digest())
        cbar_ms = kmean.get("cbar", 0.0)
        cbar_flops = 2.0 * n * (N // KAPPA) ** 4 * (KAPPA ** 4 + KAPPA ** 2)
        primal_ms = kmean.get("primal", 0.0)
        ipf_bytes = 16.0 * m * SWEEPS * n
        passes = {
            "kernel_ms": {k: round(v, 4) for k, v in kmean.items()},
            "cbar": {"bound": "alu", "achieved_tflops": cbar_flops / (cbar_ms * 1e-3) / 1e12 if cbar_ms else None,
                     "frac_of_fp32": (cbar_flops / (cbar_ms * 1e-3) / 1e12) / fp32_peak if cbar_ms else None,
                     "flops_per_launch": cbar_flops},
            "ipf": {"bound": "hbm", "algorithmic_bytes_per_launch": ipf_bytes,
                    "achieved_gbs": ipf_bytes / (primal_ms * 1e-3) / 1e9 if primal_ms else None,
                    "frac_of_hbm": (ipf_bytes / (primal_ms * 1e-3) / 1e9) / hbm if primal_ms else None,
                    "note": "L2-resident working set (180 x 256 KB per sweep); includes the certified "
                            "FP64 sweep and the upper-bound assembly"},
        }
        out = {
            "metric": METRIC, "value": round(value, 3), "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_b_max, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "pairs_per_gpu": n, "N": N, "kappa": KAPPA, "p": P,
                       "ipf_sweeps": SWEEPS, "precision": "mixed", "form": "batched",
                       "l2": "flushed between timed steps (256 MiB write)",
                       "value_scope": "device passes; exact coarse solves timed in host_solve; "
                                      "e2e includes everything"},
            "plain": {"value": round(plain_value, 3), "unit": "pairs/s",
                      "ms_per_step": round(ms_p_max, 4),
                      "batched_over_plain": round(value / plain_value, 3)},
            "roofline": {"kernel": "ctransform (lazy min-plus c-transform)", "bound": "alu",
                         "achieved": round(achieved, 3) if achieved else None,
                         "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                         "frac": round(achieved / fp32_peak, 4) if achieved else None,
                         "traffic": traffic,
                         "peak_source": "measured: fma.rn.f32 rate on this GPU x 2 flops "
                                        "(qwb_probe_fp32_rate, 8 chains per thread, one full wave)",
                         "peak_nominal": round(fp32_nominal, 2),
                         "frac_of_nominal": round(achieved / fp32_nominal, 4) if achieved else None,
                         "nominal_source": f"{sms} SMs x 128 FP32 lanes x 2 ops x {sm_max:.0f} MHz",
                         "frac_of_mix_ceiling": round(pair_ops_ct / 2 / (ct_ms * 1e-3) / alu["mix_ceiling_per_s"], 4)
                         if ct_ms > 0 else None,
                         "ops_per_launch": pair_ops_ct, "avg_launch_ms": round(ct_ms, 4)},
            "alu_rates": alu,
            "passes": passes,
            "host_solve": {"seconds": round(host_solve_s, 3),
                           "ctilde_only_seconds": round(ctilde_solve_s, 3),
                           "pairs_per_s": round(n / host_solve_s, 3),
                           "threads": args.threads or os.cpu_count(),
                           "what": "network simplex on C~ and C-bar (M = 1024) per pair"},
            "e2e": {"value": round(n * world / e2e_s, 3), "unit": "pairs/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps, "warmup": e2e_warmup, "ms_per_step": round(1e3 * e2e_s, 3),
                    "internal_d2h_bytes_per_step": n * (M_C * M_C + 2 * M_C) * 8,
                    "parts_ms": e2e_parts,
                    "parts_note": "host wall time of each API call per step: the copy of the measures and "
                                  "the asynchronous coarse pass; qwb_batch_solve (waits for the coarse "
                                  "pass, reads C-bar back, runs the host exact solves, uploads the plans); "
                                  "of which the exact solves alone; the fine passes and the results read"},
            "gpu_launches": int(launches),
            "autotune": batch.tuning(),
            "clocks": clocks,
        }
        if sep_times:
            skm = {k: statistics.mean(v) for k, v in sep_kern.items() if all(x >= 0 for x in v)}
            sct_ms = 0.5 * (skm.get("ctransform_g", 0.0) + skm.get("ctransform_f", 0.0))
            sep_ops = 2.0 * 2.0 * float(N) ** 3 * n          # 2 stages x N^3 pairs x 2 ops
            cbar_bytes = 8.0 * M_C * M_C * n                  # the FP64 C-bar written
            hbm_peak = 6700.8
            try:
                with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
                    hbm_peak = float(json.load(fh).get("hbm_gbs") or hbm_peak)
            except (OSError, ValueError):
                pass
            dlb = max(abs(a["lb"] - b["lb"]) / max(b["lb"], 1e-300) for a, b in zip(sep_res, lazy_res))
            out["separable_p2"] = {
                "value": round(n * world / (ms_sep_max * 1e-3), 3), "unit": "pairs/s",
                "ms_per_step": round(ms_sep_max, 4),
                "kernel_ms": {k: round(v, 4) for k, v in skm.items()},
                "ctransform": {"bound": "alu", "ops_per_launch": sep_ops, "avg_launch_ms": round(sct_ms, 4),
                               "achieved_tflops": round(sep_ops / (sct_ms * 1e-3) / 1e12, 3) if sct_ms else None,
                               "frac_of_fp32": round(sep_ops / (sct_ms * 1e-3) / 1e12 / fp32_peak, 4)
                               if sct_ms else None},
                "cbar": {"bound": "hbm", "bytes_per_launch": cbar_bytes,
                         "avg_launch_ms": round(skm.get("cbar", 0.0), 4),
                         "achieved_gbs": round(cbar_bytes / (skm["cbar"] * 1e-3) / 1e9, 1)
                         if skm.get("cbar") else None,
                         "frac_of_hbm": round(cbar_bytes / (skm["cbar"] * 1e-3) / 1e9 / hbm_peak, 4)
                         if skm.get("cbar") else None,
                         "note": "separable C-bar: 2 kappa^2 + 2 kappa multiply-adds per block pair; bound "
                                 "by writing the FP64 M x M matrix (bytes = 8 M^2 per pair)"},
                "max_rel_lb_diff_vs_lazy": dlb,
                "note": "QWB_FLAG_SEPARABLE: p = 2 c-transform as two 1-D transforms (2 N^3 pairs "
                        "each) instead of the N^4 lazy transform, and the C-bar sum regrouped over "
                        "the two axes (row and column sums of each block); same certified rounding"}
        if not args.skip_workloads:
            out["uneven_200"] = _uneven_workload(api, dev, args)
            out["differentiable_256"] = _differentiable_workload(api, dev, args)
            out["ipf_hbm"] = _ipf_hbm_workload(api, dev, args)
            out["ipf_hbm_76"] = _ipf_hbm_workload(api, dev, args, n_pairs=76)
            out["workload_64"] = _workload_64(api, dev, args)
            out["kernel_upscale"] = _kernel_upscale_workload(api, dev, args)
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args.cpu_seconds, args.cpu_workers)
    batch.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return out


_ALU = None


def alu_rates(api):
    """FP32 instruction rates of this GPU (qwb_probe_fp32_rate): the measured
    FP32 peak (fma.rn.f32 x 2 flops) and the c-transform's instruction-mix
    ceiling (the best two-candidate mix: packed round-down subtraction or two
    scalar ones, then a three-input min)."""
    global _ALU
    if _ALU is not None:
        return _ALU
    api.probe_fp32_rate(0, iters=16384)             # clocks up before the measured runs
    rows = [api.probe_fp32_rate(k) for k in range(8)]
    mix = max(rows[6]["per_s"], rows[7]["per_s"])
    _ALU = {"fp32_peak_tflops": round(2.0 * rows[0]["per_s"] / 1e12, 3),
            "mix_ceiling_per_s": mix,
            "mix_ceiling_tops": round(2.0 * mix / 1e12, 3),
            "per_s": {r["kind"]: round(r["per_s"] / 1e12, 4) for r in rows},
            "per_cycle_per_sm": {r["kind"]: round(r["per_clk_per_sm"], 2) for r in rows},
            "counter_mhz": {r["kind"]: round(r["counter_mhz"], 1) for r in rows},
            "ctas_per_sm": {r["kind"]: [r["ctas_per_sm"], r["most_ctas_on_one_sm"]] for r in rows},
            "what": "FP32 results (packed: 2 per instruction; mixes: candidates) per second (x1e12, CUDA "
                    "events) and per cycle of each SM's cycle counter; 8 independent chains per thread, "
                    "256-thread CTAs; ctas_per_sm = [requested, most on one SM]"}
    return _ALU


def alu_sweep(api):
    """The c-transform's instructions (kinds 3, 5, 6, 7 of qwb_probe_fp32_rate)
    at 1-8 resident 256-thread CTAs per SM: how the rates depend on the number
    of warps an SM can interleave."""
    api.probe_fp32_rate(0, iters=16384)
    out = {}
    for k in (0, 3, 5, 6, 7):
        out[api.PROBE_KINDS[k]] = {c: round(api.probe_fp32_rate(k, ctas_per_sm=c)["per_s"] / 1e12, 3)
                                   for c in (1, 2, 3, 4, 6, 8)}
    return {"per_s_x1e12_by_ctas_per_sm": out}


# ----------------------------------------------------------------------------
# secondary workloads (reported beside the headline, rank 0)
# ----------------------------------------------------------------------------
def _event_ms(fn, steps, warmup, flush):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    times = []
    for _ in range(steps):
        _flush_l2(flush)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.mean(times)


def _uneven_workload(api, dev, args):
    """200 pairs with N in {32, 64, 128, 256}, kappa in {4, 8}, p in {1, 2}, one
    batch (autotuned persistent launches replayed from CUDA graphs)."""
    import torch
    from paper_2506_00976_gb300 import synth
    W = synth.uneven_workload(200)
    mus = [torch.tensor(w["mu"], dtype=torch.float64, device=dev) for w in W]
    nus = [torch.tensor(w["nu"], dtype=torch.float64, device=dev) for w in W]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    with api.Batch([(w["N"], w["kappa"], w["p"]) for w in W], ipf_sweeps=SWEEPS, prec="mixed",
                   device=dev) as bt:
        bt.coarse(mus, nus, batched=True)
        t0 = time.perf_counter()
        bt.solve(threads=args.threads)
        solve_s = time.perf_counter() - t0

        def step():
            bt.coarse(mus, nus, batched=True)
            bt.fine(mus, nus, batched=True)
        ms = _event_ms(step, max(3, min(args.steps, 5)), 3, flush)
        kern = {k: round(v, 4) for k, v in bt.kernel_times().items()}
        res = bt.results()
        assert all(r["status"] == 0 for r in res)
        sizes = {}
        for w in W:
            sizes[w["N"]] = sizes.get(w["N"], 0) + 1
        return {"value": round(len(W) / (ms * 1e-3), 3), "unit": "pairs/s", "ms_per_step": round(ms, 4),
                "kernel_ms": kern, "pairs_by_N": sizes, "host_solve_s": round(solve_s, 3),
                "what": "device passes (SumPool, C-bar, IPF 50 sweeps + upper bound, c-transforms + "
                        "lower bound) of one batch of 200 uneven pairs; host exact solves separate",
                "autotune": bt.tuning()}


def _workload_64(api, dev, args):
    """45 pairs of each value class at 64 x 64 (kappa 4, 16 x 16 coarse) for
    p = 1 and p = 2, one batch per p: pairs/s and per-pass device times."""
    import torch
    from paper_2506_00976_gb300 import synth
    Nw, kw = 64, 4
    raw = []
    for cls in CLASSES:
        raw += synth.class_pairs(Nw, cls, 1)
    mus = [torch.tensor(a, dtype=torch.float64, device=dev) for a, _ in raw]
    nus = [torch.tensor(b, dtype=torch.float64, device=dev) for _, b in raw]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    out = {}
    for p in (1.0, 2.0):
        with api.Batch([(Nw, kw, p)] * len(raw), ipf_sweeps=SWEEPS, prec="mixed", device=dev) as bt:
            bt.coarse(mus, nus, batched=True)
            t0 = time.perf_counter()
            bt.solve(threads=args.threads)
            solve_s = time.perf_counter() - t0

            def step():
                bt.coarse(mus, nus, batched=True)
                bt.fine(mus, nus, batched=True)
            ms = _event_ms(step, max(3, min(args.steps, 5)), 3, flush)
            kern = {k: round(v, 4) for k, v in bt.kernel_times().items()}
            assert all(r["status"] == 0 for r in bt.results())
        out[f"p{int(p)}"] = {"value": round(len(raw) / (ms * 1e-3), 3), "unit": "pairs/s",
                             "ms_per_step": round(ms, 4), "kernel_ms": kern,
                             "host_solve_s": round(solve_s, 3)}
    out["what"] = ("180 pairs (4 classes x 45) of 64x64, kappa 4, MIXED, 50 IPF sweeps, batched device "
                   "passes; host exact solves separate")
    return out


def _ipf_hbm_workload(api, dev, args, n_pairs=45):
    """The IPF sweeps on a working set larger than L2: n_pairs pairs of
    512 x 512 (kappa 8, 64 x 64 coarse), 50 sweeps, 4.2 MB per pair and sweep
    (45 pairs: 189 MB per sweep > the 129 MB L2).  Only the primal pass runs
    (C-bar and the dual pass off)."""
    import torch
    from paper_2506_00976_gb300 import synth
    Nh, kh, sweeps = 512, 8, SWEEPS
    pairs = []
    for ci, cls in enumerate(CLASSES):
        pairs += synth.class_pairs(Nh, cls, 6, count=6 if n_pairs <= 60 else 8)[:(n_pairs + 3) // 4]
    pairs = pairs[:n_pairs]
    mus = [torch.tensor(a, dtype=torch.float64, device=dev) for a, _ in pairs]
    nus = [torch.tensor(b, dtype=torch.float64, device=dev) for _, b in pairs]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    with api.Batch([(Nh, kh, 2.0)] * len(pairs), ipf_sweeps=sweeps, prec="mixed", flags=1 | 4,
                   device=dev) as bt:
        bt.coarse(mus, nus, batched=True)
        t0 = time.perf_counter()
        bt.solve(threads=args.threads)
        solve_s = time.perf_counter() - t0

        def step():
            bt.fine(mus, nus, batched=True)
        ms = _event_ms(step, 3, 3, flush)
        kern = bt.kernel_times()
        res = bt.results()
        assert all(r["status"] == 0 for r in res)
        tuning = bt.tuning()
    m = Nh * Nh
    nbytes = 16.0 * m * sweeps * len(pairs)
    ipf_ms = kern.get("ipf_cluster", 0.0)
    sweep_ms = ipf_ms if ipf_ms > 0 else kern.get("primal", ms)
    hbm = 6792.1
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            hbm = float(json.load(fh).get("hbm_gbs") or hbm)
    except (OSError, ValueError):
        pass
    return {"bound": "hbm", "pairs": len(pairs), "N": Nh, "kappa": kh, "sweeps": sweeps,
            "bytes_per_sweep": 16.0 * m * len(pairs), "algorithmic_bytes": nbytes,
            "sweeps_ms": round(sweep_ms, 4), "primal_pass_ms": round(kern.get("primal", 0.0), 4),
            "achieved_gbs": round(nbytes / (sweep_ms * 1e-3) / 1e9, 1) if sweep_ms > 0 else None,
            "peak_gbs": hbm,
            "frac_of_hbm": round(nbytes / (sweep_ms * 1e-3) / 1e9 / hbm, 4) if sweep_ms > 0 else None,
            "ipf_cluster": tuning.get("ipf"), "host_solve_s": round(solve_s, 3),
            "what": "fine IPF sweeps (16 B per pixel and sweep: read mu, write a, read nu, write b) on a "
                    "working set larger than L2; sweeps_ms is the cluster sweep kernel, or the whole "
                    "primal kernel when the sweeps run inside it"}


def _kernel_upscale_workload(api, dev, args):
    """The primal pass with a general upscaling kernel (Gaussian over the
    in-block offsets, sigma = 1 px) on the headline pairs: 180 pairs of
    128 x 128, kappa 4, p 2, 50 FP32 sweeps; only the primal pass runs.  The
    same pairs with 500 sweeps, with the uniform kernel and with the
    weighted-cost bound are run beside it, and the bounds are compared."""
    import numpy as np
    import torch
    from paper_2506_00976_gb300 import synth
    mus_h, nus_h = _workload_arrays(0)
    mus = [torch.tensor(a, dtype=torch.float64, device=dev) for a in mus_h]
    nus = [torch.tensor(b, dtype=torch.float64, device=dev) for b in nus_h]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    K = synth.gaussian_offset_kernel(KAPPA, 1.0)
    out, ubs = {}, {}
    for name, kern_K, sweeps, flags in (("gaussian", K, SWEEPS, 1 | 4), ("gaussian_single_cta", K, SWEEPS, 1 | 4),
                                        ("gaussian_500", K, 500, 1 | 4), ("uniform", None, SWEEPS, 4)):
        with api.Batch([(N, KAPPA, P)] * len(mus), ipf_sweeps=sweeps, prec="mixed", flags=flags,
                       device=dev) as bt:
            if kern_K is not None:
                bt.set_upscale_kernel(KAPPA, kern_K)
            if name == "gaussian_single_cta":
                bt.set_upscale_cluster(0)          # the one-CTA-per-pair kernel, for comparison
            bt.coarse(mus, nus, batched=True)
            bt.solve(threads=args.threads)

            def step():
                bt.fine(mus, nus, batched=True)
            ms = _event_ms(step, 3 if sweeps > SWEEPS else max(3, min(args.steps, 5)), 3, flush)
            kt = bt.kernel_times()
            res = bt.results()
            assert all(r["status"] == 0 for r in res)
            form = bt.tuning().get("upscale_kernel") if kern_K is not None else None
        out[name] = {"sweeps": sweeps, "ms_per_step": round(ms, 4), "primal_pass_ms": round(kt.get("primal", 0.0), 4),
                     "ipf_cluster_ms": round(kt.get("ipf_cluster", 0.0), 4)}
        if form is not None:
            out[name]["form"] = form
        ubs[name] = np.array([r["ub_primal"] for r in res])
        if name == "uniform":
            ubs["weighted"] = np.array([r["ub_weighted"] for r in res])
    # a smaller batch, 40 pairs (at most one per SM): the cluster form spreads
    # each pair over several SMs; the tuned pass beside the one-CTA kernel
    small = {}
    for name, single in (("tuned", False), ("single_cta", True)):
        with api.Batch([(N, KAPPA, P)] * 40, ipf_sweeps=SWEEPS, prec="mixed", flags=1 | 4, device=dev) as bt:
            bt.set_upscale_kernel(KAPPA, K)
            if single:
                bt.set_upscale_cluster(0)
            bt.coarse(mus[:40], nus[:40], batched=True)
            bt.solve(threads=args.threads)

            def step():
                bt.fine(mus[:40], nus[:40], batched=True)
            ms = _event_ms(step, max(3, min(args.steps, 5)), 3, flush)
            kt = bt.kernel_times()
            assert all(r["status"] == 0 for r in bt.results())
            small[name] = {"ms_per_step": round(ms, 4), "primal_pass_ms": round(kt.get("primal", 0.0), 4),
                           "form": bt.tuning().get("upscale_kernel")}
    out["gaussian_40_pairs"] = small
    m, kk, n = N * N, KAPPA * KAPPA, len(mus)
    flops = 4.0 * m * kk * SWEEPS * n          # the K products: 2 halves x m kk FMAs per sweep
    kms = out["gaussian"]["primal_pass_ms"]
    props = torch.cuda.get_device_properties(dev)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except (OSError, ValueError):
        pass
    fp32_nominal = props.multi_processor_count * 128 * 2 * float(peaks.get("sm_max_mhz") or 2070.0) * 1e6 / 1e12
    fp32_peak = alu_rates(api)["fp32_peak_tflops"]
    achieved = flops / (kms * 1e-3) / 1e12 if kms > 0 else None
    g5 = ubs["gaussian_500"]
    out.update({
        "pairs": n, "N": N, "kappa": KAPPA, "p": P, "sweeps": SWEEPS, "sigma_px": 1.0,
        "value": round(n / (kms * 1e-3), 3) if kms > 0 else None, "unit": "pairs/s (primal pass)",
        "roofline": {"bound": "fp32", "achieved": round(achieved, 3) if achieved else None,
                     "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                     "frac": round(achieved / fp32_peak, 4) if achieved else None,
                     "peak_source": "measured fma.rn.f32 rate (qwb_probe_fp32_rate) x 2 flops",
                     "frac_of_nominal": round(achieved / fp32_nominal, 4) if achieved else None,
                     "flops_per_launch": flops},
        "ub_mean": {k: float(v.mean()) for k, v in ubs.items()},
        "gaussian_500_below": {"uniform": int((g5 < ubs["uniform"]).sum()),
                               "weighted": int((g5 < ubs["weighted"]).sum())},
        "what": "general-kernel primal pass (primalk_cl_kernel on clusters, primalk_kernel one CTA per pair, or "
                "its sweeps with the evaluation spread over one CTA per block row, as tuned; "
                "gaussian_single_cta forces the one-CTA kernel): IPF of pi~ (x) K with a Gaussian K, FP32 sweeps, "
                "certified FP64 evaluation; "
                "achieved counts the K products only (4 m kappa^2 FLOP per sweep, the plan gather's "
                "<= 4 (2M - 1) kappa^2 not counted); 'uniform' is the uniform primal pass (cluster sweeps + "
                "primal kernel) of a batch that also computes the weighted-cost bound; gaussian_500_below "
                "counts the pairs whose 500-sweep Gaussian bound is below the other bound"})
    return out


def _differentiable_workload(api, dev, args):
    """16 smooth-field pairs of 256 x 256, p = 2, kappa 4: the lower bound's
    device passes and the adjoint kernel's gradient with respect to mu."""
    import torch
    from paper_2506_00976_gb300 import synth
    Nd, kd, pd = 256, 4, 2.0
    pairs = synth.class_pairs(Nd, "field", 4)[:16]
    mus = [torch.tensor(a, dtype=torch.float64, device=dev) for a, _ in pairs]
    nus = [torch.tensor(b, dtype=torch.float64, device=dev) for _, b in pairs]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    with api.Batch([(Nd, kd, pd)] * len(pairs), ipf_sweeps=1, prec="mixed", flags=1 | 2,
                   device=dev) as bt:
        bt.coarse(mus, nus, batched=True)
        bt.solve(threads=args.threads)
        bt.fine(mus, nus, batched=True)
        res = bt.results()
        fs = [bt.potentials(t)[0] for t in range(len(pairs))]

        def fwd():
            bt.coarse(mus, nus, batched=True)
            bt.fine(mus, nus, batched=True)

        def adj():
            for t in range(len(pairs)):
                api.lb_adjoint(fs[t], mus[t], Nd, pd, res[t]["lb_p"])
        ms_f = _event_ms(fwd, 3, 3, flush)
        ms_a = _event_ms(adj, 3, 3, flush)
    return {"value": round(len(pairs) / ((ms_f + ms_a) * 1e-3), 3), "unit": "pairs/s",
            "forward_ms": round(ms_f, 4), "adjoint_ms": round(ms_a, 4),
            "what": "16 pairs of 256x256 smooth random fields, kappa 4 (64x64 coarse), p 2: lower-bound "
                    "device passes (SumPool, upsample, two lazy c-transforms, sum) plus the adjoint "
                    "kernel for every pair; host exact solves excluded"}


# ----------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ----------------------------------------------------------------------------
def _oracle_pair(args):
    """The oracle's passes for one pair with its coarse solution given."""
    mu, nu, plan, f_c = args
    from oracle import qwb_oracle as O
    t0 = time.perf_counter()
    O.coarse_cost_weighted(mu, nu, N, KAPPA, P)
    O.ub_primal(mu, nu, N, KAPPA, P, xi=1e-13, max_sweeps=SWEEPS, plan_c=plan)
    O.lb_dual(mu, nu, N, KAPPA, P, f_c=f_c)
    return time.perf_counter() - t0


def _oracle_coarse(args):
    mu, nu = args
    from oracle import qwb_oracle as O
    mt, nt = O.sumpool(mu, N, KAPPA), O.sumpool(nu, N, KAPPA)
    plan, f_c, _, _ = O.exact_ot(O.coarse_cost_centre(N, KAPPA, P), mt, nt)
    return plan, f_c


def _pool(workers):
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(workers)


def cpu_baseline(seconds, workers):
    """Oracle pairs/s on a bounded sample: `workers` pairs in parallel, one per core."""
    from oracle import build as oracle_build
    oracle_build.build()
    workers = workers or min(os.cpu_count() or 1, 16)
    mus, nus = _workload_arrays(0)
    idx = list(range(0, len(mus), max(1, len(mus) // workers)))[:workers]
    with _pool(workers) as pool:
        coarse = pool.map(_oracle_coarse, [(mus[i], nus[i]) for i in idx])
        t0 = time.perf_counter()
        pool.map(_oracle_pair, [(mus[i], nus[i], c[0], c[1]) for i, c in zip(idx, coarse)])
        wall = time.perf_counter() - t0
    return {"value": round(len(idx) / wall, 4), "unit": "pairs/s", "cores": workers,
            "kind": "oracle",
            "sample": f"{len(idx)} pairs of the 128x128 workload (one per core), oracle passes "
                      f"(C-bar, IPF + upper bound, c-transforms + lower bound), coarse solutions "
                      f"precomputed by the oracle's own solver; {wall:.1f} s wall"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    from oracle import build as oracle_build
    oracle_build.build()
    workers = args.cpu_workers or min(os.cpu_count() or 1, 16)
    mus, nus = _workload_arrays(0)
    idx = list(range(0, len(mus), max(1, len(mus) // workers)))[:workers]
    with _pool(workers) as pool:
        coarse = pool.map(_oracle_coarse, [(mus[i], nus[i]) for i in idx])
        jobs = [(mus[i], nus[i], c[0], c[1]) for i, c in zip(idx, coarse)]
        for _ in range(args.warmup):        # warm-up: one pair (imports, first-touch)
            pool.map(_oracle_pair, jobs[:1])
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            pool.map(_oracle_pair, jobs)
            times.append(time.perf_counter() - t0)
    ms = statistics.mean(times) * 1e3
    value = len(jobs) / (ms * 1e-3)
    return {"metric": METRIC, "value": round(value, 4), "unit": "pairs/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "N": N, "kappa": KAPPA, "p": P,
                       "ipf_sweeps": SWEEPS, "form": "FP64 CPU oracle",
                       "value_scope": "oracle passes with precomputed coarse solutions"},
            "cpu_baseline": {"value": round(value, 4), "unit": "pairs/s", "cores": workers,
                             "kind": "oracle",
                             "sample": f"{len(jobs)} pairs per step, one per core"},
            "e2e": {"value": round(value, 4), "unit": "pairs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def launch_ranks(n, argv):
    """`bench.py --gpus N` outside a launcher: start N ranks on this node (one
    process per GPU) with torch.distributed.run on 127.0.0.1 and return its
    exit status; each rank reads RANK / LOCAL_RANK / WORLD_SIZE from the env."""
    import socket
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__), *argv]
    return subprocess.call(cmd)


def run_dry(args):
    """The multi-rank plumbing without a GPU (gloo): every rank builds its own
    pair list (weak scaling), ranks meet at a barrier, and rank 0 reports the
    per-rank pair counts and the maximum over ranks of a per-rank time."""
    import torch.distributed as dist
    from paper_2506_00976_gb300 import shard
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world != args.gpus:
        raise SystemExit(f"bench.py: --gpus {args.gpus} but {world} rank(s) were started")
    if world > 1:
        dist.init_process_group("gloo")
    t0 = time.perf_counter()
    mus, _ = _workload_arrays(rank, args.pairs_per_class)
    local_s = time.perf_counter() - t0
    digest = hashlib.sha256(mus[0].tobytes()).hexdigest()[:12]
    counts, digests = [len(mus)] * world, [digest] * world
    if world > 1:
        gathered = [None] * world
        dist.all_gather_object(gathered, (len(mus), digest))
        counts = [g[0] for g in gathered]
        digests = [g[1] for g in gathered]
        dist.barrier()
    slowest = shard.max_over_ranks(local_s)
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return None
    return {"dry_run": True, "n_gpus": world, "pairs_per_rank": counts, "first_pair_digest": digests,
            "max_rank_seconds": round(slowest, 4), "backend": "gloo" if world > 1 else "none"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--threads", type=int, default=0, help="host solver threads (0 = all cores)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--cpu-workers", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--pairs-per-class", type=int, default=45,
                    help="pairs per value class (45 = the full workload; smaller for profiling)")
    ap.add_argument("--skip-plain", action="store_true", help="time only the batched form")
    ap.add_argument("--skip-e2e", action="store_true", help="skip the end-to-end timing")
    ap.add_argument("--only", default="", choices=["", "ipf_hbm", "ipf_hbm_76", "uneven_200", "differentiable_256",
                                                   "workload_64", "kernel_upscale", "alu_rates", "alu_sweep"],
                    help="run one secondary workload alone and print its JSON (profiling)")
    ap.add_argument("--skip-workloads", action="store_true",
                    help="skip the uneven 200-pair and differentiable 256x256 measurements")
    ap.add_argument("--skip-separable", action="store_true",
                    help="skip the separable p = 2 c-transform measurement")
    ap.add_argument("--dry-run", action="store_true",
                    help="check the multi-rank launch on the CPU (gloo), no GPU work")
    args = ap.parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ and args.impl == "native":
        sys.exit(launch_ranks(args.gpus, sys.argv[1:]))    # one process per GPU
    if args.dry_run:
        out = run_dry(args)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if args.warmup < 3 and args.impl == "native":
        args.warmup = 3
    if args.only:
        import torch
        from paper_2506_00976_gb300 import api
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        fn = {"ipf_hbm": _ipf_hbm_workload, "uneven_200": _uneven_workload,
              "ipf_hbm_76": lambda a, d, r: _ipf_hbm_workload(a, d, r, n_pairs=76),
              "differentiable_256": _differentiable_workload, "workload_64": _workload_64,
              "kernel_upscale": _kernel_upscale_workload,
              "alu_rates": lambda a, d, r: alu_rates(a),
              "alu_sweep": lambda a, d, r: alu_sweep(a)}[args.only]
        print(json.dumps({args.only: fn(api, dev, args)}), flush=True)
        return
    out = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
