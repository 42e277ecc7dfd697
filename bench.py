#!/usr/bin/env python
"""Benchmark: forward + adjoint gradient evaluations per second at 256^3.

Workload: one chain per GPU, 256^3 mesh, L = 1000 Mpc/h, ALPT (r_s = 4) + CIC,
Phi x delta web (16 regions, Table 3 bias), NB likelihood; FP32 fields with
FP64 reductions.  A step is one full log-posterior + gradient evaluation
(every stage of the forward model and of its adjoint).

  value      device-resident inputs, CUDA events on the context stream,
             max over ranks; grad evals/s for the whole job
  e2e        the same through bridge_logpost_grad_host: pinned host nu and
             counts copied in and the gradient copied out inside every step
  roofline   dominant kernel class from live CUDA-event timing of its
             launches; algorithmic bytes = each launch's distinct inputs read
             once and outputs written once; peak = measured copy bandwidth
  cpu_baseline  the FP64 oracle on the host cores (bounded sample)

`--impl reference` times the FP64 CPU oracle instead (the paper has no code).
Under torchrun (N > 1) every rank runs its own chain (replicas, weak scaling).
"""
from __future__ import annotations

import argparse
import copy
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "forward+adjoint grad evals/s at 256^3 (FP32 batched vs FP64 plain); % HBM peak"
UNIT = "grad evals/s"
WORKLOAD_INDEX = 2               # 256^3, L = 1000, Phi x delta web
SMALL_CASE_INDEX = 1             # 128^3, L = 1000, Phi x delta web (small ncu captures)
MODEL_R = {16: 226, 4: 178}      # canonical algorithmic bytes per evaluation, in units of R = 4 N^3 bytes
FALLBACK_HBM = 6800.0


# ---------------------------------------------------------------------------
# host-side helpers (also exercised by the CPU multi-process tests)
# ---------------------------------------------------------------------------
def rank_seeds(cfg, rank: int):
    """Independent chains per rank: seeds offset by the rank."""
    return cfg.seed_eval + 1000 * rank, cfg.seed_counts + 1000 * rank


def max_over_ranks(value: float, dist=None) -> float:
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": FALLBACK_HBM}, "fallback"


def csrc_hash(files=None) -> str:
    """sha1 (first 12 hex digits) over the CUDA sources: every file under csrc, or the listed
    ones (names and contents, in sorted order)."""
    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_2506_03969_gb300", "csrc")
    for name in sorted(files if files is not None else os.listdir(d)):
        path = os.path.join(d, name)
        if not os.path.isfile(path):
            return "missing"
        with open(path, "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:12]


def recorded_traffic(kernel: str, alg_bytes_per_launch: float):
    """DRAM bytes per launch from the committed ncu record, if it was taken on the current sources.

    profiles/dram_traffic.json holds, per kernel class, the source hash of the capture and the
    ratio of DRAM bytes to algorithmic bytes per launch; the ratio times the algorithmic bytes of
    the timed launch is the traffic.  A record may name the source files that define the kernel
    ("sources": its translation unit and the headers it includes); the hash then covers those
    files only, else every file under csrc.  Records of other sources give None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        data = json.load(f)
    for r in data.get("records", []):
        if r.get("kernel") == kernel and r.get("csrc_hash") == csrc_hash(r.get("sources")):
            return float(r["dram_over_algorithmic"]) * alg_bytes_per_launch
    return None


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(device_index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing
# ---------------------------------------------------------------------------
def oracle_eval_seconds(n: int, seed: int) -> float:
    import numpy as np
    import torch
    import synth
    from oracle import model
    cfg = synth.config(WORKLOAD_INDEX)
    cfg.n = n
    cfg.box = 1000.0 * n / 256.0                     # same cell size as the timed workload
    bias = synth.default_bias(cfg)
    nu = synth.white_noise(n, seed)
    counts = synth.timing_counts(n, seed + 1, cfg.mean_tracers)
    t0 = time.perf_counter()
    model.logpost_and_grad(nu, counts, cfg, bias)
    return time.perf_counter() - t0


def oracle_sample(budget_s: float):
    """Largest mesh whose single oracle gradient fits the budget; throughput scaled
    to 256^3 evaluations by the voxel count (an upper bound for the CPU)."""
    import torch
    threads = torch.get_num_threads()
    t64 = oracle_eval_seconds(64, 9000)
    n, t = 64, t64
    for cand in (128, 256):
        est = t * 8.5
        if est > budget_s:
            break
        t = oracle_eval_seconds(cand, 9000)
        n = cand
    scale = (n / 256.0) ** 3
    return {"value": scale / t, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"one FP64 oracle gradient at {n}^3 (same cell size, 16 regions) took {t:.2f} s on "
                      f"{threads} threads; scaled to 256^3 by voxel count (x{1/scale:g})",
            "seconds": t, "mesh": n}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, each step a bounded sample."""
    import torch
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    threads = torch.get_num_threads()
    # mesh per step sized so that warm-up + steps fit in about two minutes
    per_step = 120.0 / max(1, args.steps + args.warmup)
    t32 = oracle_eval_seconds(32, 9100)
    n = 32
    for cand, factor in ((64, 10.0), (128, 75.0), (256, 650.0)):
        if t32 * factor <= per_step:
            n = cand
    for _ in range(args.warmup):
        oracle_eval_seconds(n, 9100)
    times = [oracle_eval_seconds(n, 9100 + s) for s in range(args.steps)]
    total = sum(times)
    scale = (n / 256.0) ** 3
    value = args.steps * scale / total
    cfg = workload_config(1)
    cfg.update({"timed_mesh": n, "timed_box_mpc_h": 1000.0 * n / 256.0,
                "sample": f"each step is one FP64 oracle gradient at {n}^3 (same cell size as 256^3); "
                          f"value = steps / time x (n/256)^3 = {scale:g}, i.e. 256^3 evaluations per second "
                          f"if the oracle's cost grows with the voxel count; ms_per_step is the measured "
                          f"{n}^3 step"})
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"each step one FP64 oracle gradient at {n}^3 (same cell size); "
                                       f"throughput scaled to 256^3 by voxel count (x{1/scale:g})"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def workload_config(batch: int, n: int = 256):
    if n != 256:   # --small-case: the 128^3 profiling case, not the headline workload
        return {"workload": f"{n}^3 mesh, L=1000 Mpc/h, Phi x delta web (16 regions): small profiling case, "
                            "not the headline workload", "n": n, "box_mpc_h": 1000.0, "chains_per_gpu": batch,
                "regions": 16, "precision": "FP32 fields, FP64 reductions"}
    return {"workload": "256^3 mesh, L=1000 Mpc/h, ALPT r_s=4 + CIC, Phi x delta web (16 regions, Table 3 bias), "
                        "NB likelihood; forward + hand-written adjoint per step",
            "n": 256, "box_mpc_h": 1000.0, "chains_per_gpu": batch, "regions": 16,
            "precision": "FP32 fields, FP64 reductions",
            "l2": "working set ~3.7 GB per chain and ~15 GB moved per evaluation, far above the 129 MB L2"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)

    import paper_2506_03969_gb300 as pkg
    from paper_2506_03969_gb300 import build as pbuild
    import synth
    if rank == 0:
        pbuild.build()
    if world > 1:
        dist.barrier()

    cfg = synth.config(SMALL_CASE_INDEX if args.small_case else WORKLOAD_INDEX)
    bias = synth.default_bias(cfg)
    seed_nu, seed_c = rank_seeds(cfg, rank)
    nu_h = torch.tensor(synth.white_noise(cfg.n, seed_nu), dtype=torch.float32).contiguous()
    c_h = torch.tensor(synth.timing_counts(cfg.n, seed_c, cfg.mean_tracers), dtype=torch.int32).contiguous()
    ctx = pkg.Context(pkg.config_from(cfg, batch=1))
    nu = nu_h.cuda()
    counts = c_h.cuda()
    grad = torch.empty_like(nu)
    stream = ctx.stream

    # launch shapes picked on this problem before the warm-up (outside every timed region)
    tune = None
    if not args.no_autotune:
        t_tune = time.perf_counter()
        ch = ctx.bridge_autotune(nu, counts, [bias])
        torch.cuda.synchronize()
        tune = {"node_alpt_cps": ch[0], "node_alpt_adj_cps": ch[1], "node_cic_gather_cps": ch[2],
                "web_bias_adj_blocks": ch[3], "note": "0 = built-in choice",
                "seconds": round(time.perf_counter() - t_tune, 2)}

    for _ in range(args.warmup):
        ctx.bridge_logpost_grad(nu, counts, [bias], grad_out=grad, want_bias_grad=False)
    launches_per_step = ctx.launches()

    # --- timed region: device-resident inputs -------------------------------
    sampler = ClockSampler(local) if rank == 0 else None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        lp, _, _ = ctx.bridge_logpost_grad(nu, counts, [bias], grad_out=grad, want_bias_grad=False)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    elapsed = e0.elapsed_time(e1) / 1e3
    elapsed = max_over_ranks(elapsed, dist if world > 1 else None)
    value = args.steps * world / elapsed

    # --- per-kernel-class CUDA-event timing (separate pass, same work) ------
    ctx.bridge_profile_enable(True)
    prof_steps = max(1, min(args.steps, 5))
    for _ in range(prof_steps):
        ctx.bridge_logpost_grad(nu, counts, [bias], grad_out=grad, want_bias_grad=False)
    prof = ctx.bridge_profile_read()
    ctx.bridge_profile_enable(False)
    total_ms = sum(v[1] for v in prof.values())
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    dname, (dl, dms, dbytes) = dom
    peaks, peak_src = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    achieved = dbytes / (dms / 1e3) / 1e9
    alg_per_launch = dbytes / dl
    traffic = recorded_traffic(dname, alg_per_launch)
    R = 4.0 * cfg.n ** 3
    model_bytes = MODEL_R[cfg.n_regions] * R
    eval_gbs = model_bytes * value / world / 1e9

    # --- end to end through the host-buffer entry point ---------------------
    nu_p = nu_h.pin_memory()
    c_p = c_h.pin_memory()
    g_p = torch.empty_like(nu_p).pin_memory()
    for _ in range(max(1, args.warmup)):
        ctx.bridge_logpost_grad_host(nu_p, c_p, [bias], g_p)
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 50))
    for _ in range(e2e_steps):
        ctx.bridge_logpost_grad_host(nu_p, c_p, [bias], g_p)
    e2e_t = max_over_ranks(time.perf_counter() - t0, dist if world > 1 else None)
    e2e_value = e2e_steps * world / e2e_t

    extras = {}
    cpu = None
    if rank == 0 and not args.no_extras:
        extras = run_extras(pkg, synth, cfg, bias, nu, counts, args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(budget_s=args.cpu_budget)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(1, cfg.n),
            "roofline": {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic, "peak_source": peak_src + " copy bandwidth",
                         "launches_per_step": dl / prof_steps, "alg_bytes_per_launch": alg_per_launch,
                         "share_of_step": dms / total_ms},
            "path_roofline": {"model_bytes_per_eval": model_bytes, "achieved_gbs": eval_gbs,
                              "frac": eval_gbs / hbm, "model": f"{MODEL_R[cfg.n_regions]}R, R = 4 N^3 bytes"},
            "kernels": {k: {"launches_per_step": v[0] / prof_steps, "ms_per_step": v[1] / prof_steps,
                            "gbs": (v[2] / (v[1] / 1e3) / 1e9) if v[1] > 0 and v[2] > 0 else None}
                        for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(nu_h.numel() * 4 + c_h.numel() * 4),
                    "d2h_bytes_per_step": int(nu_h.numel() * 4 + 8)},
            "gpu_launches": int(launches_per_step * args.steps),
            "clocks": clocks,
            "cpu_baseline": cpu,
            "logpost": float(lp[0]),
            "autotune": tune,
            "extras": extras,
        }
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_extras(pkg, synth, cfg, bias, nu32, counts, args):
    """Comparators reported beside the headline: FP64 plain path, HMC dH at several step sizes,
    batched FP32 chains against single FP64 chains at equal dH accuracy, a cuFFT cross-check of
    the FFT passes, stored vs recomputed ALPT fields, batched and 512^3 throughput, and redshift
    space with both lines of sight."""
    import numpy as np
    import torch
    out = {}

    def timed(fn, steps):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / steps

    def rel(a, b):
        return float(torch.linalg.vector_norm(a.double() - b.double()) / torch.linalg.vector_norm(b.double()))

    # FP64 plain single chain at 256^3
    c64 = pkg.Context(pkg.config_from(cfg, precision=pkg.BRIDGE_FP64, batch=1))
    nu64 = nu32.double()
    g64 = torch.empty_like(nu64)
    t = timed(lambda: c64.bridge_logpost_grad(nu64, counts, [bias], grad_out=g64, want_bias_grad=False), 3)
    lp64, _, _ = c64.bridge_logpost_grad(nu64, counts, [bias], grad_out=g64, want_bias_grad=False)
    c32 = pkg.Context(pkg.config_from(cfg, batch=1))
    lp32, g32, _ = c32.bridge_logpost_grad(nu32, counts, [bias], want_bias_grad=False)
    out["fp64_plain_256"] = {"evals_per_s": 1.0 / t, "fp32_vs_fp64_grad_rel_l2": rel(g32, g64),
                             "fp32_vs_fp64_logpost_rel": abs(lp32[0] - lp64[0]) / abs(lp64[0])}

    # HMC at 256^3: 10 leapfrog steps, identity mass; data drawn from the model (gamma-Poisson,
    # beta = 5, around the FP64 path's nbar at nu_true); trajectories start at nu_true.
    nu_t = torch.tensor(synth.white_noise(cfg.n, cfg.seed_truth), dtype=torch.float64, device="cuda")
    _, lnnbar = c64.bridge_forward(nu_t, counts, [bias], want_ln_nbar=True)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(cfg.seed_counts)
    shape = torch.full_like(lnnbar, 5.0)
    rate = torch.exp(lnnbar) * torch._standard_gamma(shape, generator=gen) / 5.0
    counts_m = torch.poisson(rate, generator=gen).clamp_(max=65535).to(torch.int32).contiguous()
    del shape, rate, lnnbar
    p0 = torch.tensor(synth.momentum(cfg.n, cfg.seed_momentum), dtype=torch.float64, device="cuda")
    hmc = {"data": "gamma-Poisson mock (beta 5) of the model at nu_true, start at nu_true, identity mass",
           "steps": 10}
    eps_star = None
    for eps in (0.05, 0.005, 5e-4, 1e-4, 5e-5, 2e-5):
        n64, p64 = nu_t.clone(), p0.clone()
        h0a, h1a = c64.bridge_leapfrog(n64, p64, counts_m, [bias], 10, eps)
        n32, p32 = nu_t.float(), p0.float()
        t0 = time.perf_counter()
        h0b, h1b = c32.bridge_leapfrog(n32, p32, counts_m, [bias], 10, eps)
        torch.cuda.synchronize()
        tl = time.perf_counter() - t0
        d64, d32 = h1a[0] - h0a[0], h1b[0] - h0b[0]
        rec = {"dH_fp64": d64, "dH_fp32": d32, "abs_dH_fp32_minus_fp64": abs(d32 - d64),
               "H0_fp64": h0a[0], "H0_fp32_minus_fp64": h0b[0] - h0a[0], "fp32_trajectory_s": tl}
        if np.isfinite(d64) and np.isfinite(d32):
            rec["nu_rel_l2_fp32_vs_fp64"] = rel(n32, n64)
            rec["p_rel_l2_fp32_vs_fp64"] = rel(p32, p64)
            if eps_star is None and abs(d64) <= 1.0:
                eps_star = eps
        else:
            rec["diverged"] = True
        hmc[f"eps_{eps:g}"] = rec
    hmc["eps_dH_order_one"] = eps_star
    out["hmc_256"] = hmc

    # batched FP32 chains against single-chain FP64 at the step size where dH = O(1): four
    # 256^3 chains (own momenta) advanced together in FP32; each chain again alone in FP64.
    if eps_star is not None:
        B = 4
        p4 = torch.stack([torch.tensor(synth.momentum(cfg.n, cfg.seed_momentum + 10 * b), dtype=torch.float64,
                                       device="cuda") for b in range(B)])
        cb4 = pkg.Context(pkg.config_from(cfg, batch=B))
        nb, pb = nu_t.float().expand(B, -1, -1, -1).contiguous(), p4.float().contiguous()
        cnt4 = counts_m.expand(B, -1, -1, -1).contiguous()
        cb4.bridge_leapfrog(nb.clone(), pb.clone(), cnt4, [bias] * B, 10, eps_star)   # graph capture
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h0b, h1b = cb4.bridge_leapfrog(nb, pb, cnt4, [bias] * B, 10, eps_star)
        torch.cuda.synchronize()
        t32 = time.perf_counter() - t0
        del cb4, cnt4
        d64s, t64 = [], 0.0
        for b in range(B):
            n64, pp64 = nu_t.clone(), p4[b].clone()
            t0 = time.perf_counter()
            h0a, h1a = c64.bridge_leapfrog(n64, pp64, counts_m, [bias], 10, eps_star)
            torch.cuda.synchronize()
            t64 += time.perf_counter() - t0
            d64s.append(h1a[0] - h0a[0])
        d32s = [h1b[b] - h0b[b] for b in range(B)]
        # the same FP32 trajectories with their two endpoint energies from the FP64 path
        # (U = -log posterior at the FP32 start and end points, 1/2 |p|^2 summed in FP64)
        dmix = []
        for b in range(B):
            lp0, _ = c64.bridge_forward(nu_t, counts_m, [bias])
            lp1, _ = c64.bridge_forward(nb[b].double().contiguous(), counts_m, [bias])
            k0 = 0.5 * float((p4[b].float().double() ** 2).sum())
            k1 = 0.5 * float((pb[b].double() ** 2).sum())
            dmix.append((-lp1[0] + k1) - (-lp0[0] + k0))
        out["hmc_equal_accuracy_256"] = {
            "eps": eps_star, "chains": B, "dH_fp64": d64s, "dH_fp32": d32s,
            "max_abs_dH_fp32_minus_fp64": float(max(abs(a - b) for a, b in zip(d32s, d64s))),
            "dH_fp32_trajectory_fp64_endpoints": dmix,
            "max_abs_dH_fp32_traj_fp64_ends_minus_fp64": float(max(abs(a - b) for a, b in zip(dmix, d64s))),
            "fp32_batched_trajectories_per_s": B / t32, "fp64_single_trajectories_per_s": B / t64,
            "speedup": (B / t32) / (B / t64),
            "note": "10 leapfrog steps = 11 gradient evaluations per trajectory; accept/reject uses dH, so equal "
                    "accuracy means |dH_fp32 - dH_fp64| << 1"}
    del p0, counts_m, nu_t, c64, nu64, g64

    # FFT cross-check: the library's five FFT pass kernels (r2c + c2r, no operator) against
    # cuFFT through torch.fft, one 256^3 FP32 field, device-resident
    x = nu32.reshape(1, -1).contiguous()
    y = torch.empty_like(x)
    t_lib = timed(lambda: c32.bridge_fft_roundtrip(x, y), 20)
    err = rel(y, x)
    x3 = nu32.reshape(cfg.n, cfg.n, cfg.n)
    t_cufft = timed(lambda: torch.fft.irfftn(torch.fft.rfftn(x3), s=x3.shape), 20)
    R = 4.0 * cfg.n ** 3
    out["fft_crosscheck_256"] = {
        "library_r2c_c2r_ms": 1e3 * t_lib, "cufft_r2c_c2r_ms": 1e3 * t_cufft, "library_over_cufft": t_lib / t_cufft,
        "library_roundtrip_rel_l2": err,
        "library_gbs_at_4R": 4 * R / t_lib / 1e9, "cufft_gbs_at_4R": 4 * R / t_cufft / 1e9,
        "note": "4R = one real field in and out of each transform; the library's pair is 5 launches (z, y, x, y, z "
                "passes); cuFFT via torch.fft.rfftn + irfftn includes its own launches and temporaries"}
    del c32

    # stored vs recomputed ALPT spectra: 256^3 and 512^3
    rec = {}
    for tag, cc, b_ in (("256", cfg, bias), ("512", synth.config(4), synth.default_bias(synth.config(4)))):
        nu_c = nu32 if tag == "256" else torch.tensor(synth.white_noise(cc.n, cc.seed_eval), dtype=torch.float32,
                                                       device="cuda")
        cn_c = counts if tag == "256" else torch.tensor(
            synth.timing_counts(cc.n, cc.seed_counts, cc.mean_tracers, beta=2.0), dtype=torch.int32, device="cuda")
        gg = torch.empty_like(nu_c)
        for mode in (False, True):
            cfg_c = pkg.config_from(cc, batch=1, recompute_alpt=mode)
            ctx_c = pkg.Context(cfg_c)
            tt = timed(lambda: ctx_c.bridge_logpost_grad(nu_c, cn_c, [b_], grad_out=gg, want_bias_grad=False), 5)
            rec[f"{tag}_{'recompute' if mode else 'stored'}"] = {
                "evals_per_s": 1.0 / tt, "workspace_gb": pkg.lib().bridge_workspace_bytes(cfg_c) / 1e9}
            del ctx_c
        del nu_c, cn_c, gg
    out["alpt_stored_vs_recompute"] = rec

    # the batched workload's HMC: 16 FP32 chains at 128^3 advanced together against single FP64
    # chains, at the step size where the FP64 dH is O(1) (data drawn from the model at nu_true)
    cb = synth.config(3)
    bb = synth.perturbed_biases(synth.default_bias(cb), cb.batch, cb.seed_perturb)
    c64b = pkg.Context(pkg.config_from(cb, precision=pkg.BRIDGE_FP64, batch=1))
    nts = [torch.tensor(synth.white_noise(cb.n, cb.seed_truth + 100 * b), dtype=torch.float64, device="cuda")
           for b in range(cb.batch)]
    cms = []
    gen = torch.Generator(device="cuda")
    gen.manual_seed(cb.seed_counts)
    ones = torch.ones(cb.n, cb.n, cb.n, dtype=torch.int32, device="cuda")
    for b in range(cb.batch):
        _, ln = c64b.bridge_forward(nts[b], ones, [bb[b]], want_ln_nbar=True)
        beta_b = 10.0
        lam = cb.mean_tracers * torch.exp(ln) * torch._standard_gamma(torch.full_like(ln, beta_b), generator=gen) / beta_b
        cms.append(torch.poisson(lam, generator=gen).clamp_(max=65535).to(torch.int32).reshape(ones.shape))
    pms = [torch.tensor(synth.momentum(cb.n, cb.seed_momentum + b), dtype=torch.float64, device="cuda")
           for b in range(cb.batch)]
    eps_b = None
    for eps in (4e-4, 2e-4, 1e-4, 5e-5):
        h0, h1 = c64b.bridge_leapfrog(nts[0].clone(), pms[0].clone(), cms[0], [bb[0]], 10, eps)
        if np.isfinite(h1[0] - h0[0]) and abs(h1[0] - h0[0]) <= 1.0:
            eps_b = eps
            break
    if eps_b is not None:
        c32b = pkg.Context(pkg.config_from(cb))
        nb = torch.stack(nts).float().contiguous()
        pb = torch.stack(pms).float().contiguous()
        cnb = torch.stack(cms).contiguous()
        c32b.bridge_leapfrog(nb.clone(), pb.clone(), cnb, bb, 10, eps_b)   # graph capture
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h0b, h1b = c32b.bridge_leapfrog(nb, pb, cnb, bb, 10, eps_b)
        torch.cuda.synchronize()
        t32 = time.perf_counter() - t0
        d64s, t64 = [], 0.0
        for b in range(4):
            t0 = time.perf_counter()
            h0, h1 = c64b.bridge_leapfrog(nts[b].clone(), pms[b].clone(), cms[b], [bb[b]], 10, eps_b)
            torch.cuda.synchronize()
            t64 += time.perf_counter() - t0
            d64s.append(h1[0] - h0[0])
        d32s = [h1b[b] - h0b[b] for b in range(4)]
        out["hmc_equal_accuracy_16x128"] = {
            "eps": eps_b, "chains_fp32_batched": cb.batch, "compared": 4, "dH_fp64": d64s, "dH_fp32": d32s,
            "max_abs_dH_fp32_minus_fp64": float(max(abs(a - b) for a, b in zip(d32s, d64s))),
            "fp32_batched_trajectories_per_s": cb.batch / t32, "fp64_single_trajectories_per_s": 4 / t64,
            "speedup": (cb.batch / t32) / (4 / t64)}
        del c32b, nb, pb, cnb
    del c64b, nts, cms, pms, ones
    # batched: 16 chains at 128^3 in one launch per pass
    biases = synth.perturbed_biases(synth.default_bias(cb), cb.batch, cb.seed_perturb)
    ctxb = pkg.Context(pkg.config_from(cb))
    nub = torch.tensor(synth.white_noise(cb.n, cb.seed_eval, cb.batch), dtype=torch.float32, device="cuda")
    cnb = torch.tensor(synth.timing_counts(cb.n, cb.seed_counts, cb.mean_tracers, batch=cb.batch),
                       dtype=torch.int32, device="cuda")
    gb = torch.empty_like(nub)
    t = timed(lambda: ctxb.bridge_logpost_grad(nub, cnb, biases, grad_out=gb, want_bias_grad=False), 5)
    out["batched_16x128"] = {"chain_evals_per_s": cb.batch / t, "ms_per_batched_eval": 1e3 * t}
    c1 = pkg.Context(pkg.config_from(cb, batch=1))
    g1 = torch.empty_like(nub[0])
    t1 = timed(lambda: c1.bridge_logpost_grad(nub[0].contiguous(), cnb[0].contiguous(), [biases[0]], grad_out=g1,
                                              want_bias_grad=False), 5)
    out["single_128"] = {"evals_per_s": 1.0 / t1}
    del ctxb, c1, nub, cnb, gb
    # four 256^3 chains in one launch per pass
    c4 = pkg.Context(pkg.config_from(cfg, batch=4))
    nu4 = torch.tensor(synth.white_noise(cfg.n, cfg.seed_eval, 4), dtype=torch.float32, device="cuda")
    cn4 = torch.tensor(synth.timing_counts(cfg.n, cfg.seed_counts, cfg.mean_tracers, batch=4), dtype=torch.int32,
                       device="cuda")
    g4 = torch.empty_like(nu4)
    t4 = timed(lambda: c4.bridge_logpost_grad(nu4, cn4, [bias] * 4, grad_out=g4, want_bias_grad=False), 5)
    out["batched_4x256"] = {"chain_evals_per_s": 4 / t4, "ms_per_batched_eval": 1e3 * t4}
    del c4, nu4, cn4, g4
    # the large single field: 512^3, L = 2000 Mpc/h, beta = 2, 0.05 tracers per cell
    c5 = synth.config(4)
    b5 = synth.default_bias(c5)
    ctx5 = pkg.Context(pkg.config_from(c5, batch=1))
    nu5 = torch.tensor(synth.white_noise(c5.n, c5.seed_eval), dtype=torch.float32, device="cuda")
    cn5 = torch.tensor(synth.timing_counts(c5.n, c5.seed_counts, c5.mean_tracers, beta=2.0), dtype=torch.int32,
                       device="cuda")
    g5 = torch.empty_like(nu5)
    t5 = timed(lambda: ctx5.bridge_logpost_grad(nu5, cn5, [b5], grad_out=g5, want_bias_grad=False), 3)
    out["single_512"] = {"evals_per_s": 1.0 / t5, "ms_per_eval": 1e3 * t5,
                         "workspace_gb": pkg.lib().bridge_workspace_bytes(pkg.config_from(c5, batch=1)) / 1e9}
    del ctx5, g5
    # redshift space (Sect. 2.9, f = 0.8): plane-parallel and radial line of sight, 256^3 and 512^3
    rsd = {}
    for label, cbase, bx, nux, cnx in (("256", cfg, bias, nu32, counts), ("512", c5, b5, nu5, cn5)):
        for los, name in ((0, "plane_parallel"), (1, "radial")):
            cr = copy.copy(cbase)
            cr.rsd_f, cr.rsd_los = 0.8, los
            cx = pkg.Context(pkg.config_from(cr, batch=1))
            gx = torch.empty_like(nux)
            tx = timed(lambda: cx.bridge_logpost_grad(nux, cnx, [bx], grad_out=gx, want_bias_grad=False), 3)
            rsd[f"{name}_{label}"] = {"evals_per_s": 1.0 / tx, "ms_per_eval": 1e3 * tx}
            del cx, gx
    out["redshift_space"] = rsd
    # deterministic mass assignment (64-bit fixed-point CIC sums), 256^3
    cdet = pkg.Context(pkg.config_from(cfg, batch=1, deterministic=True))
    gdet = torch.empty_like(nu32)
    tdet = timed(lambda: cdet.bridge_logpost_grad(nu32, counts, [bias], grad_out=gdet, want_bias_grad=False), 5)
    out["deterministic_256"] = {"evals_per_s": 1.0 / tdet, "ms_per_eval": 1e3 * tdet}
    del cdet, gdet
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the built-in launch shapes")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=60.0, help="seconds for the oracle sample")
    ap.add_argument("--small-case", action="store_true",
                    help="time the 128^3 case instead of the 256^3 workload (for small profiler captures)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)   # at least three untimed warm-up steps
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
