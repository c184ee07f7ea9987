"""Benchmark: one step = one full compressed-sensing reconstruction of a 1.1 mm slice.

Workload (paper-scale plain method): 200x200 image (1.1 mm, FOV 220 mm), 32 coils,
single-shot spiral at R = 4 with 24 000 samples (1 us dwell), 3rd-order spherical-
harmonic field (16 terms) plus B0 within +-150 Hz, Daubechies-4 wavelet with 4 levels,
lambda = 1e-3 ||A^H y||_inf, 30 power iterations for L_f, 50 FISTA iterations.
Synthetic, seeded inputs stand in for the paper's in-vivo data.

Metric: A_exp + A_exp^H throughput in Gvoxel*sample*coil/s = (applications per step x
nr x nt x nc) / step time; seconds per slice reconstruction is reported beside it.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "A_exp+A_exp^H Gvoxel*sample*coil/s; s per 1.1mm slice recon, TC vs FP32"
UNIT = "Gvoxel*sample*coil/s"
WORKLOAD = "slice_200: 200x200 1.1mm, 32 coils, 24000-sample R=4 spiral, 3rd-order SH + B0, db4 J=4, 50 FISTA + 30 power iterations"


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(ms: float, world: int) -> float:
    """The slowest rank's time (all-reduce MAX over the process group; identity on one rank).
    Every rank must call it the same number of times in the same order."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(world: int, units_per_rank_step: float, steps: int, total_ms: float) -> float:
    """Whole-job throughput in G units/s: every rank processes its own units (its own slice),
    the job takes as long as the slowest rank."""
    return world * units_per_rank_step * steps / (total_ms / 1e3) / 1e9


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            ids = [v.strip() for v in vis.split(",") if v.strip()]
            self.gpu = ids[gpu_index] if gpu_index < len(ids) else str(gpu_index)
        else:
            self.gpu = str(gpu_index)
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [s.strip() for s in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def fp32_alu_peak_tflops(sm_mhz: float) -> float:
    """FP32 FMA pipe: 152 SMs x 128 lanes x 2 flop per FMA x SM clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def sfu_peak_gops(sm_mhz: float) -> float:
    """MUFU (sin, cos, ...): 152 SMs x 16 results per clock x SM clock, in G results/s."""
    return 152 * 16 * sm_mhz * 1e6 / 1e9


def launches_per_recon(levels: int, iters: int, n_power: int, form: str = "fp32", nx: int = 200,
                       ny: int = 200) -> int:
    """Kernel launches issued by cs_recon (mirrors the host sequence in recon.cu; checked against
    the ncu launch lists of one solve in each form)."""
    # one A^H A (power iteration or FISTA gradient step): FP32 coil weighting, contraction,
    # reduction with the residual, contraction, reduction with the gradient step; BF16 packing,
    # persistent contraction, fused reduction + residual + packing, persistent contraction,
    # reduction; FP16 hi+lo in addition a max reset and a max reduction per packing and a
    # separate packing of the residual
    aha = {"fp32": 5, "bf16": 5, "fp16x2": 10}[form]
    ahy = {"fp32": 2, "bf16": 3, "fp16x2": 5}[form]          # A^H y: the power iteration's start
    # coefficients, tiles, reference phases, coils (+ BF16: phase-GEMM operands, descriptor,
    # items; + FP16 hi+lo: the per-term scaling), then the transpose of y
    prep = {"fp32": 4, "bf16": 8, "fp16x2": 9}[form] + 1
    # wavelet prox step: level 1 each way plus levels 2..J in one launch where the level-1
    # approximation fits the middle-level kernel's shared memory, else one launch per level each way
    q = 1 << levels
    npx, npy = -(-nx // q) * q, -(-ny // q) * q
    prox = 3 if levels >= 2 and (npx // 2) * (npy // 2) <= 12800 else 2 * levels
    power = ahy + 2 + n_power * (aha + 2) + 1            # A^H y; norm + scale; per iteration A^H A + norm + scale; finalize
    fista = iters * (aha + prox)
    return prep + power + fista


def cpu_sample(p, y, seconds: float):
    """Time the oracle (as it stands) on a bounded sample of the workload's operator
    applications: forward rows and adjoint voxels in equal numbers of voxel*sample*coil."""
    import oracle
    nr, nt, nc = p["nx"] * p["ny"], p["nt"], p["nc"]
    rng = np.random.default_rng(0)
    done = 0.0
    t0 = time.perf_counter()
    rows = 0
    while time.perf_counter() - t0 < seconds:
        ts = rng.choice(nt, 16, replace=False)
        oracle.forward_rows(p, p["x_gt"], ts)
        rs = rng.choice(nr, int(round(16 * nr / nt)), replace=False)
        oracle.adjoint_rows(p, y, rs)
        done += 16 * nr * nc + len(rs) * nt * nc
        rows += 16
    dt = time.perf_counter() - t0
    return done / dt / 1e9, dt, rows


def run_reference(args):
    rank, world, local = dist_info()
    if rank != 0:
        return
    import oracle
    from paper_2211_07532_gb300 import synth
    oracle.build()
    p = synth.slice_200()
    rng = np.random.default_rng(1)
    y = synth.random_kspace(rng, p["nc"], p["nt"])
    per_step = []
    vals = []
    # each step a bounded sample: --ref-seconds, capped so that the whole run stays near 2.5 minutes
    step_s = min(args.ref_seconds, max(1.0, 150.0 / max(1, args.warmup + args.steps)))
    for i in range(args.warmup + args.steps):
        v, dt, rows = cpu_sample(p, y, step_s)
        if i >= args.warmup:
            per_step.append(dt)
            vals.append(v)
    value = float(np.mean(vals))
    cores = oracle.threads()
    sample = (f"oracle forward rows (16 random samples x all 40000 voxels x 32 coils) and adjoint voxels "
              f"(27 random voxels x all 24000 samples x 32 coils) repeated for {step_s:.1f} s per step")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(per_step)),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "bounded oracle sample"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_info()
    if world > 1:
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    side = torch.cuda.Stream(dev)      # a non-default stream, so cs_recon can capture its CUDA graph
    with torch.cuda.stream(side):
        _run_ours(args, rank, world, local, dev)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def _kernel_ms(ax, torch, prob, x, y, precision, flush, stream, reps=10, items_per_sm=0, tile_variant=0):
    """One operator application each way (packing/coil weighting + contraction + partial-sum
    reduction) in the launch shape the solve uses, CUDA events on the launching stream."""
    ws_k = ax.workspace(prob, precision, items_per_sm=items_per_sm, tile_variant=tile_variant)
    ax.prepare(prob, ws_k, precision, items_per_sm=items_per_sm, tile_variant=tile_variant)
    yo = torch.empty_like(y)
    xo = torch.empty_like(x)
    kern = {}
    for name, fn in (("a_exp_forward", lambda: ax.a_exp_forward(prob, x, ws_k, y=yo, precision=precision)),
                     ("a_exp_adjoint", lambda: ax.a_exp_adjoint(prob, y, ws_k, x=xo, precision=precision))):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        kern[name] = float(np.mean(ts))
    return kern


def _run_ours(args, rank, world, local, dev):
    import torch
    import torch.distributed as dist

    from paper_2211_07532_gb300 import build as _b
    _b.build()
    import paper_2211_07532_gb300 as ax
    from paper_2211_07532_gb300 import synth

    forms = {"fp32": ax.FP32, "bf16": ax.BF16_TC, "fp16x2": ax.FP16X2_TC}
    precision = forms[args.form]
    p = synth.slice_200(index=rank)           # each rank reconstructs its own slice (weak scaling)
    nr, nt, nc = p["nx"] * p["ny"], p["nt"], p["nc"]
    iters, levels, n_power = p["iters"], p["levels"], 30
    prob = ax.Problem.from_arrays(p, device=dev)
    x_gt = torch.as_tensor(p["x_gt"], device=dev)

    # simulated data on the device through the library's own FP32 forward model (Sec. 2.2.2)
    ws_op = ax.workspace(prob, ax.FP32)
    ax.prepare(prob, ws_op, ax.FP32)
    y0 = ax.a_exp_forward(prob, x_gt, ws_op)
    sigma = float(torch.sqrt(torch.mean(y0.abs() ** 2))) / p["snr"]
    y = (y0 + sigma * torch.as_tensor(p["noise"], device=dev)).contiguous()
    lam = 1e-3 * float(ax.a_exp_adjoint(prob, y, ws_op).abs().max())
    del ws_op

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream()
    applications = 2 * iters + 2 * n_power + 1
    vsc_per_step = applications * nr * nt * nc
    x_out = torch.empty(nr, dtype=torch.complex64, device=dev)
    L_out = torch.empty(1, dtype=torch.float64, device=dev)

    def recon_ws(prec):
        # autotuned work-item granularity (untimed); the tuner's workspace then serves the solve
        o = ax.recon_opts(precision=prec, wavelet="db4", levels=levels, n_power=n_power)
        w = torch.empty(ax.lib_autotune_workspace_size(prob, o), dtype=torch.uint8, device=dev)
        o.items_per_sm, o.tile_variant, _ = ax.autotune(prob, o, ws=w)
        return o, w

    opts, ws = recon_ws(precision)
    for _ in range(args.warmup):
        ax.cs_recon(prob, y, lam, iters, opts=opts, ws=ws, x_out=x_out, lipschitz_out=L_out)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()                     # L2 flushed between timed iterations (outside the events)
            ev[i][0].record(stream)
            ax.cs_recon(prob, y, lam, iters, opts=opts, ws=ws, x_out=x_out, lipschitz_out=L_out)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(float(sum(step_ms)), world)
    ms_per_step = total_ms / args.steps
    value = weak_scaling_value(world, vsc_per_step, args.steps, total_ms)
    status = ax.read_status(ws)
    nrmse = float(torch.linalg.vector_norm(x_out - x_gt) / torch.linalg.vector_norm(x_gt))

    # end to end through the public API from pinned host memory: H2D of y, recon, D2H of x
    y_host = y.cpu().pin_memory()
    x_host = torch.empty(nr, dtype=torch.complex64).pin_memory()
    y_dev = torch.empty_like(y)
    y_dev.copy_(y_host)
    ax.cs_recon(prob, y_dev, lam, iters, opts=opts, ws=ws, x_out=x_out, lipschitz_out=L_out)  # capture, untimed
    torch.cuda.synchronize()
    e2e_ms = []
    for i in range(max(1, args.steps)):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        y_dev.copy_(y_host, non_blocking=True)
        ax.cs_recon(prob, y_dev, lam, iters, opts=opts, ws=ws, x_out=x_out, lipschitz_out=L_out)
        x_host.copy_(x_out, non_blocking=True)
        b.record(stream)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e_total = max_over_ranks(float(sum(e2e_ms)), world)
    e2e_value = weak_scaling_value(world, vsc_per_step, len(e2e_ms), e2e_total)

    kern = _kernel_ms(ax, torch, prob, x_gt, y, precision, flush, stream, items_per_sm=opts.items_per_sm,
                      tile_variant=opts.tile_variant)
    dom = max(kern, key=kern.get)
    clocks = clk.summary()
    nterms = p["nl"] + 1
    flops_per_launch = nr * nt * (8.0 * nc + 2.0 * nterms + 4.0)   # contraction + phase FMAs + reduction
    achieved = flops_per_launch / (kern[dom] / 1e3) / 1e12
    sm_mhz_peak = measured_peaks().get("sm_max_mhz", 2070.0)
    peak = fp32_alu_peak_tflops(sm_mhz_peak)
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        import hashlib
        with open(tfile) as f:
            rec = json.load(f)
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            current = hashlib.sha256(f.read()).hexdigest()[:16]
        if current == rec.get("sha256_16"):           # counters only valid for the profiled source
            traffic = rec.get(f"{args.form}:{dom}")

    # the other forms of the same workload, same timing rules (the metric compares TC and FP32)
    bf16_peak = measured_peaks().get("bf16_tflops", 1977.2)
    contraction_flops = nr * nt * 8.0 * nc
    comparison = {}
    for other in [f for f in forms if f != args.form]:
        o_opts, o_ws = recon_ws(forms[other])
        o_ms = []
        for _ in range(args.warmup):
            ax.cs_recon(prob, y, lam, iters, opts=o_opts, ws=o_ws, x_out=x_out, lipschitz_out=L_out)
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ax.cs_recon(prob, y, lam, iters, opts=o_opts, ws=o_ws, x_out=x_out, lipschitz_out=L_out)
            b.record(stream)
            b.synchronize()
            o_ms.append(a.elapsed_time(b))
        o_nrmse = float(torch.linalg.vector_norm(x_out - x_gt) / torch.linalg.vector_norm(x_gt))
        o_kern = _kernel_ms(ax, torch, prob, x_gt, y, forms[other], flush, stream,
                            items_per_sm=o_opts.items_per_sm, tile_variant=o_opts.tile_variant)
        o_step = max_over_ranks(float(np.mean(o_ms)), world)
        c = {"s_per_slice": o_step / 1e3, "value": weak_scaling_value(world, vsc_per_step, 1, o_step), "unit": UNIT,
             "nrmse_vs_phantom": o_nrmse, "device_status": ax.read_status(o_ws), "kernels_ms": o_kern,
             "speedup_vs_primary": ms_per_step / o_step, "items_per_sm": o_opts.items_per_sm,
             "tile_variant": o_opts.tile_variant}
        if other != "fp32":
            o_dom = max(o_kern, key=o_kern.get)
            passes = 3 if other == "fp16x2" else 1    # hi.hi2 + hi.lo' + lo.hi2 MMA passes
            cb_tc = 8 if nc <= 8 else 16 if nc <= 16 else 32
            lp = next(v for v in (4, 8, 12, 20, 32) if nterms <= v)
            ks = (lp + 15) // 16
            # executed on the tensor pipe per (sample, voxel): the contraction (N = 2 C_pad, two
            # flops per MAC, K = 2 per voxel or sample) per pass, and the phase GEMM (3 products,
            # K = 16 per step)
            exec_pair = passes * 8.0 * cb_tc + 3 * 2 * 16 * ks
            ach = contraction_flops / (o_kern[o_dom] / 1e3) / 1e12
            tp_ach = nr * nt * exec_pair / (o_kern[o_dom] / 1e3) / 1e12
            c["tensor_pipe"] = {
                "achieved": tp_ach, "unit": "TFLOP/s", "peak": bf16_peak, "frac": tp_ach / bf16_peak,
                "algorithmic_contraction_tflops": ach, "mma_passes": passes, "phase_k_steps": ks,
                "flops_per_pair_executed": exec_pair,
                "note": "executed MMA flops per (sample, voxel): contraction passes x 8 C_pad + phase GEMM "
                        "3 x 2 x 16 x K steps; FP16 and BF16 share the dense rate of the measured BF16 peak"}
            # SFU: one sincos (2 MUFU results) per (sample, voxel)
            sfu_ach = 2.0 * nr * nt / (o_kern[o_dom] / 1e3) / 1e9
            sfu_peak = sfu_peak_gops(sm_mhz_peak)
            sfu = {"bound": "sfu", "achieved": sfu_ach, "peak": sfu_peak, "unit": "G MUFU results/s",
                   "frac": sfu_ach / sfu_peak, "kernel": o_dom, "kernel_ms": o_kern[o_dom],
                   "peak_basis": f"152 SM x 16 MUFU results/clk at {sm_mhz_peak:.0f} MHz"}
            tensor = {"bound": "tensor", "achieved": tp_ach, "peak": bf16_peak, "unit": "TFLOP/s",
                      "frac": tp_ach / bf16_peak, "kernel": o_dom, "kernel_ms": o_kern[o_dom],
                      "peak_basis": "measured dense BF16 (MEASURED_PEAKS.json bf16_tflops; FP16 has the same rate)"}
            # the roofline of a form is the unit it comes closest to saturating
            c["roofline"] = sfu if sfu["frac"] >= tensor["frac"] else tensor
        comparison[other] = c
        del o_ws

    # the paper's LS baseline on the same data: CGLS from x = 0, 20 iterations (41 applications)
    ls_baseline = {}
    for f in ("fp32", "bf16"):
        lo = ax.recon_opts(precision=forms[f])
        lws = torch.empty(ax.cgls_workspace_size(prob, lo), dtype=torch.uint8, device=dev)
        for _ in range(max(1, args.warmup)):
            ax.cgls_recon(prob, y, 20, opts=lo, ws=lws, x_out=x_out)
        torch.cuda.synchronize()
        l_ms = []
        for i in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ax.cgls_recon(prob, y, 20, opts=lo, ws=lws, x_out=x_out)
            b.record(stream)
            b.synchronize()
            l_ms.append(a.elapsed_time(b))
        cs_s = ms_per_step / 1e3 if f == args.form else comparison[f]["s_per_slice"]
        ls_s = max_over_ranks(float(np.mean(l_ms)), world) / 1e3
        ls_baseline[f] = {"s_per_slice": ls_s, "iterations": 20, "applications": 41,
                          "nrmse_vs_phantom": float(torch.linalg.vector_norm(x_out - x_gt) / torch.linalg.vector_norm(x_gt)),
                          "cs_over_ls_time": cs_s / ls_s, "device_status": ax.read_status(lws)}
        del lws

    # the paper's own regulariser: one-level undecimated db4, lambda = sigma / 2 from W A^H y,
    # the paper's 100 FISTA iterations (Sec. 2.1; Supporting Information S1, S2)
    paper_cs = {}
    for f in ("fp32", "bf16"):
        lam_dev = torch.zeros(1, dtype=torch.float64, device=dev)
        po = ax.recon_opts(precision=forms[f], wavelet="db4", n_power=n_power, undecimated=True,
                           lambda_rule=ax.LAMBDA_RAYLEIGH, lambda_out=lam_dev,
                           items_per_sm=(opts.items_per_sm if f == args.form else comparison[f]["items_per_sm"]),
                           tile_variant=(opts.tile_variant if f == args.form else comparison[f]["tile_variant"]))
        pws = ax.recon_workspace(prob, po)
        for _ in range(max(1, args.warmup)):
            ax.cs_recon(prob, y, 0.0, 100, opts=po, ws=pws, x_out=x_out, lipschitz_out=L_out)
        torch.cuda.synchronize()
        p_ms = []
        for i in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ax.cs_recon(prob, y, 0.0, 100, opts=po, ws=pws, x_out=x_out, lipschitz_out=L_out)
            b.record(stream)
            b.synchronize()
            p_ms.append(a.elapsed_time(b))
        paper_cs[f] = {"s_per_slice": max_over_ranks(float(np.mean(p_ms)), world) / 1e3, "fista_iters": 100,
                       "power_iters": n_power,
                       "applications": 2 * 100 + 2 * n_power + 2, "lambda": float(lam_dev.cpu()[0]),
                       "nrmse_vs_phantom": float(torch.linalg.vector_norm(x_out - x_gt) / torch.linalg.vector_norm(x_gt)),
                       "device_status": ax.read_status(pws)}
        del pws

    # coil compression (Sec. 2.2.1: 20 virtual coils to speed the reconstruction up): principal
    # components of the data on the device, then the same reconstruction with nv coils
    def solve_ms(pr, yy, lm, f):
        """Mean event time of the 50-iteration solve of problem pr in form f (L2 flushed between runs)."""
        o = ax.recon_opts(precision=forms[f], wavelet="db4", levels=levels, n_power=n_power)
        w = ax.recon_workspace(pr, o)
        for _ in range(max(1, args.warmup)):
            ax.cs_recon(pr, yy, lm, iters, opts=o, ws=w, x_out=x_out, lipschitz_out=L_out)
        torch.cuda.synchronize()
        t_ms = []
        for i in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ax.cs_recon(pr, yy, lm, iters, opts=o, ws=w, x_out=x_out, lipschitz_out=L_out)
            b.record(stream)
            b.synchronize()
            t_ms.append(a.elapsed_time(b))
        return max_over_ranks(float(np.mean(t_ms)), world), ax.read_status(w)

    virtual = {}
    for f, nv in (("fp32", 20), ("bf16", 16), ("bf16", 20)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pv, yv, eig = ax.coil_compress(prob, y, nv)
        b.record(stream)
        b.synchronize()
        comp_ms = a.elapsed_time(b)
        v_ms, v_st = solve_ms(pv, yv, lam, f)
        e = eig.cpu().numpy()
        virtual[f"{f}_vc{nv}"] = {
            "s_per_slice": v_ms / 1e3, "compression_ms": comp_ms, "energy_kept": float(e[:nv].sum() / e.sum()),
            "nrmse_vs_phantom": float(torch.linalg.vector_norm(x_out - x_gt) / torch.linalg.vector_norm(x_gt)),
            "device_status": v_st}

    # field model beyond 3rd order: 4th-order harmonics + concomitant rows + B0 = 30 terms
    pe = synth.slice_200_expanded(index=rank)
    prob_e = ax.Problem.from_arrays(pe, device=dev)
    xe_gt = torch.as_tensor(pe["x_gt"], device=dev)
    ws_e = ax.workspace(prob_e, ax.FP32)
    ax.prepare(prob_e, ws_e, ax.FP32)
    ye = ax.a_exp_forward(prob_e, xe_gt, ws_e)
    ye = (ye + float(torch.sqrt(torch.mean(ye.abs() ** 2))) / pe["snr"] * torch.as_tensor(pe["noise"], device=dev))
    ye = ye.contiguous()
    lam_e = 1e-3 * float(ax.a_exp_adjoint(prob_e, ye, ws_e).abs().max())
    del ws_e
    expanded = {"terms": pe["nl"] + 1, "workload": "200x200 slice, 4th-order harmonics + 4 concomitant rows + B0, "
                                                   "tilted 20 deg, 32 coils, 24k samples"}
    for f in ("fp32", "bf16"):
        e_ms, e_st = solve_ms(prob_e, ye, lam_e, f)
        expanded[f] = {"s_per_slice": e_ms / 1e3, "device_status": e_st,
                       "nrmse_vs_phantom": float(torch.linalg.vector_norm(x_out - xe_gt) / torch.linalg.vector_norm(xe_gt))}

    # the ragged many-problem batch and the unrolled-FISTA gradients, one timed step each
    ragged = diff = None
    if not args.no_extras:
        if world > 1:
            dist.barrier()
        ragged = measure_ragged(ax, torch, dev, args.volumes, 1, 1)
        diff = measure_diff(ax, torch, 1, 1)

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            import oracle
            oracle.build()
            v, dt, rows = cpu_sample(p, y.cpu().numpy(), args.cpu_seconds)
            cpu = {"value": v, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                   "sample": f"{rows} forward sample rows + matching adjoint voxels of the same workload, "
                             f"{dt:.1f} s of FP64 oracle work"}
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16", "fp16x2": "f16x2"}[args.form],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": args.form, "nx": p["nx"], "nt": nt, "nc": nc,
                       "terms": nterms, "fista_iters": iters, "power_iters": n_power,
                       "applications_per_step": applications, "l2": "flushed between timed steps (512 MB write)",
                       "items_per_sm": opts.items_per_sm, "tile_variant": opts.tile_variant,
                       "parallelism": f"replicas x{world} (independent slices)"},
            "s_per_slice": ms_per_step / 1e3,
            "nrmse_vs_phantom": nrmse,
            "device_status": status,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(y.numel() * 8),
                    "d2h_bytes_per_step": int(nr * 8), "s_per_slice": e2e_total / len(e2e_ms) / 1e3},
            "gpu_launches": launches_per_recon(levels, iters, n_power, args.form, p["nx"], p["ny"]) * args.steps,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": dom,
                         "kernel_ms": kern[dom],
                         "peak_basis": f"FP32 FMA pipe 152 SM x 128 lanes x 2 flop at {sm_mhz_peak:.0f} MHz "
                                       "(sm_max_mhz of MEASURED_PEAKS.json)"},
            "kernels_ms": kern,
            "comparison": comparison,
            "ls_baseline_cgls20": ls_baseline,
            "paper_regulariser_cs100": paper_cs,
            "virtual_coils": virtual,
            "field_terms_30": expanded,
            "ragged_batch": ragged,
            "diff": diff,
        }
        # compact summaries last, so that a reader of the line's tail sees them
        summary = {}
        for f, c in comparison.items():
            summary[f] = {"s_per_slice": round(c["s_per_slice"], 4), "speedup_vs_fp32": round(ms_per_step / 1e3 /
                                                                                                 c["s_per_slice"], 2)
                          if args.form == "fp32" else None,
                          "nrmse": round(c["nrmse_vs_phantom"], 4),
                          "bound": c["roofline"]["bound"] if "roofline" in c else None,
                          "roofline_frac": round(c["roofline"]["frac"], 3) if "roofline" in c else None,
                          "tensor_pipe_frac": round(c["tensor_pipe"]["frac"], 3) if "tensor_pipe" in c else None,
                          "op_ms": round(c["roofline"]["kernel_ms"], 3) if "roofline" in c else None}
        out["tc_summary"] = {"fp32_s_per_slice": round(ms_per_step / 1e3, 4), "fp32_nrmse": round(nrmse, 4),
                             "fp32_fma_frac": round(achieved / peak, 3),
                             "fp32_tile_variant": opts.tile_variant, **summary}
        if ragged:
            out["ragged_summary"] = {"problems": ragged["config"]["problems"], "s_per_batch": round(ragged["ms_per_step"] / 1e3, 2),
                                     "s_per_slice": round(ragged["s_per_slice"], 4), "gvsc_per_s": round(ragged["value"], 1),
                                     "sfu_frac_whole_step": round(ragged["sfu_frac_whole_step"], 3),
                                     "nrmse_median": round(ragged["nrmse_vs_phantom_median"], 4),
                                     "device_status": ragged["device_status"]}
        if diff:
            out["diff_summary"] = {"forward_ms": round(diff["forward_ms"], 1), "backward_ms": round(diff["backward_ms"], 1),
                                   "backward_over_forward": round(diff["backward_over_forward"], 2)}
        out["clocks"] = clocks
        out["cpu_baseline"] = cpu
        print(json.dumps(out))


def measure_ragged(ax, torch, dev, volumes: int, steps: int, warmup: int, form: str = "bf16"):
    """372 ragged problems (148/170/200 px x `volumes` diffusion volumes x 4 slices, 32 coils,
    3rd-order field + B0, each volume with its own coefficients), tensor cores, one persistent
    launch per operator application, whole 30-power + 50-FISTA solve captured in one CUDA graph.
    Returns the full record (inputs generated on the device, autotuned layout, CUDA events)."""
    from paper_2211_07532_gb300 import synth
    nvol, nsl = volumes, 4
    t0 = time.time()
    probs, ys, lams, gts, vsc, pairs = [], [], [], [], 0, 0
    ws_sim = None
    for res in range(3):
        for sl in range(nsl):
            for vol in range(nvol):
                p = synth.ragged_problem(res, vol, sl)
                pr = ax.Problem.from_arrays(p, device=dev)
                need = ax.workspace_size(pr)
                if ws_sim is None or ws_sim.numel() < need:
                    ws_sim = torch.empty(need, dtype=torch.uint8, device=dev)
                ax.prepare(pr, ws_sim)
                xg = torch.as_tensor(p["x_gt"], device=dev)
                y0 = ax.a_exp_forward(pr, xg, ws_sim)
                sigma = float(torch.sqrt(torch.mean(y0.abs() ** 2))) / p["snr"]
                y = (y0 + sigma * torch.as_tensor(p["noise"], device=dev)).contiguous()
                lams.append(1e-3 * float(ax.a_exp_adjoint(pr, y, ws_sim).abs().max()))
                probs.append(pr)
                ys.append(y)
                gts.append(xg)
                vsc += pr.nr * pr.nt * pr.nc
                pairs += pr.nr * pr.nt
    del ws_sim
    gen_s = time.time() - t0
    iters, n_power, levels = 50, 30, 4
    opts = ax.recon_opts(precision={"bf16": ax.BF16_TC, "fp16x2": ax.FP16X2_TC}[form], wavelet="db4",
                         levels=levels, n_power=n_power)
    # one workspace serves the autotuner (every candidate layout) and the solve
    ws = torch.empty(ax.lib_autotune_workspace_size(probs, opts), dtype=torch.uint8, device=dev)
    t0 = time.time()
    best_ips, best_var, best_ms = ax.autotune(probs, opts, ws=ws)
    tune_s = time.time() - t0
    opts.items_per_sm = best_ips
    opts.tile_variant = best_var
    xs = [torch.empty(pr.nr, dtype=torch.complex64, device=dev) for pr in probs]
    L = torch.empty(len(probs), dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(max(1, warmup)):
        ax.cs_recon_batched(probs, ys, lams, iters, opts=opts, ws=ws, x_outs=xs, lipschitz_out=L)
    torch.cuda.synchronize()
    ms = []
    with ClockSampler(dev.index or 0) as clk:
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ax.cs_recon_batched(probs, ys, lams, iters, opts=opts, ws=ws, x_outs=xs, lipschitz_out=L)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
    status = ax.read_status(ws)
    nrmse = [float(torch.linalg.vector_norm(x - g) / torch.linalg.vector_norm(g)) for x, g in zip(xs, gts)]
    ws_gb = ws.numel() / 1e9
    del ws, xs, ys, probs, flush
    torch.cuda.empty_cache()
    step = float(np.mean(ms))
    applications = 2 * iters + 2 * n_power + 1
    sm_mhz = measured_peaks().get("sm_max_mhz", 2070.0)
    sfu = 2.0 * pairs * applications / (step / 1e3) / 1e9
    return {
        "value": applications * vsc / (step / 1e3) / 1e9, "unit": UNIT, "steps": steps, "warmup": max(1, warmup),
        "ms_per_step": step, "s_per_slice": step / 1e3 / len(gts), "dtype": {"bf16": "bf16", "fp16x2": "f16x2"}[form],
        "nrmse_vs_phantom_median": float(np.median(nrmse)), "device_status": status,
        "sfu_frac_whole_step": sfu / sfu_peak_gops(sm_mhz),
        "config": {"workload": f"ragged batch: 3 resolutions (148/170/200) x {nvol} volumes x {nsl} slices = "
                               f"{len(gts)} problems, 32 coils, 3rd-order SH + B0, db4 J=4, 50 FISTA + 30 power",
                   "problems": len(gts), "vsc_per_application": vsc, "applications_per_step": applications,
                   "workspace_gb": ws_gb, "generation_s": gen_s,
                   "autotune": {"items_per_sm": best_ips, "tile_variant": best_var, "ms_per_AhA": best_ms,
                                "seconds": tune_s}},
        "clocks": clk.summary()}


def run_ragged(args):
    import torch
    from paper_2211_07532_gb300 import build as _b
    _b.build()
    import paper_2211_07532_gb300 as ax
    dev = torch.device("cuda", 0)
    form = args.form if args.form != "fp32" else "bf16"   # the batched path runs on the tensor cores
    with torch.cuda.stream(torch.cuda.Stream(dev)):
        r = measure_ragged(ax, torch, dev, args.volumes, args.steps, args.warmup, form)
    r.update(metric=METRIC, workload="ragged", n_gpus=1, higher_is_better=True, data="synthetic")
    print(json.dumps(r))


def measure_diff(ax, torch, steps: int, warmup: int, B: int = 8):
    """Unrolled-FISTA gradients: 170x170, 16 coils, 12k samples, 2nd order + B0, 10 iterations,
    batch of B slices; forward unroll and backward (x0, lambda, k) timed with CUDA events."""
    from paper_2211_07532_gb300 import synth
    from paper_2211_07532_gb300.autograd import unrolled_fista

    iters = 10
    slices = []
    for i in range(B):
        p = synth.diff_170(index=i)
        prob = ax.Problem.from_arrays(p)
        ws = ax.workspace(prob)
        ax.prepare(prob, ws)
        xg = torch.as_tensor(p["x_gt"], device="cuda")
        y0 = ax.a_exp_forward(prob, xg, ws)
        y = (y0 + float(torch.sqrt(torch.mean(y0.abs() ** 2))) / p["snr"]
             * torch.as_tensor(p["noise"], device="cuda")).contiguous()
        _, L = ax.cs_recon(prob, y, 0.0, 0, n_power=30)
        lam = 1e-3 * float(ax.a_exp_adjoint(prob, y, ws).abs().max())
        slices.append((p, y, xg, float(L.cpu()[0]), lam))
    stream = torch.cuda.current_stream()

    def run():
        x0s = [torch.zeros(170 * 170, dtype=torch.complex64, device="cuda").requires_grad_(True) for _ in slices]
        lam_s = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
        ks = [torch.as_tensor(s[0]["k"], device="cuda").requires_grad_(True) for s in slices]
        a, m, b = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        loss = 0.0
        for (p, y, xg, L, lam), x0, k in zip(slices, x0s, ks):
            xK = unrolled_fista(p, y, x0, lam_s * lam, k, iters, L, wavelet="db4", levels=4)
            loss = loss + torch.mean(torch.abs(xK - xg) ** 2)
        m.record(stream)
        (loss / B).backward()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(m), m.elapsed_time(b)

    for _ in range(max(1, warmup)):
        run()
    f, bw = zip(*[run() for _ in range(steps)])
    vsc = 170 * 170 * 12000 * 16
    return {"forward_ms": float(np.mean(f)), "backward_ms": float(np.mean(bw)),
            "backward_over_forward": float(np.mean(bw) / np.mean(f)),
            "forward_gvsc_per_s": B * iters * 2 * vsc / (np.mean(f) / 1e3) / 1e9, "dtype": "f32",
            "steps": steps, "warmup": max(1, warmup),
            "config": {"workload": f"170x170, 16 coils, 12k samples, 2nd-order SH + B0, 10 unrolled FISTA, batch of {B}",
                       "applications_forward": B * iters * 2,
                       "applications_backward": B * iters * 4 + B * iters * 2}}


def run_diff(args):
    import torch
    from paper_2211_07532_gb300 import build as _b
    _b.build()
    import paper_2211_07532_gb300 as ax
    r = measure_diff(ax, torch, args.steps, args.warmup)
    r.update(workload="diff", metric="unrolled FISTA forward + backward time", unit="ms")
    print(json.dumps(r))


def run_op_only(args):
    """Operator applications alone on the bench workload (a small, bounded profiling target)."""
    import torch
    from paper_2211_07532_gb300 import build as _b
    _b.build()
    import paper_2211_07532_gb300 as ax
    from paper_2211_07532_gb300 import synth

    precision = {"fp32": ax.FP32, "bf16": ax.BF16_TC, "fp16x2": ax.FP16X2_TC}[args.form]
    p = synth.slice_200()
    prob = ax.Problem.from_arrays(p)
    ws = ax.workspace(prob, precision, tile_variant=args.tiling)
    ax.prepare(prob, ws, precision, tile_variant=args.tiling)
    x = torch.as_tensor(p["x_gt"], device="cuda")
    y = torch.as_tensor(p["noise"], device="cuda")
    ms = {"a_exp_forward": [], "a_exp_adjoint": []}
    for _ in range(args.reps):
        for name, fn in (("a_exp_forward", lambda: ax.a_exp_forward(prob, x, ws, precision=precision)),
                         ("a_exp_adjoint", lambda: ax.a_exp_adjoint(prob, y, ws, precision=precision))):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            out = fn()
            b.record()
            b.synchronize()
            ms[name].append(a.elapsed_time(b))
            if name == "a_exp_forward":
                yo = out
            else:
                xo = out
    torch.cuda.synchronize()
    assert ax.read_status(ws) == 0
    vsc = p["nx"] * p["ny"] * p["nt"] * p["nc"]
    best = {k: min(v) for k, v in ms.items()}
    print(json.dumps({"mode": "op", "form": args.form, "tiling": args.tiling, "reps": args.reps, "ms_min": best,
                      "gvsc_per_s": {k: vsc / (v / 1e3) / 1e9 for k, v in best.items()},
                      "y_norm": float(yo.abs().sum()), "x_norm": float(xo.abs().sum())}))


def run_solve_only(args):
    """One reconstruction of the bench slice in the chosen form (a bounded profiling target:
    preparation, 30 power + 50 FISTA iterations, no autotuning, no graph replay)."""
    import torch
    from paper_2211_07532_gb300 import build as _b
    _b.build()
    import paper_2211_07532_gb300 as ax
    from paper_2211_07532_gb300 import synth
    precision = {"fp32": ax.FP32, "bf16": ax.BF16_TC, "fp16x2": ax.FP16X2_TC}[args.form]
    dev = torch.device("cuda")
    with torch.cuda.stream(torch.cuda.Stream(dev)):
        p = synth.slice_200()
        prob = ax.Problem.from_arrays(p, device=dev)
        x = torch.as_tensor(p["x_gt"], device=dev)
        ws = ax.workspace(prob)
        ax.prepare(prob, ws)
        y = ax.a_exp_forward(prob, x, ws)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        xr, _ = ax.cs_recon(prob, y, 1.0, p["iters"], precision=precision, wavelet="db4", levels=p["levels"],
                            n_power=30, use_graph=False)
        b.record()
        b.synchronize()
    print(json.dumps({"mode": "solve", "form": args.form, "ms": a.elapsed_time(b)}))


def run_kernel_classes(args):
    """One small invocation of every kernel class outside the operator (a bounded profiling
    target): the orthogonal wavelet levels and FP64 norms of a 2-iteration FISTA on the 200^2
    slice, the undecimated wavelet and lambda-rule kernels, coil compression 32 -> 20, two CGLS
    iterations, one
    unrolled-FISTA step and its VJP on the 170^2 / 16-coil slice (k-gradient kernel), and a
    2-iteration batched solve of six ragged problems (persistent batch kernels)."""
    import torch
    from paper_2211_07532_gb300 import build as _b
    _b.build()
    import paper_2211_07532_gb300 as ax
    from paper_2211_07532_gb300 import synth
    from paper_2211_07532_gb300.autograd import unrolled_fista

    dev = torch.device("cuda")
    with torch.cuda.stream(torch.cuda.Stream(dev)):
        p = synth.slice_200()
        prob = ax.Problem.from_arrays(p, device=dev)
        x = torch.as_tensor(p["x_gt"], device=dev)
        ws = ax.workspace(prob)
        ax.prepare(prob, ws)
        y = ax.a_exp_forward(prob, x, ws)
        ax.cs_recon(prob, y, 1.0, 2, wavelet="db4", levels=4, n_power=2, use_graph=False)
        lam = torch.zeros(1, dtype=torch.float64, device=dev)
        ax.cs_recon(prob, y, 0.0, 2, wavelet="db4", undecimated=True, lambda_rule=ax.LAMBDA_RAYLEIGH,
                    lambda_out=lam, n_power=2, use_graph=False)
        ax.coil_compress(prob, y, 20)
        ax.cgls_recon(prob, y, 2)
        q = synth.diff_170()
        pq = ax.Problem.from_arrays(q, device=dev)
        wq = ax.workspace(pq)
        ax.prepare(pq, wq)
        yq = ax.a_exp_forward(pq, torch.as_tensor(q["x_gt"], device=dev), wq)
        x0 = torch.zeros(170 * 170, dtype=torch.complex64, device=dev).requires_grad_(True)
        k = torch.as_tensor(q["k"], device=dev).requires_grad_(True)
        lam_t = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
        xK = unrolled_fista(q, yq, x0, lam_t, k, 1, 1e6, wavelet="db4", levels=4)
        torch.mean(torch.abs(xK) ** 2).backward()
        probs, ys = [], []
        for res in range(3):
            for vol in range(2):
                r = synth.ragged_problem(res, vol, 0)
                pr = ax.Problem.from_arrays(r, device=dev)
                w = ax.workspace(pr)
                ax.prepare(pr, w)
                probs.append(pr)
                ys.append(ax.a_exp_forward(pr, torch.as_tensor(r["x_gt"], device=dev), w))
        ax.cs_recon_batched(probs, ys, [1.0] * len(probs), 2, precision=ax.BF16_TC, wavelet="db4", levels=4,
                            n_power=2)
        torch.cuda.synchronize()
        assert ax.read_status(ws) == 0
    print(json.dumps({"mode": "kernels", "ok": True}))


def run_trends(args):
    """NRMSE tables of the simulation study (Sec. 2.2.2, Figs. 4 and 5): no timing."""
    import torch
    from paper_2211_07532_gb300 import build as _b
    _b.build()
    import paper_2211_07532_gb300 as ax
    from paper_2211_07532_gb300 import trends
    t0 = time.time()
    out = trends.run(ax, eddy_scale=args.eddy_scale)
    torch.cuda.synchronize()
    out.update(kind="trends", data="synthetic", wall_s=time.time() - t0,
               workload="148x148 (1.5 mm), 32 physical coils, single-shot spiral at R, 2nd-order field + B0")
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--form", choices=["fp32", "bf16", "fp16x2"], default="fp32")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the ragged-batch and gradient sub-measurements of the default run")
    ap.add_argument("--mode", choices=["recon", "op", "kernels", "solve"], default="recon",
                    help="op: only prepare + `--reps` forward/adjoint applications (profiling target); "
                         "kernels: one small run of every non-operator kernel class; solve: one reconstruction "
                         "in --form (profiling targets)")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--tiling", type=int, default=0, help="kernel tiling of --mode op (aexp_recon_opts.tile_variant)")
    ap.add_argument("--workload", choices=["slice", "ragged", "diff"], default="slice",
                    help="slice: the 200x200 paper-scale slice (default); ragged: the 372-problem batch; "
                         "diff: unrolled-FISTA gradients")
    ap.add_argument("--volumes", type=int, default=31, help="diffusion volumes per slice (ragged workload)")
    ap.add_argument("--trends", action="store_true",
                    help="the simulation study of Figs. 4-5 (NRMSE vs R, coils, SNR, model) instead of timing")
    ap.add_argument("--eddy-scale", type=float, default=0.1, help="eddy amplitude of the trend inputs")
    args = ap.parse_args()
    if args.trends:
        run_trends(args)
    elif args.mode == "op":
        run_op_only(args)
    elif args.mode == "kernels":
        run_kernel_classes(args)
    elif args.mode == "solve":
        run_solve_only(args)
    elif args.workload == "ragged" and args.impl == "ours":
        run_ragged(args)
    elif args.workload == "diff" and args.impl == "ours":
        run_diff(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
