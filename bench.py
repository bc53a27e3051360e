#!/usr/bin/env python
"""Benchmark of the EM multi-frame deconvolution hot path (Sec. 2, Eq. (2)).

One step is one EM iteration over the whole frame set: for every exposure
the forward model, the 1/v weighting, the adjoint correlation summed over
exposures, and the multiplicative update. The default workload is the
HSC-shaped frame set (4096^2 exposures, n = 33, 43 x 43 PSFs, 5% masked),
synthetic and seeded. The metric is Gpix.exposure-iters/s: latent pixels x
exposures x iterations per second / 1e9.

Arms:
  --impl ours        the CUDA library through its C ABI (default)
  --impl reference   the FP64 CPU oracle on a bounded crop of the same
                     workload (host cores of this machine)

Multi-GPU: the path does not shard (one GPU per frame set), so N ranks run N
independent replicas; value = all ranks' work / max-over-ranks time.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "EM Gpix·exposure-iters/s"
UNIT = "Gpix·exposure-iters/s"
FP32_LANES_PER_SM = 128   # FP32 FMA lanes per SM (Blackwell)
# tile shapes of the FP32 halo-exchange kernel (emd_tile_shape values)
TILE_SHAPES = {"64": 1, "48": 2, "32": 3}
TILE_NAMES = {1: "64 x 128 tiles, 4 x 16 outputs per thread",
              2: "48 x 128 tiles, 3 x 16 outputs per thread",
              3: "32 x 128 tiles, 2 x 16 outputs per thread"}
# kernels one emd_iterate(ctx, 1) call launches: the halo-exchange (or
# CTA-pair) kernel (FP32); the x split and the tensor-core forward and adjoint
# kernels (BF16 modes); the x maximum, the power-of-two scales, the split and
# the two tensor-core kernels (FP16 modes); the FFT forward and adjoint kernels
LAUNCHES_PER_STEP = {"fp32": 1, "fp32_pair": 1, "bf16": 3, "split_bf16": 3, "fp16": 5,
                     "split_fp16": 5, "fft": 2}
# sources whose change invalidates a committed DRAM-traffic record, per kernel
KERNEL_SOURCES = {
    "halo": ["paper_2302_05804_gb300/csrc/emd_halo.cu",
             "paper_2302_05804_gb300/csrc/emd_halo.cuh",
             "paper_2302_05804_gb300/csrc/emd_corr.cuh",
             "paper_2302_05804_gb300/csrc/emd_internal.cuh"],
    "fused": ["paper_2302_05804_gb300/csrc/emd_direct.cu",
              "paper_2302_05804_gb300/csrc/emd_corr.cuh",
              "paper_2302_05804_gb300/csrc/emd_internal.cuh"],
    "fft": ["paper_2302_05804_gb300/csrc/emd_fft.cu",
            "paper_2302_05804_gb300/csrc/emd_fft.cuh",
            "paper_2302_05804_gb300/csrc/emd_internal.cuh"],
}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return int(os.environ.get("RANK", "0")), ws, int(os.environ.get("LOCAL_RANK", "0"))


def fp32_peak(device_index):
    """Derived FP32 FMA peak of the device in TFLOP/s: SMs (queried) x 128
    lanes x 2 flop x the maximum SM clock (nvidia-smi clocks.max.sm; the
    GB300's 2070 MHz when nvidia-smi cannot be asked). Returns (peak,
    description, sms, max_mhz)."""
    import torch
    sms = torch.cuda.get_device_properties(device_index).multi_processor_count
    mhz, src = 2070.0, "2070 MHz (nvidia-smi unavailable)"
    try:
        out = subprocess.run(["nvidia-smi", f"--id={device_index}", "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True,
                             timeout=30).stdout.strip()
        mhz, src = float(out.splitlines()[0]), "nvidia-smi clocks.max.sm"
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        pass
    peak = sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    return peak, (f"derived: {sms} SMs (queried) x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x "
                  f"{mhz:.0f} MHz ({src})"), sms, mhz


def workload_shape(name):
    import synth
    _, d = synth.RECIPES[name]
    return d


def algorithmic_flops(H, W, n, K, r):
    """flops of one iteration: forward + adjoint, each n * H * W * (K+r-1)^2
    FMA on the exposure grid (the polyphase count; r = 1 gives K^2)."""
    return 2.0 * 2.0 * n * H * W * (K + r - 1) ** 2


def aggregate_over_ranks(local_ms, units_per_rank, world, device="cuda"):
    """Whole-job throughput of N independent replicas: every rank processed
    units_per_rank; the job took the slowest rank's time. Returns
    (max_ms over ranks, value in units/s / 1e9)."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    max_ms = float(t.item())
    return max_ms, units_per_rank * world / (max_ms / 1e3) / 1e9


def tc_executed_flops(H, W, n, K, r, nprod):
    """Tensor-core flops one iteration issues: per 128 x 128 tile, exposure,
    phase and filter row (Kc of them), one forward and one adjoint GEMM of
    M = N = 128 over a band of Kd = rup(128 + 2 hc + hc mod 8, 16) columns
    (the banded Toeplitz operand, zeros included), for each product of the
    split."""
    rup = lambda a, b: (a + b - 1) // b * b
    hc = ((K - 1) // 2 + r - 1) // r
    Kc = 2 * hc + 1
    Kd = rup(128 + 2 * hc + (hc & 7), 16)
    tiles = ((W + 127) // 128) * ((H + 127) // 128)
    return tiles * n * r * r * Kc * nprod * 2 * (128 * 128 * Kd) * 2


def fft_flops(H, W, n, K, r, nu):
    """flops one FFT-form iteration runs: 128^2 real transforms (2.5 N log2 N
    each, N = 128^2) on overlap-save tiles of 128 - 2 hc outputs, and the
    spectrum products. Forward: R2 + n transforms per tile; adjoint: n + R2,
    or 2 n + 2 R2 with the heavy-tailed numerator planes."""
    hc = ((K - 1) // 2 + r - 1) // r
    B = 128 - 2 * hc
    tiles = -(-H // B) * -(-W // B)
    m = 2 if nu > 0 else 1
    ffts = tiles * ((1 + m) * (n + r * r))
    return ffts * 2.5 * 16384 * 14 + tiles * (1 + m) * n * r * r * 6 * 128 * 65


def fft_kernels(H, W, n, K, r, nu, sms):
    """Names of the two kernels an FFT-form iteration launches: the split
    forms (persistent, one CTA per SM) for r = 1 Gaussian with at least as
    many tiles as SMs, else one CTA per tile."""
    hc = ((K - 1) // 2 + r - 1) // r
    B = 128 - 2 * hc
    tiles = -(-H // B) * -(-W // B)
    if r == 1 and nu == 0 and tiles >= sms:
        return "fft_forward_split_kernel + fft_adjoint_split_kernel"
    return "fft_forward_kernel + fft_adjoint_kernel"


def bf16_peak():
    """(TFLOP/s, description) of the measured dense BF16 peak (burst)."""
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(mp["bf16_tflops"]), "measured bf16_tflops (burst), of measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback 1.9 PFLOP/s bf16 burst"


def variant_roofline(name, p, launch_s, peak32, peak32_src, sms):
    """Roofline record of one timed variant (same conventions as the
    headline's): FMA pipe for the direct forms, FP32 issue for the FFT form,
    the tensor pipe (executed flops) for the tensor-core forms."""
    flops = algorithmic_flops(p.H, p.W, p.n, p.K, p.r)
    nu = 3.0 if name.startswith("student") else 0.0
    if name.startswith("student"):
        flops *= 1.5
    if "fft" in name:
        fl = fft_flops(p.H, p.W, p.n, p.K, p.r, nu)
        ex = fl / launch_s / 1e12
        rec = {"bound": "alu", "achieved": ex, "peak": peak32, "unit": "TFLOP/s",
               "frac": ex / peak32, "peak_source": peak32_src,
               "kernel": fft_kernels(p.H, p.W, p.n, p.K, p.r, nu, sms),
               "fft_tflop_per_iteration": fl / 1e12,
               "direct_equivalent_tflops": flops / launch_s / 1e12}
        tr = committed_traffic("fft", "hsc") if nu == 0 else None
        if tr:
            rec["traffic"] = tr
            rec["hbm_gbs"] = tr / launch_s / 1e9
        return rec
    if name in ("split_bf16", "bf16", "split_fp16", "fp16"):
        nprod = 3 if name.startswith("split") else 1
        ex = tc_executed_flops(p.H, p.W, p.n, p.K, p.r, nprod) / launch_s / 1e12
        pk, src = bf16_peak()
        return {"bound": "tensor", "achieved": ex, "peak": pk, "unit": "TFLOP/s",
                "frac": ex / pk, "peak_source": src, "kernel": "tc_fwd_kernel + tc_adj_kernel",
                "useful_tflops": flops / launch_s / 1e12}
    ach = flops / launch_s / 1e12
    return {"bound": "alu", "achieved": ach, "peak": peak32, "unit": "TFLOP/s",
            "frac": ach / peak32, "peak_source": peak32_src,
            "kernel": "fused_kernel" if name == "fp32_pair" else "halo_kernel"}


def kernel_source_hash(kernel):
    h = hashlib.sha256()
    for p in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, p), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic(kernel, workload):
    """DRAM bytes per iteration of a kernel ("halo", "fused"; "fft": its
    forward and adjoint launches together) from the committed ncu summary
    profiles/<kernel>_<workload>_traffic.json, or None when the kernel's
    source changed since it was taken."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}_traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    if rec.get("source_hash") != kernel_source_hash(kernel):
        return None
    return rec.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, on a bounded crop
# ---------------------------------------------------------------------------

def crop_problem(p, side):
    """Fresh zero-padded sub-problem: a centred side x side crop of every
    exposure (and of the latent grid)."""
    import synth
    c0 = (p.H - side) // 2
    sl = slice(c0, c0 + side)
    r = p.r
    return synth.Problem(y=np.ascontiguousarray(p.y[:, sl, sl]),
                         v=np.ascontiguousarray(p.v[:, sl, sl]), f=p.f,
                         mask=np.ascontiguousarray(p.mask[:, sl, sl]),
                         x_true=p.x_true[r * c0:r * (c0 + side), r * c0:r * (c0 + side)], r=r)


def oracle_steps(p, side, steps, warmup, min_seconds=0.0):
    import oracle
    q = crop_problem(p, side)
    u, y, N, c = oracle.prepare(q)
    x = np.full((q.r * side, q.r * side), c)
    for _ in range(warmup):
        x = oracle.em_step(x, N, u, q.f, q.r)
    times = []
    t_all = time.perf_counter()
    while len(times) < steps or (time.perf_counter() - t_all) < min_seconds:
        t0 = time.perf_counter()
        x = oracle.em_step(x, N, u, q.f, q.r)
        times.append(time.perf_counter() - t0)
        if len(times) >= max(steps, 1) and min_seconds == 0.0:
            break
    units = (q.r * side) ** 2 * q.n
    total = sum(times)
    return {"value": units * len(times) / total / 1e9, "unit": UNIT,
            "cores": oracle.num_threads(), "kind": "oracle",
            "sample": (f"{side}x{side} centred crop (all {q.n} exposures, zero-padded, "
                       f"K={q.K}, r={q.r}) of the workload, {len(times)} EM iteration(s) "
                       f"of the FP64 C oracle"),
            "seconds": total, "steps": len(times)}


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import synth
    # a bounded sample of the workload: the same recipe (source densities,
    # PSFs, noise, masks) drawn at side x side
    side = args.ref_crop
    p = synth.make_problem(args.workload, H=side, W=side)
    res = oracle_steps(p, side, args.steps, args.warmup)
    ms = res["seconds"] / res["steps"] * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": res["value"], "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": config_of(args, extra={"sample_crop": side}),
        "cpu_baseline": {k: res[k] for k in ("value", "unit", "cores", "kind", "sample")},
        "e2e": {"value": res["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_serving(p, args, precision=0, jobs=2000):
    """Continuous-batching run: `jobs` jobs with sides log-uniform in
    [128, 2048], 4-40 exposures, odd PSF sides 15-43, 50 iterations each, cut
    from the resident frame set; an 80 GB budget. First all jobs at t=0
    (saturated jobs/s, seed 4004), then Poisson streams of `jobs` jobs (seed
    4005) at 0.5x, 0.7x and 0.9x that rate for p50/p99 latency (the
    top-level figures are the 0.7x stream's)."""
    from paper_2302_05804_gb300 import serve
    pool = serve.DataPool(p)
    kw = dict(s_range=(128, min(2048, p.H)), n_range=(4, 40), k_range=(15, min(43, p.K)),
              iters=50)
    sat_trace = serve.poisson_trace(jobs, rate=1e9, seed=4004, **kw)
    srv = serve.Server(hbm_budget=80e9, max_slots=64, precision=precision)
    t0 = time.perf_counter()
    try:
        res = srv.run(sat_trace, pool.make, realtime=False)
    finally:
        srv.close()
    sat = serve.Server.summary(res)
    print(f"serving ({'fft' if precision == 5 else 'direct'}): {len(res)} jobs saturated, "
          f"{sat['jobs_per_s']:.1f} jobs/s, {time.perf_counter() - t0:.0f} s", file=sys.stderr,
          flush=True)
    per_rate = {}
    for frac in (0.5, 0.7, 0.9):
        rate_f = frac * sat["jobs_per_s"]
        trace_f = serve.poisson_trace(jobs, rate=rate_f, seed=4005, **kw)
        srv = serve.Server(hbm_budget=80e9, max_slots=64, precision=precision)
        try:
            res_f = srv.run(trace_f, pool.make, realtime=True)
        finally:
            srv.close()
        per_rate[frac] = (rate_f, trace_f, res_f, serve.Server.summary(res_f))
        print(f"serving at {frac}x: p50 {per_rate[frac][3]['p50_s']:.3f} s, "
              f"p99 {per_rate[frac][3]['p99_s']:.3f} s over {len(res_f)} jobs", file=sys.stderr,
              flush=True)
    rate, trace, res, live = per_rate[0.7]
    fma = sum(2.0 * s.n * s.H * s.W * s.K ** 2 * s.iters for s in trace)
    return {"form": "fft" if precision == 5 else "direct fp32",
            "jobs": len(res), "saturated_jobs_per_s": sat["jobs_per_s"],
            "saturated_jobs": sat["jobs"],
            "by_load": {f"{frac}x": {"jobs": v[3]["jobs"], "arrival_rate_jobs_per_s": v[0],
                                     "p50_latency_s": v[3]["p50_s"],
                                     "p99_latency_s": v[3]["p99_s"], "jobs_per_s": v[3]["jobs_per_s"],
                                     "span_s": v[3]["span_s"]}
                        for frac, v in per_rate.items()},
            "arrival_rate_jobs_per_s": rate, "jobs_per_s": live["jobs_per_s"],
            "p50_latency_s": live["p50_s"], "p99_latency_s": live["p99_s"],
            "mean_latency_s": live["mean_s"], "gpix_exposure_iters_per_s":
                sum(s.H * s.W * s.n * s.iters for s in trace) / live["span_s"] / 1e9,
            "useful_tflops": 2 * fma / live["span_s"] / 1e12,
            "workload": "sides log-uniform 128-2048, n 4-40, K odd 15-43, 50 iterations, "
                        "Poisson arrivals at 0.5x/0.7x/0.9x the saturated rate, 80 GB budget, "
                        "64 slots"}


def run_variants(p, peak32, peak32_src, steps=5, warmup=2):
    """The other built forms of the iteration on the same frame set, each in
    its own context: CUDA events per iteration on the context's stream, and a
    roofline record for each."""
    import torch
    from paper_2302_05804_gb300 import emd
    forms = [("fp32_pair", emd.EMD_PREC_FP32_PAIR, 0.0),
             ("fft", emd.EMD_PREC_FFT_FP32, 0.0), ("split_bf16", emd.EMD_PREC_SPLIT_BF16, 0.0),
             ("bf16", emd.EMD_PREC_BF16, 0.0), ("split_fp16", emd.EMD_PREC_SPLIT_FP16, 0.0),
             ("fp16", emd.EMD_PREC_FP16, 0.0), ("student_t_nu3", emd.EMD_PREC_FP32, 3.0),
             ("student_t_nu3_fft", emd.EMD_PREC_FFT_FP32, 3.0)]
    out = {}
    for name, prec, nu in forms:
        st = torch.cuda.Stream()
        d = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r, stream=st)
        try:
            d.set_frames(p.y, p.v, p.f, p.mask)
            if prec:
                d.set_precision(prec)
            if nu > 0:
                d.set_noise(emd.EMD_NOISE_STUDENT_T, nu)
            d.iterate(warmup)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            d.iterate(steps)
            e1.record(st)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
        finally:
            d.close()
        out[name] = {"ms_per_iteration": ms,
                     "value": p.r * p.r * p.H * p.W * p.n / (ms / 1e3) / 1e9, "unit": UNIT,
                     "roofline": variant_roofline(name, p, ms / 1e3, peak32, peak32_src,
                                                  torch.cuda.get_device_properties(
                                                      torch.cuda.current_device()).multi_processor_count)}
    return out


def run_psf_fit(p, iters):
    """Eq. (4) fit of super-resolved PSFs for every exposure: the workload's
    coarse PSFs (n x K x K) to r = 2 fine PSFs (2 (K-1) + 1 per side), g a
    Gaussian of FWHM one coarse pixel, lambda 1e-3, lr 1e-4. Device buffers;
    CUDA events on the legacy default stream around the call."""
    import torch
    import synth
    from paper_2302_05804_gb300 import emd
    r, lam, lr = 2, 1e-3, 1e-4
    n, K = p.f.shape[0], p.f.shape[1]
    Kh = r * (K - 1) + 1
    g = synth.gaussian_kernel(r).astype(np.float32)
    Kg = g.shape[0]
    fd = torch.from_numpy(np.ascontiguousarray(p.f, dtype=np.float32)).cuda()
    gd = torch.from_numpy(g).cuda()
    hd = torch.empty((n, Kh, Kh), dtype=torch.float32, device="cuda")
    ld = torch.empty(n, dtype=torch.float32, device="cuda")
    emd.emd_fit_psf(fd, gd, r, lam, lr, 10, h_out=hd, loss_out=ld)  # warm
    s0 = torch.cuda.default_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s0)
    emd.emd_fit_psf(fd, gd, r, lam, lr, iters, h_out=hd, loss_out=ld)
    e1.record(s0)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # useful FMAs: in-grid taps of h * g and of its adjoint (equal counts)
    hg = (Kg - 1) // 2
    taps1d = sum(sum(1 for a in range(Kg) if 0 <= P + hg - a < Kh) for P in range(Kh))
    flops = 2.0 * 2.0 * taps1d ** 2 * n * iters
    peak = fp32_peak(torch.cuda.current_device())[0]
    tf = flops / (ms / 1e3) / 1e12
    return {"workload": f"{n} coarse {K}x{K} PSFs -> {Kh}x{Kh} (r = {r}), Kg = {Kg}, "
                        f"{iters} projected Adam iterations",
            "ms": ms, "us_per_iteration": ms * 1e3 / iters, "useful_tflops": tf,
            "alu_frac": tf / peak, "ctas": n,
            "final_loss_median": float(ld.median().item())}


def config_of(args, extra=None):
    d = workload_shape(args.workload)
    H, W, n, K, r = d["H"], d["W"], d["n"], d["K"], d["r"]
    if getattr(args, "size", 0) and args.impl == "ours":
        H = W = args.size
    c = {"workload": f"{args.workload}: {n} exposures of {H}x{W}, "
                     f"{K}x{K} PSFs, r={r}, latent {r * H}x{r * W}",
         "H": H, "W": W, "n": n, "K": K, "r": r,
         "precision": args.precision,
         "noise": (f"student-t nu={args.nu:g}" if getattr(args, "nu", 0) > 0 else "gaussian"),
         "l2": (f"no flush: each step streams the u planes ({n * H * W * 4 / 1e9:.2f} GB), "
                + ("far above" if n * H * W * 4 > 4 * 129e6 else "not far above")
                + " the 129 MB L2"),
         "parallelism": "replicas"}
    if extra:
        c.update(extra)
    return c


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import synth
    from paper_2302_05804_gb300 import emd

    over = {"H": args.size, "W": args.size} if args.size else {}
    p = synth.make_problem(args.workload, **over)
    Hf, Wf = p.r * p.H, p.r * p.W
    prec = {"fp32": 0, "bf16": 1, "fp16": 2, "split_bf16": 3, "split_fp16": 4,
            "fft": 5, "fp32_pair": 6}[args.precision]

    stream = torch.cuda.Stream()
    d = emd.Deconvolver(p.H, p.W, p.n, p.K, p.r, stream=stream)
    d.set_frames(p.y, p.v, p.f, p.mask)
    if prec:
        d.set_precision(prec)
    if args.nu > 0:
        d.set_noise(emd.EMD_NOISE_STUDENT_T, args.nu)
    if args.tile_shape:
        d.set_tile_shape(TILE_SHAPES[args.tile_shape])

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # warm-up; the FP32 direct form's autotuner times its tile shapes on the
    # first iterations of a new problem shape, so warm up until it has decided
    for _ in range(args.warmup):
        d.iterate(1)
    torch.cuda.synchronize()
    if prec == 0:
        for _ in range(16):
            if d.tile_shape()[1]:
                break
            d.iterate(1)
            torch.cuda.synchronize()
    tile = d.tile_shape() if prec == 0 else None

    # timed region: K steps, one fused-kernel launch each, events per step
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    ev[0].record(stream)
    for k in range(args.steps):
        d.iterate(1)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms, value = aggregate_over_ranks(ev[0].elapsed_time(ev[-1]), Hf * Wf * p.n * args.steps,
                                           world)

    # the heavy-tailed step needs the forward model once and two adjoints
    # (of u'z and of u'y): 1.5x the Gaussian step's convolutions
    flops = algorithmic_flops(p.H, p.W, p.n, p.K, p.r) * (1.5 if args.nu > 0 else 1)
    launch_s = statistics.mean(per) / 1e3
    achieved = flops / launch_s / 1e12
    peak32, peak32_src, _, sm_max_mhz = fp32_peak(local)
    if prec == 5:
        # FFT form: flops of the transforms it runs (a real 128^2 transform
        # = 2.5 N log2 N, N = 128^2) and of the spectrum products, against
        # the FP32 peak; the direct-form flops it replaces are reported beside
        peak = peak32
        fl = fft_flops(p.H, p.W, p.n, p.K, p.r, args.nu)
        ex = fl / launch_s / 1e12
        traffic = committed_traffic("fft", args.workload) if args.nu == 0 else None
        roofline = {"bound": "alu", "achieved": ex, "peak": peak, "unit": "TFLOP/s",
                    "frac": ex / peak, "traffic": traffic,
                    "kernel": fft_kernels(p.H, p.W, p.n, p.K, p.r, args.nu,
                                          fp32_peak(local)[2]) + " (FP32 FFT)",
                    "peak_source": peak32_src,
                    "direct_equivalent_tflops": achieved,
                    "fft_tflop_per_iteration": fl / 1e12}
    elif prec in (0, 6):
        peak = peak32
        kern = "halo" if prec == 0 else "fused"
        # the committed DRAM records are of the Gaussian instances
        traffic = committed_traffic(kern, args.workload) if args.nu == 0 else None
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": traffic,
                    "kernel": {"halo": "halo_kernel (FP32 FMA, persistent, w ring in L2)",
                               "fused": "fused_kernel (FP32 FMA, CTA pairs)"}[kern] +
                              (" heavy-tailed instance" if args.nu > 0 else ""),
                    "peak_source": peak32_src}
        if prec == 0:
            how = ("fixed by --tile-shape" if args.tile_shape else
                   "autotuned" if tile[1] else "autotuner undecided")
            roofline["tile"] = f"{TILE_NAMES[tile[0]]} ({how})"
        if traffic:
            hbm_peak, hsrc = 6800.0, "fallback 6.8 TB/s"
            try:
                hbm_peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
                hsrc = "measured hbm_gbs, of measured"
            except (OSError, KeyError, ValueError):
                pass
            roofline["hbm_gbs"] = traffic / launch_s / 1e9
            roofline["hbm_frac"] = roofline["hbm_gbs"] / hbm_peak
            roofline["hbm_peak_source"] = hsrc
        if clocks.get("sm_mhz"):
            roofline["frac_at_sampled_clock"] = achieved / (peak * clocks["sm_mhz"] / sm_max_mhz)
        fma = emd.emd_measure_fma_rate()
        roofline["fma_chain_measured_tflops"] = fma
        roofline["frac_of_measured_fma"] = achieved / fma
    else:
        nprod = 3 if args.precision.startswith("split") else 1
        ex = tc_executed_flops(p.H, p.W, p.n, p.K, p.r, nprod) / launch_s / 1e12
        peak, src = bf16_peak()
        roofline = {"bound": "tensor", "achieved": ex, "peak": peak, "unit": "TFLOP/s",
                    "frac": ex / peak, "traffic": None,
                    "kernel": "tc_fwd_kernel + tc_adj_kernel (tcgen05)",
                    "useful_tflops": achieved, "peak_source": src}

    # end to end through the public API from pinned host memory
    e2e = None
    if args.e2e_iters > 0:
        pin = lambda a: torch.from_numpy(a).pin_memory()
        hy, hv, hf, hm = pin(p.y), pin(p.v), pin(p.f), pin(p.mask)
        hx = torch.empty((Hf, Wf), dtype=torch.float32).pin_memory()
        h2d = sum(a.numel() * a.element_size() for a in (hy, hv, hf, hm))
        d2h = hx.numel() * 4 + 8

        parts = {"set_frames_s": 0.0, "iterations_and_loglik_s": 0.0, "get_x_s": 0.0}

        def job(record):
            # host timestamps between the calls; every call that returns to
            # the host already synchronises the stream (set_frames from host
            # buffers, loglik, get_x), so none is added here
            ta = time.perf_counter()
            d.set_frames(hy, hv, hf, hm)
            tb = time.perf_counter()
            d.iterate(args.e2e_iters)
            d.loglik()
            tc = time.perf_counter()
            emd.emd_get_x(d.ctx, hx)
            td = time.perf_counter()
            if record:
                parts["set_frames_s"] += tb - ta
                parts["iterations_and_loglik_s"] += tc - tb
                parts["get_x_s"] += td - tc

        job(False)  # warm
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_jobs):
            job(True)
        torch.cuda.synchronize()
        el = torch.tensor([time.perf_counter() - t0], device="cuda")
        if world > 1:
            torch.distributed.all_reduce(el, op=torch.distributed.ReduceOp.MAX)
        e2e = {"value": Hf * Wf * p.n * args.e2e_iters * args.e2e_jobs * world / el.item() / 1e9,
               "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "iters_per_step": args.e2e_iters,
               "step": "set_frames + iterations + loglik + get_x, host pinned buffers",
               "components_s_per_step": {k: v / args.e2e_jobs for k, v in parts.items()}}
    d.close()

    serving = serving_direct = None
    if args.serve_jobs > 0 and prec == 0:
        serving = run_serving(p, args, precision=5, jobs=args.serve_jobs)
    if args.serve_jobs_direct > 0 and prec == 0:
        serving_direct = run_serving(p, args, precision=0, jobs=args.serve_jobs_direct)
    psf_fit = None
    if args.psf_iters > 0 and prec == 0:
        psf_fit = run_psf_fit(p, args.psf_iters)
    variants = None
    if args.variants and prec == 0 and args.nu == 0:
        variants = run_variants(p, peak32, peak32_src)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res = oracle_steps(p, args.cpu_crop, 1, 0, min_seconds=args.cpu_seconds)
        cpu = {k: res[k] for k in ("value", "unit", "cores", "kind", "sample")}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp32_pair": "f32", "bf16": "bf16", "split_bf16": "bf16x3",
                      "fp16": "f16", "split_fp16": "f16x3", "fft": "f32"}[args.precision],
            "data": "synthetic",
            "config": config_of(args), "roofline": roofline, "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps * LAUNCHES_PER_STEP[args.precision] *
                            (2 if args.nu > 0 and args.precision == "fp32_pair" else 1),
            "clocks": clocks,
            "serving": serving, "serving_direct_fp32": serving_direct, "psf_fit": psf_fit,
            "variants": variants,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["hsc", "sr2", "parity"], default="hsc")
    ap.add_argument("--size", type=int, default=0,
                    help="override the exposure side (profiling of small cases)")
    ap.add_argument("--precision", default="fp32",
                    choices=["fp32", "fp32_pair", "bf16", "fp16", "split_bf16", "split_fp16",
                             "fft"])
    ap.add_argument("--e2e-iters", type=int, default=10)
    ap.add_argument("--e2e-jobs", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-jobs", type=int, default=2000,
                    help="jobs of each serving run in the FFT form (0 disables it)")
    ap.add_argument("--serve-jobs-direct", type=int, default=200,
                    help="jobs of each serving run in the direct FP32 form (0 disables it; "
                         "2000 would take about 20 minutes at its 10 jobs/s)")
    ap.add_argument("--no-variants", dest="variants", action="store_false",
                    help="skip timing the FFT, tensor-core and heavy-tailed forms")
    ap.add_argument("--nu", type=float, default=0.0,
                    help="Student-t degrees of freedom of the heavy-tailed noise model "
                         "(0: Gaussian, Eq. (1))")
    ap.add_argument("--psf-iters", type=int, default=20000,
                    help="Adam iterations of the Eq. (4) PSF fit sample (0 disables it)")
    ap.add_argument("--tile-shape", default="", choices=[""] + list(TILE_SHAPES),
                    help="tile shape of the FP32 halo-exchange kernel (default: autotuned)")
    ap.add_argument("--cpu-crop", type=int, default=512)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-crop", type=int, default=256)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    return run_reference(args) if args.impl == "reference" else run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
