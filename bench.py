#!/usr/bin/env python3
"""Benchmark of the Fourier LLF hot path on GB300 (one JSON line on stdout).

Workload: one 3840 x 2160 RGB frame (planar float32, synthetic, seeded;
40 polygons, texture and noise), every channel filtered independently,
8 pyramid levels, K = 8 Fourier orders, m = 3, sigma_r = 0.2, T = 2.
A step is one pass of the whole path (all kernels) over one frame.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp16|bf16]
    python bench.py --impl reference ...     # the float64 CPU oracle, timed on host cores

Multi-GPU runs (torchrun, one rank per GPU) are replicas: each rank filters
its own frames, no collective on the data path (weak scaling); the timed
region is bracketed by barriers and the slowest rank's time is reported.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpixel/s Fourier LLF K=8 4K RGB at PSNR≥60dB vs FP64; serving p50/p99 ms"
UNIT = "Mpixel/s"
WORKLOAD = dict(H=2160, W=3840, C=3, polygons=40, seed=2, levels=8, K=8, m=3.0, sigma_r=0.2, T=2.0)
N_FRAMES = 4          # distinct input/output frames cycled per step (4 x 99.5 MB > 129 MB L2)
STAGES = ("up0", "up", "down", "down0", "chain", "down_s")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "fp16", "bf16"], default="fp32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--workload", choices=["uhd", "batch", "serve"], default="uhd",
                    help="uhd: the 4K RGB headline (plus fast LLF at the same pyramid count and a "
                         "short served stream); batch: 64 mixed images, batched vs looped; serve: "
                         "Poisson request streams.  Accuracy against the float64 oracle is "
                         "measured by tests/accuracy.py")
    ap.add_argument("--serve-seconds", type=float, default=None,
                    help="length of each served stream (default 30 s; 4 s in the uhd line)")
    ap.add_argument("--serve-rates", type=str, default=None,
                    help="comma-separated arrival rates in requests/s, or max for a backlog "
                         "(default 50,100,200,400,max)")
    ap.add_argument("--serve-precision", choices=["fp32", "fp16", "bf16"], default="fp16")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the launch-shape autotuner (default settings)")
    return ap.parse_args()


def level_sizes(H, W, L):
    out, h, w = [], H, W
    for _ in range(L):
        out.append((h, w))
        h, w = (h + 1) // 2, (w + 1) // 2
    return out


CHAIN_PIXELS = 0         # default: levels whose pixels over all planes fit this run chained
SMALL_PIXELS = 1 << 40   # default: other combines at levels >= 2 this small run on 32 x 16 tiles


def stage_split(cfg, chain_px=CHAIN_PIXELS, small_px=SMALL_PIXELS):
    """Which levels each stage kind covers, as the library launches them.

    Returns (up_levels, chain_up, chain_down, down_levels, small_levels,
    fused): REDUCE l -> l+1 for l in up_levels / chain_up, level-l combines
    for l in chain_down / down_levels (64 x 32 tiles) / small_levels (32 x 16
    tiles), and whether the level-0 stage also runs the level-1 combine
    (levels >= 3)."""
    L, C = cfg["levels"], cfg["C"]
    sz = level_sizes(cfg["H"], cfg["W"], L)
    c0 = L - 1
    for l in range(2, L - 1):
        if sz[l][0] * sz[l][1] * C <= chain_px:
            c0 = l
            break
    c0 = max(c0, L - 1 - 12)
    up_levels = [l for l in range(1, L - 1) if l < c0]
    chain_up = list(range(c0, L - 1)) if c0 <= L - 2 else []
    chain_down = list(range(L - 2, c0 - 1, -1)) if c0 <= L - 2 else []
    fused = L >= 3
    hi = c0 - 1 if c0 <= L - 2 else L - 2
    down_all = list(range(hi, (2 if fused else 1) - 1, -1))
    small_levels = [l for l in down_all if l >= 2 and sz[l][0] * sz[l][1] * C <= small_px]
    down_levels = [l for l in down_all if l not in small_levels]
    return up_levels, chain_up, chain_down, down_levels, small_levels, fused


def stage_work(cfg, zbytes, chain_px=CHAIN_PIXELS, small_px=SMALL_PIXELS):
    """Algorithmic FP32 ops and bytes per stage kind for one frame (all planes).

    Ops (FMA = 1; the method's separable stencil count with Horner's rule
    over the orders):
      trig per evaluated pixel      16 (sincospi and its fix-up); the REDUCE of
                                    level 0 adds 2 (K - 1) for the recurrence
                                    over the orders
      REDUCE per output per image   13 (2 horizontal x 4 + vertical 4 + scale)
      combine per pixel and order   10 at level 0 (6 EXPAND + 4 complex
                                    multiply-add), 12 at level >= 1 (+2 for
                                    Z_l - up(Z_{l+1}))
      residual EXPAND + add         4 per pixel
    Bytes: each input element read once and each output written once; the
    level-1 combine inside the level-0 stage reads G_1, Z_1 (shared with the
    level-0 EXPAND), Z_2 and E_2, and writes nothing.
    """
    L, K, C = cfg["levels"], cfg["K"], cfg["C"]
    sz = level_sizes(cfg["H"], cfg["W"], L)
    n = [h * w for h, w in sz]
    trig = 16
    up_levels, chain_up, chain_down, down_levels, small_levels, fused = stage_split(cfg, chain_px, small_px)
    ops = dict.fromkeys(STAGES, 0.0)
    byt = dict.fromkeys(STAGES, 0.0)

    def reduce_work(l):
        g = 1 if l + 1 <= L - 2 else 0
        return (n[l + 1] * 13 * (2 * K + g),
                (4 * n[l] * g + zbytes * K * n[l]) + (4 * n[l + 1] * g + zbytes * K * n[l + 1]))

    def combine_work(l):
        e = 1 if l + 1 <= L - 2 else 0
        return (n[l] * (trig + 12 * K + 4 * e),
                4 * n[l] + zbytes * K * n[l] + zbytes * K * n[l + 1] + 4 * n[l + 1] * e + 4 * n[l])

    if L >= 2:
        ops["up0"] = n[0] * (trig + 2 * (K - 1)) + n[1] * 13 * (2 * K + 1)
        byt["up0"] = 4 * n[0] + 4 * n[1] + zbytes * K * n[1]
    for l in up_levels:
        o, b = reduce_work(l)
        ops["up"] += o
        byt["up"] += b
    for l in chain_up:
        o, b = reduce_work(l)
        ops["chain"] += o
        byt["chain"] += b
    for l in chain_down:
        o, b = combine_work(l)
        ops["chain"] += o
        byt["chain"] += b
    for l in down_levels:
        o, b = combine_work(l)
        ops["down"] += o
        byt["down"] += b
    for l in small_levels:
        o, b = combine_work(l)
        ops["down_s"] += o
        byt["down_s"] += b
    if L >= 2:
        e1 = 1 if L >= 3 else 0
        ops["down0"] = n[0] * (trig + 10 * K + 4 * e1)
        byt["down0"] = 4 * n[0] + zbytes * K * n[1] + 4 * n[0]
        if fused:
            e2 = 1 if L >= 4 else 0
            ops["down0"] += n[1] * (trig + 12 * K + 4 * e2)
            byt["down0"] += 4 * n[1] + zbytes * K * n[2] + 4 * n[2] * e2
        else:
            byt["down0"] += 4 * n[1] * e1
    return {k: v * C for k, v in ops.items()}, {k: v * C for k, v in byt.items()}


def hbm_min_bytes(cfg):
    """Input read + output write + guide pyramid (levels >= 1) written once and read once."""
    sz = level_sizes(cfg["H"], cfg["W"], cfg["levels"])
    guide = sum(h * w for h, w in sz[1:])
    return cfg["C"] * (4 * cfg["H"] * cfg["W"] * 2 + 2 * 4 * guide)


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        loaded = [s for s in sm if mx and s >= 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def cpu_oracle_sample():
    """Float64 oracle on channel 0 of the 4K frame (one of three planes)."""
    import numpy as np
    import oracle
    from paper_2206_04681_gb300.synth import synth_image
    cfg = WORKLOAD
    img = synth_image(cfg["H"], cfg["W"], cfg["C"], cfg["polygons"], cfg["seed"])
    a = oracle.coeffs_quadrature(cfg["m"], cfg["sigma_r"], cfg["T"], cfg["K"])
    t0 = time.perf_counter()
    oracle.fourier_llf(img[0].astype(np.float64), cfg["levels"], a, cfg["T"])
    dt = time.perf_counter() - t0
    frame_s = dt * cfg["C"]
    return {"value": cfg["H"] * cfg["W"] / frame_s / 1e6, "unit": UNIT, "cores": 1,
            "kind": "oracle",
            "sample": f"float64 numpy oracle, channel 0 of the 3840x2160x3 frame "
                      f"({dt:.1f} s; frame time = 3 x plane time)"}


def run_reference(args):
    """Reference arm: the float64 CPU oracle as it stands, on host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    from paper_2206_04681_gb300.synth import synth_image
    cfg = WORKLOAD
    img = synth_image(cfg["H"], cfg["W"], cfg["C"], cfg["polygons"], cfg["seed"])
    a = oracle.coeffs_quadrature(cfg["m"], cfg["sigma_r"], cfg["T"], cfg["K"])
    # each step: one plane of a 960 x 540 crop (a bounded sample of the frame)
    crop = img[0, 810:1350, 1440:2400].astype(np.float64)
    for _ in range(args.warmup):
        oracle.fourier_llf(crop, cfg["levels"], a, cfg["T"])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.fourier_llf(crop, cfg["levels"], a, cfg["T"])
    dt = (time.perf_counter() - t0) / args.steps
    value = crop.size / (dt * cfg["C"]) / 1e6   # a pixel counts once over its 3 channels
    sample = "float64 numpy oracle on one plane of a 960x540 crop per step (RGB time = 3 x plane)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "uhd_rgb_3840x2160x3_L8_K8", "H": cfg["H"], "W": cfg["W"],
                       "C": cfg["C"], "levels": cfg["levels"], "K": cfg["K"], "m": cfg["m"],
                       "sigma_r": cfg["sigma_r"], "T": cfg["T"], "sample": "960x540 crop, 1 plane"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---- replicas over ranks (one process per GPU) ---------------------------------------
def rank_env():
    """(world, rank, local rank) from the torchrun environment (1, 0, 0 alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(cfg, rank):
    """Each rank filters its own synthetic frames: the workload seed plus the rank."""
    return cfg["seed"] + rank


def max_over_ranks(x, world, device):
    """The largest value of x over the ranks (the slowest rank's time); x itself alone."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mpixel_s(world, pixels_per_rank_step, seconds_per_step):
    """Whole-job throughput: every rank filters one frame per step (weak scaling)."""
    return world * pixels_per_rank_step / seconds_per_step / 1e6


def time_precision(pkg, torch, cfg, precision, frames, steps, warmup, stream, device, params=None):
    """ms per frame of a plan (autotuned), back to back over the cycled frames."""
    p = params or pkg.make_params(cfg["H"], cfg["W"], cfg["C"], cfg["levels"], cfg["K"], cfg["m"],
                                  cfg["sigma_r"], cfg["T"], precision)
    plan = pkg.fllf_plan_create(p, device)
    outs = [torch.empty_like(f) for f in frames]
    try:
        pkg.fllf_plan_autotune(plan, frames[0].data_ptr(), outs[0].data_ptr(), reps=8,
                               stream=stream.cuda_stream)
        with torch.cuda.stream(stream):
            for i in range(warmup):
                pkg.fllf_run(plan, frames[i % len(frames)].data_ptr(),
                             outs[i % len(frames)].data_ptr(), stream.cuda_stream)
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for i in range(steps):
                pkg.fllf_run(plan, frames[i % len(frames)].data_ptr(),
                             outs[i % len(frames)].data_ptr(), stream.cuda_stream)
            e1.record(stream)
            e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
    finally:
        pkg.fllf_plan_destroy(plan)
    return ms


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2206_04681_gb300 as pkg
    from paper_2206_04681_gb300 import build
    from paper_2206_04681_gb300.synth import synth_image

    world, rank, local = rank_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    device = local

    build.build_library()
    cfg = WORKLOAD
    img = synth_image(cfg["H"], cfg["W"], cfg["C"], cfg["polygons"], rank_seed(cfg, rank))
    base = torch.from_numpy(img).cuda()
    frames = [base.clone() for _ in range(N_FRAMES)]
    outs = [torch.empty_like(base) for _ in range(N_FRAMES)]
    stream = torch.cuda.Stream()

    p = pkg.make_params(cfg["H"], cfg["W"], cfg["C"], cfg["levels"], cfg["K"], cfg["m"],
                        cfg["sigma_r"], cfg["T"], args.precision)
    plan = pkg.fllf_plan_create(p, device)
    # launch-shape autotuner (setup, outside the timed region, like plan creation)
    tuning = None
    if not args.no_autotune:
        t0 = time.perf_counter()
        tun, tuned_ms = pkg.fllf_plan_autotune(plan, frames[0].data_ptr(), outs[0].data_ptr(), reps=8,
                                               stream=stream.cuda_stream)
        tuning = dict(tun.as_dict(), tuned_ms_per_run=tuned_ms, seconds=time.perf_counter() - t0)

    def barrier():
        if world > 1:
            dist.barrier()

    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            pkg.fllf_run(plan, frames[i % N_FRAMES].data_ptr(), outs[i % N_FRAMES].data_ptr(),
                         stream.cuda_stream)
    stream.synchronize()
    torch.cuda.synchronize()

    # Pre-pass with every stage kind timed: the per-stage breakdown and the
    # dominant kernel.  The timed region below records events only around the
    # dominant kernel's launches, so the events cost the other launches nothing.
    pre_steps = max(10, min(100, args.steps // 10))
    pkg.fllf_plan_enable_timing(plan, True)
    pkg.fllf_plan_stage_times(plan)                  # clear
    with torch.cuda.stream(stream):
        for i in range(pre_steps):
            pkg.fllf_run(plan, frames[i % N_FRAMES].data_ptr(), outs[i % N_FRAMES].data_ptr(),
                         stream.cuda_stream)
    stream.synchronize()
    pre = pkg.fllf_plan_stage_times(plan)
    dom = max(STAGES, key=lambda s: pre[s][0])
    pkg.fllf_plan_set_timing_mask(plan, [dom])
    pkg.fllf_plan_stage_times(plan)                  # clear
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for i in range(args.steps):
            pkg.fllf_run(plan, frames[i % N_FRAMES].data_ptr(), outs[i % N_FRAMES].data_ptr(),
                         stream.cuda_stream)
        e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    total_ms = e0.elapsed_time(e1)
    stage = pkg.fllf_plan_stage_times(plan)
    pkg.fllf_plan_enable_timing(plan, False)
    total_ms = max_over_ranks(total_ms, world, "cuda")
    ms_step = total_ms / args.steps
    pixels = cfg["H"] * cfg["W"]
    value = whole_job_mpixel_s(world, pixels, ms_step * 1e-3)

    # end to end through the C ABI with host buffers (copies inside the timed region)
    hin = torch.from_numpy(img).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    e2e_steps = max(20, min(50, args.steps // 20))
    for _ in range(5):
        pkg.fllf_run_host(plan, hin.data_ptr(), hout.data_ptr(), stream.cuda_stream)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        pkg.fllf_run_host(plan, hin.data_ptr(), hout.data_ptr(), stream.cuda_stream)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world, "cuda")
    tn = pkg.fllf_plan_get_tuning(plan)
    pkg.fllf_plan_destroy(plan)

    zbytes = 8 if args.precision == "fp32" else 4
    ops, byt = stage_work(cfg, zbytes, tn.chain_pixels, tn.small_pixels)
    dom_ms, dom_launches = stage[dom]                  # timed region, dominant kernel only
    per_launch_s = dom_ms / max(dom_launches, 1) * 1e-3
    launches_per_step = {s: pre[s][1] / pre_steps for s in STAGES}
    ops_launch = ops[dom] / max(launches_per_step[dom], 1)
    byt_launch = byt[dom] / max(launches_per_step[dom], 1)
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    mhz = (clk or {}).get("sm_mhz") or peaks.get("clocks_under_load", {}).get("sm_mhz_median") or 1900.0
    alu_peak = sms * 128 * mhz * 1e6 / 1e12           # FP32 lane-ops/s (FMA = 1), in T
    alu_ach = ops_launch / per_launch_s / 1e12
    hbm_ach = byt_launch / per_launch_s / 1e9
    alu_frac, hbm_frac = alu_ach / alu_peak, hbm_ach / hbm_peak
    if alu_frac >= hbm_frac:
        roof = {"bound": "alu", "achieved": alu_ach, "peak": alu_peak, "unit": "Top/s",
                "frac": alu_frac, "traffic": None, "kernel": dom,
                "peak_source": f"{sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz (median SM clock "
                               "sampled in this run)",
                "hbm_alt": {"achieved": hbm_ach, "peak": hbm_peak, "unit": "GB/s",
                            "frac": hbm_frac, "peak_source": hbm_src}}
    else:
        roof = {"bound": "hbm", "achieved": hbm_ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": hbm_frac, "traffic": None, "kernel": dom, "peak_source": hbm_src,
                "alu_alt": {"achieved": alu_ach, "peak": alu_peak, "unit": "Top/s",
                            "frac": alu_frac}}
    traffic_file = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        tr = json.load(open(traffic_file))
        key = f"{dom}:{args.precision}"
        if key in tr and tr[key].get("kernel_rev") == kernel_revision():
            roof["traffic"] = tr[key]["bytes_per_launch"]
    except (OSError, ValueError):
        pass
    hbm_min = hbm_min_bytes(cfg)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "uhd_rgb_3840x2160x3_L8_K8", "H": cfg["H"], "W": cfg["W"],
                   "C": cfg["C"], "levels": cfg["levels"], "K": cfg["K"], "m": cfg["m"],
                   "sigma_r": cfg["sigma_r"], "T": cfg["T"],
                   "pyramid_storage": args.precision,
                   "launch_tuning": tuning or "default (no autotune)",
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": f"inputs cycled over {N_FRAMES} frames ({N_FRAMES * 99.5:.0f} MB) plus "
                         "the plan scratch per step; working set > 129 MB L2"},
        "e2e": {"value": whole_job_mpixel_s(world, pixels, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": int(hin.numel() * 4), "d2h_bytes_per_step": int(hout.numel() * 4)},
        "gpu_launches": int(round(sum(launches_per_step.values()) * args.steps)),
        "roofline": roof,
        "hbm_min_roofline": {"bytes_per_step": hbm_min, "achieved": hbm_min / (ms_step * 1e-3) / 1e9,
                             "peak": hbm_peak, "unit": "GB/s",
                             "frac": hbm_min / (ms_step * 1e-3) / 1e9 / hbm_peak},
        "stages_ms_per_step": {s: pre[s][0] / pre_steps for s in STAGES},
        "stages_note": (f"per-stage times from a {pre_steps}-step pre-pass with every launch timed; "
                        f"the timed region records events around the {dom} launches only"),
        "clocks": clk,
    }
    if rank == 0 and not args.no_variants and world == 1:
        variants = {}
        for prec in ("fp32", "fp16", "bf16"):
            if prec == args.precision:
                continue
            ms = time_precision(pkg, torch, cfg, prec, frames, min(args.steps, 500), 10, stream, device)
            variants[prec] = {"ms_per_step": ms, "value": pixels / (ms * 1e-3) / 1e6}
        line["precision_variants"] = variants
        # fast LLF (Sec. II-D) at the same number of pyramids: S = 2K samples
        S = 2 * cfg["K"]
        fp = pkg.make_fast_params(cfg["H"], cfg["W"], cfg["C"], cfg["levels"], S, cfg["m"], cfg["sigma_r"],
                                  args.precision)
        ms = time_precision(pkg, torch, cfg, args.precision, frames, min(args.steps, 500), 10, stream,
                            device, params=fp)
        line["fast_llf"] = {"samples": S, "pyramids": S + 1, "ms_per_step": ms,
                            "value": pixels / (ms * 1e-3) / 1e6, "unit": UNIT,
                            "pyramid_storage": args.precision,
                            "note": "fast LLF (Sec. II-D) on the same frame, same levels, m and sigma_r, "
                                    "with 2K samples: the paper's comparison at an equal pyramid count "
                                    "(2K + 1)"}
    if rank == 0 and world == 1 and not args.no_serve:
        line["serving"] = serving_summary(pkg, torch, device, args.serve_precision,
                                          seconds=args.serve_seconds or 4.0)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_sample()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def kernel_revision():
    """Hash of the kernel sources and of the launch path, to tell whether
    stored ncu traffic still describes the kernels that run."""
    import hashlib
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2206_04681_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.startswith(("fllf_kernels", "fllf_device", "fllf_path")):
            h.update(open(os.path.join(csrc, name), "rb").read())
    return h.hexdigest()[:12]


def run_batch(args):
    """64 mixed-size images (own K, sigma_r, m, levels): one batched pass per
    step (one launch per stage kind, CUDA graph) against looping fllf_run."""
    import torch
    import paper_2206_04681_gb300 as pkg
    from paper_2206_04681_gb300 import build
    from paper_2206_04681_gb300.synth import batch_workload, synth_image
    build.build_library()
    torch.cuda.set_device(0)
    items = batch_workload(64, seed=4)
    plans, ins, outs = [], [], []
    for it in items:
        p = pkg.make_params(it["H"], it["W"], it["C"], it["levels"], it["K"], it["m"],
                            it["sigma_r"], it["T"], args.precision)
        plans.append(pkg.fllf_plan_create(p, 0))
        x = torch.from_numpy(synth_image(it["H"], it["W"], it["C"], it["polygons"], it["seed"])).cuda()
        ins.append(x)
        outs.append(torch.empty_like(x))
    pixels = sum(it["H"] * it["W"] for it in items)
    stream = torch.cuda.Stream()
    batch = pkg.fllf_batch_create(plans)
    pin = [x.data_ptr() for x in ins]
    pout = [y.data_ptr() for y in outs]

    def timed(step, steps, warmup):
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                step()
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                step()
            e1.record(stream)
            e1.synchronize()
        return e0.elapsed_time(e1) / steps

    steps = max(3, min(args.steps, 50))
    warm = max(3, min(args.warmup, 5))
    caps = None
    if not args.no_autotune:   # the batch's launch shapes (setup, outside the timed region)
        caps, _ = pkg.fllf_batch_autotune(batch, pin, pout, reps=3, stream=stream.cuda_stream)
        for pl, x, y in zip(plans, pin, pout):
            pkg.fllf_plan_autotune(pl, x, y, reps=3, stream=stream.cuda_stream)
    clocks = ClockSampler(0)
    clocks.start()
    ms_batch = timed(lambda: pkg.fllf_batch_run(batch, pin, pout, stream.cuda_stream), steps, warm)
    clk = clocks.stop()
    pkg.fllf_batch_check(batch)
    ms_loop = timed(lambda: [pkg.fllf_run(p, a, b, stream.cuda_stream)
                             for p, a, b in zip(plans, pin, pout)], steps, warm)
    pkg.fllf_batch_destroy(batch)
    for p in plans:
        pkg.fllf_plan_destroy(p)
    line = {"metric": "Mpixel/s Fourier LLF, 64 mixed-size images (batched)", "value": pixels / ms_batch / 1e3,
            "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": warm, "ms_per_step": ms_batch,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "batch64_mixed_sizes", "images": len(items), "pixels": pixels,
                       "sides": "log-uniform 256..4096, aspect 0.5..2", "K": "4 or 8",
                       "pyramid_storage": args.precision,
                       "batch_ctas_per_sm": caps or "default (no autotune)"},
            "looped_per_image": {"ms_per_step": ms_loop, "value": pixels / ms_loop / 1e3},
            "speedup_vs_loop": ms_loop / ms_batch, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0

SERVE = dict(rates=(50, 100, 200, 400, "max"), seconds=30.0, seed=5, budget=120 << 30,
             max_slots=64, max_queue=256, max_waves=3)


def serve_canvas(torch, device):
    """8192 x 8192 x 3 synthetic canvas on the device (a 4096^2 frame, 40
    polygons, mirrored 2 x 2); requests are cropped from it."""
    from paper_2206_04681_gb300.synth import synth_image
    img = torch.from_numpy(synth_image(4096, 4096, 3, 40, seed=SERVE["seed"])).to(device)
    top = torch.cat([img, img.flip(2)], 2)
    return torch.cat([top, top.flip(1)], 1).contiguous()


def serve_stream(pkg, torch, server, canvas, reqs, precision, keep, saturate=False):
    """Replays an arrival schedule in real time against the server.

    At each arrival the client crops its image from the canvas into a fresh
    device buffer and submits it; finished tickets are polled without
    blocking.  With `saturate`, every request is due at once and a full
    queue (FLLF_EBUSY) makes the client wait and retry instead of dropping
    the request.  Returns client-side latencies (scheduled arrival -> poll
    OK), the count of rejected submissions and the kept (input, output)
    pairs."""
    import numpy as np
    rng = np.random.default_rng(SERVE["seed"] + 1)
    copy_stream = torch.cuda.Stream()
    inflight, kept, lat, rejected = {}, {}, [], 0
    pkg.fllf_server_stats_reset(server)
    t0 = time.perf_counter()
    i = 0
    while i < len(reqs) or inflight:
        now = time.perf_counter() - t0
        while i < len(reqs) and (saturate or reqs[i]["t"] <= now):
            if saturate and len(inflight) >= 96:   # client window: bounds the buffers held
                break
            r = reqs[i]
            H, W, C = r["H"], r["W"], r["C"]
            y0 = int(rng.integers(0, canvas.shape[1] - H + 1))
            x0 = int(rng.integers(0, canvas.shape[2] - W + 1))
            with torch.cuda.stream(copy_stream):
                x = canvas[:C, y0:y0 + H, x0:x0 + W].contiguous()
                y = torch.empty_like(x)
            copy_stream.synchronize()
            p = pkg.make_params(H, W, C, r["levels"], r["K"], r["m"], r["sigma_r"], r["T"], precision)
            try:
                t = pkg.fllf_server_submit(server, p, x.data_ptr(), y.data_ptr())
                inflight[t] = (i, x, y)
            except pkg.FllfError as e:
                if e.status != pkg.FLLF_EBUSY:
                    raise
                if saturate:
                    break           # queue full: poll, then retry this request
                rejected += 1
            i += 1
        for t in list(inflight):
            if pkg.fllf_server_poll(server, t, 0) == pkg.FLLF_OK:
                idx, x, y = inflight.pop(t)
                lat.append((time.perf_counter() - t0 - (0.0 if saturate else reqs[idx]["t"])) * 1e3)
                if idx in keep:
                    kept[idx] = (x.cpu().numpy(), y.cpu().numpy())
        if saturate:
            nxt = 5e-5
        else:
            nxt = reqs[i]["t"] - (time.perf_counter() - t0) if i < len(reqs) else 1.0
        time.sleep(min(max(nxt, 0.0), 2e-4))
    return lat, rejected, kept


def serve_warmup(pkg, torch, server, canvas, precision):
    """Untimed requests first: module loading, first-touch of the pool and
    the caching allocator's blocks stay out of the measured latencies."""
    from paper_2206_04681_gb300.synth import request_stream
    serve_stream(pkg, torch, server, canvas, request_stream(200, 0.3, seed=SERVE["seed"] + 100),
                 precision, set(), saturate=True)


def serve_rate(pkg, torch, server, canvas, rate, seconds, precision, keep=()):
    """One Poisson stream at `rate` requests/s (rate "max": the same stream at
    400/s submitted as a backlog, to measure capacity); a JSON-ready summary,
    the request list and the (input, output) pairs of the requests in `keep`."""
    import numpy as np
    from paper_2206_04681_gb300.synth import request_stream
    saturate = rate == "max"
    reqs = request_stream(400 if saturate else rate, seconds, seed=SERVE["seed"])
    keep = set(keep)
    serve_warmup(pkg, torch, server, canvas, precision)
    lat, rejected, kept = serve_stream(pkg, torch, server, canvas, reqs, precision, keep, saturate)
    st = pkg.fllf_server_stats_get(server)
    offered = None if saturate else sum(r["H"] * r["W"] for r in reqs) / seconds / 1e6
    out = {"rate_per_s": rate, "seconds": seconds, "requests": len(reqs), "rejected": rejected,
           "completed": st["completed"], "mpixel_per_s": st["mpixel_per_s"],
           "offered_mpixel_per_s": offered,
           "latency_ms": {"p50": st["p50_ms"], "p99": st["p99_ms"], "mean": st["mean_ms"],
                          "max": st["max_ms"], "measured": "submit -> completion (server)"},
           "client_latency_ms": {"p50": float(np.percentile(lat, 50)) if lat else None,
                                 "p99": float(np.percentile(lat, 99)) if lat else None,
                                 "measured": "scheduled arrival -> poll OK (client)"},
           "waves": st["waves"], "max_active": st["max_active"],
           "pool_peak_gb": st["pool_peak_bytes"] / 1e9}
    return out, reqs, kept


def make_server(pkg, device):
    return pkg.fllf_server_create(SERVE["budget"], SERVE["max_slots"], SERVE["max_queue"],
                                  SERVE["max_waves"], device)


def serving_summary(pkg, torch, device, precision, rate=200, seconds=4.0):
    """A short served stream for the headline line."""
    server = make_server(pkg, device)
    try:
        canvas = serve_canvas(torch, device)
        out, _, _ = serve_rate(pkg, torch, server, canvas, rate, seconds, precision)
    finally:
        pkg.fllf_server_destroy(server)
    out["pyramid_storage"] = precision
    out["budget_gb"] = SERVE["budget"] / 2 ** 30
    return out


def run_serve(args):
    """Poisson streams of mixed requests (sides 512..8192, C 1 or 3, K 4/8/16,
    random remap) through the continuous-batching server, one per rate."""
    import torch
    import paper_2206_04681_gb300 as pkg
    from paper_2206_04681_gb300 import build
    build.build_library()
    torch.cuda.set_device(0)
    rates = ([r if r == "max" else float(r) for r in args.serve_rates.split(",")]
             if args.serve_rates else list(SERVE["rates"]))
    seconds = args.serve_seconds or SERVE["seconds"]
    server = make_server(pkg, 0)
    clocks = ClockSampler(0)
    try:
        canvas = serve_canvas(torch, 0)
        clocks.start()
        runs = [serve_rate(pkg, torch, server, canvas, r, seconds, args.serve_precision)[0] for r in rates]
        clk = clocks.stop()
    finally:
        pkg.fllf_server_destroy(server)
    best = max(runs, key=lambda r: r["mpixel_per_s"])   # the backlog run: capacity
    line = {"metric": "Mpixel/s and p50/p99 ms, served Fourier LLF requests (Poisson arrivals)",
            "value": best["mpixel_per_s"], "unit": UNIT, "n_gpus": 1, "steps": len(runs),
            "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "served_poisson_512_8192", "rates": list(rates),
                       "seconds_per_rate": seconds, "pyramid_storage": args.serve_precision,
                       "budget_gb": SERVE["budget"] / 2 ** 30, "max_slots": SERVE["max_slots"],
                       "max_waves": SERVE["max_waves"],
                       "value": "highest Mpixel/s over the runs (the backlog run measures capacity)",
                       "requests": "sides log-uniform 512..8192, aspect 0.5..2, C 1 or 3, "
                                   "K 4/8/16, sigma_r U[0.05,0.4], m U[0.5,4], T 2"},
            "runs": runs, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
