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
E2E_DEPTH = 4         # frames in flight in the end-to-end stream (host buffers)
FRAMES_IN_FLIGHT = 3  # plans and streams filtering successive frames (N_FRAMES is a multiple)
N_FRAMES = 6          # distinct input/output frames cycled per step (6 x 99.5 MB > 129 MB L2)
STAGES = ("up0", "up", "down", "down0", "chain", "down_s", "graph")


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
                         "short served stream, and the timed frame's accuracy against the float64 "
                         "oracle); batch: 64 mixed images, batched vs looped; serve: Poisson "
                         "request streams.  The precision sweep and the served-request accuracy "
                         "are in tests/accuracy.py")
    ap.add_argument("--serve-seconds", type=float, default=None,
                    help="length of each served stream (default 30 s; 2.5 s per rate in the uhd line)")
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


def level_ops(cfg):
    """Algorithmic FP32 ops (FMA = 1) per level-l pixel of one plane, by part.

    The design-independent lower-bound count of the method (Eq. (14) with
    2K + 1 pyramids), split by the level it is spent on:
      trig0      level 0 only: one sincospi and 4 (K - 1) for the rotation
                 to the higher orders                                   4K + 16
      reduce     REDUCE l -> l+1 of the 2K + 1 images: symmetric 5-tap, 4 ops
                 per 1-D output, N/2 horizontal + N/4 vertical outputs  3 (2K + 1)
      combine    EXPAND of the 2K images (1.5 ops per 1-D output over
                 N/2 + N outputs), the Laplacian difference and the
                 product with the coefficient pair, per image  2K (2.25 + 1 + 1)
      gtrig      the coefficient pairs (cos, sin)(w_k g) at a level l >= 1
                                                                        4K + 16
      resid      the residual EXPAND and the per-pixel remainder         11.25
    Summed over the levels (x 4/3 for the per-level parts, x 1/3 for gtrig)
    this is 24.7 K + 40 per value: 237 at K = 8, the count 25 K + 35 of the
    method's op table up to its rounding."""
    K = cfg["K"]
    return {"trig0": 4 * K + 16, "reduce": 3 * (2 * K + 1), "combine": 2 * K * 4.25,
            "gtrig": 4 * K + 16, "resid": 11.25}


def stage_accounts(cfg, zbytes, chain_px=CHAIN_PIXELS, small_px=SMALL_PIXELS, dataflow=0):
    """Per stage kind, for one frame (all planes): algorithmic ops, the
    minimum HBM bytes of the stage's image and guide operands, and the bytes
    of the Fourier and residual pyramid operands it reads and writes.

    ops: ``level_ops`` per level, attributed to the stage that spends them
    (the level-0 trig and REDUCE to up0; REDUCE l -> l+1 to up / chain; the
    combine, its coefficient pairs and the residual EXPAND of level l to the
    stage that combines level l).
    hbm_min: the input read, the output write and each guide level G_l read
    or written by the stage, 4 B per value: the algorithmic bytes.
    pyramid: Z_l (zbytes per complex sample, K per pixel) and E_l (4 B)
    operand bytes, each element read once and written once: traffic the
    method's algorithm does not need (the path materialises the pyramids).
    Returns (ops, hbm_min, pyramid), dicts keyed by stage kind."""
    L, K, C = cfg["levels"], cfg["K"], cfg["C"]
    sz = level_sizes(cfg["H"], cfg["W"], L)
    n = [h * w for h, w in sz]
    lo = level_ops(cfg)
    up_levels, chain_up, chain_down, down_levels, small_levels, fused = stage_split(cfg, chain_px, small_px)
    ops = dict.fromkeys(STAGES, 0.0)
    hbm = dict.fromkeys(STAGES, 0.0)
    pyr = dict.fromkeys(STAGES, 0.0)

    def add(stage, o, h, p):
        ops[stage] += o
        hbm[stage] += h
        pyr[stage] += p

    def reduce_acc(l):   # l -> l+1, l >= 1
        g = 1 if l + 1 <= L - 2 else 0
        return (n[l] * lo["reduce"], 4 * n[l] * g + 4 * n[l + 1] * g,
                zbytes * K * (n[l] + n[l + 1]))

    def combine_acc(l):  # level l >= 1 on its own tiles: G_l read; Z_l, Z_{l+1}, E_{l+1} read, E_l written
        e = 1 if l + 1 <= L - 2 else 0
        return (n[l] * (lo["combine"] + lo["gtrig"] + lo["resid"]), 4 * n[l],
                zbytes * K * (n[l] + n[l + 1]) + 4 * n[l + 1] * e + 4 * n[l])

    if L >= 2:
        add("up0", n[0] * (lo["trig0"] + lo["reduce"]), 4 * n[0] + 4 * n[1] * (1 if L >= 3 else 0),
            zbytes * K * n[1])
    for l in up_levels:
        add("up", *reduce_acc(l))
    for l in chain_up:
        add("chain", *reduce_acc(l))
    for l in chain_down:
        add("chain", *combine_acc(l))
    for l in down_levels:
        add("down", *combine_acc(l))
    for l in small_levels:
        add("down_s", *combine_acc(l))
    if L >= 2:
        # level 0: I read, O written, Z_1 (and E_1 when levels >= 3, unless fused) read
        add("down0", n[0] * (lo["combine"] + lo["resid"]), 8 * n[0],
            zbytes * K * n[1] + (4 * n[1] if L >= 3 and not fused else 0))
        if fused:
            # level 1 inside the level-0 tiles: G_1 read, Z_2 and E_2 read (Z_1 shared)
            e2 = 1 if L >= 4 else 0
            add("down0", n[1] * (lo["combine"] + lo["gtrig"] + lo["resid"]), 4 * n[1],
                zbytes * K * n[2] + 4 * n[2] * e2)
    if dataflow:
        # one dataflow launch runs every stage (dataflow 1), or every stage but
        # the fused level-1/level-0 combine, which follows as its own kernel (2)
        keep = ("down0",) if dataflow == 2 and L >= 3 else ()
        for d in (ops, hbm, pyr):
            d["graph"] = sum(v for k, v in d.items() if k not in keep and k != "graph")
            for k in STAGES:
                if k != "graph" and k not in keep:
                    d[k] = 0.0
    f = lambda d: {k: v * C for k, v in d.items()}
    return f(ops), f(hbm), f(pyr)


def step_ops(cfg):
    """Algorithmic ops of one whole step (every level of every plane)."""
    ops, _, _ = stage_accounts(cfg, 8)
    return sum(ops.values())


# kernel launched by each stage kind (the level-0 stage is the fused
# level-1/level-0 combine when levels >= 3)
STAGE_KERNEL = {"up0": "k_up0", "up": "k_up", "down": "k_down", "down0": "k_down10",
                "chain": "k_chain", "down_s": "k_down_s", "graph": "k_graph"}


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


# ---- the float64 oracle on the host cores (cpu_baseline, accuracy, --impl reference) ----
def host_cores():
    """Cores this process may run on (the pool's worker count)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_warm(_):
    import oracle  # noqa: F401  (the import is the warm-up)
    time.sleep(0.2)
    return os.getpid()


def _oracle_job(job):
    """Worker: the float64 oracle, as it stands, on one plane (or a tile of
    one) of the frame in shared memory; with ``ref`` set, the result is
    written into the shared float64 reference frame."""
    import numpy as np
    from multiprocessing import shared_memory
    import oracle
    name, shape, c, y0, y1, x0, x1, levels, a, T, ref = job
    shm = shared_memory.SharedMemory(name=name)
    try:
        x = np.ndarray(shape, dtype=np.float32, buffer=shm.buf)[c, y0:y1, x0:x1].astype(np.float64)
    finally:
        shm.close()
    y = oracle.fourier_llf(x, levels, a, T)
    if ref is not None:
        rs = shared_memory.SharedMemory(name=ref)
        try:
            np.ndarray(shape, dtype=np.float64, buffer=rs.buf)[c, y0:y1, x0:x1] = y
        finally:
            rs.close()
    return 0


class OraclePool:
    """A spawned process pool over the host cores that runs the float64
    oracle on the planes of a frame held in shared memory."""

    def __init__(self, img, cores=None):
        import multiprocessing as mp
        from multiprocessing import shared_memory
        import numpy as np
        self.cores = cores or host_cores()
        self.shape = img.shape
        self.shm = shared_memory.SharedMemory(create=True, size=img.nbytes)
        np.ndarray(img.shape, dtype=np.float32, buffer=self.shm.buf)[:] = img
        self.ref = shared_memory.SharedMemory(create=True, size=img.size * 8)
        self.pool = mp.get_context("spawn").Pool(self.cores)
        self.pool.map(_oracle_warm, range(self.cores), chunksize=1)

    def jobs(self, specs, cfg, a):
        return [(self.shm.name, self.shape, c, y0, y1, x0, x1, cfg["levels"], a, cfg["T"],
                 self.ref.name if keep else None) for c, y0, y1, x0, x1, keep in specs]

    def run(self, specs, cfg, a):
        """Wall seconds of the oracle over the given (plane, tile, keep) specs."""
        jobs = self.jobs(specs, cfg, a)
        t0 = time.perf_counter()
        if len(jobs) == 1:
            self.pool.apply(_oracle_job, (jobs[0],))
        else:
            self.pool.map(_oracle_job, jobs, chunksize=1)
        return time.perf_counter() - t0

    def reference(self):
        import numpy as np
        return np.ndarray(self.shape, dtype=np.float64, buffer=self.ref.buf)

    def close(self):
        self.pool.close()
        self.pool.join()
        for s in (self.shm, self.ref):
            s.close()
            s.unlink()


def accuracy_of(out, ref):
    """max |GPU - oracle| and PSNR (peak 1, over every value) of a frame."""
    import numpy as np
    d = np.asarray(out, np.float64) - ref
    mse = float(np.mean(d * d))
    return {"max_abs": float(np.max(np.abs(d))),
            "psnr_db": None if mse == 0 else float(10 * np.log10(1.0 / mse))}


def cpu_baseline_and_accuracy(img, outs):
    """The float64 oracle on the host cores: the 4K RGB frame's planes, one
    per worker, on every core at once, and channel 0 alone on one core.
    Both are bounded samples of the workload (one plane per core).  The
    oracle's output for the three planes of the frame also gives the
    accuracy of each GPU output in ``outs`` ({name: (C, H, W) array})."""
    import oracle
    cfg = WORKLOAD
    a = oracle.coeffs_quadrature(cfg["m"], cfg["sigma_r"], cfg["T"], cfg["K"])
    H, W, C = cfg["H"], cfg["W"], cfg["C"]
    op = OraclePool(img)
    try:
        cores = op.cores
        one = op.run([(0, 0, H, 0, W, True)], cfg, a)
        specs = [(i % C, 0, H, 0, W, i < C) for i in range(max(cores, C))]
        t_all = op.run(specs, cfg, a)
        ref = op.reference().copy()
    finally:
        op.close()
    planes = len(specs)
    base = {"value": planes * H * W / C / t_all / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "nproc": os.cpu_count(),
            "sample": f"float64 numpy oracle, unchanged, in a spawned pool of {cores} processes on "
                      f"{cores} host cores: {planes} planes of the 3840x2160x3 frame at once, one "
                      f"per process ({t_all:.1f} s wall; Mpixel/s counts a pixel once over its "
                      f"{C} planes)",
            "one_core": {"value": H * W / C / one / 1e6, "unit": UNIT, "cores": 1,
                         "sample": f"channel 0 of the frame on one core ({one:.1f} s)"}}
    acc = {name: dict(accuracy_of(o, ref), vs="float64 oracle, all 3 planes of the frame")
           for name, o in outs.items()}
    return base, acc


def run_reference(args):
    """Reference arm: the float64 CPU oracle as it stands, on every host core.

    Each step filters one tile-plane per core at once (960 x 540 tiles of the
    3840 x 2160 x 3 frame, cycled over its 48 tile-planes; smaller tiles when
    the step count is large, so that the run stays within a few minutes)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_2206_04681_gb300.synth import synth_image
    cfg = WORKLOAD
    img = synth_image(cfg["H"], cfg["W"], cfg["C"], cfg["polygons"], cfg["seed"])
    a = oracle.coeffs_quadrature(cfg["m"], cfg["sigma_r"], cfg["T"], cfg["K"])
    n = args.steps + args.warmup
    div = 4 if n <= 150 else 8 if n <= 600 else 16
    th, tw = cfg["H"] // div, cfg["W"] // div
    tiles = [(c, ty * th, (ty + 1) * th, tx * tw, (tx + 1) * tw)
             for c in range(cfg["C"]) for ty in range(div) for tx in range(div)]
    op = OraclePool(img)
    k = 0

    def step():
        nonlocal k
        specs = [tiles[(k + j) % len(tiles)] + (False,) for j in range(op.cores)]
        k += op.cores
        return op.run(specs, cfg, a)

    try:
        for _ in range(args.warmup):
            step()
        dt = sum(step() for _ in range(args.steps)) / args.steps
    finally:
        op.close()
    value = op.cores * th * tw / cfg["C"] / dt / 1e6   # a pixel counts once over its 3 channels
    sample = (f"float64 numpy oracle, unchanged, in a spawned pool of {op.cores} processes on {op.cores} "
              f"host cores; each step filters {op.cores} tile-planes of {tw}x{th} of the frame at once")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "uhd_rgb_3840x2160x3_L8_K8", "H": cfg["H"], "W": cfg["W"],
                       "C": cfg["C"], "levels": cfg["levels"], "K": cfg["K"], "m": cfg["m"],
                       "sigma_r": cfg["sigma_r"], "T": cfg["T"],
                       "sample": f"{op.cores} tile-planes of {tw}x{th} per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": op.cores, "nproc": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
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
    """ms per frame of a plan (autotuned), back to back over the cycled
    frames, and the plan's output of the first frame (host array)."""
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
        with torch.cuda.stream(stream):
            pkg.fllf_run(plan, frames[0].data_ptr(), outs[0].data_ptr(), stream.cuda_stream)
        stream.synchronize()
        out0 = outs[0].cpu().numpy()
    finally:
        pkg.fllf_plan_destroy(plan)
    return ms, out0


def launch_modes(pkg, torch, cfg, frames, steps, stream, device, precision):
    """ms per frame of the same plan under each launch mode, all computing the
    same bits: the per-stage kernels (the default), the dataflow launch of
    every stage, the dataflow launch followed by the fused level-1/level-0
    combine, the per-stage kernels with one dataflow launch for the levels
    from 3 up, and the level-0 / level 1 -> 2 REDUCE in 4 row bands."""
    p = pkg.make_params(cfg["H"], cfg["W"], cfg["C"], cfg["levels"], cfg["K"], cfg["m"], cfg["sigma_r"],
                        cfg["T"], precision)
    plan = pkg.fllf_plan_create(p, device)
    outs = [torch.empty_like(f) for f in frames]
    res = {}
    try:
        for name, mode, level, bands in (("per_stage", 0, 0, 1), ("dataflow", 1, 0, 1),
                                          ("dataflow_then_fused_combine", 2, 0, 1),
                                          ("dataflow_levels_from_3", 3, 3, 1), ("reduce_bands_4", 0, 0, 4)):
            t = pkg.fllf_plan_get_tuning(plan)
            t.dataflow, t.dataflow_level, t.reduce_bands = mode, level, bands
            pkg.fllf_plan_set_tuning(plan, t)
            with torch.cuda.stream(stream):
                for i in range(10):
                    pkg.fllf_run(plan, frames[i % len(frames)].data_ptr(), outs[i % len(frames)].data_ptr(),
                                 stream.cuda_stream)
                stream.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for i in range(steps):
                    pkg.fllf_run(plan, frames[i % len(frames)].data_ptr(), outs[i % len(frames)].data_ptr(),
                                 stream.cuda_stream)
                e1.record(stream)
                e1.synchronize()
            res[name] = e0.elapsed_time(e1) / steps
    finally:
        pkg.fllf_plan_destroy(plan)
    res["note"] = "ms per frame, default task sizes and CTA caps, no autotune; every mode gives the same bits"
    return res


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
    total_ms = e0.elapsed_time(e1)
    stage = pkg.fllf_plan_stage_times(plan)
    pkg.fllf_plan_enable_timing(plan, False)
    total_ms = max_over_ranks(total_ms, world, "cuda")
    ms_single = total_ms / args.steps
    pixels = cfg["H"] * cfg["W"]
    tn = pkg.fllf_plan_get_tuning(plan)


    # the timed frames are copies of one frame: its output is every timed step's
    with torch.cuda.stream(stream):
        pkg.fllf_run(plan, frames[0].data_ptr(), outs[0].data_ptr(), stream.cuda_stream)
    stream.synchronize()
    out_acc = outs[0].cpu().numpy()

    # End to end through the C ABI with host buffers, every step's copies in
    # the timed region: a stream of frames through fllf_submit_host (the
    # plan's staging slots in turn, E2E_DEPTH frames in flight, each host
    # buffer reused only after its frame's ticket is done), then one frame at
    # a time through the synchronous fllf_run_host (the latency of a frame).
    hins = [torch.from_numpy(img).pin_memory() for _ in range(E2E_DEPTH)]
    houts = [torch.empty_like(hins[0]).pin_memory() for _ in range(E2E_DEPTH)]

    def e2e_stream(n):
        pending = []
        for i in range(n):
            if len(pending) == E2E_DEPTH:
                pkg.fllf_poll(pending.pop(0), -1)
            pending.append(pkg.fllf_submit_host(plan, hins[i % E2E_DEPTH].data_ptr(),
                                                houts[i % E2E_DEPTH].data_ptr(), stream.cuda_stream))
        for t in pending:
            pkg.fllf_poll(t, -1)

    e2e_steps = max(50, min(300, args.steps // 10))
    e2e_stream(2 * E2E_DEPTH + 1)
    barrier()
    t0 = time.perf_counter()
    e2e_stream(e2e_steps)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world, "cuda")
    e2e_same = all(bool(np.array_equal(h.numpy(), out_acc)) for h in houts)
    sync_steps = max(10, min(50, args.steps // 20))
    for _ in range(3):
        pkg.fllf_run_host(plan, hins[0].data_ptr(), houts[0].data_ptr(), stream.cuda_stream)
    barrier()
    t0 = time.perf_counter()
    for _ in range(sync_steps):
        pkg.fllf_run_host(plan, hins[0].data_ptr(), houts[0].data_ptr(), stream.cuda_stream)
    sync_s = max_over_ranks((time.perf_counter() - t0) / sync_steps, world, "cuda")

    # Frames in flight: FRAMES_IN_FLIGHT plans (each with its own scratch and
    # the same tuning) filter successive frames on as many streams, as a
    # pipeline over a stream of frames does, so that the latency-bound small
    # levels of one frame overlap the first stages of the next.  The line's
    # value is this throughput; the one-stream time above is reported beside
    # it, and the roofline of the dominant kernel comes from that region.
    fplans = [plan] + [pkg.fllf_plan_create(p, device) for _ in range(FRAMES_IN_FLIGHT - 1)]
    for q in fplans[1:]:
        pkg.fllf_plan_set_tuning(q, tn)
    fstreams = [stream] + [torch.cuda.Stream() for _ in fplans[1:]]

    def run_in_flight(n):
        for i in range(n):
            j = i % FRAMES_IN_FLIGHT
            pkg.fllf_run(fplans[j], frames[i % N_FRAMES].data_ptr(), outs[i % N_FRAMES].data_ptr(),
                         fstreams[j].cuda_stream)

    run_in_flight(max(args.warmup, 2 * FRAMES_IN_FLIGHT))
    torch.cuda.synchronize()
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for fs in fstreams[1:]:
        fs.wait_event(f0)
    run_in_flight(args.steps)
    for fs in fstreams[1:]:
        ev = torch.cuda.Event()
        ev.record(fs)
        stream.wait_event(ev)
    f1.record(stream)
    f1.synchronize()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms_step = max_over_ranks(f0.elapsed_time(f1), world, "cuda") / args.steps
    value = whole_job_mpixel_s(world, pixels, ms_step * 1e-3)
    for q in fplans[1:]:
        pkg.fllf_plan_destroy(q)
    pkg.fllf_plan_destroy(plan)

    zbytes = 8 if args.precision == "fp32" else 4
    ops, hbm_b, pyr_b = stage_accounts(cfg, zbytes, tn.chain_pixels, tn.small_pixels, tn.dataflow)
    dom_ms, dom_launches = stage[dom]                  # timed region, dominant kernel only
    per_launch_s = dom_ms / max(dom_launches, 1) * 1e-3
    launches_per_step = {s: pre[s][1] / pre_steps for s in STAGES}
    per = max(launches_per_step[dom], 1)
    ops_launch, hbm_launch, pyr_launch = ops[dom] / per, hbm_b[dom] / per, pyr_b[dom] / per
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "of measured" if "hbm_gbs" in peaks else "of fallback"
    mhz = (clk or {}).get("sm_mhz") or peaks.get("clocks_under_load", {}).get("sm_mhz_median") or 1900.0
    alu_peak = sms * 128 * mhz * 1e6 / 1e12           # FP32 lane-ops/s (FMA = 1), in T
    alu_ach = ops_launch / per_launch_s / 1e12
    roof = {"bound": "alu", "kernel": STAGE_KERNEL[dom], "achieved": alu_ach, "peak": alu_peak,
            "unit": "Top/s", "frac": alu_ach / alu_peak, "traffic": None,
            "ops_per_launch": ops_launch, "launch_us": per_launch_s * 1e6,
            "peak_source": f"{sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz, the median SM clock sampled "
                           "in this run (FMA = 1 op)",
            "ops_source": "the method's per-level op count (bench.level_ops; 24.7 K + 40 per value "
                          "summed over the levels)",
            "hbm_min": {"bytes_per_launch": hbm_launch, "achieved": hbm_launch / per_launch_s / 1e9,
                        "peak": hbm_peak, "unit": "GB/s",
                        "frac": hbm_launch / per_launch_s / 1e9 / hbm_peak, "peak_source": hbm_src,
                        "bytes": "input read, output write and the guide levels the kernel reads"},
            "pyramid_traffic": {"bytes_per_launch": pyr_launch,
                                "note": "operand bytes of the Fourier and residual pyramids the "
                                        "kernel reads and writes: materialised intermediates, not "
                                        "algorithmic bytes"}}
    traffic_file = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        tr = json.load(open(traffic_file))
        key = f"{dom}:{args.precision}"
        if key in tr and tr[key].get("kernel_rev") == kernel_revision():
            roof["traffic"] = tr[key]["bytes_per_launch"]
    except (OSError, ValueError):
        pass
    all_ops = sum(ops.values())
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
                   "frames_in_flight": FRAMES_IN_FLIGHT,
                   "l2": f"inputs cycled over {N_FRAMES} frames ({N_FRAMES * 99.5:.0f} MB) plus "
                         "the plan scratch per step; working set > 129 MB L2"},
        "e2e": {"value": whole_job_mpixel_s(world, pixels, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": int(hins[0].numel() * 4), "d2h_bytes_per_step": int(houts[0].numel() * 4),
                "ms_per_step": e2e_s * 1e3, "steps": e2e_steps,
                "api": f"fllf_submit_host + fllf_poll from pinned host buffers, {E2E_DEPTH} frames in flight "
                       "(host clock around the whole stream)",
                "outputs_equal_device_run": e2e_same,
                "one_frame_at_a_time": {"api": "fllf_run_host (synchronous; planes pipelined)",
                                        "ms_per_frame": sync_s * 1e3,
                                        "value": whole_job_mpixel_s(world, pixels, sync_s)}},
        "one_stream": {"ms_per_step": ms_single, "value": whole_job_mpixel_s(world, pixels, ms_single * 1e-3),
                       "note": "the same steps on one plan and one stream, one frame after another (the "
                               "region the dominant kernel's roofline is measured in)"},
        "gpu_launches": int(round(sum(launches_per_step.values()) * args.steps)),
        "roofline": roof,
        "alu_roofline_step": {"ops_per_step": all_ops, "achieved": all_ops / (ms_step * 1e-3) / 1e12,
                              "peak": alu_peak, "unit": "Top/s",
                              "frac": all_ops / (ms_step * 1e-3) / 1e12 / alu_peak},
        "hbm_min_roofline": {"bytes_per_step": hbm_min, "achieved": hbm_min / (ms_step * 1e-3) / 1e9,
                             "peak": hbm_peak, "unit": "GB/s",
                             "frac": hbm_min / (ms_step * 1e-3) / 1e9 / hbm_peak,
                             "peak_source": hbm_src},
        "stages_ms_per_step": {s: pre[s][0] / pre_steps for s in STAGES},
        "stages_note": (f"per-stage times from a {pre_steps}-step pre-pass with every launch timed; "
                        f"the timed region records events around the {dom} launches only"),
        "clocks": clk,
    }
    gpu_outs = {args.precision: out_acc}
    if rank == 0 and not args.no_variants and world == 1:
        variants = {}
        for prec in ("fp32", "fp16", "bf16"):
            if prec == args.precision:
                continue
            ms, o = time_precision(pkg, torch, cfg, prec, frames, min(args.steps, 500), 10, stream, device)
            variants[prec] = {"ms_per_step": ms, "value": pixels / (ms * 1e-3) / 1e6}
            gpu_outs[prec] = o
        line["precision_variants"] = variants
        line["launch_modes"] = launch_modes(pkg, torch, cfg, frames, min(args.steps, 300), stream, device,
                                            args.precision)
        # fast LLF (Sec. II-D) at the same number of pyramids: S = 2K samples
        S = 2 * cfg["K"]
        fp = pkg.make_fast_params(cfg["H"], cfg["W"], cfg["C"], cfg["levels"], S, cfg["m"], cfg["sigma_r"],
                                  args.precision)
        ms, _ = time_precision(pkg, torch, cfg, args.precision, frames, min(args.steps, 500), 10, stream,
                               device, params=fp)
        line["fast_llf"] = {"samples": S, "pyramids": S + 1, "ms_per_step": ms,
                            "value": pixels / (ms * 1e-3) / 1e6, "unit": UNIT,
                            "pyramid_storage": args.precision,
                            "note": "fast LLF (Sec. II-D) on the same frame, same levels, m and sigma_r, "
                                    "with 2K samples: the paper's comparison at an equal pyramid count "
                                    "(2K + 1)"}
    if rank == 0 and world == 1 and not args.no_serve:
        line["serving"] = serving_summary(pkg, torch, device, args.serve_precision,
                                          seconds=args.serve_seconds or 2.5)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"], acc = cpu_baseline_and_accuracy(img, gpu_outs)
        line["accuracy"] = acc[args.precision]
        for prec, v in line.get("precision_variants", {}).items():
            v["accuracy"] = acc[prec]
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
    # every launch mode of the batch, each timed with every CTA cap at "as many
    # as fit": 0 one launch per stage kind and level, 1 one dataflow launch,
    # 2 the dataflow launch and the batched fused level-1/level-0 combine
    modes = {}
    for mode in (0, 1, 2):
        pkg.fllf_batch_set_mode(batch, mode)
        modes[mode] = timed(lambda: pkg.fllf_batch_run(batch, pin, pout, stream.cuda_stream), steps, warm)
        pkg.fllf_batch_check(batch)
    pkg.fllf_batch_set_mode(batch, 0)
    caps = None
    if not args.no_autotune:   # the batch's launch shapes (setup, outside the timed region)
        caps, _ = pkg.fllf_batch_autotune(batch, pin, pout, reps=3, stream=stream.cuda_stream)
        for pl, x, y in zip(plans, pin, pout):
            pkg.fllf_plan_autotune(pl, x, y, reps=3, stream=stream.cuda_stream)
    mode, task_items = pkg.fllf_batch_get_mode(batch)
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
                       "batch_ctas_per_sm": caps or "default (no autotune)",
                       "batch_mode": mode, "task_items": task_items},
            "modes_ms_per_step": {"per_stage_levels": modes[0], "dataflow": modes[1],
                                  "dataflow_then_fused_combine": modes[2],
                                  "note": "each mode with every CTA cap at 'as many as fit', before "
                                          "the autotuner"},
            "looped_per_image": {"ms_per_step": ms_loop, "value": pixels / ms_loop / 1e3,
                                 "note": "fllf_run per image, each plan autotuned"},
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
           "pool_peak_gb": st["pool_peak_bytes"] / 1e9,
           "plan_cache": {"hits": st["plan_cache_hits"], "misses": st["plan_cache_misses"],
                          "admission_quadratures": st["admission_quadratures"]}}
    return out, reqs, kept


def make_server(pkg, device):
    return pkg.fllf_server_create(SERVE["budget"], SERVE["max_slots"], SERVE["max_queue"],
                                  SERVE["max_waves"], device)


def serving_summary(pkg, torch, device, precision, rates=(50, 200, 400), seconds=2.5):
    """Short served streams at a low, middle and high arrival rate for the
    headline line."""
    server = make_server(pkg, device)
    runs = []
    try:
        canvas = serve_canvas(torch, device)
        for rate in rates:
            out, _, _ = serve_rate(pkg, torch, server, canvas, rate, seconds, precision)
            runs.append(out)
    finally:
        pkg.fllf_server_destroy(server)
    return {"pyramid_storage": precision, "budget_gb": SERVE["budget"] / 2 ** 30, "runs": runs}


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
