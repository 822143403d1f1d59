#!/usr/bin/env python
"""Benchmark of the dirty-imaging hot path: dirty images/s on the full-band streaming workload.

Workload (one step): one 50 ms chunk of the full-band observation - 144 tiles, 2 polarisations,
24 coarse x 128 fine channels at 10 kHz averaged by 4 into 768 channels of 40 kHz, 500 voltage samples
of 100 us integrated to 1 ms (K = 40) - imaged into 50 x 768 = 38,400 Stokes-I dirty images of 512^2.
The step is the whole path: correlation (FP8 tensor cores by default), gridding, 2D inverse FFT.

`value`: images/s with voltages resident in HBM.  `e2e`: the same metric through the host-buffer entry
point (pinned voltages in, images back to pinned host memory, both copies timed) on a 5 ms sub-chunk.
Inputs (442 MB of voltages) and outputs (40 GB of images) are far larger than L2, so no flush is needed.

Multi-GPU (torchrun): every rank images its own chunk (chunks are dealt round-robin from chunk 4), with
no collective on the data path; the timing is the max over ranks and `value` counts all ranks' images
(weak scaling).

`--impl reference` times the CPU oracle (the only other implementation of the method here) on a
bounded sample of the same workload, on the host cores.

`--workload` runs one of the other synthetic workloads instead (tiny, coarse, precision, uneven; the
default is the full-band one above); the uneven workload, four channel sets with their own flagged tiles
and image sides, goes through `blink_pipeline_sets`.  `--cpu-threads` sets the oracle's thread count.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "dirty images/s (512² px, 144 tiles) mixed-prec vs FP32 at ≤1e-4 rel RMS"
WORKLOAD = "fullband"
PROFILES = os.path.join(ROOT, "profiles")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--arith", choices=["fp8", "fp32"], default="fp8")
    ap.add_argument("--mode", choices=["batched", "plain"], default="batched")
    ap.add_argument("--precision", choices=["fp32", "bf16"], default="fp32", help="grid / FFT storage")
    ap.add_argument("--fused", action="store_true",
                    help="correlate inside the imaging launch (one persistent launch per step)")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the comparison forms (plain FP32, batched FP32, cuFFT, four-product correlation)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--samples", type=int, default=0, help="voltage samples per step (default: the 50 ms chunk)")
    ap.add_argument("--int-samples", type=int, default=0,
                    help="samples per integration (default: the workload's; e.g. 200 gives the paper's 20 ms "
                         "integrations, K = 800 on the full-band workload)")
    ap.add_argument("--workload", default=WORKLOAD, choices=["tiny", "coarse", "precision", "uneven", "fullband"])
    ap.add_argument("--n-pix", type=int, default=0,
                    help="image side for every channel set instead of the workload's (e.g. 1200, 8192)")
    ap.add_argument("--average", type=int, nargs=2, default=None, metavar=("T_AVG", "F_AVG"),
                    help="image means over T_AVG integrations and F_AVG channels (blink_pipeline_averaged); the "
                         "metric then counts the images averaged")
    ap.add_argument("--cpu-threads", type=int, default=0, help="oracle threads (default: every host core)")
    ap.add_argument("--dedisperse", action="store_true",
                    help="also time blink_dedisperse on the step's images (a DM sweeping half the chunk)")
    ap.add_argument("--jones", action="store_true",
                    help="apply seeded full 2x2 Jones matrices (30 %% leakage) in the correlation")
    ap.add_argument("--support", type=int, default=0,
                    help="gridding kernel width in cells: Kaiser-Bessel on a grid of twice the image side; 0 = nearest cell")
    ap.add_argument("--pointing", type=float, nargs=2, default=(0.0, 0.0), metavar=("L", "M"),
                    help="phase centre: direction cosines in the local East, North, Up frame (default zenith)")
    ap.add_argument("--gains", action="store_true",
                    help="apply seeded per-channel, per-tile, per-polarisation calibration gains in the correlation")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_id: str):
        self.dev = dev_id
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.dev, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
                pw.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(pw) if pw else None}


# ---------------------------------------------------------------------------------------------------
# roofline of the dominant kernel
# ---------------------------------------------------------------------------------------------------

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def measured_bf16():
    """Dense BF16 GEMM TFLOP/s measured on this machine's GPUs (burst), else the fallback figure."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            v = json.load(f).get("bf16_tflops")
        if v:
            return float(v), "measured"
    return 1900.0, "fallback"


def fast_side(n: int) -> bool:
    """Sides the side-specialised kernels cover (the others run the two mixed-radix passes)."""
    return 64 <= n <= 2048 and n & (n - 1) == 0


def stage_bytes(stage: int, n_tiles: int, n_pix: int, K: int) -> float:
    """Algorithmic bytes per image of each pipeline stage (what the step must move, not what it moves)."""
    B = n_tiles * (n_tiles + 1) // 2
    half = n_pix * (n_pix // 2)                       # complex entries of the u >= 0 half plane (no Nyquist)
    if stage == 0:                                    # voltages in, Stokes-I visibilities out
        return K * 2 * n_tiles + 8 * B
    if not fast_side(n_pix):                          # mixed-radix passes: the column results cannot stay on
        h = n_pix * (n_pix // 2 + 1)                  # chip, so each pass moves them once (to L2 or DRAM)
        return 8 * B + 8 * h if stage == 1 else 8 * h + 4 * n_pix * n_pix
    if stage == 1:                                    # visibilities in, images out (intermediate on chip / L2)
        return 8 * B + 4 * n_pix * n_pix
    if stage == 3:                                    # fused: the image's voltage share in, the image out
        return K * 2 * n_tiles + 4 * n_pix * n_pix
    return 8 * half + 4 * n_pix * n_pix               # half plane in, image out


STAGE_NAMES = ["correlate", "grid + 2D FFT", "row c2r FFT", "correlate + grid + 2D FFT (fused)"]
STAGE_KERNELS = ["k_corr_tc", "k_fft_persistent", "k_rowpass", "k_fft_persistent"]
STAGE_SOURCES = ["correlate_tc.cu", "fft_persistent.cu", "grid_fft.cu", "fft_persistent.cu"]
# on mixed-radix sides: the gather-gridding column pass and the complex-to-real row pass
MIXED_NAMES = ["correlate", "grid + column FFT (mixed radix)", "row c2r FFT (mixed radix)", None]
MIXED_KERNELS = ["k_corr_tc", "k_mixed_col", "k_mixed_row", None]
MIXED_SOURCES = ["correlate_tc.cu", "fft_mixed.cu", "fft_mixed.cu", None]


def source_hash(name: str) -> str:
    with open(os.path.join(ROOT, "paper_2505_15204_gb300", "csrc", name), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def traffic_for(kernel: str, source: str, shape=None, side=None):
    """DRAM bytes per launch of `kernel` (at the tuned launch shape, where traffic depends on it, and at the
    image side it was captured on, where recorded) from the committed ncu summary, if its source is
    unchanged."""
    p = os.path.join(PROFILES, "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel)
    if not e or e.get("source_sha256_16") != source_hash(source):
        return None
    if "side" in e and e["side"] != side:
        return None
    by_shape = e.get("dram_bytes_per_launch_fullsize_by_shape")
    if by_shape is not None:
        return by_shape.get(",".join(str(x) for x in shape)) if shape else None
    return e.get("dram_bytes_per_launch_fullsize")


# ---------------------------------------------------------------------------------------------------
# the reference arm: the CPU oracle on a bounded sample
# ---------------------------------------------------------------------------------------------------

def workload_of(args):
    """The workload, with the integration length of --int-samples, and the samples of one step (a whole number
    of integrations)."""
    import dataclasses
    import blinksynth as bs
    w = bs.WORKLOADS[args.workload]
    if args.int_samples:
        if args.int_samples < 1:
            raise SystemExit("--int-samples must be >= 1")
        w = dataclasses.replace(w, samples_per_int=args.int_samples)
    ns = args.samples or (w.samples_per_chunk // w.samples_per_int) * w.samples_per_int
    if ns < w.samples_per_int or ns % w.samples_per_int:
        raise SystemExit("the samples of a step must be a positive multiple of the samples per integration")
    return w, ns


def workload_label(name: str, w, n_pix=0) -> str:
    if name == "fullband":
        side = n_pix or 512
        T = w.samples_per_chunk // w.samples_per_int
        return ("fullband: 50 ms chunk, 144 tiles x 2 pol, 768 x 40 kHz (10 kHz averaged by 4), "
                f"{T} x {w.samples_per_int * 0.1:g} ms (K = {w.k}), {side}^2 Stokes-I images")
    return f"{name}: {w.description}" + (f"; imaged at {n_pix}^2" if n_pix else "")


def bench_config(args, w, ns, chunk, n_img, in_bytes, out_bytes):
    """The workload description both arms print (the reference arm times a sample of the same workload)."""
    L2_BYTES = 129 * 2 ** 20
    small = in_bytes + out_bytes < 2 * L2_BYTES
    return {"workload": workload_label(args.workload, w, args.n_pix), "n_pix": args.n_pix or None,
            "images_per_step": n_img, "samples_per_step": ns, "samples_per_int": w.samples_per_int, "K": w.k,
            "chunk": chunk, "arith": args.arith,
            "mode": args.mode, "precision": args.precision, "gains": bool(args.gains), "fused": bool(args.fused),
            "jones": bool(args.jones), "support": args.support, "pointing": list(args.pointing),
            "average": list(args.average) if args.average else None,
            "l2": (f"inputs {in_bytes / 1e6:.3g} MB and outputs {out_bytes / 1e6:.3g} MB per step fit L2: "
                   "each step timed alone after a 516 MB buffer overwrite") if small else
                  (f"inputs {in_bytes / 1e6:.3g} MB and outputs {out_bytes / 1e9:.3g} GB per step exceed L2; "
                   "no flush")}


def image_sets(inp, w, ns, n_pix=0):
    """(set, first image, images, side) of every channel set of the workload, images packed per set;
    n_pix > 0 images every set at that side instead of the workload's."""
    T = ns // w.samples_per_int
    out, first = [], 0
    for st in inp["sets"]:
        n = T * (st.n_fine // w.chan_avg)
        out.append((st, first, n, n_pix or st.n_pix))
        first += n
    return out


def bench_gains(n_out_chan: int, n_tiles: int) -> np.ndarray:
    """Seeded calibration gains, complex64 [channels][tiles][2]: amplitude 0.5-1.5, any phase."""
    rng = np.random.default_rng(2505152040)
    amp = rng.uniform(0.5, 1.5, size=(n_out_chan, n_tiles, 2))
    return (amp * np.exp(1j * rng.uniform(-np.pi, np.pi, size=amp.shape))).astype(np.complex64)


def bench_jones(n_out_chan: int, n_tiles: int) -> np.ndarray:
    """Seeded Jones matrices, complex64 [channels][tiles][2][2]: identity plus about 30 % random leakage."""
    rng = np.random.default_rng(2505152041)
    z = rng.normal(size=(n_out_chan, n_tiles, 2, 2)) + 1j * rng.normal(size=(n_out_chan, n_tiles, 2, 2))
    return (np.eye(2) + 0.3 * z).astype(np.complex64)


def oracle_sets_images(oracle, inp, w, sets, picks, threads, gains=None, support=0, pointing=(0.0, 0.0)):
    """The oracle's images for the picked (set index, local image id) pairs, in order."""
    out = []
    for q, (st, _, _, side) in enumerate(sets):
        ids = np.array([i for s_, i in picks if s_ == q], dtype=np.int64)
        if len(ids) == 0:
            continue
        kw = {} if len(sets) == 1 else {"flags": st.flags, "fine0": st.fine0, "n_fine": st.n_fine}
        if support:
            kw["support"] = support
        if tuple(pointing) != (0.0, 0.0):
            kw["phase_centre"] = tuple(pointing)
        if gains is not None:
            f0 = st.fine0 // w.chan_avg
            kw["gains"] = gains[f0:f0 + st.n_fine // w.chan_avg].astype(np.complex128)
        ref = oracle.pipeline(inp["volt"], inp["enu"], inp["freqs"], w.samples_per_int, w.chan_avg, side, ids=ids,
                              n_threads=threads, **kw)
        out.extend(ref["images"])
    return out


def pick_images(sets, n):
    """About n (set, local id) pairs spread evenly over every set's images."""
    total = sum(c for _, _, c, _ in sets)
    picks = []
    for q, (_, _, cnt, _) in enumerate(sets):
        k = max(1, round(n * cnt / total))
        picks += [(q, int(i)) for i in oracle_sample_ids(cnt, min(k, cnt))]
    return picks


def oracle_sample_ids(n_total: int, n: int) -> np.ndarray:
    return np.unique(np.linspace(0, n_total - 1, n).round().astype(np.int64))


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    import blinksynth as bs
    import oracle
    w, ns = workload_of(args)
    cores = args.cpu_threads or os.cpu_count() or 1
    chunk = min(4, w.n_chunks - 1)
    inp = bs.build_workload(args.workload, chunk=chunk, workers=min(16, os.cpu_count() or 1), n_samples=ns)
    sets = image_sets(inp, w, ns, args.n_pix)
    n_total = sum(c for _, _, c, _ in sets)
    img_floats = sum(c * side * side for _, _, c, side in sets)
    config = bench_config(args, w, ns, chunk, n_total, int(inp["volt"].size), img_floats * 4)
    n_per = max(2, cores)
    picks = pick_images(sets, n_per * (args.steps + args.warmup))
    times = []
    for s_ in range(args.warmup + args.steps):
        sel = picks[s_::args.warmup + args.steps][:n_per]
        if not sel:
            sel = picks[:1]
        t = time.perf_counter()
        cal = (bench_jones(w.n_out_chan, w.n_tiles) if args.jones else
               bench_gains(w.n_out_chan, w.n_tiles) if args.gains else None)
        oracle_sets_images(oracle, inp, w, sets, sel, cores, cal, args.support, args.pointing)
        dt = time.perf_counter() - t
        if s_ >= args.warmup:
            times.append((len(sel), dt))
    n = sum(a for a, _ in times)
    tt = sum(b for _, b in times)
    v = n / tt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "images/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tt / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64/f64", "data": "synthetic",
        "config": config,
        "cpu_baseline": {"value": v, "unit": "images/s", "cores": cores, "kind": "oracle",
                         "sample": f"{n_per} images per step, ids evenly spaced over the {n_total}-image chunk"},
        "e2e": {"value": v, "unit": "images/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------------------

def run_ours(args, world, rank, local):
    import blinksynth as bs
    w, ns = workload_of(args)
    cores = args.cpu_threads or os.cpu_count() or 1
    from paper_2505_15204_gb300.shard import chunks_for_rank, job_rate, max_over_ranks
    chunk = chunks_for_rank(w.n_chunks, rank, world, first=min(4, w.n_chunks - 1))[0]
    t_gen = time.perf_counter()
    host = os.cpu_count() or 1
    inp = bs.build_workload(args.workload, chunk=chunk, workers=max(1, min(16, host // max(1, world))), n_samples=ns)
    t_gen = time.perf_counter() - t_gen

    import torch
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    from paper_2505_15204_gb300 import blink as B

    n_tiles, K = w.n_tiles, w.k
    sets = image_sets(inp, w, ns, args.n_pix)
    multi = len(sets) > 1
    n_pix = sets[0][3]
    n_img = sum(c for _, _, c, _ in sets)
    img_floats = sum(c * side * side for _, _, c, side in sets)
    T_int = ns // w.samples_per_int
    avg = tuple(args.average) if args.average else None
    if avg:
        if multi or T_int % avg[0] or w.n_out_chan % avg[1]:
            raise SystemExit("--average: one channel set, T_AVG and F_AVG dividing the integrations and channels")
        n_out = (T_int // avg[0]) * (w.n_out_chan // avg[1])
        img_floats = n_out * n_pix * n_pix
    arith = B.BLINK_CORR_FP8 if args.arith == "fp8" else B.BLINK_CORR_FP32
    mode = B.BLINK_MODE_BATCHED if args.mode == "batched" else B.BLINK_MODE_PLAIN
    if multi and mode != B.BLINK_MODE_BATCHED:
        raise SystemExit("several channel sets run only in the batched mode")
    ctx = B.blink_create(local)
    if args.fused:
        B.blink_set_fused(ctx, True)
    prec = B.BLINK_PREC_BF16 if args.precision == "bf16" else B.BLINK_PREC_FP32
    gains = bench_gains(w.n_out_chan, n_tiles) if args.gains else None
    jones = bench_jones(w.n_out_chan, n_tiles) if args.jones else None
    arr = B.Array(inp["enu"], None, gains, jones)
    obs = B.Obs(inp["freqs"], w.chan_avg, w.samples_per_int, ns)
    pc = tuple(args.pointing)
    im = B.Imaging(n_pix, precision=prec, support=args.support, phase_centre=pc)
    bsets = [B.Set(fine0=st.fine0, n_fine=st.n_fine,
                   imaging=B.Imaging(side, precision=prec, support=args.support, phase_centre=pc),
                   flags=st.flags) for st, _, _, side in sets]
    stream = torch.cuda.current_stream()
    volt = torch.from_numpy(inp["volt"]).cuda()
    if multi:
        img = torch.empty(img_floats, dtype=torch.float32, device="cuda")
    elif avg:
        img = torch.empty((n_out, n_pix, n_pix), dtype=torch.float32, device="cuda")
    else:
        img = torch.empty((n_img, n_pix, n_pix), dtype=torch.float32, device="cuda")
    wts = torch.empty(n_img, dtype=torch.float32, device="cuda")

    def step(weights=None):
        if avg:
            B.blink_pipeline_averaged(ctx, arr, obs, im, arith, avg[0], avg[1], volt, img, stream)
        elif multi:
            B.blink_pipeline_sets(ctx, arr, obs, bsets, arith, volt, img, img_floats, stream)
        else:
            B.blink_pipeline(ctx, arr, obs, im, arith, mode, volt, img, weights, stream)

    t_plan = time.perf_counter()
    step(wts)
    B.blink_sync(ctx, stream)
    t_plan = time.perf_counter() - t_plan
    for _ in range(args.warmup):
        step()
    B.blink_sync(ctx, stream)

    props = torch.cuda.get_device_properties(local)
    dev_id = str(getattr(props, "uuid", local))
    if dev_id and not dev_id.startswith("GPU-") and len(dev_id) == 36:
        dev_id = "GPU-" + dev_id
    sampler = ClockSampler(dev_id)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    B.blink_read_profile(ctx, stream, reset=True)
    B.blink_set_profiling(ctx, True)
    sampler.start()
    time.sleep(0.3)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    L2_BYTES = 129 * 2 ** 20
    in_bytes, out_bytes = volt.numel(), img_floats * 4
    small = in_bytes + out_bytes < 2 * L2_BYTES
    if small:
        # the step's data fit L2: time each step alone and overwrite L2 with a larger buffer in between
        flush = torch.empty(4 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for a, b in ev:
            flush.fill_(1.0)
            a.record(stream)
            step()
            b.record(stream)
        torch.cuda.synchronize()
        ms_steps = sum(a.elapsed_time(b) for a, b in ev)
    e0.record(stream)
    if not small:
        for _ in range(args.steps):
            step()
    e1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = sampler.stop()
    B.blink_set_profiling(ctx, False)
    B.blink_sync(ctx, stream)
    stage_ms, stage_n = B.blink_read_profile(ctx, stream, reset=True)
    ms_total = ms_steps if small else e0.elapsed_time(e1)
    ms_step = max_over_ranks(ms_total / args.steps, pg, "cuda")
    value = job_rate(n_img, world, ms_step / 1e3)

    # roofline of the dominant stage (live CUDA-event times of its launches in the timed region)
    dom = int(np.argmax(stage_ms)) if mode == B.BLINK_MODE_BATCHED else 1
    peak, peak_kind = measured_peaks()
    roof = None
    def set_bytes(stage):
        if avg:                                   # per output: fa channels' sums in, one transform
            Bn = n_tiles * (n_tiles + 1) // 2
            h = n_pix * (n_pix // 2 + 1)
            if stage == 0:
                return (n_img // avg[0]) * (K * avg[0] * 2 * n_tiles + 8 * Bn)
            return n_out * ((avg[1] * 8 * Bn + 8 * h) if stage == 1 else (8 * h + 4 * n_pix * n_pix))
        return sum(stage_bytes(stage, n_tiles, side, K) * c for _, _, c, side in sets)

    if stage_n[dom]:
        bytes_total = set_bytes(dom) * args.steps
        per_launch = bytes_total / stage_n[dom]
        avg_s = stage_ms[dom] / 1e3 / stage_n[dom]
        ach = per_launch / avg_s / 1e9
        mixed = bool(avg) or not fast_side(sets[0][3] * (2 if args.support else 1))
        names, kerns, srcs = (MIXED_NAMES, MIXED_KERNELS, MIXED_SOURCES) if mixed else (STAGE_NAMES, STAGE_KERNELS,
                                                                                          STAGE_SOURCES)
        kern = kerns[dom] if (dom or arith == B.BLINK_CORR_FP8) else "k_corr_fp32"
        src = srcs[dom] if (dom or arith == B.BLINK_CORR_FP8) else "correlate.cu"
        # the committed DRAM counters are those of the nearest-cell, two-launch, unaveraged forms
        shape = B.blink_tuned_shape(ctx)
        traffic = (traffic_for(kern, src, shape, sets[0][3])
                   if not (args.support or args.fused or avg or args.gains or args.jones) else None)
        roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": traffic, "kernel": kern, "stage": names[dom],
                "bytes_per_launch": per_launch, "avg_launch_ms": avg_s * 1e3, "peak_kind": f"{peak_kind} hbm_gbs",
                "tuned_shape": {"ring": shape[0], "lag": shape[1], "ctas_per_sm": shape[2]}}
    # the correlation against both of its bounds: the FP8 tensor peak (the measured BF16 GEMM peak times the
    # nominal FP8 / BF16 ratio of 2) on the method's flops, 8 per complex product and polarisation, XX and YY
    # for Stokes I (16 B K per image, 8 B K for XX), and the HBM copy peak on its bytes
    corr_roof = None
    if stage_n[0] and arith == B.BLINK_CORR_FP8 and not avg:
        Bn = n_tiles * (n_tiles + 1) // 2
        flops = (16 if im.pol == B.BLINK_POL_I else 8) * Bn * K * n_img * args.steps
        t_s = stage_ms[0] / 1e3
        bf16, kind16 = measured_bf16()
        tf_peak = 2.0 * bf16
        tf = flops / t_s / 1e12
        gbs = set_bytes(0) * args.steps / t_s / 1e9
        t_tensor, t_hbm = flops / (tf_peak * 1e12), set_bytes(0) / (peak * 1e9)
        corr_roof = {"bound": "tensor" if t_tensor >= t_hbm else "hbm", "kernel": "k_corr_tc", "K": K,
                     "tensor": {"achieved": tf, "peak": tf_peak, "unit": "TFLOP/s", "frac": tf / tf_peak,
                                "peak_kind": f"{kind16} bf16_tflops x 2 (nominal fp8 / bf16 ratio)"},
                     "hbm": {"achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak},
                     "flops_per_image": flops / (n_img * args.steps), "bytes_per_image": set_bytes(0) / n_img}
    stages = {STAGE_NAMES[s]: {"ms_per_step": stage_ms[s] / args.steps, "launches_per_step": stage_n[s] / args.steps,
                               "GBps": (set_bytes(s) * args.steps / (stage_ms[s] / 1e3) / 1e9)
                               if stage_ms[s] else None}
              for s in range(B.BLINK_N_STAGES)}

    # full-size parity on sampled images, and the oracle's own throughput on them (rank 0, one GPU)
    parity = None
    cpu = None
    if rank == 0 and not args.no_cpu and not avg:
        import oracle
        n_s = max(4, 4 * cores)
        picks = pick_images(sets, n_s)
        t = time.perf_counter()
        refs = oracle_sets_images(oracle, inp, w, sets, picks, cores, jones if jones is not None else gains,
                                  args.support, args.pointing)
        dt = time.perf_counter() - t
        flat = img.reshape(-1)
        got = []
        for q, i in picks:
            _, first, _, side = sets[q]
            off = sum(c * sd * sd for _, _, c, sd in sets[:q]) + i * side * side
            got.append(flat[off:off + side * side].reshape(side, side).cpu().numpy())
        errs = [float(np.linalg.norm(g - r) / np.linalg.norm(r)) for g, r in zip(got, refs)]
        gate = 1e-4 if args.precision == "fp32" else None
        parity = {"images_checked": len(picks), "max_rel_rms": max(errs), "gate": gate,
                  "pass": (max(errs) <= 1e-4) if gate else None,
                  "max_abs": float(max(np.abs(g - r).max() for g, r in zip(got, refs)))}
        if world == 1:
            cpu = {"value": len(picks) / dt, "unit": "images/s", "cores": cores, "kind": "oracle",
                   "sample": f"{len(picks)} images, ids evenly spaced over the {n_img}-image chunk"}

    # incoherent dedispersion of the step's image cube: a dispersion measure whose sweep across the band
    # fills half the chunk, delays rounded to whole integrations
    dedisp = None
    if args.dedisperse and rank == 0 and not multi and not avg:
        T_int, F = ns // w.samples_per_int, n_img // (ns // w.samples_per_int)
        t_int = w.samples_per_int * 100e-6
        nu = inp["freqs"].reshape(F, w.chan_avg).mean(axis=1) / 1e6          # MHz
        per_dm = 4.148808e3 * (nu.min() ** -2 - nu.max() ** -2)               # s per pc cm^-3
        dm = (T_int // 2) * t_int / per_dm
        delays = np.rint(4.148808e3 * dm * (nu ** -2 - nu.max() ** -2) / t_int).astype(np.int32)
        n_out = T_int - int(delays.max())
        dd = torch.empty((n_out, n_pix, n_pix), dtype=torch.float32, device="cuda")
        for _ in range(2):
            B.blink_dedisperse(ctx, img, T_int, F, n_pix, delays, dd, stream)
        reps = 10
        e0.record(stream)
        for _ in range(reps):
            B.blink_dedisperse(ctx, img, T_int, F, n_pix, delays, dd, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_d = e0.elapsed_time(e1) / reps
        byts = n_out * (F + 1) * n_pix * n_pix * 4
        dedisp = {"dm_pc_cm3": round(float(dm), 4), "max_delay_integrations": int(delays.max()), "outputs": n_out,
                  "ms": ms_d, "GBps": byts / (ms_d / 1e3) / 1e9, "frac": byts / (ms_d / 1e3) / 1e9 / peak,
                  "bytes_per_launch": byts, "kernel": "k_dedisperse"}
        del dd

    # the forms the headline is compared with, on the same chunk (rank 0, single set, the default form only):
    # plain FP32 per-image path, batched FP32-correlation path, cuFFT's batched c2r transform of grids of the
    # same shape (the FFT stage alone), and the ABI correlation entry point's four-product visibilities
    comparison = None
    if rank == 0 and not multi and not avg and not args.no_compare and args.mode == "batched" and args.arith == "fp8":
        def timed(fn, reps, warm=1):
            for _ in range(warm):
                fn()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps
        ms_b32 = timed(lambda: B.blink_pipeline(ctx, arr, obs, im, B.BLINK_CORR_FP32, B.BLINK_MODE_BATCHED, volt, img,
                                                None, stream), 3)
        B.blink_set_fused(ctx, not args.fused)                    # the other of the two batched mixed forms
        ms_alt = timed(lambda: B.blink_pipeline(ctx, arr, obs, im, B.BLINK_CORR_FP8, B.BLINK_MODE_BATCHED, volt, img,
                                                None, stream), 3)
        B.blink_set_fused(ctx, args.fused)
        ns_p = min(ns, 2 * w.samples_per_int)                     # the per-image form on two integrations
        n_p = (ns_p // w.samples_per_int) * w.n_out_chan
        obs_p = B.Obs(inp["freqs"], w.chan_avg, w.samples_per_int, ns_p)
        ms_p32 = timed(lambda: B.blink_pipeline(ctx, arr, obs_p, im, B.BLINK_CORR_FP32, B.BLINK_MODE_PLAIN, volt,
                                                img, None, stream), 2)
        B.blink_sync(ctx, stream)
        nb = 768
        g = torch.randn((nb, n_pix, n_pix // 2 + 1), dtype=torch.complex64, device="cuda")
        ms_cf = timed(lambda: torch.fft.irfft2(g, s=(n_pix, n_pix)), 10, warm=3)
        del g
        Bn = n_tiles * (n_tiles + 1) // 2
        vis4 = torch.empty(n_img * Bn * 8, dtype=torch.float32, device="cuda")
        ms_v4 = timed(lambda: B.blink_correlate(ctx, arr, obs, B.BLINK_CORR_FP8, volt, vis4, stream), 3)
        del vis4
        B.blink_sync(ctx, stream)
        plain = n_p / (ms_p32 / 1e3)
        comparison = {
            "plain_fp32_per_image": {"images_per_s": plain, "images_per_step": n_p,
                                     "note": "correlate (CUDA cores) -> atomic grid -> column and row FFT, per image"},
            "batched_fp32": {"images_per_s": n_img / (ms_b32 / 1e3), "ms_per_step": ms_b32},
            "batched_mixed": {"images_per_s": value, "ms_per_step": ms_step,
                              "form": "fused single launch" if args.fused else "correlate launch + imaging launch"},
            ("batched_mixed_two_launches" if args.fused else "batched_mixed_fused"): {
                "images_per_s": n_img / (ms_alt / 1e3), "ms_per_step": ms_alt},
            "cufft_irfft2": {"images_per_s": nb / (ms_cf / 1e3), "batch": nb,
                             "note": "torch.fft.irfft2 (cuFFT) of random half-plane grids: the FFT stage alone"},
            "correlate_vis4": {"vis_per_s": n_img * Bn * 4 / (ms_v4 / 1e3), "ms_per_step": ms_v4,
                               "note": "blink_correlate, FP8 tensor cores: XX, XY, YX, YY of every baseline, V = S / K"},
            "multiple_vs_plain_fp32": value / plain,
        }

    # end to end through the host-buffer entry point (pinned voltages in, pinned images out)
    e2e = None
    if not args.no_e2e and not multi and not avg:
        ns_e = min(5 * w.samples_per_int, ns)
        n_e = (ns_e // w.samples_per_int) * w.n_out_chan
        obs_e = B.Obs(inp["freqs"], w.chan_avg, w.samples_per_int, ns_e)
        h_volt = torch.from_numpy(np.ascontiguousarray(inp["volt"][:ns_e])).pin_memory()
        h_img = torch.empty((n_e, n_pix, n_pix), dtype=torch.float32).pin_memory()
        B.blink_pipeline_host(ctx, arr, obs_e, im, arith, h_volt, h_img, 0, stream)
        B.blink_sync(ctx, stream)
        reps = max(3, min(args.steps, 10))
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            B.blink_pipeline_host(ctx, arr, obs_e, im, arith, h_volt, h_img, 0, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_e = max_over_ranks(e0.elapsed_time(e1) / reps, pg, "cuda")
        # the ingest alone (the paper's data-loading column): the step's voltages copied host -> device
        d_volt_e = torch.empty(h_volt.numel(), dtype=torch.uint8, device="cuda")
        d_volt_e.copy_(h_volt.view(-1), non_blocking=True)
        e0.record(stream)
        for _ in range(reps):
            d_volt_e.copy_(h_volt.view(-1), non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_h2d = e0.elapsed_time(e1) / reps
        del d_volt_e
        e2e = {"value": job_rate(n_e, world, ms_e / 1e3), "unit": "images/s", "h2d_bytes_per_step": int(h_volt.numel()),
               "d2h_bytes_per_step": int(h_img.numel() * 4), "images_per_step": n_e, "ms_per_step": ms_e,
               "h2d_ms": ms_h2d,
               "workload": f"{ns_e // w.samples_per_int} integrations x {w.n_out_chan} channels of the same chunk"}

    launches = int(sum(stage_n))
    line = {
        "metric": METRIC, "value": value, "unit": "images/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("e4m3->f32 correlation" if arith == B.BLINK_CORR_FP8 else "f32 correlation")
                 + (", bf16-stored f32 grid/FFT" if args.precision == "bf16" else ", f32 grid/FFT"),
        "data": "synthetic",
        "config": bench_config(args, w, ns, chunk, n_img, in_bytes, out_bytes),
        "setup_s": {"generate": round(t_gen, 2), "plan": round(t_plan, 3)},
        "roofline": roof, "corr_roofline": corr_roof, "stages": stages, "clocks": clocks, "gpu_launches": launches,
        "cpu_baseline": cpu, "parity": parity, "e2e": e2e, "comparison": comparison, "dedisperse": dedisp,
        "baselines_per_s": value * (n_tiles * (n_tiles + 1) // 2),
        "xx_yy_products_per_s": value * (n_tiles * (n_tiles + 1) // 2) * 2,
        "rates_note": ("per image the imaging path correlates every baseline incl. autos (baselines_per_s) and forms "
                       "its XX and YY products (xx_yy_products_per_s); the four-product visibilities of the "
                       "correlation entry point are comparison.correlate_vis4"),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    B.blink_destroy(ctx)
    if pg:
        pg.destroy_process_group()
    return 0


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
