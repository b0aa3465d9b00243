#!/usr/bin/env python
"""DARE benchmark: resliced Mpix/s and slice latency, 512^2 planes from a 256^3
directional volume, against the plain FP32 path.

One step = one pass of the whole hot path over one batch of synthetic input:
empty the volume, rebuild it from the 1600 tracked sweep frames (scatter +
finalize, Fig. 1), then reslice the 1000-pose trajectory (Eq. 1 / Eq. 2
weight tables + the tiled reslice, Fig. 2) into 512 x 512 FP32 images and
coverage masks.  Inputs are resident on the device when the timed region
starts; the volume (1.3 GB), frames (210 MB) and outputs (1 GB) are all
larger than L2, so no extra flush is needed.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs its own
independent workload (weak scaling: sessions do not exchange data).
"""
import argparse
import hashlib
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

METRIC = "resliced Mpix/s and p50/p99 slice latency (512² from 256³) vs plain FP32 path"
WORKLOAD = "dare_256cube_1600f_512px"
DTYPE_NAMES = {"u8": 0, "f16": 1, "bf16": 2, "f32": 3}
VALUE_BYTES = {"u8": 1, "f16": 2, "bf16": 2, "f32": 4}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["dare", "reference"], default="dare")
    ap.add_argument("--poses", type=int, default=1000)
    ap.add_argument("--dtype", choices=list(DTYPE_NAMES), default="f32")
    ap.add_argument("--slots", type=int, default=12)
    ap.add_argument("--path", choices=["tiled", "plain"], default="tiled")
    ap.add_argument("--radius", type=int, default=1, help="interpolation radius in voxels (default 1)")
    ap.add_argument("--kernel", choices=["tent", "box", "exp"], default="tent", help="distance kernel (default tent)")
    ap.add_argument("--probe", choices=["linear", "curvilinear"], default="linear",
                    help="probe of the frames and of the virtual planes (curvilinear: a fan from 40 mm above the face)")
    ap.add_argument("--workload", choices=["working", "batched", "serving"], default="working",
                    help="working: the 256^3 step (default); batched: 64 uneven volumes through a graph-replayed "
                         "plan; serving: 16 sessions under Poisson pose streams with live ingestion")
    ap.add_argument("--duration", type=float, default=10.0, help="seconds of the serving run")
    ap.add_argument("--coalesce-us", type=int, default=300,
                    help="serving: a batch that is not full waits until its oldest request is this old")
    ap.add_argument("--volumes", type=int, default=64, help="volumes of the batched workload")
    ap.add_argument("--quick", action="store_true", help="main timed loop only (for profiler runs)")
    ap.add_argument("--frames", type=int, default=0,
                    help="build from the first N frames only (profiler runs on a smaller build; 0 = all 1600)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--build-chunk", type=int, default=0,
                    help="append the frames in calls of this many frames (same volume, smaller build workspace; "
                         "for profiler runs that must stay small); 0 = one call")
    return ap.parse_args()


# ---------------------------------------------------------------- distributed plumbing

class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            backend = "nccl" if self._cuda() else "gloo"
            dist.init_process_group(backend)
            self.pg = dist

    @staticmethod
    def _cuda():
        import torch
        return torch.cuda.is_available()

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x):
        if not self.pg:
            return x
        import torch
        t = torch.tensor([float(x)], device=f"cuda:{self.local}" if self._cuda() else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", str(self.device)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=5)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------- helpers

def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


def kernel_source_hash():
    """Hash of what the tiled reslice kernel is built from: its source, the
    device helpers, and the parts of the internal header it uses (the job
    layout and the fixed-point / tile constants); other declarations in that
    header do not change the kernel."""
    csrc = os.path.join(ROOT, "paper_2605_26325_b300", "csrc")
    h = hashlib.sha256()
    for f in ("kernels_tiled.cu", "device_common.cuh"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    hdr = open(os.path.join(csrc, "dare_internal.h")).read()
    a = hdr.index("struct ResliceJob {")
    h.update(hdr[a:hdr.index("};", a) + 2].encode())
    for line in hdr.splitlines():
        if line.startswith("constexpr") and any(k in line for k in ("kFixBits", "kFixOne", "kTileW", "kTileH",
                                                                      "kTiledColMax", "kTiledSlotMax")):
            h.update(line.encode())
    return h.hexdigest()[:16]


def profiled_counters(kernel, n_slices):
    """Per-launch DRAM and L2 bytes from the committed ncu summary of the tiled
    kernel, scaled per slice to n_slices; None when the kernel's sources changed
    since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "reslice_tiled_dram_traffic.txt")
    try:
        kv = dict(line.split("=", 1) for line in open(path).read().split("\n") if "=" in line and not line.startswith("#"))
    except OSError:
        return None
    if kv.get("kernel", "").strip() != kernel or kv.get("src_sha256_16", "").strip() != kernel_source_hash():
        return None
    out = {}
    for key, name in (("dram_bytes_per_slice", "dram"), ("l2_bytes_per_slice", "l2")):
        try:
            out[name] = float(kv[key]) * n_slices
        except (KeyError, ValueError):
            out[name] = None
    return out


def build_source_hash():
    """Hash of what the reconstruction kernels are built from (their source and
    the internal header)."""
    csrc = os.path.join(ROOT, "paper_2605_26325_b300", "csrc")
    h = hashlib.sha256()
    for f in ("kernels_build.cu", "dare_internal.h"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def build_counters(n_frames):
    """Per-launch DRAM bytes of the count and full-write finalize kernels from the
    committed ncu summary of the full rebuild; None when the sources changed since
    the counters were taken or the rebuild is not the one captured."""
    path = os.path.join(ROOT, "profiles", "build_kernels_dram_traffic.txt")
    try:
        kv = dict(line.split("=", 1) for line in open(path).read().split("\n") if "=" in line and not line.startswith("#"))
        if kv.get("src_sha256_16", "").strip() != build_source_hash() or int(kv["frames"]) != n_frames:
            return None
        return {k: float(kv[f"{k}_dram_bytes"]) for k in ("scatter_count", "finalize")}
    except (OSError, KeyError, ValueError):
        return None


def host_cores():
    """Host threads this process may run on (its CPU affinity), as nproc reports."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def omp_threads(n):
    """Thread count of the oracle's OpenMP loops (libgomp's own setting)."""
    import ctypes
    try:
        ctypes.CDLL("libgomp.so.1").omp_set_num_threads(int(n))
    except OSError:
        pass


def workload_config(args, n_frames, P, W, H, world):
    """The working workload's config, identical in both arms."""
    return {"workload": WORKLOAD, "grid": "256^3 @ 0.4 mm", "frames": int(n_frames),
            "frame_px": "256x512 @ 0.2 mm", "poses": P, "out_px": f"{W}x{H} @ 0.2 mm",
            "storage": args.dtype, "slots": args.slots, "path": args.path, "weights": "f32",
            "distance_kernel": f"{args.kernel} R={args.radius}", "probe": args.probe,
            "step": "reset + rebuild volume from all frames + reslice every pose",
            "l2": "inputs larger than L2 (volume, frames and outputs each > 126 MB); no flush",
            "parallelism": f"replicas x{world}"}


def percentile(xs, q):
    return float(np.percentile(np.asarray(xs), q))


# ---------------------------------------------------------------- CPU oracle (baseline / reference arm)

def cpu_baseline(w, n_poses, slots, n_sub=16):
    """The FP64 oracle on the host: the tiny workload in full (200 frames of
    128 x 128 into 64^3, 16 planes of 128 x 128), and the working workload's
    full reconstruction plus a fixed subset of n_sub of its planes (every
    (n_poses / n_sub)-th), each reslice set single-threaded and on every core
    this process may use.  The reconstruction loop is sequential in the
    oracle.  value: the working step (rebuild + n_poses planes) at the
    measured all-core reslice rate."""
    import oracle
    import synth
    cores = host_cores()
    out = {"cores": cores, "kind": "oracle", "unit": "Mpix/s"}
    tiny = synth.tiny_workload(0)
    t = time.perf_counter()
    tv = oracle.build(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world, tiny.frames, tiny.frame_poses,
                      tiny.frame_px, oracle.F32, 8)
    tb = time.perf_counter() - t
    tiny_res = {}
    for threads in (1, cores):
        omp_threads(threads)
        t = time.perf_counter()
        for T in tiny.reslice_poses:
            oracle.reslice(tv, T, tiny.out_w, tiny.out_h, tiny.out_px)
        tiny_res[threads] = (time.perf_counter() - t) / len(tiny.reslice_poses)
    px_t = len(tiny.reslice_poses) * tiny.out_w * tiny.out_h
    out["tiny_full"] = {"build_s": tb, "ms_per_slice_1_thread": tiny_res[1] * 1e3,
                        "ms_per_slice_all_cores": tiny_res[cores] * 1e3,
                        "mpix_s_all_cores": px_t / (tb + len(tiny.reslice_poses) * tiny_res[cores]) / 1e6,
                        "mpix_s_1_thread": px_t / (tb + len(tiny.reslice_poses) * tiny_res[1]) / 1e6}
    del tv
    t = time.perf_counter()
    vol = oracle.build(w.grid.dims, w.grid.spacing, w.grid.vol_to_world, w.frames, w.frame_poses, w.frame_px,
                       oracle.F32, slots)
    t_build = time.perf_counter() - t
    sub = w.reslice_poses[::max(1, n_poses // n_sub)][:n_sub]
    res = {}
    for threads in (1, cores):
        omp_threads(threads)
        t = time.perf_counter()
        for T in sub:
            oracle.reslice(vol, T, w.out_w, w.out_h, w.out_px)
        res[threads] = (time.perf_counter() - t) / len(sub)
    omp_threads(cores)
    px = n_poses * w.out_w * w.out_h
    full = t_build + n_poses * res[cores]
    out["working"] = {"build_s_1_thread": t_build, "planes_timed": len(sub),
                      "ms_per_slice_1_thread": res[1] * 1e3, "ms_per_slice_all_cores": res[cores] * 1e3,
                      "mpix_s_reslice_only_all_cores": w.out_w * w.out_h / res[cores] / 1e6,
                      "mpix_s_reslice_only_1_thread": w.out_w * w.out_h / res[1] / 1e6}
    out["value"] = px / full / 1e6
    out["ms_per_step"] = full * 1e3
    out["sample"] = (f"FP64 oracle on the host ({cores} cores by CPU affinity): the tiny workload in full "
                     f"(build {tb:.2f} s, {len(tiny.reslice_poses)} planes of 128x128) and the working workload's full "
                     f"reconstruction of {len(w.frames)} frames (single-threaded, {t_build:.1f} s) + {len(sub)} of its "
                     f"{n_poses} 512x512 planes (every {max(1, n_poses // n_sub)}th; {res[cores] * 1e3:.0f} ms each on "
                     f"{cores} threads, {res[1] * 1e3:.0f} ms on 1); value = one working step at those rates")
    return out


def run_reference(args, dist):
    """The reference arm: the FP64 oracle as it stands, on the host cores.  Each
    step is 1/16 of the working step with the same frames-to-planes ratio: a
    fresh reconstruction of 100 consecutive frames (1600 / 16) and the reslice
    of 62 or 63 planes (1000 / 16) on the full volume, built once before timing.
    value = planes resliced x 512^2 / step time."""
    if dist.rank != 0:
        return
    import oracle
    import synth
    w = synth.working_workload(1, n_poses=args.poses)
    cores = host_cores()
    omp_threads(cores)
    log("reference: building the full oracle volume (untimed)")
    vol = oracle.build(w.grid.dims, w.grid.spacing, w.grid.vol_to_world, w.frames, w.frame_poses, w.frame_px,
                       oracle.F32, args.slots)
    parts = 16
    nf = len(w.frames) // parts

    def step(k):
        j = k % parts
        a = j * nf
        planes = range(j * args.poses // parts, (j + 1) * args.poses // parts)
        t = time.perf_counter()
        oracle.build(w.grid.dims, w.grid.spacing, w.grid.vol_to_world, w.frames[a:a + nf], w.frame_poses[a:a + nf],
                     w.frame_px, oracle.F32, args.slots)
        for i in planes:
            oracle.reslice(vol, w.reslice_poses[i], w.out_w, w.out_h, w.out_px)
        return time.perf_counter() - t, len(planes)

    for k in range(args.warmup):
        step(k)
    times, planes = [], 0
    for k in range(args.steps):
        dt, n = step(args.warmup + k)
        times.append(dt)
        planes += n
    total = sum(times)
    value = planes * w.out_w * w.out_h / total / 1e6
    sample = (f"each step: the FP64 oracle's fresh reconstruction of {nf} consecutive frames of the {len(w.frames)} "
              f"(single-threaded) + the reslice of {args.poses // parts} or {args.poses // parts + 1} of the "
              f"{args.poses} 512x512 planes (OpenMP over {cores} threads) on the full oracle volume built before "
              f"timing: 1/{parts} of a working step; successive steps take successive sixteenths")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, len(w.frames), args.poses, w.out_w, w.out_h, dist.world),
            "cpu_baseline": {"value": value, "unit": "Mpix/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "work_per_step": {"frames_built": nf, "planes_resliced": planes / args.steps,
                              "fraction_of_working_step": 1.0 / parts}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm

def run_dare(args, dist):
    import torch

    import paper_2605_26325_b300 as dare
    import synth

    dev = dist.local
    torch.cuda.set_device(dev)
    device = f"cuda:{dev}"
    seed = 1 + dist.rank
    t0 = time.perf_counter()
    w = synth.working_workload(seed, n_poses=args.poses)
    if args.frames > 0:
        w.frames, w.frame_poses = w.frames[:args.frames], w.frame_poses[:args.frames]
    log(f"rank {dist.rank}: workload ready in {time.perf_counter() - t0:.1f} s")
    P, W, H = args.poses, w.out_w, w.out_h
    dtype = DTYPE_NAMES[args.dtype]
    s = dare.Session(w.grid.dims, w.grid.spacing, w.grid.vol_to_world, dtype=dtype, max_slots=args.slots,
                     device=dev)  # the comparators' totals are kept by a session of their own (extras)
    curv_apex = (0.0, -40.0) if args.probe == "curvilinear" else None
    if curv_apex is not None:
        s.set_probe(dare.DARE_PROBE_CURVILINEAR, curv_apex)
    stream = torch.cuda.current_stream()
    frames_d = torch.from_numpy(w.frames).to(device)
    outs = torch.empty((P, H, W), dtype=torch.float32, device=device)
    masks = torch.empty((P, H, dare.mask_words(W)), dtype=torch.int32, device=device)
    reqs = dare.make_requests([(s, w.reslice_poses[i], outs[i], masks[i], w.out_px) for i in range(P)])
    path = dare.DARE_PATH_TILED if args.path == "tiled" else dare.DARE_PATH_PLAIN
    params = dare.params_default(path=path, radius_vox=args.radius, probe_apex_mm=curv_apex,
                                 dist_kernel={"tent": dare.DARE_TENT, "box": dare.DARE_BOX, "exp": dare.DARE_EXP}[args.kernel])

    chunk = args.build_chunk if args.build_chunk > 0 else len(w.frames)

    def step():
        s.reset(stream)
        for a in range(0, len(w.frames), chunk):
            s.build(frames_d[a:a + chunk], w.frame_poses[a:a + chunk], w.frame_px, stream)
        dare.reslice_batch(reqs, params, stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    info = s.info()
    if info.overflow_voxels:
        log(f"warning: {info.overflow_voxels} voxels hit the {args.slots}-slot capacity")
    dist.barrier()
    torch.cuda.synchronize()
    dare.trace_read()
    dare.trace_counters(reset=True)  # (reads a device counter: synchronises)
    clocks = ClockSampler(dev)
    clocks.start()
    # untimed steps while the sampler starts: a GPU left idle for that long comes
    # back to the timed region slower (about 0.05 ms a step on a B300); nothing
    # between them and the timed steps waits for the device
    t_warm, n_warm = time.perf_counter(), 0
    while time.perf_counter() - t_warm < 0.15:
        step()
        n_warm += 1
    dare.trace_enable(True)
    n0 = dare.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = dare.launch_count() - n0
    clk = clocks.stop()
    dare.trace_enable(False)
    trace = dare.trace_read()
    counters = dare.trace_counters(reset=True)
    dist.barrier()
    ms_total = dist.max(e0.elapsed_time(e1))
    ms_step = ms_total / args.steps
    px_step = P * W * H * dist.world
    value = px_step / (ms_step * 1e-3) / 1e6

    # roofline of the dominant kernel.  Algorithmic bytes per plane: every record of
    # its footprint read once (the record's data, 2 B id + value per slot; the
    # 16-byte stride's padding is layout, not the method's bytes), the image and
    # mask written, the weight table read.
    top = max(trace.items(), key=lambda kv: kv[1][1])
    per_launch_ms = {k: v[1] / max(v[0], 1) for k, v in trace.items()}
    fp = s.footprint(w.reslice_poses, W, H, w.out_px)
    rec_stride = info.record_bytes
    rec_data = args.slots * (2 + VALUE_BYTES[args.dtype])
    out_bytes = P * (W * H * 4 + H * dare.mask_words(W) * 4)
    reslice_alg = float(fp.sum() * rec_data + out_bytes + P * info.n_frames * 4)
    alg = {"reslice_tiled": reslice_alg, "reslice_plain": reslice_alg}
    if args.radius == 1 and args.kernel == "tent":  # the footprint counts the TENT R = 1 support
        alg["reslice_curv"] = reslice_alg
    peak, peak_kind = peaks()
    roof = None
    if top[0] in alg:
        t_launch = per_launch_ms[top[0]] * 1e-3
        achieved = alg[top[0]] / t_launch / 1e9
        prof = profiled_counters(top[0], P) or {}
        dram, l2b = prof.get("dram"), prof.get("l2")
        roof = {"kernel": top[0], "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": peak_kind, "traffic": dram,
                "algorithmic_bytes_per_launch": alg[top[0]], "launch_ms": per_launch_ms[top[0]],
                "footprint_voxels_per_slice": float(fp.mean()), "record_bytes": rec_data,
                "record_stride_bytes": rec_stride,
                "note": "achieved/frac: algorithmic bytes (each plane's footprint read once, cold) over the "
                        "launch time; dram_*: bytes DRAM actually moved (ncu, scaled per plane); l2: bytes "
                        "through L2 (ncu lts__t_bytes) against the measured L2 read bandwidth"}
        if dram:
            roof["dram_achieved"] = dram / t_launch / 1e9
            roof["dram_frac"] = roof["dram_achieved"] / peak
        l2_peak = None
        try:
            l2_peak = dare.measure_l2_bandwidth(dev, 32 << 20, 200)
        except dare.DareError as e:
            log(f"L2 bandwidth measurement failed: {e}")
        roof["l2"] = {"peak_gbs": l2_peak, "peak_kind": "measured: dare_measure_l2_bandwidth, 32 MiB x 200 passes",
                      "bytes_per_launch": l2b}
        if l2b and l2_peak:
            roof["l2"]["achieved_gbs"] = l2b / t_launch / 1e9
            roof["l2"]["frac"] = roof["l2"]["achieved_gbs"] / l2_peak
        t_hbm = alg[top[0]] / (peak * 1e9)
        t_l2 = l2b / (l2_peak * 1e9) if (l2b and l2_peak) else 0.0
        roof["roofline_ms"] = max(t_hbm, t_l2) * 1e3
        roof["binding_term"] = "l2" if t_l2 > t_hbm else "hbm"
        roof["roofline_frac"] = max(t_hbm, t_l2) / t_launch
    # the reconstruction as a whole (count + scan + place + finalize): its method's
    # bytes are the frames read and every voxel's record data and npix row written
    build_kernels = ("scatter_count", "exclusive_scan", "overflow_alloc", "scatter_place", "finalize",
                     "finalize_deferred")
    build_ms = sum(trace[k][1] for k in build_kernels if k in trace) / args.steps
    n_vox = int(np.prod(w.grid.dims))
    build_bytes = float(w.frames.size + n_vox * rec_data + n_vox * args.slots * 2)
    build_roof = {"ms_per_step": build_ms, "bytes": build_bytes,
                  "achieved": build_bytes / (build_ms * 1e-3) / 1e9 if build_ms > 0 else None, "peak": peak,
                  "unit": "GB/s", "kernels": list(build_kernels),
                  "note": "frames read + record data and npix of every voxel written (a reset volume is rewritten "
                          "whole); intermediate pair and entry lists are not the method's bytes"}
    if build_roof["achieved"]:
        build_roof["frac"] = build_roof["achieved"] / peak
    # DRAM bytes the two large build kernels move (ncu, one launch each), against
    # their CUDA-event launch times here
    bc = build_counters(len(w.frames))
    build_roof["traffic"] = None if bc is None else {
        k: {"dram_bytes": v, "launch_ms": trace[k][1] / max(trace[k][0], 1),
            "dram_gbs": v / (trace[k][1] / max(trace[k][0], 1) * 1e-3) / 1e9,
            "dram_frac": v / (trace[k][1] / max(trace[k][0], 1) * 1e-3) / 1e9 / peak}
        for k, v in bc.items() if k in trace}
    line = {"metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(args, len(w.frames), P, W, H, dist.world),
            "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"],
                       "samples": clk["samples"], "power_w_max": clk.get("power_w_max")},
            "gpu_launches": int(launches),
            "roofline": roof,
            "build_roofline": build_roof,
            "path_counters": dict(counters, steps=args.steps + n_warm,
                                  note="planes by path over the timed steps and the untimed steps run while "
                                       "the clock sampler starts"),
            "kernels_ms_per_step": {k: v[1] / args.steps for k, v in sorted(trace.items())}}

    if not args.quick:
        extras(args, dist, dare, torch, s, w, stream, frames_d, outs, masks, reqs, params, line, step, P, W, H)
        # the other configurations of the workload family: storage precision against
        # the FP64 oracle, the uneven batch through a graph-replayed plan, the serving loop
        line["precision"] = precision_leg(dare, torch, w, frames_d, outs, masks, stream, P, W, H, args.slots)
        bres, bclk = batched_leg(args, dist, 300, args.warmup)
        bres["clocks"] = {"sm_mhz": bclk["sm_mhz"], "sm_max_mhz": bclk["sm_max_mhz"], "reasons": bclk["reasons"]}
        line["batched"] = bres
        sres, sclk = serving_leg(args, dist, args.duration, args.coalesce_us)
        sres["clocks"] = {"sm_mhz": sclk["sm_mhz"], "sm_max_mhz": sclk["sm_max_mhz"], "reasons": sclk["reasons"]}
        line["serving"] = sres
        if dist.rank == 0 and dist.world == 1 and not args.no_cpu:
            del s
            torch.cuda.synchronize()
            cb = cpu_baseline(w, P, args.slots)
            line["cpu_baseline"] = cb
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


def workload_hash(w):
    """Digest of the working workload's grid, frames, frame poses and planes (the
    stored FP64 reference values of the precision sweep name the workload they
    were computed on by this digest)."""
    h = hashlib.sha256()
    h.update(np.asarray(w.grid.dims, np.int64).tobytes())
    h.update(np.float64(w.grid.spacing).tobytes())
    h.update(np.ascontiguousarray(w.grid.vol_to_world, np.float64).tobytes())
    h.update(np.ascontiguousarray(w.frames).tobytes())
    h.update(np.ascontiguousarray(w.frame_poses, np.float64).tobytes())
    h.update(np.asarray(w.frame_px, np.float64).tobytes())
    h.update(np.ascontiguousarray(w.reslice_poses, np.float64).tobytes())
    h.update(np.asarray([w.out_w, w.out_h], np.int64).tobytes())
    h.update(np.asarray(w.out_px, np.float64).tobytes())
    return h.hexdigest()[:32]


# storage half-ulp for values in [128, 256) plus FP32 accumulation of a convex combination of values
# <= 255 (a few ulp of 255); the FP16 weight table adds 2 eps / (1 - eps) (max I - min I), eps = 2^-11
PRECISION_BOUND = {"u8": 0.5 + 4e-5, "f16": 0.0625 + 4e-5, "bf16": 0.5 + 4e-5, "f32": 2.0 ** -17 + 4e-5}


def precision_leg(dare, torch, w, frames_d, outs, masks, stream, P, W, H, slots):
    """Storage precision on the working workload: every plane resliced from
    volumes stored as u8, f16, bf16 (FP16 weight tables) and f32 (FP32 weights),
    compared at 64 covered pixels of each plane with the FP64 oracle's values on
    the exact, unrounded means (tests/golden/precision_working.npz, written by
    tests/golden/make_precision_reference.py from the oracle alone)."""
    path = os.path.join(ROOT, "tests", "golden", "precision_working.npz")
    try:
        g = np.load(path)
    except OSError:
        return {"unavailable": "no stored reference values"}
    if str(g["workload"]) != workload_hash(w) or g["uv"].shape[0] != P:
        return {"unavailable": "the stored reference values were computed on another workload"}
    uv, ref, cnt = g["uv"].astype(np.int64), g["value"], g["count"]
    pidx = np.repeat(np.arange(P), uv.shape[1])
    keep = (np.arange(uv.shape[1])[None, :] < cnt[:, None]).reshape(-1)
    pi, u, v = pidx[keep], uv[:, :, 0].reshape(-1)[keep], uv[:, :, 1].reshape(-1)[keep]
    refv = ref.reshape(-1)[keep]
    ti = torch.from_numpy(pi).to(outs.device)
    tv = torch.from_numpy(v).to(outs.device)
    tu = torch.from_numpy(u).to(outs.device)
    eps = 2.0 ** -11
    res = {"planes": P, "pixels": int(keep.sum()), "pixels_per_plane": int(uv.shape[1]),
           "reference": "FP64 oracle on exact per-(voxel, frame) means (tests/golden/precision_working.npz)"}
    for name in ("u8", "f16", "bf16", "f32"):
        wd = dare.DARE_WEIGHTS_F32 if name == "f32" else dare.DARE_WEIGHTS_F16
        sp = dare.Session(w.grid.dims, w.grid.spacing, w.grid.vol_to_world, dtype=DTYPE_NAMES[name], max_slots=slots,
                          device=outs.device.index)
        sp.build(frames_d, w.frame_poses, w.frame_px, stream)
        rq = dare.make_requests([(sp, w.reslice_poses[i], outs[i], masks[i], w.out_px) for i in range(P)])
        dare.reslice_batch(rq, dare.params_default(weight_dtype=wd), stream)
        torch.cuda.synchronize()
        got = outs[ti, tv, tu].double().cpu().numpy()
        words = masks[ti, tv, tu // 32].cpu().numpy().view(np.uint32)
        covered = ((words >> (u % 32).astype(np.uint32)) & 1).astype(bool)
        e = np.abs(got - refv)
        bound = PRECISION_BOUND[name] + (0.0 if name == "f32" else 2 * eps / (1 - eps) * 255.0)
        res[name] = {"max_abs": float(e.max()), "psnr_db": float(10 * np.log10(255.0 ** 2 / max(np.mean(e ** 2), 1e-30))),
                     "mean_abs": float(e.mean()), "bound": bound, "within_bound": bool(e.max() <= bound),
                     "mask_agrees": bool(covered.all()), "weights": "f32" if name == "f32" else "f16",
                     "overflow_voxels": int(sp.info().overflow_voxels)}
        sp.close()
    return res


def _ssim_map(a, b):
    """SSIM (7 x 7 uniform windows, constants for 8-bit data) of two images."""
    from scipy.ndimage import uniform_filter
    c1, c2 = (0.01 * 255) ** 2, (0.03 * 255) ** 2
    ma, mb = uniform_filter(a, 7), uniform_filter(b, 7)
    va = uniform_filter(a * a, 7) - ma * ma
    vb = uniform_filter(b * b, 7) - mb * mb
    cab = uniform_filter(a * b, 7) - ma * mb
    return ((2 * ma * mb + c1) * (2 * cab + c2)) / ((ma * ma + mb * mb + c1) * (va + vb + c2))


def _ncc(a, b):
    a = a - a.mean()
    b = b - b.mean()
    return float((a * b).sum() / np.sqrt((a * a).sum() * (b * b).sum()))


def quality(dare, torch, s, w, stream, params, n=16, fill=(2, 1)):
    """Median NCC and SSIM of DARE, of the scalar comparator and of the scalar
    comparator after hole filling (radius, min_neighbours = fill) against the
    phantom rendered at n poses spread over the trajectory: over every pixel
    DARE and the unfilled comparator both cover, and over the specular pixels
    among them -- where the phantom's direction-dependent echo, rendered alone
    at the virtual pose (no speckle), is at least 10 of its 200 (dilated by
    one pixel) -- which is where orientation weighting can differ from mean
    compounding."""
    import dataclasses

    import synth
    from scipy.ndimage import binary_dilation, binary_erosion
    W, H = w.out_w, w.out_h
    poses = w.reslice_poses[np.linspace(0, len(w.reslice_poses) - 1, n).astype(int)]
    gt = synth.render_frames(w.phantom, poses, W, H, *w.out_px).astype(np.float64)
    spec = synth.render_frames(dataclasses.replace(w.phantom, sigma=0.0), poses, W, H, *w.out_px)
    out = torch.empty((H, W), dtype=torch.float32, device=stream.device)
    mask = torch.empty((H, dare.mask_words(W)), dtype=torch.int32, device=stream.device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.fill_holes(*fill, stream=stream)
    torch.cuda.synchronize()
    fill_ms = (time.perf_counter() - t0) * 1e3
    names = ("dare", "scalar", "scalar_filled")
    res = {k: {"ncc": [], "ssim": [], "ncc_spec": [], "ssim_spec": []} for k in names}
    cover, spec_share = [], []
    cov_each = {k: [] for k in names}
    for k, T in enumerate(poses):
        imgs = {}
        for name in names:
            if name == "dare":
                s.reslice(T, out, mask, w.out_px, params, stream=stream)
            elif name == "scalar":
                s.reslice_scalar(T, out, mask, w.out_px, stream=stream)
            else:
                s.reslice_scalar_filled(T, out, mask, w.out_px, stream=stream)
            torch.cuda.synchronize()
            imgs[name] = (out.cpu().numpy().astype(np.float64), dare.unpack_mask(mask.cpu().numpy(), W).astype(bool))
            cov_each[name].append(float(imgs[name][1].mean()))
        both = imgs["dare"][1] & imgs["scalar"][1]
        cover.append(float(both.mean()))
        if both.sum() < 1000:
            continue
        sp = binary_dilation(spec[k] >= 10, np.ones((3, 3), bool)) & both
        spec_share.append(float(sp.sum() / both.sum()))
        inner = binary_erosion(both, np.ones((7, 7), bool))
        for name, (img, _) in imgs.items():
            res[name]["ncc"].append(_ncc(img[both], gt[k][both]))
            smap = _ssim_map(np.where(both, img, 0.0), np.where(both, gt[k], 0.0)) if inner.any() else None
            if smap is not None:
                res[name]["ssim"].append(float(smap[inner].mean()))
            if sp.sum() >= 200:
                res[name]["ncc_spec"].append(_ncc(img[sp], gt[k][sp]))
                if smap is not None and (sp & inner).sum() >= 100:
                    res[name]["ssim_spec"].append(float(smap[sp & inner].mean()))
    med = lambda xs: float(np.median(xs)) if xs else None
    return {"ncc_median": {k: med(v["ncc"]) for k, v in res.items()},
            "ssim_median": {k: med(v["ssim"]) for k, v in res.items()},
            "specular": {"ncc_median": {k: med(v["ncc_spec"]) for k, v in res.items()},
                         "ssim_median": {k: med(v["ssim_spec"]) for k, v in res.items()},
                         "poses_scored": len(res["dare"]["ncc_spec"]),
                         "share_of_covered_pixels_median": med(spec_share)},
            "poses": n, "scored": len(res["dare"]["ncc"]), "coverage_median": med(cover),
            "coverage_each_median": {k: med(v) for k, v in cov_each.items()},
            "hole_fill": {"radius_vox": fill[0], "min_neighbours": fill[1], "ms": fill_ms},
            "note": "ground truth: the phantom rendered at each virtual probe pose (speckle + specular echoes "
                    "that depend on the beam direction); scalar = mean compounding with trilinear interpolation, "
                    "scalar_filled = the same after hole filling (the PLUS baseline's configuration); scored over "
                    "the pixels DARE and the unfilled comparator both cover, and over the specular ones among "
                    "them; the paper's medians on its own data: SSIM 0.465 vs 0.430, NCC 0.376 vs 0.215 (DARE "
                    "vs PLUS)"}


def extras(args, dist, dare, torch, s, w, stream, frames_d, outs, masks, reqs, params, line, step, P, W, H):
    """End-to-end arm, per-slice latency, the comparators (plain FP32 and scalar
    trilinear) and the L2-resident mode on a small volume."""
    import synth
    # --- end to end through the C ABI's host-buffer calls: frames uploaded from
    # page-locked host memory (overlapping the scatter), images and masks
    # downloaded to page-locked host memory (overlapping the next reslices)
    frames_h = torch.from_numpy(w.frames).pin_memory()
    outs_h = torch.empty(outs.shape, dtype=outs.dtype).pin_memory()
    masks_h = torch.empty(masks.shape, dtype=masks.dtype).pin_memory()
    reqs_h = dare.make_requests([(s, w.reslice_poses[i], outs_h[i], masks_h[i], w.out_px) for i in range(P)],
                                host=True)

    # consecutive steps alternate between two streams: the library orders the
    # session's kernels, so step k+1's reset and build run while step k's
    # downloads finish
    e2e_streams = [stream, torch.cuda.Stream(device=stream.device)]
    e2e_k = [0]

    def e2e_step():
        st = e2e_streams[e2e_k[0] & 1]
        e2e_k[0] += 1
        s.reset(st)
        s.build_host(frames_h, w.frame_poses, w.frame_px, st)
        dare.reslice_batch_host(reqs_h, params, st)

    n_e2e = max(2, min(args.steps, 10))
    e2e_step()
    torch.cuda.synchronize()
    dist.barrier()
    t = time.perf_counter()
    for _ in range(n_e2e):
        e2e_step()
    torch.cuda.synchronize()
    dt = dist.max((time.perf_counter() - t) / n_e2e)
    h2d = frames_h.numel() + w.frame_poses.nbytes + P * 16 * 8
    d2h = outs_h.numel() * 4 + masks_h.numel() * 4
    line["e2e"] = {"value": P * W * H * dist.world / dt / 1e6, "unit": "Mpix/s", "h2d_bytes_per_step": int(h2d),
                   "d2h_bytes_per_step": int(d2h), "ms_per_step": dt * 1e3,
                   "note": "dare_build_volume_host + dare_reslice_batch_host: H2D of the frames from pinned host "
                           "memory, poses from host arrays, D2H of every image and mask to pinned host memory, all "
                           "inside the timed region; steps queued back to back on two alternating streams"}

    # --- reslice-only throughput of each path (volume resident) and build-only time
    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def timed_on(fn, reps, st):
        fn()
        st.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(reps):
            fn()
        b.record(st)
        st.synchronize()
        return a.elapsed_time(b) / reps

    plain = dare.params_default(path=dare.DARE_PATH_PLAIN)
    tiled = dare.params_default(path=dare.DARE_PATH_TILED)
    ms_tiled = timed(lambda: dare.reslice_batch(reqs, tiled, stream), 5)
    ms_plain = timed(lambda: dare.reslice_batch(reqs, plain, stream), 3)

    def build_only():
        s.reset(stream)
        s.build(frames_d, w.frame_poses, w.frame_px, stream)

    ms_build = timed(build_only, 5)
    # the comparators' session: the same volume plus the mean-compounding totals
    # (kept apart so that the timed step rebuilds only what DARE reslices)
    sc = dare.Session(w.grid.dims, w.grid.spacing, w.grid.vol_to_world, dtype=DTYPE_NAMES[args.dtype],
                      max_slots=args.slots, device=dist.local, flags=dare.DARE_SESSION_SCALAR)
    sc.build(frames_d, w.frame_poses, w.frame_px, stream)
    ms_scalar = timed(lambda: [sc.reslice_scalar(w.reslice_poses[i], outs[i], masks[i], w.out_px, stream=stream)
                               for i in range(P)], 2)
    px = P * W * H
    line["paths_mpix_s"] = {"tiled_batched": px / ms_tiled / 1e3, "plain_fp32_batched": px / ms_plain / 1e3,
                            "scalar_trilinear": px / ms_scalar / 1e3}
    line["build_ms"] = ms_build

    # --- per-slice latency: query (host call) to image ready on the device, as the
    # caller sees it through the library's own wait on the session
    def lat(p, n=200):
        out1 = outs[0]
        m1 = masks[0]
        for i in range(5):  # untimed: a kernel's first use loads it
            s.reslice(w.reslice_poses[i % P], out1, m1, w.out_px, p, stream=stream)
            s.sync()
        xs = []
        for i in range(n):
            T = w.reslice_poses[i % P]
            torch.cuda.synchronize()
            t = time.perf_counter()
            s.reslice(T, out1, m1, w.out_px, p, stream=stream)
            s.sync()
            xs.append((time.perf_counter() - t) * 1e3)
        return {"p50_ms": percentile(xs, 50), "p99_ms": percentile(xs, 99), "samples": n}

    # L2-resident mode: a 128^3 f16 K=8 volume (67 MB of records) built from the same frames
    side = torch.cuda.Stream()
    l2 = {}
    for name, flags in (("default", 0), ("l2_persist", dare.DARE_SESSION_L2_PERSIST)):
        g = synth.centred_grid((128, 128, 128), 0.8)
        sm = dare.Session(g.dims, g.spacing, g.vol_to_world, dtype=dare.DARE_F16, max_slots=8, device=dist.local,
                          flags=flags)
        sm.build(frames_d, w.frame_poses, w.frame_px, stream)
        torch.cuda.synchronize()
        rq = dare.make_requests([(sm, w.reslice_poses[i], outs[i], masks[i], w.out_px) for i in range(P)])
        with torch.cuda.stream(side):
            l2[name] = timed_on(lambda: dare.reslice_batch(rq, tiled, side), 5, side)
        l2["volume_mb"] = sm.info().record_bytes * 128 ** 3 / 1e6
        sm.close()
    line["l2_mode"] = {"volume_mb": l2["volume_mb"], "default_ms": l2["default"], "l2_persist_ms": l2["l2_persist"],
                       "planes": P}

    # --- the same volume in mapped host memory (DARE_SESSION_HOST_VOLUME): reset +
    # rebuild and the 1000-plane reslice, every record access over the host link
    hv = dare.Session(w.grid.dims, w.grid.spacing, w.grid.vol_to_world, dtype=DTYPE_NAMES[args.dtype],
                      max_slots=args.slots, device=dist.local, flags=dare.DARE_SESSION_HOST_VOLUME)

    def hv_build():
        hv.reset(stream)
        hv.build(frames_d, w.frame_poses, w.frame_px, stream)

    hv_build_ms = timed(hv_build, 2)
    rq_hv = dare.make_requests([(hv, w.reslice_poses[i], outs[i], masks[i], w.out_px) for i in range(P)])
    hv_res_ms = timed(lambda: dare.reslice_batch(rq_hv, params, stream), 2)
    line["host_volume"] = {"host_bytes": int(hv.info().record_bytes) * int(np.prod(w.grid.dims)),
                           "device_bytes": int(hv.info().volume_bytes), "build_ms": hv_build_ms,
                           "reslice_ms_per_plane": hv_res_ms / P, "mpix_s": P * W * H / (hv_res_ms * 1e-3) / 1e6}
    # the same host volume with a device brick cache of a quarter of its bytes:
    # bricks of each plane's footprint paged in as the trajectory moves
    cache_bytes = int(hv.info().record_bytes) * int(np.prod(w.grid.dims)) // 4
    hv.set_cache(cache_bytes)
    n_pg = min(P, 500)
    rq_pg = (dare.dare_reslice_req * n_pg)(*rq_hv[:n_pg])
    pg_ms = timed(lambda: dare.reslice_batch(rq_pg, params, stream), 2)
    stats = hv.cache_stats()
    line["host_volume"]["paged"] = {"cache_bytes": cache_bytes, "planes": n_pg,
                                    "reslice_ms_per_plane": pg_ms / n_pg,
                                    "mpix_s": n_pg * W * H / (pg_ms * 1e-3) / 1e6, "cache": stats,
                                    "note": "dare_session_set_cache: 8^3-voxel bricks of the plane footprints paged "
                                            "into device memory, the per-pixel gather reading the cache; planes in "
                                            "groups of up to 64 whose bricks fit the cache, one launch per group"}
    hv.close()

    # --- the paper's timing axis (Sec. 3): interpolation radius.  BOX gives its
    # cubic neighbourhoods (3^3, 5^3, 9^3 voxels); TENT the 2R-wide support
    radius = {}
    for kname, kern in (("box", dare.DARE_BOX), ("tent", dare.DARE_TENT)):
        for R in (1, 2, 4):
            pr = dare.params_default(path=dare.DARE_PATH_TILED, radius_vox=R, dist_kernel=kern)
            n = P if R < 4 else min(P, 200)
            rq = (dare.dare_reslice_req * n)(*reqs[:n])
            ms = timed(lambda: dare.reslice_batch(rq, pr, stream), 3 if R < 4 else 2) / n
            side_n = 2 * R + 1 if kern == dare.DARE_BOX else 2 * R
            radius[f"{kname}_R{R}"] = {"neighbourhood": f"{side_n}^3", "ms_per_plane_batched": ms,
                                       "mpix_s": W * H / (ms * 1e-3) / 1e6, "latency": lat(pr, 50)}
    radius["note"] = ("tiled path, 512x512 planes from the resident 256^3 volume; the paper's laptop-GPU medians "
                      "(image and volume size not stated) are 50 / 100 / 300 ms for 3^3 / 5^3 / 9^3")
    line["radius_axis"] = radius

    # --- curvilinear probes: the same frames as a fan from an apex 40 mm above the
    # transducer face, resliced by a curvilinear virtual probe (per-sample Eq. 1 /
    # Eq. 2 kernel); and the linear volume under the curvilinear virtual probe
    apex = (0.0, -40.0)
    cs = dare.Session(w.grid.dims, w.grid.spacing, w.grid.vol_to_world, dtype=DTYPE_NAMES[args.dtype],
                      max_slots=args.slots, device=dist.local)
    cs.set_probe(dare.DARE_PROBE_CURVILINEAR, apex)

    def cs_build():
        cs.reset(stream)
        cs.build(frames_d, w.frame_poses, w.frame_px, stream)

    c_build_ms = timed(cs_build, 2)
    pc = dare.params_default(probe_apex_mm=apex)
    rq_c = dare.make_requests([(cs, w.reslice_poses[i], outs[i], masks[i], w.out_px) for i in range(P)])
    c_ms = timed(lambda: dare.reslice_batch(rq_c, pc, stream), 2)
    v_ms = timed(lambda: dare.reslice_batch(reqs, pc, stream), 2)
    c_lat = []
    for i in range(5):  # untimed: a kernel's first use loads it
        cs.reslice(w.reslice_poses[i % P], outs[0], masks[0], w.out_px, pc, stream=stream)
        cs.sync()
    for i in range(50):
        torch.cuda.synchronize()
        t = time.perf_counter()
        cs.reslice(w.reslice_poses[i % P], outs[0], masks[0], w.out_px, pc, stream=stream)
        cs.sync()
        c_lat.append((time.perf_counter() - t) * 1e3)
    line["curvilinear"] = {"apex_mm": list(apex), "build_ms": c_build_ms, "reslice_ms": c_ms,
                           "mpix_s": P * W * H / (c_ms * 1e-3) / 1e6,
                           "virtual_probe_only_mpix_s": P * W * H / (v_ms * 1e-3) / 1e6,
                           "latency": {"p50_ms": percentile(c_lat, 50), "p99_ms": percentile(c_lat, 99),
                                       "samples": len(c_lat)},
                           "note": "curvilinear frames and virtual probe; the second figure is the linear "
                                   "volume under the curvilinear virtual probe; both gather per pixel"}
    cs.close()

    # --- image quality on synthetic ground truth (the paper's Sec. 3 comparison,
    # NCC / SSIM against the acquired image, on rendered data): the phantom
    # rendered at the virtual probe's pose vs DARE and the mean-compounding
    # (orientation-blind, trilinear) comparator, over the pixels both cover
    line["quality"] = quality(dare, torch, sc, w, stream, tiled)
    sc.close()

    line["latency"] = {"tiled": lat(tiled), "plain_fp32": lat(plain),
                       "note": "wall time from the host call to the 512x512 image and mask on the device, "
                               "one plane per call, waited for with dare_session_sync"}


def batched_leg(args, dist, steps, warmup):
    """Uneven batch (64 volumes of dims U(96..384, 96..384, 96..256), 8-32
    planes each of 128^2 .. 640^2): every plane through one autotuned plan
    replayed as a CUDA graph (volumes built untimed).  Returns the measurements
    and the clock record."""
    import torch

    import paper_2605_26325_b300 as dare
    import synth

    dev = dist.local
    torch.cuda.set_device(dev)
    device = f"cuda:{dev}"
    t0 = time.perf_counter()
    vols = synth.batched_workload(3 + dist.rank, n_volumes=args.volumes)
    log(f"rank {dist.rank}: batched workload ready in {time.perf_counter() - t0:.1f} s")
    stream = torch.cuda.current_stream()
    sessions, items = [], []
    overflow = 0
    for v in vols:
        s = dare.Session(v.grid.dims, v.grid.spacing, v.grid.vol_to_world, dtype=dare.DARE_F16, max_slots=8,
                         device=dev)
        fr = torch.from_numpy(v.frames).to(device)
        s.build(fr, v.frame_poses, v.frame_px, stream)
        torch.cuda.synchronize()
        del fr
        overflow += s.info().overflow_voxels
        sessions.append(s)
        for T, (W, H) in zip(v.plane_poses, v.plane_sizes):
            out = torch.empty((H, W), dtype=torch.float32, device=device)
            mask = torch.empty((H, dare.mask_words(W)), dtype=torch.int32, device=device)
            items.append((s, T, out, mask, v.plane_px))
    px = sum(o.numel() for _, _, o, _, _ in items)
    reqs = dare.make_requests(items)
    t = time.perf_counter()
    plan = dare.Plan(reqs, dare.params_default(path=dare.DARE_PATH_AUTO), stream)
    tune_s = time.perf_counter() - t

    def timed(fn, reps):
        for _ in range(max(warmup, 3)):
            fn()
        torch.cuda.synchronize()
        dist.barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return dist.max(a.elapsed_time(b) / reps)

    clocks = ClockSampler(dev)
    clocks.start()
    n0 = dare.launch_count()
    ms_plan = timed(lambda: plan.launch(stream), steps)
    launches = (dare.launch_count() - n0) // (steps + max(warmup, 3))
    clk = clocks.stop()
    dare.trace_counters(reset=True)
    ms_batch = timed(lambda: dare.reslice_batch(reqs, dare.params_default(), stream), 20)
    counters = dare.trace_counters(reset=True)
    ms_plain = timed(lambda: dare.reslice_batch(reqs, dare.params_default(path=dare.DARE_PATH_PLAIN), stream), 5)
    info = plan.info()
    pitch = [max(v.plane_px) / v.grid.spacing for v in vols]
    res = {"mpix_s": px * dist.world / ms_plan / 1e3, "ms_per_replay": ms_plan, "replays": steps,
           "volumes": len(vols), "planes": len(items), "out_mpix": px / 1e6, "overflow_voxels": int(overflow),
           "pixel_pitch_vox": [min(pitch), max(pitch)],
           "plan": {"groups": info["n_groups"], "choice": info["choice"],
                    "tune_ms": {"plain": info["tune_ms"][0][0], "tiled_rows_le_64": info["tune_ms"][0][1],
                                "tiled_rows_le_32": info["tune_ms"][0][2], "tiled_rows_le_16": info["tune_ms"][0][3]},
                    "tune_s": tune_s, "kernel": "persistent tiled (work queue over every plane's tiles)"
                    if info["choice"] and info["choice"][0] else "plain"},
           "gpu_launches_per_replay": int(launches),
           "paths_mpix_s": {"plan_graph": px / ms_plan / 1e3, "batch_call_tiled": px / ms_batch / 1e3,
                            "batch_call_plain": px / ms_plain / 1e3},
           "batch_call_path_counters": {k: v // (max(warmup, 3) + 20) for k, v in counters.items()}}
    plan.close()
    for s in sessions:
        s.close()
    return res, clk


def run_batched(args, dist):
    reps = max(args.steps, 300)  # about a second of replays, long enough for the clock sampler
    res, clk = batched_leg(args, dist, reps, args.warmup)
    line = {"metric": "resliced Mpix/s, uneven batch of 64 volumes through one graph-replayed plan",
            "value": res["mpix_s"], "unit": "Mpix/s", "n_gpus": dist.world, "steps": reps,
            "warmup": args.warmup, "ms_per_step": res["ms_per_replay"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"dare_batch_{res['volumes']}vol_uneven", "volumes": res["volumes"],
                       "planes": res["planes"], "out_mpix": res["out_mpix"], "storage": "f16", "slots": 8,
                       "dims": "U(96..384, 96..384, 96..256) @ 0.4 mm", "sizes": "{128,256,512,640}^2",
                       "overflow_voxels": res["overflow_voxels"]},
            "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]},
            "gpu_launches": res["gpu_launches_per_replay"], "plan": res["plan"], "paths_mpix_s": res["paths_mpix_s"],
            "batch_call_path_counters": res["batch_call_path_counters"]}
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


def serving_leg(args, dist, duration, coalesce_us):
    """16 sessions (dims 128^3 .. 512x512x384, u8/f16) admitted under a 120 GB
    device-memory budget; each session's poses arrive as a Poisson stream at
    60-1000 Hz with a fixed output size in 256^2 .. 640^2; two sessions ingest
    new sweep frames live (30 frames/s in batches of 3).  Returns throughput,
    submit-to-done latency percentiles, batching figures and the clocks."""
    import torch

    import paper_2605_26325_b300 as dare
    import synth

    dev = dist.local
    torch.cuda.set_device(dev)
    device = f"cuda:{dev}"
    rng = np.random.default_rng(np.random.SeedSequence([11, dist.rank]))
    dare.set_memory_budget(120 * 10**9)
    t0 = time.perf_counter()
    sessions, meta, rejected = [], [], 0
    for k in range(16):
        dims = (int(rng.integers(128, 513)), int(rng.integers(128, 513)), int(rng.integers(128, 385)))
        grid = synth.centred_grid(dims, 0.4)
        ext = grid.extent
        W, H = int(np.ceil(ext[0] / 0.4)), int(np.ceil(ext[2] * 1.1 / 0.4))
        tilts = [float(rng.uniform(-40, 40)) for _ in range(int(rng.integers(2, 5)))]
        nf = int(ext[1] / 0.8)
        vseed = int(rng.integers(0, 2**31 - 1))
        ph = synth.make_phantom(vseed, float(min(ext)), 6, 1)
        poses = np.concatenate([synth.sweep_poses(vseed, i, nf, H, 0.4, t, float(ext[1])) for i, t in enumerate(tilts)])
        dtype = dare.DARE_U8 if k % 2 == 0 else dare.DARE_F16
        try:
            s = dare.Session(dims, 0.4, grid.vol_to_world, dtype=dtype, max_slots=8, device=dev)
        except dare.DareError as e:
            if e.status != dare.DARE_E_ADMISSION:
                raise
            rejected += 1
            continue
        frames = torch.from_numpy(synth.render_frames(ph, poses, W, H, 0.4, 0.4)).to(device)
        s.build(frames, poses, (0.4, 0.4))
        torch.cuda.synchronize()
        del frames
        live = None
        if len(meta) < 2:  # the first two admitted sessions get a live sweep
            lp = synth.sweep_poses(vseed, 99, int(30 * duration) + 6, H, 0.4, float(rng.uniform(-40, 40)),
                                   float(ext[1]))
            live = (torch.from_numpy(synth.render_frames(ph, lp, W, H, 0.4, 0.4)).to(device), lp)
        size = int(rng.choice([256, 320, 384, 448, 512, 576, 640]))
        rate = float(rng.uniform(60, 1000))
        traj = synth.smooth_trajectory(vseed, int(duration * 1000) + 10, 1000.0, size, size, 0.3, 0.3, tilts,
                                       pos_sigma_mm=0.15 * float(min(ext)))
        sessions.append(s)
        meta.append({"dims": dims, "dtype": "u8" if dtype == dare.DARE_U8 else "f16", "size": size, "rate": rate,
                     "traj": traj, "live": live, "W": W, "H": H})
    log(f"rank {dist.rank}: {len(sessions)} sessions admitted ({rejected} rejected), in use "
        f"{dare.memory_in_use() / 1e9:.1f} GB, set-up {time.perf_counter() - t0:.1f} s")
    # arrivals: merged Poisson streams
    arrivals = []
    for i, m in enumerate(meta):
        t = 0.0
        while True:
            t += float(rng.exponential(1.0 / m["rate"]))
            if t >= duration:
                break
            arrivals.append((t, i))
    arrivals.sort()
    ring = 64
    bufs = [[(torch.empty((m["size"], m["size"]), dtype=torch.float32, device=device),
              torch.empty((m["size"], dare.mask_words(m["size"])), dtype=torch.int32, device=device))
             for _ in range(ring)] for m in meta]
    free = [list(range(ring)) for _ in meta]
    server = dare.Server(device=dev, lanes=3, max_batch=64, coalesce_us=coalesce_us)
    tag_of = {}
    lat, ingest_lat, px_done, dropped = [], [], 0, 0

    detail = []  # per request: latency, queue wait, on-stream time, batch, session (ms)

    def collect():
        nonlocal px_done
        for tag, status, kind, t_sub, t_done, t_iss, nb, lane in server.poll():
            if status != dare.DARE_OK:
                raise RuntimeError(f"request {tag} failed with status {status}")
            if kind == 1:
                ingest_lat.append((t_done - t_sub) * 1e3)
                continue
            i, b = tag_of.pop(tag)
            free[i].append(b)
            lat.append((t_done - t_sub) * 1e3)
            detail.append(((t_done - t_sub) * 1e3, (t_iss - t_sub) * 1e3, (t_done - t_iss) * 1e3, nb, i))
            px_done += meta[i]["size"] ** 2

    # untimed warm-up: every session's kernels once (CUDA loads kernels lazily on first launch) and one
    # ingest per live session
    tag = 1 << 50
    for i, m in enumerate(meta):
        out, mask = bufs[i][0]
        server.submit(sessions[i], m["traj"][0], out, mask, (0.3, 0.3), tag)
        tag += 1
    ingest_idx = [0, 0]
    for j in range(min(2, len(meta))):
        fr, lp = meta[j]["live"]
        server.ingest(sessions[j], fr[0:3], lp[0:3], (0.4, 0.4), tag=tag)
        ingest_idx[j] = 3
        tag += 1
    server.drain(60.0)
    server.poll()
    tag = 0
    dist.barrier()
    clocks = ClockSampler(dev)
    clocks.start()
    start = dare.clock_seconds()
    next_ingest = 0.0
    k = 0
    while k < len(arrivals):
        now = dare.clock_seconds() - start
        while k < len(arrivals) and arrivals[k][0] <= now:
            t_arr, i = arrivals[k]
            k += 1
            if not free[i]:
                collect()
            if not free[i]:
                dropped += 1
                continue
            b = free[i].pop()
            out, mask = bufs[i][b]
            traj = meta[i]["traj"]
            server.submit(sessions[i], traj[min(int(t_arr * 1000), len(traj) - 1)], out, mask, (0.3, 0.3), tag)
            tag_of[tag] = (i, b)
            tag += 1
        while now >= next_ingest and next_ingest < duration:
            for j in range(min(2, len(meta))):
                fr, lp = meta[j]["live"]
                a = ingest_idx[j]
                if a + 3 <= fr.shape[0]:
                    server.ingest(sessions[j], fr[a:a + 3], lp[a:a + 3], (0.4, 0.4), tag=(1 << 40) + tag)
                    ingest_idx[j] = a + 3
                    tag += 1
            next_ingest += 0.1
        collect()
        if k < len(arrivals):
            wait = arrivals[k][0] - (dare.clock_seconds() - start)
            if wait > 2e-4:
                time.sleep(min(wait, 1e-3))
    server.drain(60.0)
    collect()
    wall = dare.clock_seconds() - start
    clk = clocks.stop()
    st = server.stats()
    server.close()
    lat = np.asarray(lat)
    det = np.asarray(detail) if detail else np.zeros((0, 5))
    slow = det[det[:, 0] >= np.percentile(det[:, 0], 99.9)] if det.size else det
    worst = det[np.argsort(det[:, 0])[-8:][::-1]] if det.size else det
    tail = {"requests": int(slow.shape[0]),
            "worst": [{"latency_ms": float(r[0]), "queue_wait_ms": float(r[1]), "on_stream_ms": float(r[2]),
                       "batch": int(r[3]), "session": int(r[4])} for r in worst],
            "queue_wait_ms_median": float(np.median(slow[:, 1])) if slow.size else None,
            "on_stream_ms_median": float(np.median(slow[:, 2])) if slow.size else None,
            "batch_median": float(np.median(slow[:, 3])) if slow.size else None,
            "live_session_share": float(np.mean(slow[:, 4] < 2)) if slow.size else None,
            "note": "requests at or above the p99.9 latency: time queued before the dispatcher issued them, time "
                    "from issue to completion on their lane, their batch size, and the share that belongs to the "
                    "two sessions ingesting live"}
    res = {"mpix_s": px_done / wall / 1e6 * dist.world, "duration_s": duration, "wall_s": wall,
           "requests": int(lat.size), "dropped_no_buffer": int(dropped),
           "latency_ms": {"p50": percentile(lat, 50), "p99": percentile(lat, 99), "p99.9": percentile(lat, 99.9),
                          "max": float(lat.max()), "mean": float(lat.mean())},
           "ingest_latency_ms": {"p50": percentile(ingest_lat, 50), "max": float(max(ingest_lat))}
           if ingest_lat else None,
           "server": {k2: int(v) for k2, v in st.items()},
           "mean_batch": (st["completed"] - st["ingests"]) / max(st["batches"], 1),
           "queue_wait_ms": {"p50": percentile(det[:, 1], 50), "p99": percentile(det[:, 1], 99)} if det.size else None,
           "on_stream_ms": {"p50": percentile(det[:, 2], 50), "p99": percentile(det[:, 2], 99)} if det.size else None,
           "tail": tail,
           "coalesce_us": coalesce_us, "lanes": 3, "max_batch": 64,
           "sessions": len(sessions), "rejected_by_budget": rejected, "budget_gb": 120,
           "device_gb_in_use": dare.memory_in_use() / 1e9,
           "rates_hz": [round(m["rate"]) for m in meta], "sizes": [m["size"] for m in meta],
           "dims": [m["dims"] for m in meta], "storage": [m["dtype"] for m in meta],
           "live_ingest_sessions": min(2, len(meta))}
    for s in sessions:
        s.close()
    return res, clk


def run_serving(args, dist):
    res, clk = serving_leg(args, dist, args.duration, args.coalesce_us)
    line = {"metric": "serving: resliced Mpix/s and submit-to-done latency over 16 sessions",
            "value": res["mpix_s"], "unit": "Mpix/s", "n_gpus": dist.world, "steps": res["requests"], "warmup": 0,
            "ms_per_step": res["latency_ms"]["mean"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "dare_serving_16sessions", "duration_s": args.duration,
                       "coalesce_us": args.coalesce_us},
            "serving": res,
            "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"],
                       "samples": clk["samples"]}}
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    dist = Dist()
    try:
        if args.impl == "reference":
            run_reference(args, dist)
        elif args.workload == "batched":
            run_batched(args, dist)
        elif args.workload == "serving":
            run_serving(args, dist)
        else:
            run_dare(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
