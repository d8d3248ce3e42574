#!/usr/bin/env python
"""Benchmark of the masked keypoint detector on one GB300 (or N, one per rank).

Workload (one step): the 640x480 synthetic clip of 300 frames (4 octaves +
intra-octaves, 16 x 12 bins, t = 30, T_I = 4, intensity-difference mask),
processed from its first frame through the C ABI in one fkd_push_frames call
with frames already resident in HBM; the stream is reset before each step so
every step does the same work. value = frames/s over all ranks.

Also reported: the same clip with plain full-frame detection (all bins
active), per-frame latency of frame-by-frame pushes (p50 / p99), an
end-to-end figure through the C ABI with pinned host buffers (host->device
copies of the frames and device->host copies of the keypoints inside the
timed region), the roofline of the dominant kernel from CUDA events recorded
around each kernel on the launching stream (in further steps after the timed
ones, so that the timed steps run plain launches) -- for the detection
kernel its integer-ALU pipe from the committed ncu counters, with the HBM
view on active bytes nested as "hbm" -- the SM clocks sampled
during the timed region, variants (mask on c_0, per-pixel masks, scale-space
suppression, detection + masked description), and the CPU oracle timed on a
bounded sample on this host.

The default line also carries "config3" (64 mixed-resolution streams, 120
frames each, one group tick per frame) and "config5" (8 streams of
3840x2160, 100 moving then 100 static frames) at their stated sizes: masked
against full-frame frames/s, Mpixel/s, tick latency p50 / p99, the
detection kernel's roofline on active bytes and their own clock records
(--no-groups leaves them out).

--config 3|4|5: one of those alone, or the serving loop (256 streams at 30
fps, 600 frames each, then a sweep of the rate) with its clocks. --sweep: the T_I / T_H
trade-off against full-frame detection. --describe masked|full|both:
detection + description alone on the 640x480 clip.
--impl reference times the CPU oracle (single-threaded C, the correctness
reference) on the same workload, a bounded number of frames per step.
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1503_06959_gb300 import synth  # noqa: E402

PEAKS_FALLBACK = {"hbm_gbs": 6800.0}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return PEAKS_FALLBACK, "fallback"


KERNEL_SOURCES = {
    "detect": ["k_detect.cu", "fkd_internal.cuh"],
    "pyramid": ["k_pyramid.cu", "fkd_internal.cuh"],
    "count": ["k_assemble.cu", "fkd_internal.cuh"],
}


def profile_counters(kernel: str, shape: dict | None = None):
    """Counters of the committed ncu summary of `kernel` on this workload, if
    the kernel's sources are unchanged since it was taken and, for the
    detection kernel, it was taken at the launch shape in use (else None)."""
    import hashlib
    import re
    if kernel not in KERNEL_SOURCES:
        return None
    path = os.path.join(ROOT, "profiles", f"k_{kernel}_masked_clip_640x480x300.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        m.update(open(os.path.join(ROOT, "paper_1503_06959_gb300", "csrc", f), "rb").read())
    sha = re.search(r"source_sha256: (\S+)", text)
    if not sha or sha.group(1) != m.hexdigest()[:16]:
        return None
    if kernel == "detect" and shape is not None:
        # one line of counters per captured launch shape: "counters th,w,c: key value key value ..."
        want = f"{shape['tile_h']},{shape['warps_per_cta']},{shape['ctas_per_sm']}"
        c = re.search(r"counters " + re.escape(want) + r": ([^\n]+)", text)
        if not c:
            return None
        toks = c.group(1).split()
        return {k: float(v) for k, v in zip(toks[0::2], toks[1::2])}
    got = {k: re.search(k + r": (\S+)", text)
           for k in ("traffic_bytes_per_launch", "alu_warp_inst_per_launch", "alu_peak_warp_inst_per_sm_cycle")}
    return {k: float(v.group(1)) for k, v in got.items() if v}


# --- multi-GPU plumbing: one independent stream per rank, timings max-reduced
def rank_env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_clip(cfg, rank: int, frames: int):
    """The clip rank `rank` processes: its own seeded stream (streams are
    independent, so the ranks share no data and exchange nothing)."""
    return synth.source_for(cfg, 2, stream=rank).frames(frames)


def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise maximum of per-rank timings (the slowest rank decides)."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def whole_job_fps(world: int, frames_per_step: int, steps: int, ms_max: float) -> float:
    """Frames of all ranks over the slowest rank's time (weak scaling)."""
    return world * frames_per_step * steps / (ms_max / 1e3)


def workload_desc(cfg, frames):
    return (f"{cfg.W}x{cfg.H} uint8 synthetic video, {frames} frames per step, O={cfg.O}"
            f"{' + intra-octaves' if cfg.intra else ''}, {cfg.N_c}x{cfg.N_r} bins (cols x rows), "
            f"t={cfg.t}, T_I={cfg.T_I}, intensity-difference mask on "
            f"{'the coarsest octave' if cfg.mask_layer == -1 else 'layer %d' % cfg.mask_layer}")


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons (200 ms)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.file.seek(0)
        sm, smax, reasons, pw = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
                pw.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.file.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(pw) if pw else None}


def cpu_oracle_fps(frames, cfg, seconds: float = 12.0):
    """The oracle as it stands, one thread, on the clip's first frames until
    about `seconds` of CPU work: frames/s."""
    import oracle
    s = oracle.Stream(cfg.W, cfg.H, N_r=cfg.N_r, N_c=cfg.N_c, T_I=cfg.T_I, O=cfg.O,
                      intra=cfg.intra, t=cfg.t, mask_mode=oracle.MASK_ID, mask_layer=cfg.mask_layer)
    t0 = time.perf_counter()
    n = 0
    while n < len(frames) and (time.perf_counter() - t0) < seconds:
        s.push(frames[n])
        s.keypoints()
        n += 1
    dt = time.perf_counter() - t0
    return n / dt, n, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cfg = synth.config2()
    frames_per_step = args.ref_frames
    frames = synth.source_for(cfg, 2).frames(frames_per_step * 2)
    import oracle
    oracle.build()

    def one_step():
        s = oracle.Stream(cfg.W, cfg.H, N_r=cfg.N_r, N_c=cfg.N_c, T_I=cfg.T_I, O=cfg.O,
                          intra=cfg.intra, t=cfg.t, mask_mode=oracle.MASK_ID, mask_layer=cfg.mask_layer)
        for f in frames[:frames_per_step]:
            s.push(f)
            s.keypoints()

    for _ in range(args.warmup):
        one_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one_step()
    dt = time.perf_counter() - t0
    fps = frames_per_step * args.steps / dt
    sample = (f"first {frames_per_step} frames of the clip per step, from its first frame, "
              f"one thread")
    line = {
        "impl": "reference", "metric": "frames/s (masked detection, bit-exact keypoints)",
        "value": fps, "unit": "frames/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": workload_desc(cfg, frames_per_step)},
        "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# --- synthetic clips generated in parallel (spawned processes write into
# shared memory; the generator is sequential within a stream)
def gen_clips(jobs, torch, device):
    """jobs: (count, W, H, seed, source kwargs). Returns one device tensor
    (count x H x W uint8) per job and the first frames of each on the host."""
    import concurrent.futures
    import multiprocessing
    from multiprocessing import shared_memory
    shms = [shared_memory.SharedMemory(create=True, size=max(1, c * W * H)) for c, W, H, _, _ in jobs]
    try:
        workers = max(1, min(len(jobs), os.cpu_count() or 1))
        with concurrent.futures.ProcessPoolExecutor(workers, mp_context=multiprocessing.get_context("spawn")) as ex:
            futs = [ex.submit(synth.fill_shared, s.name, *j) for s, j in zip(shms, jobs)]
            for f in futs:
                f.result()
        dev, heads = [], []
        for s, (c, W, H, _, _) in zip(shms, jobs):
            arr = np.ndarray((c, H, W), np.uint8, buffer=s.buf)
            dev.append(torch.from_numpy(arr).to(device, copy=True))
            heads.append(arr[:4].copy())
            del arr
        if torch.device(device).type == "cuda":
            torch.cuda.synchronize()
        return dev, heads
    finally:
        for s in shms:
            s.close()
            s.unlink()


# --- the active bytes of the detection step (the pixels that must be read:
# every pixel within 4 px -- the ring radius 3 plus the suppression
# neighbour -- of a pixel whose bin is active, on every layer)
def layer_dims(W, H, O, intra):
    """(w, h, S) of every layer: c_0 = W x H, c_{i+1} = c_i halved (floor),
    d_0 = 2 floor(W/3) x 2 floor(H/3), d_{i+1} = d_i halved; S = 2 sigma."""
    out = []
    for i in range(O):
        out.append((W >> i, H >> i, 2 << i))
        if intra:
            out.append(((W // 3) * 2 >> i, (H // 3) * 2 >> i, 3 << i))
    return out


class ActiveBytes:
    """Active layer pixels plus a `halo`-pixel border, per frame mask: the
    bytes the masked detection must read at least once. A layer pixel (x, y)
    of scale code S lies in bin (floor(floor(y S/2) N_r / H), floor(floor(x
    S/2) N_c / W)) (Eq. 3); it must be read when a bin of a pixel within
    `halo` of it (Chebyshev distance, inside the layer) is active. Because the
    bin index is monotone in x and y, the bins within reach of a pixel form a
    rectangle of bins, and pixels with the same rectangle are counted
    together through a prefix sum of the mask."""

    def __init__(self, W, H, O, intra, N_r, N_c, halo=4):
        self.N_r, self.N_c = N_r, N_c
        self.classes = []
        for w, h, S in layer_dims(W, H, O, intra):
            if w < 1 or h < 1:
                continue
            cb = ((np.arange(w) * S) // 2) * N_c // W
            rb = ((np.arange(h) * S) // 2) * N_r // H
            xs, ys = np.arange(w), np.arange(h)
            cu, cc = np.unique(cb[np.maximum(0, xs - halo)] * 65536 + cb[np.minimum(w - 1, xs + halo)],
                               return_counts=True)
            ru, rc = np.unique(rb[np.maximum(0, ys - halo)] * 65536 + rb[np.minimum(h - 1, ys + halo)],
                               return_counts=True)
            self.classes.append((ru >> 16, ru & 0xffff, rc, cu >> 16, cu & 0xffff, cc))

    def __call__(self, mask) -> int:
        m = np.asarray(mask, np.int64).reshape(self.N_r, self.N_c)
        P = np.zeros((self.N_r + 1, self.N_c + 1), np.int64)
        P[1:, 1:] = m.cumsum(0).cumsum(1)
        total = 0
        for r0, r1, rc, c0, c1, cc in self.classes:
            rect = (P[r1 + 1][:, c1 + 1] - P[r0][:, c1 + 1] - P[r1 + 1][:, c0] + P[r0][:, c0])
            total += int(((rect > 0) * rc[:, None] * cc[None, :]).sum())
        return total


def keypoint_keys(rec):
    """(layer, y, x) of records as one int64 each."""
    return (rec["layer"].astype(np.int64) << 32) | (rec["y"].astype(np.int64) << 16) | rec["x"].astype(np.int64)


def recall_precision(masked_frames, full_frames):
    """Mean over frames of |D_n and F_n| / |F_n| and |D_n and F_n| / |D_n|,
    D_n the masked set and F_n full-frame detection, over (layer, y, x)."""
    rec, prec = [], []
    for a, f in zip(masked_frames, full_frames):
        ka, kf = keypoint_keys(a), keypoint_keys(f)
        both = np.intersect1d(ka, kf).size
        rec.append(both / max(1, kf.size))
        prec.append(both / max(1, ka.size))
    return float(np.mean(rec)), float(np.mean(prec))


def group_workload(cfgs, clips, segments, warm, mode, fkd, torch, mask_layer=None, pattern=None,
                   with_latency=True, with_profile=True, profile_ticks=12):
    """One group of streams (cfgs[i] fed clips[i], device frames), one frame of
    every stream per tick. The detection launch shape is autotuned on the
    first ticks. Per segment (name, tick range; the ticks before the first
    segment are warm-up): frames/s from back-to-back graph replays between two
    CUDA events (the faster of two passes); then, in a second group, the tick latency (tick + wait, host
    clock) of the same ticks; then, in a third, stage times from CUDA events
    around every kernel and the masks (for the detection step's active bytes)."""
    O, intra = cfgs[0].O, cfgs[0].intra
    mpix = sum(c.W * c.H for c in cfgs) / 1e6

    def make():
        st = torch.cuda.Stream()
        g = fkd.Group(O, intra, cuda_stream=st.cuda_stream)
        ids = [g.add_stream(c.W, c.H, N_r=c.N_r, N_c=c.N_c, T_I=c.T_I, t=c.t, mask_mode=mode,
                            mask_layer=c.mask_layer if mask_layer is None else mask_layer,
                            K_max=1 << 20 if c.W * c.H > 4_000_000 else 1 << 17)[0] for c in cfgs]
        if pattern is not None:
            for i in ids:
                g.set_descriptor(i, pattern)
        return st, g, ids

    def tick(g, ids, n):
        g.tick(ids, [f[n] for f in clips])

    st, g, ids = make()
    shape, tune_ms = g.autotune(ids, [[f[n] for f in clips] for n in range(min(3, warm))], reps=2)
    res = {"launch_shape": dict(shape, tuned_ms_for_ticks=[min(3, warm), tune_ms]), "segments": {}}
    # Two passes, each in a group of its own from the first frame on; a
    # segment reports the faster pass (a stall of the host between two
    # ticks idles the GPU) and lists both.
    passes = {name: [] for name, _ in segments}
    for rep in range(2):
        if rep:
            st, g, ids = make()
            g.set_launch_config(shape)
        for n in range(warm):
            tick(g, ids, n)
        gc.disable()
        for name, rng in segments:
            g.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for n in rng:
                tick(g, ids, n)
            e1.record(st)
            e1.synchronize()
            passes[name].append(e0.elapsed_time(e1) / 1e3)
        gc.enable()
        g.close()
    for name, rng in segments:
        sec = min(passes[name])
        fps = len(cfgs) * len(rng) / sec
        res["segments"][name] = {"frames_per_s": fps, "mpix_per_s": fps / len(cfgs) * mpix,
                                 "ms_per_tick": sec / len(rng) * 1e3, "ticks": len(rng),
                                 "passes_ms_per_tick": [x / len(rng) * 1e3 for x in passes[name]]}
    if with_latency:
        st, g, ids = make()
        g.set_launch_config(shape)
        for n in range(warm):
            tick(g, ids, n)
        g.synchronize()
        for name, rng in segments:
            lat = []
            for n in rng:
                t0 = time.perf_counter()
                tick(g, ids, n)
                g.synchronize()
                lat.append((time.perf_counter() - t0) * 1e3)
            res["segments"][name]["tick_latency_ms"] = {
                "p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                "what": "fkd_group_tick of every stream + fkd_group_synchronize, host clock, one tick at a time"}
        g.close()
    if with_profile:
        pk, pk_kind = peaks()
        st, g, ids = make()
        g.set_launch_config(shape)
        counters = [ActiveBytes(c.W, c.H, c.O, c.intra, c.N_r, c.N_c) for c in cfgs]
        for n in range(warm):
            tick(g, ids, n)
        g.synchronize()
        g.profile_enable(True)
        for name, rng in segments:
            g.profile_read()
            sampled = set(list(rng)[::max(1, len(rng) // profile_ticks)])
            ms = {}
            act_bytes, act_bins, nb, tiles_px, nt = 0, 0, 0, 0, 0
            for n in rng:
                tick(g, ids, n)
                g.synchronize()
                prof = g.profile_read()
                if n not in sampled:
                    continue
                nt += 1
                for k, v in prof["ms"].items():
                    ms[k] = ms.get(k, 0.0) + v
                tiles_px += prof["tile_pixels"]
                for i, cnt in zip(ids, counters):
                    m = g.get_mask(i)
                    act_bytes += cnt(m)
                    act_bins += int(m.sum())
                    nb += m.size
            det_ms = ms.get("detect", 0.0) / max(1, nt)
            ab = act_bytes / max(1, nt)
            ach = ab / (det_ms / 1e3) / 1e9 if det_ms else None
            seg = res["segments"][name]
            seg["stage_ms_per_tick"] = {k: v / max(1, nt) for k, v in ms.items()}
            seg["active_bin_fraction"] = act_bins / max(1, nb)
            seg["detect_roofline"] = {
                "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": ach / pk["hbm_gbs"] if ach else None, "peak_source": f"{pk_kind} hbm_gbs",
                "active_bytes_per_tick": ab, "launch_ms": det_ms, "ticks_sampled": nt,
                "processed_tile_pixels_per_tick": tiles_px / max(1, nt),
                "bytes": "layer pixels within 4 px of an active bin's pixels, every layer of every stream "
                         "(1 byte read each), from the sampled ticks' masks; launch_ms from CUDA events "
                         "around the detection kernel of the same ticks"}
        g.close()
    return res


def config3_workload(torch, fkd, device, F=120, per_res=16):
    """64 streams (16 of each of 320x240 .. 1920x1080), F frames each, moving
    area U[5 %, 60 %] per stream: masked (intensity difference on the
    coarsest octave) against full-frame detection, one group tick per frame."""
    cfgs = synth.config3_streams(per_res)
    jobs = [(F, c.W, c.H, 1000 + 300 + j, c.source) for j, c in enumerate(cfgs)]
    t0 = time.perf_counter()
    clips, heads = gen_clips(jobs, torch, device)
    gen_s = time.perf_counter() - t0
    warm = 3
    segs = [("all", range(warm, F))]
    clocks = ClockSampler(torch.cuda.current_device())
    masked = group_workload(cfgs, clips, segs, warm, fkd.FKD_MASK_ID, fkd, torch)
    full = group_workload(cfgs, clips, segs, warm, fkd.FKD_MASK_FULL, fkd, torch)
    clk = clocks.stop()
    mpix = sum(c.W * c.H for c in cfgs) / 1e6
    out = {"workload": f"{len(cfgs)} streams ({per_res} each of 320x240, 640x480, 1280x720, 1920x1080), "
                       f"{F} frames each resident in HBM, O=4 + intra-octaves, 16x12 bins, t=30, T_I=4, "
                       f"moving area U[5%,60%]; one group tick = one frame of every stream "
                       f"({mpix:.1f} Mpixel of c_0); {warm} warm-up ticks, {F - warm} timed",
           "l2": f"inputs larger than L2 ({(F - warm) * mpix:.0f} MB of distinct frames over the timed ticks)",
           "masked": dict(masked["segments"]["all"], launch_shape=masked["launch_shape"]),
           "full_frame": dict(full["segments"]["all"], launch_shape=full["launch_shape"]),
           "clocks": clk, "frame_generation_s": gen_s}
    out["masked_over_full"] = out["masked"]["frames_per_s"] / out["full_frame"]["frames_per_s"]
    del clips
    return out, cfgs, heads


def config5_workload(torch, fkd, device, seg=100, n_streams=8):
    """8 streams of 3840x2160, 2 * seg frames: seg frames of motion (12
    movers of 700x700) then seg static frames (sensor noise only), O=5 +
    intra-octaves: masked against full-frame detection per segment."""
    cfg = synth.config5()
    F = 2 * seg
    src = dict(cfg.source, static_segments=(seg, 0))
    jobs = [(F, cfg.W, cfg.H, 1000 + 500 + j, src) for j in range(n_streams)]
    t0 = time.perf_counter()
    clips, heads = gen_clips(jobs, torch, device)
    gen_s = time.perf_counter() - t0
    warm = 2
    segs = [("moving", range(warm, seg)), ("static", range(seg, F))]
    cfgs = [cfg] * n_streams
    clocks = ClockSampler(torch.cuda.current_device())
    masked = group_workload(cfgs, clips, segs, warm, fkd.FKD_MASK_ID, fkd, torch)
    full = group_workload(cfgs, clips, segs, warm, fkd.FKD_MASK_FULL, fkd, torch)
    clk = clocks.stop()
    out = {"workload": f"{n_streams} streams of 3840x2160, {F} frames each resident in HBM: {seg} moving "
                       f"(12 movers of 700x700 at 2-6 px/frame) then {seg} static, N(0,2) noise, O=5 + "
                       f"intra-octaves (10 layers), 16x12 bins, t=30, T_I=4; one tick = one frame of every "
                       f"stream; ticks 0-{warm - 1} warm-up",
           "l2": "inputs larger than L2 (66 MB of c_0 per tick, distinct frames every tick)",
           "masked": dict(masked["segments"], launch_shape=masked["launch_shape"]),
           "full_frame": dict(full["segments"], launch_shape=full["launch_shape"]),
           "clocks": clk, "frame_generation_s": gen_s}
    out["masked_over_full"] = {p: out["masked"][p]["frames_per_s"] / out["full_frame"][p]["frames_per_s"]
                               for p in ("moving", "static")}
    del clips
    return out, cfg, heads


def run_config3(args):
    """The 64-stream group alone, as one JSON line (plus the describe variants)."""
    import torch
    from paper_1503_06959_gb300 import fkd
    dev = torch.device("cuda", 0)
    F = args.frames or 120
    sub, cfgs, heads = config3_workload(torch, fkd, dev, F=F, per_res=args.streams_per_res)
    line = {"metric": "frames/s (group of mixed-resolution streams, bit-exact keypoints)",
            "value": sub["masked"]["frames_per_s"], "unit": "frames/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "u8", "data": "synthetic", **sub}
    if args.describe_groups:
        clips, _ = gen_clips([(F, c.W, c.H, 1000 + 300 + j, c.source) for j, c in enumerate(cfgs)], torch, dev)
        pattern = synth.descriptor_pattern(256)
        segs = [("all", range(3, F))]
        dm = group_workload(cfgs, clips, segs, 3, fkd.FKD_MASK_ID, fkd, torch, pattern=pattern, with_latency=False)
        df = group_workload(cfgs, clips, segs, 3, fkd.FKD_MASK_FULL, fkd, torch, pattern=pattern, with_latency=False)
        line["describe"] = {"masked": dm["segments"]["all"], "full": df["segments"]["all"], "bits": 256,
                            "masked_over_full": dm["segments"]["all"]["frames_per_s"] /
                            df["segments"]["all"]["frames_per_s"]}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = group_cpu_baseline(cfgs, heads, per_res=args.streams_per_res)
    print(json.dumps(line))
    return 0


def group_cpu_baseline(cfgs, heads, per_res=16, seconds=3.0):
    """The oracle on the first frames of one stream per resolution (about
    `seconds` each): frames/s of the equal-count mix, one thread."""
    per_frame = []
    for j in range(0, len(cfgs), per_res):
        fps_r, _, _ = cpu_oracle_fps(heads[j], cfgs[j], seconds=seconds)
        per_frame.append(1.0 / fps_r)
    return {"value": 1.0 / (sum(per_frame) / len(per_frame)), "unit": "frames/s", "cores": 1, "kind": "oracle",
            "sample": "first frames (about 3 s each) of one stream per resolution, masked, one thread; "
                      "frames/s of the equal-count mix"}


def run_config5(args):
    """8 streams of 3840x2160 alone, as one JSON line."""
    import torch
    from paper_1503_06959_gb300 import fkd
    sub, cfg, heads = config5_workload(torch, fkd, torch.device("cuda", 0), seg=args.segment,
                                       n_streams=args.streams_5)
    line = {"metric": "frames/s and tick latency (3840x2160 stress: moving vs static segments)",
            "value": sub["masked"]["moving"]["frames_per_s"], "unit": "frames/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "u8", "data": "synthetic", **sub}
    if not args.no_cpu_baseline:
        fps_o, n_o, dt_o = cpu_oracle_fps(heads[0], cfg, seconds=10.0)
        line["cpu_baseline"] = {"value": fps_o, "unit": "frames/s", "cores": 1, "kind": "oracle",
                                "sample": f"first {n_o} frames of stream 0 (moving segment), masked, "
                                          f"one thread, {dt_o:.1f} s"}
    print(json.dumps(line))
    return 0


def run_sweep(args):
    """Threshold sweep (the paper's energy-accuracy trade-off, Sec. 4): on the
    640x480 clip, for each T_I (intensity-difference mask on the coarsest
    octave) and each T_H (keypoint binning), the active-bin fraction, frames/s
    and the agreement of D_n with full-frame detection: recall = |D_n and
    F_n| / |F_n| and precision = |D_n and F_n| / |D_n| over (layer, x, y),
    averaged over the frames."""
    import torch
    from paper_1503_06959_gb300 import fkd
    cfg = synth.config2()
    T = args.frames or 120
    frames = torch.from_numpy(synth.source_for(cfg, 2).frames(T)).cuda()
    st = torch.cuda.current_stream()
    base = dict(N_r=cfg.N_r, N_c=cfg.N_c, O=cfg.O, intra=cfg.intra, t=cfg.t, mask_layer=cfg.mask_layer,
                cuda_stream=st.cuda_stream)

    def run(mode, T_I=cfg.T_I, T_H=1):
        s = fkd.Stream(cfg.W, cfg.H, mask_mode=mode, T_I=T_I, T_H=T_H, T_max=T, **base)
        out = torch.empty(T * 65536, dtype=torch.int64, device="cuda")
        off = torch.empty(T + 1, dtype=torch.int32, device="cuda")
        msk = torch.empty((T, cfg.N_r, cfg.N_c), dtype=torch.uint8, device="cuda")
        for _ in range(2):
            s.reset()
            s.push_frames(frames, out=out, offsets=off, masks=msk)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        s.reset()
        s.push_frames(frames, out=out, offsets=off, masks=msk)
        e1.record(st)
        s.synchronize()
        ms = e0.elapsed_time(e1)
        o = off.cpu().numpy().astype(np.int64)
        rec = out[:o[T]].cpu().numpy().view(np.uint8).reshape(-1, 8)
        keys = (rec[:, 4].astype(np.int64) << 32) | (rec[:, 2].astype(np.int64) | rec[:, 3].astype(np.int64) << 8) << 16 \
            | (rec[:, 0].astype(np.int64) | rec[:, 1].astype(np.int64) << 8)
        per_frame = [keys[o[k]:o[k + 1]] for k in range(T)]
        return {"fps": T / (ms / 1e3), "active": float(msk.float().mean().item()), "kp": per_frame}

    full = run(fkd.FKD_MASK_FULL)

    def agree(r):
        rec_, prec_ = [], []
        for a, f in zip(r["kp"], full["kp"]):
            both = np.intersect1d(a, f).size
            rec_.append(both / max(1, f.size))
            prec_.append(both / max(1, a.size))
        return float(np.mean(rec_)), float(np.mean(prec_))

    rows = []
    for T_I in (1, 2, 4, 8, 16, 32):
        r = run(fkd.FKD_MASK_ID, T_I=T_I)
        rc, pc = agree(r)
        rows.append({"mask": "ID", "T_I": T_I, "active_bin_fraction": r["active"], "frames_per_s": r["fps"],
                     "time_vs_full": full["fps"] / r["fps"], "recall": rc, "precision": pc})
    # keypoint binning needs D_{n-1} before frame n's mask: one stream runs its
    # batch in spans of 16 frames (detected on the bins still active at the
    # span's start, masks resolved from the detection counts); beside it, 64
    # streams (stream 0 = the clip above) in one group, one frame each per tick
    n_grp = 64
    clips = [frames] + [torch.from_numpy(synth.source_for(cfg, 2, stream=j).frames(T)).cuda()
                        for j in range(1, n_grp)]

    def group_fps(mode, T_H=1):
        gst = torch.cuda.Stream()
        g = fkd.Group(cfg.O, cfg.intra, cuda_stream=gst.cuda_stream)
        ids = [g.add_stream(cfg.W, cfg.H, N_r=cfg.N_r, N_c=cfg.N_c, T_I=cfg.T_I, T_H=T_H, t=cfg.t,
                            mask_mode=mode, mask_layer=cfg.mask_layer)[0] for _ in range(n_grp)]
        for n in range(3):
            g.tick(ids, [c[n] for c in clips])
        g.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(gst)
        for n in range(3, T):
            g.tick(ids, [c[n] for c in clips])
        e1.record(gst)
        e1.synchronize()
        g.close()
        return n_grp * (T - 3) / (e0.elapsed_time(e1) / 1e3)

    full_grp = group_fps(fkd.FKD_MASK_FULL)
    for T_H in (1, 2, 3, 4):
        r = run(fkd.FKD_MASK_KB, T_H=T_H)
        rc, pc = agree(r)
        fg = group_fps(fkd.FKD_MASK_KB, T_H)
        rows.append({"mask": "KB", "T_H": T_H, "active_bin_fraction": r["active"],
                     "frames_per_s_one_stream": r["fps"], "frames_per_s": fg,
                     "frames_per_s_what": f"{n_grp} streams in one group, one frame of each per tick",
                     "time_vs_full": full_grp / fg, "recall": rc, "precision": pc})
    line = {"metric": "threshold sweep: active bins, frames/s and agreement with full detection",
            "unit": "frames/s", "n_gpus": 1, "dtype": "u8", "data": "synthetic",
            "config": {"workload": workload_desc(cfg, T) + "; KB in spans of 16 frames (its mask needs D_{n-1})"},
            "full_frame_fps": full["fps"], "full_frame_group_fps": full_grp, "rows": rows}
    print(json.dumps(line))
    return 0


def run_describe(args):
    """Detection + masked description alone on the 640x480 clip (Sec. 3:
    descriptors only for newly detected keypoints, carried ones copied),
    against full-frame detection + description of every keypoint; 256-bit
    descriptors. One JSON line; also the case the describe profiles use."""
    import torch
    from paper_1503_06959_gb300 import fkd
    cfg = synth.config2()
    T = args.frames or cfg.frames
    frames = torch.from_numpy(synth.source_for(cfg, 2).frames(T)).cuda()
    st = torch.cuda.current_stream()
    base = dict(N_r=cfg.N_r, N_c=cfg.N_c, T_I=cfg.T_I, O=cfg.O, intra=cfg.intra, t=cfg.t,
                mask_layer=cfg.mask_layer, T_max=T, cuda_stream=st.cuda_stream,
                pattern=synth.descriptor_pattern(256))
    cap = T * 32768
    out = torch.empty(cap, dtype=torch.int64, device="cuda")
    off = torch.empty(T + 1, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    res = {}
    modes = {"masked": fkd.FKD_MASK_ID, "full": fkd.FKD_MASK_FULL}
    for name in (modes if args.describe == "both" else [args.describe]):
        s = fkd.Stream(cfg.W, cfg.H, mask_mode=modes[name], **base)
        if args.shape:
            th, wp, cp = (int(v) for v in args.shape.split(","))
            s.set_launch_config(dict(tile_h=th, warps_per_cta=wp, ctas_per_sm=cp))
        for _ in range(args.warmup):
            s.reset()
            s.push_frames(frames, out=out, offsets=off)
        s.synchronize()
        ms = 0.0
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            s.reset()
            s.push_frames(frames, out=out, offsets=off)
            e1.record(st)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        s.synchronize()
        # stage times from one more step with CUDA events around every kernel
        s.profile_read(reset=True)
        s.profile_enable(True)
        s.reset()
        s.push_frames(frames, out=out, offsets=off)
        s.synchronize()
        prof = s.profile_read(reset=True)
        s.profile_enable(False)
        o = off.cpu().numpy().astype(np.int64)
        rec = out[:int(o[T])].cpu().numpy().view(fkd.KEYPOINT_DTYPE)
        res[name] = {"value": T * args.steps / (ms / 1e3), "unit": "frames/s", "records_per_step": int(o[T]),
                     "described_per_step": int(((rec["flags"] & fkd.FKD_KP_PROPAGATED) == 0).sum()),
                     "stage_ms_per_step": {k: v / max(1, prof["batches"]) for k, v in prof["ms"].items()}}
        s.close()
    line = {"metric": "frames/s (detection + masked description, bit-exact)", "unit": "frames/s",
            "steps": args.steps, "warmup": args.warmup, "bits": 256,
            "config": {"workload": workload_desc(cfg, T), "frames_per_step": T,
                       "l2": "flushed between steps (256 MB write outside the timed events)"},
            **res}
    if "masked" in res and "full" in res:
        line["masked_over_full"] = res["masked"]["value"] / res["full"]["value"]
    print(json.dumps(line))
    return 0


def run_config4(args):
    """Serving: 256 streams of mixed resolution producing frames with Poisson
    arrivals, continuous batching. Frames come from a pinned pool (12 per
    resolution; stream j's n-th frame is pool frame (7 j + n) mod 12) and are
    submitted by reference at their arrival times by the library's own load
    generator (fkd_server_replay), so no interpreter sits in the arrival
    loop. The nominal run offers 30 fps per stream (600 frames each); the
    sweep multiplies the per-stream rate until the offered load exceeds what
    the loop serves, for masked and full-frame detection alike."""
    import torch
    from paper_1503_06959_gb300 import fkd
    per_res = args.serve_streams_per_res
    frames_per_stream = args.serve_frames
    res_list = [(320, 240), (640, 480), (1280, 720), (1920, 1080)]
    pool = {}
    for k, (W, H) in enumerate(res_list):
        src = synth.VideoSource(W, H, seed=1000 + 400 + k, n_movers=4,
                                mover_size=int(math.sqrt(0.3 * W * H / 4)), speed=(1, 4))
        pool[(W, H)] = torch.from_numpy(src.frames(args.pool)).pin_memory()

    def serve(mode, rate_mult, seed):
        srv = fkd.Server(4, 1, budget_bytes=args.budget_gb << 30, max_tick_keypoints=1 << 23)
        srv.keep_results(False)
        streams, rejected = [], 0
        for k, (W, H) in enumerate(res_list):
            for j in range(per_res):
                try:
                    sid = srv.open_stream(W, H, N_r=12, N_c=16, T_I=4, t=30, mask_mode=mode,
                                          mask_layer=-1, K_max=1 << 17)
                    streams.append((sid, W, H, k * per_res + j))
                except fkd.FkdError as e:
                    if e.code != fkd.FKD_E_BUDGET:
                        raise
                    rejected += 1
        # warm-up outside the statistics: two frames of every stream (loads the
        # kernels, captures the tick graphs)
        t_w = time.monotonic_ns() + 50_000_000
        warm = [(t_w + (n * len(streams) + i) * 20_000, sid, W, H, (j * 7 + n) % args.pool)
                for n in range(2) for i, (sid, W, H, j) in enumerate(streams)]
        srv.replay([w[1] for w in warm], [pool[(w[2], w[3])][w[4]].data_ptr() for w in warm],
                   [pool[(w[2], w[3])].stride(1) for w in warm], [w[0] for w in warm])
        srv.drain(600000)
        srv.stats(reset=True)
        rng = np.random.default_rng(seed)
        rate = 30.0 * rate_mult
        t_start = time.monotonic_ns() + 300_000_000
        ts, ids, ptrs, pitches = [], [], [], []
        for sid, W, H, j in streams:
            gaps = rng.exponential(1.0 / rate, frames_per_stream)
            gaps[0] = rng.uniform(0, 1.0 / rate)
            ts.append(t_start + (np.cumsum(gaps) * 1e9).astype(np.int64))
            ids.append(np.full(frames_per_stream, sid, np.int32))
            pf = pool[(W, H)]
            idx = (j * 7 + np.arange(frames_per_stream)) % args.pool
            ptrs.append(pf.data_ptr() + idx.astype(np.uint64) * np.uint64(pf.stride(0)))
            pitches.append(np.full(frames_per_stream, pf.stride(1), np.uint64))
        ts, ids, ptrs, pitches = (np.concatenate(v) for v in (ts, ids, ptrs, pitches))
        order = np.argsort(ts, kind="stable")
        offered_s = (ts.max() - t_start) / 1e9
        refused = srv.replay(ids[order], ptrs[order], pitches[order], ts[order])
        srv.drain(600000)
        st = srv.stats()
        srv.close()
        return {"rate_per_stream_fps": rate, "offered_fps": len(ts) / offered_s, "fps": st["fps"],
                "frames_offered": int(len(ts)), "frames_done": st["frames_done"], "frames_dropped": int(refused),
                "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
                "mean_batch": st["mean_batch"], "ticks": st["ticks"], "streams_admitted": len(streams),
                "streams_rejected": rejected, "device_bytes": st["bytes_in_use"]}

    out, sweep = {}, {"masked": [], "full": []}
    clocks = ClockSampler(0)
    for name, mode in (("masked", fkd.FKD_MASK_ID), ("full", fkd.FKD_MASK_FULL)):
        out[name] = serve(mode, 1.0, 4)
        for m in args.serve_sweep:
            sweep[name].append(serve(mode, float(m), 5))
    clk = clocks.stop()

    def knee(points):
        """The highest offered load the loop kept up with (served >= 98 % of
        it, at most 0.1 % of its frames dropped: with four queued frames per
        stream a Poisson burst can drop a frame well below capacity), and the
        largest served rate seen."""
        kept = [p for p in points
                if p["frames_dropped"] <= 0.001 * p["frames_offered"] and p["fps"] >= 0.98 * p["offered_fps"]]
        return {"kept_up_to_offered_fps": max((p["offered_fps"] for p in kept), default=None),
                "p99_ms_there": max(kept, key=lambda p: p["offered_fps"])["p99_ms"] if kept else None,
                "max_served_fps": max(p["fps"] for p in points)}
    # admission under a small budget: streams of the mix, round robin, until
    # the budget refuses them; closing one frees room for the next
    small = args.small_budget_mb << 20
    srv = fkd.Server(4, 1, budget_bytes=small, max_tick_keypoints=1 << 20)
    admitted = {f"{W}x{H}": 0 for W, H in res_list}
    refused = {f"{W}x{H}": 0 for W, H in res_list}
    open_ids = []
    for j in range(per_res):
        for W, H in res_list:
            try:
                open_ids.append((srv.open_stream(W, H, N_r=12, N_c=16, T_I=4, t=30, mask_mode=fkd.FKD_MASK_ID,
                                                 mask_layer=-1, K_max=1 << 17), W, H))
                admitted[f"{W}x{H}"] += 1
            except fkd.FkdError as e:
                if e.code != fkd.FKD_E_BUDGET:
                    raise
                refused[f"{W}x{H}"] += 1
    in_use = srv.stats()["bytes_in_use"]
    readmit = None
    big = [sid for sid, W, H in open_ids if W == 1920]
    if big:
        srv.close_stream(big[0])
        try:
            srv.open_stream(1920, 1080, N_r=12, N_c=16, T_I=4, t=30, mask_mode=fkd.FKD_MASK_ID,
                            mask_layer=-1, K_max=1 << 17)
            readmit = True
        except fkd.FkdError:
            readmit = False
    srv.close()
    admission = {"budget_bytes": small, "admitted": admitted, "refused": refused,
                 "bytes_in_use": in_use, "readmitted_after_close": readmit}
    line = {"metric": "frames/s and p99 latency (serving, continuous batching)",
            "value": out["masked"]["fps"], "unit": "frames/s", "n_gpus": 1, "dtype": "u8",
            "data": "synthetic", "admission_small_budget": admission,
            "config": {"workload": f"{4 * per_res} streams ({per_res} each of 320x240 .. 1920x1080), "
                                   f"{frames_per_stream} frames each, Poisson arrivals at 30 fps per stream "
                                   f"(sweep: x{', x'.join(str(m) for m in args.serve_sweep)}), O=4 + "
                                   f"intra-octaves, 16x12 bins, t=30, T_I=4, mask on the coarsest octave, "
                                   f"budget {args.budget_gb} GB; frames from a pinned pool submitted by "
                                   f"reference by fkd_server_replay",
                       "latency": "arrival (scheduled) to the frame's keypoints on the host"},
            "masked": out["masked"], "full_frame": out["full"],
            "sweep": sweep, "knee": {"masked": knee(sweep["masked"]), "full": knee(sweep["full"])},
            "clocks": clk}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames", type=int, default=0, help="frames per step (default: the clip)")
    ap.add_argument("--ref-frames", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--latency-frames", type=int, default=300)
    ap.add_argument("--config", type=int, default=2, choices=[2, 3, 4, 5],
                    help="2: the 640x480 clip (default line); 3: stream group; 4: serving; 5: 4K stress")
    ap.add_argument("--sweep", action="store_true", help="threshold sweep of T_I and T_H on the 640x480 clip")
    ap.add_argument("--streams-per-res", type=int, default=16)
    ap.add_argument("--serve-streams-per-res", type=int, default=64)
    ap.add_argument("--serve-frames", type=int, default=600, help="frames per served stream")
    ap.add_argument("--serve-sweep", type=float, nargs="*", default=[2, 4, 8, 10, 12, 14, 16, 32, 64],
                    help="multiples of 30 fps per stream offered in the serving sweep")
    ap.add_argument("--pool", type=int, default=12)
    ap.add_argument("--budget-gb", type=int, default=8)
    ap.add_argument("--small-budget-mb", type=int, default=256)
    ap.add_argument("--segment", type=int, default=100)
    ap.add_argument("--no-groups", action="store_true",
                    help="default run: leave out the config 3 and config 5 sub-objects")
    ap.add_argument("--describe-groups", action="store_true",
                    help="--config 3: add detection + description in the group")
    ap.add_argument("--streams-5", type=int, default=8)
    ap.add_argument("--describe", default="", choices=["", "masked", "full", "both"],
                    help="detection + description on the 640x480 clip only (masked, full or both)")
    ap.add_argument("--shape", default="",
                    help="detection launch shape tile_h,warps_per_cta,ctas_per_sm (default: autotune)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        return run_sweep(args)
    if args.describe:
        return run_describe(args)
    if args.config == 3:
        return run_config3(args)
    if args.config == 4:
        return run_config4(args)
    if args.config == 5:
        return run_config5(args)

    import torch
    from paper_1503_06959_gb300 import fkd

    world, rank, local = rank_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    cfg = synth.config2()
    T = args.frames or cfg.frames
    frames_np = rank_clip(cfg, rank, T)
    frames = torch.from_numpy(frames_np).to(dev)
    torch_stream = torch.cuda.current_stream()
    handle = torch_stream.cuda_stream
    common = dict(N_r=cfg.N_r, N_c=cfg.N_c, T_I=cfg.T_I, O=cfg.O, intra=cfg.intra, t=cfg.t,
                  mask_layer=cfg.mask_layer,
                  T_max=T, cuda_stream=handle)
    cap = T * 32768
    out = torch.empty(cap, dtype=torch.int64, device=dev)
    offsets = torch.empty(T + 1, dtype=torch.int32, device=dev)
    masks = torch.empty((T, cfg.N_r, cfg.N_c), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(stream_obj, steps, warmup, profile=False):
        """Milliseconds of `steps` plain steps (no events between the
        kernels); with `profile`, also the stage times of further steps run
        with CUDA events around every kernel."""
        def step():
            stream_obj.reset()
            stream_obj.push_frames(frames, out=out, offsets=offsets, masks=masks)
        for _ in range(warmup):
            step()
        stream_obj.synchronize()
        evs = []
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        for _ in range(steps):
            flush.zero_()  # L2 flush between steps (outside the events)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(torch_stream)
            step()
            e1.record(torch_stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        stream_obj.synchronize()  # raises on a capacity overflow
        ms = sum(a.elapsed_time(b) for a, b in evs)
        prof = None
        if profile:
            stream_obj.profile_read(reset=True)
            stream_obj.profile_enable(True)
            for _ in range(max(3, steps // 2)):
                flush.zero_()
                step()
            stream_obj.synchronize()
            prof = stream_obj.profile_read(reset=True)
            stream_obj.profile_enable(False)
        return ms, prof

    masked = fkd.Stream(cfg.W, cfg.H, mask_mode=fkd.FKD_MASK_ID, **common)
    full = fkd.Stream(cfg.W, cfg.H, mask_mode=fkd.FKD_MASK_FULL, **common)
    # detection launch shape: autotuned per stream on the step's own frames
    if args.shape:
        th, wp, cp = (int(v) for v in args.shape.split(","))
        shape_masked = shape_full = dict(tile_h=th, warps_per_cta=wp, ctas_per_sm=cp)
        masked.set_launch_config(shape_masked)
        full.set_launch_config(shape_full)
        tune_ms_masked = tune_ms_full = None
    else:
        shape_masked, tune_ms_masked = masked.autotune(frames, reps=2)
        shape_full, tune_ms_full = full.autotune(frames, reps=2)

    # the headline: plain launches, no events between the kernels (the stage
    # times and the dominant kernel's launch duration come from further steps
    # run with events, after the timed ones)
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    t_wall0 = time.perf_counter()
    ms, _ = timed(masked, args.steps, args.warmup)
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop() if clocks else None
    off_masked = offsets.cpu().numpy().astype(np.int64)
    kp_masked = int(off_masked[T] - off_masked[0])
    rec_masked = out[:kp_masked].cpu().numpy().view(fkd.KEYPOINT_DTYPE)
    masks_np = masks.cpu().numpy()
    act = float(masks_np.mean())
    act_counter = ActiveBytes(cfg.W, cfg.H, cfg.O, cfg.intra, cfg.N_r, cfg.N_c)
    act_bytes = sum(act_counter(m) for m in masks_np)  # per step (one launch of each kernel)
    _, prof = timed(masked, 0, 0, profile=True)

    ms_full, prof_full = timed(full, max(3, args.steps // 2), 3, profile=True)
    off_full = offsets.cpu().numpy().astype(np.int64)
    kp_full = int(off_full[T] - off_full[0])
    rec_full = out[:kp_full].cpu().numpy().view(fkd.KEYPOINT_DTYPE)
    # how much of full-frame detection the masked sets keep (a statistic of
    # the method, not parity: each mode is bit-exact with its own oracle mode)
    m_recall, m_precision = recall_precision(fkd.split_frames(rec_masked, off_masked),
                                             fkd.split_frames(rec_full, off_full))
    del rec_masked, rec_full

    # the same masked detection with the intensity test on c_0 (the library's
    # default layer) beside the coarsest octave (the paper's experiments)
    c0_common = dict(common, mask_layer=0)
    masked_c0 = fkd.Stream(cfg.W, cfg.H, mask_mode=fkd.FKD_MASK_ID, **c0_common)
    if args.shape:
        masked_c0.set_launch_config(shape_masked)
        shape_c0 = shape_masked
    else:
        shape_c0, _ = masked_c0.autotune(frames, reps=2)
    ms_c0, prof_c0 = timed(masked_c0, max(3, args.steps // 2), 3, profile=True)
    act_c0 = masks.float().mean().item()

    # Eq. 2 per pixel of every layer (option (i) of Sec. 3.1)
    masked_px = fkd.Stream(cfg.W, cfg.H, mask_mode=fkd.FKD_MASK_IDP, **common)
    masked_px.set_launch_config(shape_masked)
    ms_px, prof_px = timed(masked_px, max(3, args.steps // 2), 3, profile=True)
    px_tiles = prof_px["tile_pixels"] / max(1, prof_px["batches"])

    # the masked detection with scale-space suppression (Sec. 2)
    masked_xs = fkd.Stream(cfg.W, cfg.H, mask_mode=fkd.FKD_MASK_ID, nms_scale=1, **common)
    masked_xs.set_launch_config(shape_masked)
    ms_xs, prof_xs = timed(masked_xs, max(3, args.steps // 2), 3, profile=True)
    off_xs = offsets.cpu().numpy().astype(np.int64)
    kp_xs = int(off_xs[T] - off_xs[0])

    # detection and description (Sec. 3): masked (descriptors only for new
    # keypoints, carried ones copied) against full-frame (every keypoint
    # described every frame), 256-bit descriptors
    pattern = synth.descriptor_pattern(256)
    desc_m = fkd.Stream(cfg.W, cfg.H, mask_mode=fkd.FKD_MASK_ID, pattern=pattern, **common)
    desc_m.set_launch_config(shape_masked)
    ms_dm, prof_dm = timed(desc_m, max(3, args.steps // 2), 3, profile=True)
    off_dm = offsets.cpu().numpy().astype(np.int64)
    rec_dm = out[:int(off_dm[T])].cpu().numpy().view(fkd.KEYPOINT_DTYPE)
    new_dm = int(((rec_dm["flags"] & fkd.FKD_KP_PROPAGATED) == 0).sum())
    desc_f = fkd.Stream(cfg.W, cfg.H, mask_mode=fkd.FKD_MASK_FULL, pattern=pattern, **common)
    desc_f.set_launch_config(shape_full)
    ms_df, prof_df = timed(desc_f, max(3, args.steps // 2), 3, profile=True)

    # max over ranks
    ms, ms_full, ms_c0, ms_xs, ms_px, ms_dm, ms_df = max_over_ranks(
        [ms, ms_full, ms_c0, ms_xs, ms_px, ms_dm, ms_df], dist, dev)
    value = whole_job_fps(world, T, args.steps, ms)
    full_fps = whole_job_fps(world, T, max(3, args.steps // 2), ms_full)
    c0_fps = whole_job_fps(world, T, max(3, args.steps // 2), ms_c0)
    xs_fps = whole_job_fps(world, T, max(3, args.steps // 2), ms_xs)
    px_fps = whole_job_fps(world, T, max(3, args.steps // 2), ms_px)
    dm_fps = whole_job_fps(world, T, max(3, args.steps // 2), ms_dm)
    df_fps = whole_job_fps(world, T, max(3, args.steps // 2), ms_df)

    # frame-by-frame latency (device frames): push_frame + get_keypoints per frame
    lat = fkd.Stream(cfg.W, cfg.H, mask_mode=fkd.FKD_MASK_ID, N_r=cfg.N_r, N_c=cfg.N_c, mask_layer=cfg.mask_layer,
                     T_I=cfg.T_I, O=cfg.O, intra=cfg.intra, t=cfg.t, cuda_stream=handle)
    lat.set_launch_config(shape_masked)
    nlat = min(args.latency_frames, T)
    lat_ms = []
    for n in range(nlat):
        t0 = time.perf_counter()
        lat.push_frame(frames[n])
        lat.get_keypoints()
        lat_ms.append((time.perf_counter() - t0) * 1e3)
    lat_ms = lat_ms[3:] if len(lat_ms) > 10 else lat_ms
    p50 = float(np.percentile(lat_ms, 50)) if lat_ms else None
    p99 = float(np.percentile(lat_ms, 99)) if lat_ms else None

    # end to end through the C ABI with pinned host buffers
    host_frames = torch.from_numpy(frames_np).pin_memory()
    host_out = torch.empty(cap, dtype=torch.int64).pin_memory()
    host_off = torch.empty(T + 1, dtype=torch.int32).pin_memory()
    host_masks = torch.empty((T, cfg.N_r, cfg.N_c), dtype=torch.uint8).pin_memory()
    hf, ho = host_frames.numpy(), host_out.numpy()
    hoff, hm = host_off.numpy().view(np.uint32), host_masks.numpy()
    e2e_stream = fkd.Stream(cfg.W, cfg.H, mask_mode=fkd.FKD_MASK_ID, **common)
    e2e_stream.set_launch_config(shape_masked)
    for _ in range(2):
        e2e_stream.reset()
        e2e_stream.push_frames(hf, out=ho, offsets=hoff, masks=hm)
    e2e_steps = max(3, args.steps // 2)
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_stream.reset()
        e2e_stream.push_frames(hf, out=ho, offsets=hoff, masks=hm)
    e2e_s = time.perf_counter() - t0
    (e2e_s,) = max_over_ranks([e2e_s], dist, dev)
    e2e_fps = whole_job_fps(world, T, e2e_steps, e2e_s * 1e3)
    h2d = T * cfg.W * cfg.H
    d2h = int(hoff[T] - hoff[0]) * 8 + (T + 1) * 4 + T * cfg.N_r * cfg.N_c

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # roofline of the dominant kernel (CUDA events around each launch, in the
    # steps run with events after the timed ones; one launch per step)
    pk, pk_kind = peaks()
    stage_ms = prof["ms"]
    dom = max(stage_ms, key=stage_ms.get)
    launches = max(1, prof["launches"][dom])
    dur_s = stage_ms[dom] / launches / 1e3
    layer_px = sum(masked.layer_info(l)[0] * masked.layer_info(l)[1]
                   for l in range(masked.num_layers()))
    if dom == "detect":
        bytes_per_launch = act_bytes
        bytes_desc = ("active bytes: layer pixels within 4 px (ring radius 3 + the suppression neighbour) "
                      "of a pixel of an active bin, every layer of every frame of the step, 1 byte read each; "
                      "counted from the step's masks")
    elif dom == "pyramid":
        bytes_per_launch = prof["frames"] / launches * (cfg.W * cfg.H + (layer_px - cfg.W * cfg.H))
        bytes_desc = "per frame: c_0 read, layers >= 1 written"
    else:
        bytes_per_launch = prof["frames"] / launches * layer_px / 8 * 2
        bytes_desc = "per frame: keypoint bitmap words read and written"
    achieved = bytes_per_launch / dur_s / 1e9
    counters = profile_counters(dom, shape_masked) if T == cfg.frames else None
    # the HBM view: algorithmic bytes per launch over the launch time
    hbm = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
           "frac": achieved / pk["hbm_gbs"], "peak_source": f"{pk_kind} hbm_gbs",
           "bytes_per_launch": bytes_per_launch, "bytes": bytes_desc}
    roof = dict(kernel=dom, **hbm)
    alu_inst = counters.get("alu_warp_inst_per_launch") if counters else None
    alu_rate = counters.get("alu_peak_warp_inst_per_sm_cycle") if counters else None
    if alu_inst and alu_rate and clk and clk.get("sm_mhz"):
        # the integer ALU pipe, the detection kernel's bound: warp instructions
        # the kernel issued to it (ncu smsp__inst_executed_pipe_alu.sum) per
        # launch duration, against the pipe's issue rate per SM and cycle (ncu
        # sm__inst_executed_pipe_alu.avg.peak_sustained) x SMs x the median SM
        # clock sampled during the timed steps; the HBM view beside it
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        peak_alu = n_sm * alu_rate * clk["sm_mhz"] * 1e6 / 1e9
        ach_alu = alu_inst / dur_s / 1e9
        roof = {"kernel": dom, "bound": "alu", "achieved": ach_alu, "peak": peak_alu,
                "unit": "G warp-instructions/s (integer ALU pipe)", "frac": ach_alu / peak_alu,
                "peak_source": f"{n_sm} SMs x {alu_rate} ALU warp-instructions/cycle/SM (ncu peak_sustained) "
                               f"x {clk['sm_mhz']:.0f} MHz (median sampled)",
                "alu_warp_inst_per_launch": alu_inst, "hbm": hbm}
    roof.update({"traffic": counters.get("traffic_bytes_per_launch") if counters else None,
                 "launch_ms": dur_s * 1e3,
                 "processed_tile_pixels_per_launch": prof["tile_pixels"] / launches if dom == "detect" else None})

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        fps_cpu, n_cpu, dt_cpu = cpu_oracle_fps(frames_np, cfg)
        cpu = {"value": fps_cpu, "unit": "frames/s", "cores": 1, "kind": "oracle",
               "sample": f"first {n_cpu} frames of the clip from frame 0, one thread, {dt_cpu:.1f} s"}

    line = {
        "metric": "frames/s (masked detection, bit-exact keypoints)", "value": value,
        "unit": "frames/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": workload_desc(cfg, T), "frames_per_step": T,
                   "l2": "flushed between steps (256 MB write outside the timed events)",
                   "parallelism": f"one stream per GPU x {world}",
                   "launch_shape": {"masked": shape_masked, "full": shape_full,
                                    "tuned_step_ms": {"masked": tune_ms_masked, "full": tune_ms_full}}},
        "mpix_per_s": value * cfg.W * cfg.H / 1e6,
        "full_frame": {"value": full_fps, "unit": "frames/s", "keypoints_per_step": kp_full,
                       "stage_ms_per_step": {k: v / max(1, prof_full["batches"])
                                             for k, v in prof_full["ms"].items()}},
        "masked_over_full": value / full_fps,
        "masked_recall": {"recall": m_recall, "precision": m_precision,
                          "what": "mean over frames of |D_n and F_n| / |F_n| (recall) and / |D_n| (precision), "
                                  "D_n masked, F_n full-frame detection, over (layer, y, x)"},
        "active_bytes_per_step": act_bytes,
        "masked_c0": {"value": c0_fps, "unit": "frames/s", "active_bin_fraction": act_c0,
                      "masked_over_full": c0_fps / full_fps, "launch_shape": shape_c0,
                      "what": "the intensity-difference test on c_0 instead of the coarsest octave",
                      "stage_ms_per_step": {k: v / max(1, prof_c0["batches"])
                                            for k, v in prof_c0["ms"].items()}},
        "masked_pixel": {"value": px_fps, "unit": "frames/s", "masked_over_full": px_fps / full_fps,
                         "tile_pixels_per_step": px_tiles,
                         "what": "Eq. 2 per pixel of every layer (each layer's own mask), T_I as above",
                         "stage_ms_per_step": {k: v / max(1, prof_px["batches"])
                                               for k, v in prof_px["ms"].items()}},
        "masked_nms_scale": {"value": xs_fps, "unit": "frames/s", "keypoints_per_step": kp_xs,
                             "what": "masked, with scale-space suppression against the adjacent layers "
                                     "(its pass is timed in the detect stage)",
                             "stage_ms_per_step": {k: v / max(1, prof_xs["batches"])
                                                   for k, v in prof_xs["ms"].items()}},
        "describe": {"masked": dm_fps, "full": df_fps, "unit": "frames/s", "masked_over_full": dm_fps / df_fps,
                     "bits": 256, "described_per_step": {"masked": new_dm, "full": kp_full},
                     "records_per_step": {"masked": int(off_dm[T]), "full": kp_full},
                     "what": "detection + masked description (descriptors for new keypoints, carried "
                             "ones copied) against full-frame detection + description of every keypoint",
                     "stage_ms_per_step": {"masked": {k: v / max(1, prof_dm["batches"])
                                                      for k, v in prof_dm["ms"].items()},
                                           "full": {k: v / max(1, prof_df["batches"])
                                                    for k, v in prof_df["ms"].items()}}},
        "active_bin_fraction": act, "keypoints_per_step": kp_masked,
        "stage_ms_per_step": {k: v / max(1, prof["batches"]) for k, v in stage_ms.items()},
        "latency_ms": {"p50": p50, "p99": p99, "frames": len(lat_ms),
                       "what": "fkd_push_frame (device frame) + fkd_get_keypoints, host clock"},
        "e2e": {"value": e2e_fps, "unit": "frames/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "roofline": roof,
        # per step: pyramid, (layer sums for a mask layer above c_0), mask,
        # worklist, detect, count, emit
        "gpu_launches": (6 + (1 if cfg.mask_layer != 0 else 0)) * args.steps,
        "clocks": clk,
        "cpu_baseline": cpu,
        "wall_s_timed_region": t_wall,
    }
    if world == 1 and not args.no_groups:
        # the batched and the stress workloads at their stated sizes, each with
        # its own clock record (one GPU: under torchrun only the clip runs)
        line["config3"], _, _ = config3_workload(torch, fkd, dev)
        line["config5"], _, _ = config5_workload(torch, fkd, dev)
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
