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
around each kernel on the launching stream, the SM clocks sampled during the
timed region, and the CPU oracle timed on a bounded sample on this host.

--impl reference times the CPU oracle (single-threaded C, the correctness
reference) on the same workload, a bounded number of frames per step.
"""
from __future__ import annotations

import argparse
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


def profile_counters(kernel: str):
    """Counters of the committed ncu summary of `kernel` on this workload, if
    the kernel's sources are unchanged since it was taken (else None)."""
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
    got = {k: re.search(k + r": (\S+)", text) for k in
           ("source_sha256", "traffic_bytes_per_launch", "alu_warp_inst_per_launch")}
    if not got["source_sha256"] or got["source_sha256"].group(1) != m.hexdigest()[:16]:
        return None
    return {k: float(v.group(1)) for k, v in got.items() if v and k != "source_sha256"}


def workload_desc(cfg, frames):
    return (f"{cfg.W}x{cfg.H} uint8 synthetic video, {frames} frames per step, O={cfg.O}"
            f"{' + intra-octaves' if cfg.intra else ''}, {cfg.N_c}x{cfg.N_r} bins (cols x rows), "
            f"t={cfg.t}, T_I={cfg.T_I}, intensity-difference mask")


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
                      intra=cfg.intra, t=cfg.t, mask_mode=oracle.MASK_ID)
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
                          intra=cfg.intra, t=cfg.t, mask_mode=oracle.MASK_ID)
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
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_1503_06959_gb300 import fkd

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
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
    frames_np = synth.source_for(cfg, 2, stream=rank).frames(T)
    frames = torch.from_numpy(frames_np).to(dev)
    torch_stream = torch.cuda.current_stream()
    handle = torch_stream.cuda_stream
    common = dict(N_r=cfg.N_r, N_c=cfg.N_c, T_I=cfg.T_I, O=cfg.O, intra=cfg.intra, t=cfg.t,
                  T_max=T, cuda_stream=handle)
    cap = T * 32768
    out = torch.empty(cap, dtype=torch.int64, device=dev)
    offsets = torch.empty(T + 1, dtype=torch.int32, device=dev)
    masks = torch.empty((T, cfg.N_r, cfg.N_c), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(stream_obj, steps, warmup, profile=False):
        def step():
            stream_obj.reset()
            stream_obj.push_frames(frames, out=out, offsets=offsets, masks=masks)
        for _ in range(warmup):
            step()
        stream_obj.synchronize()
        if profile:
            stream_obj.profile_read(reset=True)
            stream_obj.profile_enable(True)
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
        prof = None
        if profile:
            prof = stream_obj.profile_read(reset=True)
            stream_obj.profile_enable(False)
        ms = sum(a.elapsed_time(b) for a, b in evs)
        return ms, prof

    masked = fkd.Stream(cfg.W, cfg.H, mask_mode=fkd.FKD_MASK_ID, **common)
    full = fkd.Stream(cfg.W, cfg.H, mask_mode=fkd.FKD_MASK_FULL, **common)

    # warm up and check parity of the first frames against the oracle once
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    t_wall0 = time.perf_counter()
    ms, prof = timed(masked, args.steps, args.warmup, profile=True)
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop() if clocks else None
    off_masked = offsets.cpu().numpy().astype(np.int64)
    kp_masked = int(off_masked[T] - off_masked[0])
    act = masks.float().mean().item()

    ms_full, prof_full = timed(full, max(3, args.steps // 2), 3, profile=True)
    off_full = offsets.cpu().numpy().astype(np.int64)
    kp_full = int(off_full[T] - off_full[0])

    # max over ranks
    t_local = torch.tensor([ms, ms_full], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(t_local, op=dist.ReduceOp.MAX)
    ms, ms_full = t_local.tolist()
    value = world * T * args.steps / (ms / 1e3)
    full_fps = world * T * max(3, args.steps // 2) / (ms_full / 1e3)

    # frame-by-frame latency (device frames): push_frame + get_keypoints per frame
    lat = fkd.Stream(cfg.W, cfg.H, mask_mode=fkd.FKD_MASK_ID, N_r=cfg.N_r, N_c=cfg.N_c,
                     T_I=cfg.T_I, O=cfg.O, intra=cfg.intra, t=cfg.t, cuda_stream=handle)
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
    e2e_t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_fps = world * T * e2e_steps / e2e_t.item()
    h2d = T * cfg.W * cfg.H
    d2h = int(hoff[T] - hoff[0]) * 8 + (T + 1) * 4 + T * cfg.N_r * cfg.N_c

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # roofline of the dominant kernel (CUDA events around each launch)
    pk, pk_kind = peaks()
    stage_ms = prof["ms"]
    dom = max(stage_ms, key=stage_ms.get)
    launches = max(1, prof["launches"][dom])
    dur_s = stage_ms[dom] / launches / 1e3
    layer_px = sum(masked.layer_info(l)[0] * masked.layer_info(l)[1]
                   for l in range(masked.num_layers()))
    if dom == "detect":
        # one input byte per pixel of each processed tile, one bitmap bit out
        bytes_per_launch = prof["tile_pixels"] / launches * (1 + 1 / 8)
        bytes_desc = "layer pixels of the processed detection tiles x (1 B read + 1/8 B bitmap)"
    elif dom == "pyramid":
        bytes_per_launch = prof["frames"] / launches * (2 * cfg.W * cfg.H + (layer_px - cfg.W * cfg.H))
        bytes_desc = "per frame: c0 of I_n and I_{n-1} read, layers >= 1 written"
    else:
        bytes_per_launch = prof["frames"] / launches * layer_px / 8 * 2
        bytes_desc = "per frame: keypoint bitmap words read and written"
    achieved = bytes_per_launch / dur_s / 1e9
    counters = profile_counters(dom) if T == cfg.frames else None
    hbm = {"achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
           "frac": achieved / pk["hbm_gbs"], "peak_source": f"{pk_kind} hbm_gbs",
           "bytes_per_launch": bytes_per_launch, "bytes": bytes_desc}
    traffic = counters.get("traffic_bytes_per_launch") if counters else None
    alu_inst = counters.get("alu_warp_inst_per_launch") if counters else None
    if alu_inst:
        # integer ALU pipe: 2 warp instructions per clock per SM (measured with a
        # throughput probe of IADD3 / PRMT / 16-bit min-max), 152 SMs, max SM clock
        sm_clk = pk.get("sm_max_mhz", 2070.0) * 1e6
        peak_alu = 152 * 2 * sm_clk / 1e9
        ach_alu = alu_inst / dur_s / 1e9
        roof = {"kernel": dom, "bound": "alu", "achieved": ach_alu, "peak": peak_alu,
                "unit": "G warp-instructions/s (integer ALU pipe)", "frac": ach_alu / peak_alu,
                "traffic": traffic, "alu_warp_inst_per_launch": alu_inst,
                "peak_source": "152 SMs x 2 ALU warp-instructions/clk x sm_max_mhz",
                "launch_ms": dur_s * 1e3, "hbm": hbm}
    else:
        roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / pk["hbm_gbs"], "traffic": traffic,
                "peak_source": f"{pk_kind} hbm_gbs", "bytes_per_launch": bytes_per_launch,
                "bytes": bytes_desc, "launch_ms": dur_s * 1e3}

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
                   "parallelism": f"one stream per GPU x {world}"},
        "mpix_per_s": value * cfg.W * cfg.H / 1e6,
        "full_frame": {"value": full_fps, "unit": "frames/s", "keypoints_per_step": kp_full,
                       "stage_ms_per_step": {k: v / max(1, prof_full["batches"])
                                             for k, v in prof_full["ms"].items()}},
        "masked_over_full": value / full_fps,
        "active_bin_fraction": act, "keypoints_per_step": kp_masked,
        "stage_ms_per_step": {k: v / max(1, prof["batches"]) for k, v in stage_ms.items()},
        "latency_ms": {"p50": p50, "p99": p99, "frames": len(lat_ms),
                       "what": "fkd_push_frame (device frame) + fkd_get_keypoints, host clock"},
        "e2e": {"value": e2e_fps, "unit": "frames/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "roofline": roof,
        "gpu_launches": 6 * args.steps,
        "clocks": clk,
        "cpu_baseline": cpu,
        "wall_s_timed_region": t_wall,
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
