"""Oracle runs in a pool of CPU processes, for the parity tests at the
benchmark sizes (many streams, large frames).

Test infrastructure only: every function here runs the CPU oracle on frames
it is given (or regenerates from the seeded generator) and returns keypoint
sets and masks; nothing here touches the CUDA library. The pool uses the
"spawn" start method, so a worker never inherits a CUDA context.
"""
from __future__ import annotations

import concurrent.futures
import multiprocessing
import os

import numpy as np


def pool(max_workers: int | None = None) -> concurrent.futures.ProcessPoolExecutor:
    n = max_workers or max(1, min(16, os.cpu_count() or 1))
    return concurrent.futures.ProcessPoolExecutor(max_workers=n,
                                                  mp_context=multiprocessing.get_context("spawn"))


def run_frames(W: int, H: int, params: dict, frames: np.ndarray):
    """Keypoint sets and masks of `frames` (in order, from the stream's first
    frame) through one oracle stream."""
    import oracle
    s = oracle.Stream(W, H, **params)
    kps, masks = [], []
    for f in frames:
        s.push(f)
        kps.append(s.keypoints())
        masks.append(s.mask())
    s.close()
    return kps, masks


def run_generated(cfg, config_id: int, stream: int, count: int, params: dict):
    """As run_frames on the first `count` frames of stream `stream` of a
    workload, regenerated in the worker from its seed."""
    from paper_1503_06959_gb300 import synth
    frames = synth.source_for(cfg, config_id, stream).frames(count)
    return run_frames(cfg.W, cfg.H, params, frames)


def params_of(cfg, mask_mode: int, mask_layer: int | None = None) -> dict:
    """Oracle parameters of a workload's stream configuration."""
    return dict(N_r=cfg.N_r, N_c=cfg.N_c, T_I=cfg.T_I, O=cfg.O, intra=cfg.intra, t=cfg.t,
                mask_mode=mask_mode, mask_layer=cfg.mask_layer if mask_layer is None else mask_layer)
