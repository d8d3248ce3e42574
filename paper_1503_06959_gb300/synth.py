"""Seeded synthetic video shaped like the paper's hand-held VGA-class clips.

This module only makes inputs: frames and the descriptor's sample pattern.
It holds none of the detector's arithmetic, and both the CUDA path and the
CPU oracle read the same bytes.

Scene recipe (one stream):
  * background: a mid-grey field with 40 rectangles, position and size
    uniform in the frame, intensity uniform in 0..255, Gaussian-blurred with
    sigma 2, rounded and clamped;
  * movers: opaque squares whose texture is uniform 0..255 noise blurred with
    sigma 1, each moving with a seeded direction and speed and bouncing at
    the frame edges;
  * optional camera jitter: every ``jitter_every`` frames the whole scene
    steps by a seeded +-1 px in x and y and stays there;
  * per-frame sensor noise N(0, noise_sigma), rounded and clamped to 0..255;
  * optional static segments: frames inside a static segment freeze the
    movers and the camera (only the sensor noise changes).

Seeds: 1000 + 100 * config + stream.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.ndimage import gaussian_filter


@dataclasses.dataclass
class Mover:
    size: int
    tex: np.ndarray  # float32 (size, size)
    x: float
    y: float
    vx: float
    vy: float


class VideoSource:
    """Frame generator for one stream; ``frame(n)`` must be called in order."""

    def __init__(self, W: int, H: int, *, seed: int, n_rect: int = 40, n_movers: int = 3,
                 mover_size: int | list[int] = 40, speed: tuple[int, int] = (2, 2),
                 noise_sigma: float = 3.0, jitter_every: int = 0,
                 static_segments: tuple[int, int] | None = None):
        self.W, self.H = W, H
        self.rng = np.random.default_rng(seed)
        rng = self.rng
        self.noise_sigma = noise_sigma
        self.jitter_every = jitter_every
        self.static_segments = static_segments  # (segment length, phase: 0 = moving first)
        self.margin = 8
        m = self.margin
        bg = np.full((H + 2 * m, W + 2 * m), 128.0, np.float32)
        for _ in range(n_rect):
            x0, y0 = rng.integers(0, W), rng.integers(0, H)
            w, h = rng.integers(1, W + 1), rng.integers(1, H + 1)
            bg[m + y0:m + y0 + h, m + x0:m + x0 + w] = float(rng.integers(0, 256))
        self.bg = gaussian_filter(bg, 2.0, mode="nearest").astype(np.float32)
        sizes = mover_size if isinstance(mover_size, list) else [mover_size] * n_movers
        self.movers: list[Mover] = []
        for s in sizes:
            s = int(min(s, W - 2, H - 2))
            tex = gaussian_filter(rng.integers(0, 256, (s, s)).astype(np.float32), 1.0,
                                  mode="nearest")
            sp = float(rng.integers(speed[0], speed[1] + 1))
            ang = float(rng.uniform(0.0, 2.0 * math.pi))
            self.movers.append(Mover(s, tex, float(rng.integers(0, W - s + 1)),
                                     float(rng.integers(0, H - s + 1)),
                                     sp * math.cos(ang), sp * math.sin(ang)))
        self.cam = [0, 0]
        self.n = 0

    def _moving(self, n: int) -> bool:
        if self.static_segments is None:
            return True
        seg, phase = self.static_segments
        return ((n // seg) + phase) % 2 == 0

    def _advance(self):
        W, H = self.W, self.H
        for mv in self.movers:
            mv.x += mv.vx
            mv.y += mv.vy
            if mv.x < 0 or mv.x > W - mv.size:
                mv.vx = -mv.vx
                mv.x = min(max(mv.x, 0.0), float(W - mv.size))
            if mv.y < 0 or mv.y > H - mv.size:
                mv.vy = -mv.vy
                mv.y = min(max(mv.y, 0.0), float(H - mv.size))

    def frame(self, n: int) -> np.ndarray:
        assert n == self.n, "frames are generated in order"
        rng = self.rng
        if n > 0 and self._moving(n):
            self._advance()
            if self.jitter_every and n % self.jitter_every == 0:
                self.cam[0] = int(np.clip(self.cam[0] + rng.choice([-1, 1]), -self.margin, self.margin))
                self.cam[1] = int(np.clip(self.cam[1] + rng.choice([-1, 1]), -self.margin, self.margin))
        m, W, H = self.margin, self.W, self.H
        cx, cy = self.cam
        img = self.bg[m + cy:m + cy + H, m + cx:m + cx + W].copy()
        for mv in self.movers:
            x, y = int(round(mv.x)), int(round(mv.y))
            img[y:y + mv.size, x:x + mv.size] = mv.tex[:H - y, :W - x]
        img += rng.normal(0.0, self.noise_sigma, img.shape).astype(np.float32)
        self.n += 1
        return np.clip(np.rint(img), 0, 255).astype(np.uint8)

    def frames(self, count: int) -> np.ndarray:
        return np.stack([self.frame(self.n) for _ in range(count)])


@dataclasses.dataclass(frozen=True)
class StreamConfig:
    W: int
    H: int
    frames: int
    O: int
    intra: int
    t: int
    N_r: int
    N_c: int
    T_I: int
    source: dict
    # layer of the intensity-difference test: -1 = the coarsest octave, the
    # layer the paper's experiments use (Sec. 4); 0 = c_0
    mask_layer: int = -1


def config1() -> StreamConfig:
    """320x240, 20 frames, 3 textured 40x40 movers at 2 px/frame, 1 octave,
    t = 20, 8x8 grid, T_I = 4."""
    return StreamConfig(320, 240, 20, 1, 0, 20, 8, 8, 4,
                        dict(n_movers=3, mover_size=40, speed=(2, 2), noise_sigma=3.0))


def config2() -> StreamConfig:
    """640x480, 300 frames, 6 movers of about 101x101 (20 % of the area) at
    1-4 px/frame, camera jitter every 30 frames, 4 octaves + intra-octaves,
    t = 30, 16 columns x 12 rows, T_I = 4."""
    return StreamConfig(640, 480, 300, 4, 1, 30, 12, 16, 4,
                        dict(n_movers=6, mover_size=101, speed=(1, 4), noise_sigma=3.0,
                             jitter_every=30))


def config3_streams(count_per_res: int = 16) -> list[StreamConfig]:
    """Mixed resolutions, 120 frames, moving-area fraction U[5 %, 60 %]."""
    out = []
    rng = np.random.default_rng(1000 + 300)
    for (W, H) in [(320, 240), (640, 480), (1280, 720), (1920, 1080)]:
        for _ in range(count_per_res):
            frac = float(rng.uniform(0.05, 0.60))
            n_mv = 4
            size = int(math.sqrt(frac * W * H / n_mv))
            out.append(StreamConfig(W, H, 120, 4, 1, 30, 12, 16, 4,
                                    dict(n_movers=n_mv, mover_size=size, speed=(1, 4),
                                         noise_sigma=3.0)))
    return out


def config5() -> StreamConfig:
    """3840x2160, 200 frames alternating 100-frame moving and static segments,
    5 octaves + intra-octaves, sensor noise N(0, 2)."""
    return StreamConfig(3840, 2160, 200, 5, 1, 30, 12, 16, 4,
                        dict(n_movers=12, mover_size=700, speed=(2, 6), noise_sigma=2.0,
                             static_segments=(100, 0)))


def source_for(cfg: StreamConfig, config_id: int, stream: int = 0) -> VideoSource:
    return VideoSource(cfg.W, cfg.H, seed=1000 + 100 * config_id + stream, **cfg.source)


def fill_shared(name: str, count: int, W: int, H: int, seed: int, source: dict) -> None:
    """Write the first `count` frames of the stream VideoSource(W, H, seed,
    **source) into the existing shared-memory block `name` (count x H x W
    uint8), so that several processes can generate streams in parallel."""
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(name=name)  # the creating process unlinks it
    arr = np.ndarray((count, H, W), np.uint8, buffer=shm.buf)
    src = VideoSource(W, H, seed=seed, **source)
    for n in range(count):
        arr[n] = src.frame(n)
    del arr
    shm.close()


DESC_RADIUS = 13  # largest |offset| of a descriptor sample the library accepts


def descriptor_pattern(D: int = 256, seed: int = 7) -> np.ndarray:
    """D sample pairs (ax, ay, bx, by) for the binary descriptor, int8 D x 4.

    The paper names no pattern. This draws each coordinate from an isotropic
    Gaussian of standard deviation (2 * DESC_RADIUS + 1) / 5, rounded and
    clipped to +-DESC_RADIUS (the usual choice for BRIEF-style pair tests).
    These are inputs of the method, drawn once and passed to both sides.
    """
    rng = np.random.default_rng(seed)
    sigma = (2 * DESC_RADIUS + 1) / 5.0
    p = np.rint(rng.normal(0.0, sigma, size=(D, 4)))
    return np.clip(p, -DESC_RADIUS, DESC_RADIUS).astype(np.int8)
