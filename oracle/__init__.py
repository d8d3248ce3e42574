"""CPU oracle of the masked keypoint detector of arXiv 1503.06959.

TEST INFRASTRUCTURE ONLY. The oracle is a plain single-threaded C library
(``fkd_oracle.c``) that restates the paper's method step by step; this module
compiles it with gcc and wraps it with ctypes. Only the test suite, the smoke
check and the benchmark's CPU-baseline leg may import it. It shares no code
with the CUDA library and never imports it.

Pinned by ``tests/test_oracle_pins.py`` against what the paper and the
mathematics fix (brute-force segment tests, closed forms, symmetries, Eq. 1
special cases, hand-computed pyramids and bins, descriptor bits against a
library box filter, a hand-computed edge and rotations). The whole-pipeline keypoint
sets are not pinned to any value the paper prints: the paper prints none.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fkd_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

KEYPOINT_DTYPE = np.dtype(
    [("x", "<u2"), ("y", "<u2"), ("layer", "u1"), ("score", "u1"), ("flags", "<u2")]
)

MASK_FULL, MASK_ID, MASK_KB, MASK_IDP = 0, 1, 2, 3


class _Params(ctypes.Structure):
    _fields_ = [
        ("N_r", ctypes.c_int), ("N_c", ctypes.c_int), ("T_I", ctypes.c_int),
        ("T_H", ctypes.c_int), ("O", ctypes.c_int), ("intra", ctypes.c_int),
        ("t", ctypes.c_int), ("mask_mode", ctypes.c_int), ("mask_layer", ctypes.c_int),
        ("nms_scale", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liborc.so`` (plain C11, -O2)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    c_int, c_size, vp = ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p
    ip = ctypes.POINTER(ctypes.c_int)
    lib.orc_num_layers.argtypes = [c_int, c_int]
    lib.orc_layer_geom.argtypes = [c_int, c_int, c_int, c_int, c_int, ip, ip, ip]
    lib.orc_pyramid_bytes.argtypes = [c_int, c_int, c_int, c_int]
    lib.orc_pyramid_bytes.restype = c_size
    lib.orc_build_pyramid.argtypes = [vp, c_int, c_int, c_int, c_int, vp]
    lib.orc_score.argtypes = [vp, c_int, c_int, c_int, c_int]
    lib.orc_score_image.argtypes = [vp, c_int, c_int, vp]
    lib.orc_block_of.argtypes = [c_int] * 7
    lib.orc_stream_create.argtypes = [ctypes.POINTER(_Params), c_int, c_int, ctypes.POINTER(vp)]
    lib.orc_stream_destroy.argtypes = [vp]
    lib.orc_stream_push.argtypes = [vp, vp, c_size, vp]
    lib.orc_stream_num_keypoints.argtypes = [vp]
    lib.orc_stream_num_keypoints.restype = c_size
    lib.orc_stream_keypoints.argtypes = [vp, vp]
    lib.orc_describe.argtypes = [vp, c_int, c_int, c_int, c_int, vp, c_int, vp]
    lib.orc_stream_set_descriptor.argtypes = [vp, vp, c_int]
    lib.orc_stream_descriptors.argtypes = [vp, vp]
    lib.orc_stream_mask.argtypes = [vp, vp]
    lib.orc_stream_block_sums.argtypes = [vp, vp]
    lib.orc_stream_frame_index.argtypes = [vp]
    lib.orc_stream_frame_index.restype = ctypes.c_long
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def num_layers(O: int, intra: int) -> int:
    return _load().orc_num_layers(O, intra)


def layer_geom(W: int, H: int, O: int, intra: int, layer: int):
    """(w, h, S) of a pyramid layer; S = 2 * scale."""
    w, h, S = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    rc = _load().orc_layer_geom(W, H, O, intra, layer, ctypes.byref(w), ctypes.byref(h), ctypes.byref(S))
    if rc != 0:
        raise ValueError("layer out of range")
    return w.value, h.value, S.value


def pyramid(frame: np.ndarray, O: int, intra: int):
    """List of uint8 layers (layer 0 is the frame itself)."""
    frame = np.ascontiguousarray(frame, dtype=np.uint8)
    H, W = frame.shape
    lib = _load()
    out = np.zeros(lib.orc_pyramid_bytes(W, H, O, intra), np.uint8)
    lib.orc_build_pyramid(_ptr(frame), W, H, O, intra, _ptr(out))
    layers, off = [], 0
    for l in range(num_layers(O, intra)):
        w, h, _ = layer_geom(W, H, O, intra, l)
        layers.append(out[off:off + w * h].reshape(h, w))
        off += w * h
    return layers


def score(img: np.ndarray, x: int, y: int) -> int:
    img = np.ascontiguousarray(img, dtype=np.uint8)
    h, w = img.shape
    return _load().orc_score(_ptr(img), w, h, x, y)


def score_image(img: np.ndarray) -> np.ndarray:
    img = np.ascontiguousarray(img, dtype=np.uint8)
    h, w = img.shape
    out = np.zeros((h, w), np.uint8)
    _load().orc_score_image(_ptr(img), w, h, _ptr(out))
    return out


def describe(img: np.ndarray, x: int, y: int, pattern: np.ndarray) -> np.ndarray:
    """Binary descriptor of pixel (x, y) of a layer: D/8 bytes, bit i in byte
    i // 8 at bit i % 8 (pattern: D x 4 int8 rows (ax, ay, bx, by))."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    pat = np.ascontiguousarray(pattern, dtype=np.int8)
    h, w = img.shape
    D = pat.shape[0]
    out = np.zeros(D // 8, np.uint8)
    if _load().orc_describe(_ptr(img), w, h, x, y, _ptr(pat), D, _ptr(out)) != 0:
        raise ValueError("invalid descriptor arguments")
    return out


def block_of(x: int, y: int, S: int, W: int, H: int, N_r: int, N_c: int) -> int:
    return _load().orc_block_of(x, y, S, W, H, N_r, N_c)


class Stream:
    """One video stream run through the oracle, frame by frame."""

    def __init__(self, W: int, H: int, *, N_r: int, N_c: int, T_I: int = 4, T_H: int = 1,
                 O: int = 1, intra: int = 0, t: int = 20, mask_mode: int = MASK_ID,
                 mask_layer: int = 0, nms_scale: int = 0, pattern: np.ndarray | None = None):
        self.W, self.H, self.N_r, self.N_c = W, H, N_r, N_c
        p = _Params(N_r, N_c, T_I, T_H, O, intra, t, mask_mode, mask_layer, nms_scale)
        self._O, self._intra = O, intra
        h = ctypes.c_void_p()
        if _load().orc_stream_create(ctypes.byref(p), W, H, ctypes.byref(h)) != 0:
            raise ValueError("invalid oracle stream parameters")
        self._h = h
        self._D = 0
        if pattern is not None:
            pat = np.ascontiguousarray(pattern, dtype=np.int8)
            if _load().orc_stream_set_descriptor(h, _ptr(pat), pat.shape[0]) != 0:
                raise ValueError("invalid descriptor pattern")
            self._D = pat.shape[0]

    def push(self, frame: np.ndarray, mask_override: np.ndarray | None = None):
        frame = np.ascontiguousarray(frame, dtype=np.uint8)
        assert frame.shape == (self.H, self.W)
        m = None
        if mask_override is not None:
            m = np.ascontiguousarray(mask_override, dtype=np.uint8).reshape(-1)
            assert m.size == self.N_r * self.N_c
        rc = _load().orc_stream_push(self._h, _ptr(frame), self.W,
                                     _ptr(m) if m is not None else None)
        if rc != 0:
            raise RuntimeError("oracle push failed")

    def pixel_mask(self, layer: int) -> np.ndarray:
        """IDP mode: the last frame's per-pixel mask of a layer (h x w, 0/1)."""
        lib = _load()
        W, H = self.W, self.H
        w, h, _ = layer_geom(W, H, self._O, self._intra, layer)
        out = np.zeros((h, w), np.uint8)
        if lib.orc_stream_pixel_mask(self._h, layer, _ptr(out)) != 0:
            raise ValueError("layer out of range")
        return out

    def keypoints(self) -> np.ndarray:
        lib = _load()
        n = lib.orc_stream_num_keypoints(self._h)
        out = np.zeros(n, KEYPOINT_DTYPE)
        if n:
            lib.orc_stream_keypoints(self._h, _ptr(out))
        return out

    def descriptors(self) -> np.ndarray:
        """Descriptors of the last frame's keypoints (n x D/8 uint8, their order)."""
        lib = _load()
        n = lib.orc_stream_num_keypoints(self._h)
        out = np.zeros((n, self._D // 8), np.uint8)
        if not self._D or lib.orc_stream_descriptors(self._h, _ptr(out)) != 0:
            raise ValueError("description is off")
        return out

    def mask(self) -> np.ndarray:
        out = np.zeros(self.N_r * self.N_c, np.uint8)
        _load().orc_stream_mask(self._h, _ptr(out))
        return out.reshape(self.N_r, self.N_c)

    def block_sums(self) -> np.ndarray:
        out = np.zeros(self.N_r * self.N_c, np.uint64)
        _load().orc_stream_block_sums(self._h, _ptr(out))
        return out.reshape(self.N_r, self.N_c)

    def close(self):
        if self._h:
            _load().orc_stream_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
