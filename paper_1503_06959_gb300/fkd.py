"""ctypes binding of the C ABI in ``include/fkd.h`` (names kept).

Argument marshalling only: every step of the detector runs in ``libfkd.so``.
Host frames are numpy arrays; device frames and outputs are torch CUDA
tensors (torch is used only for device memory and streams). There is no
fallback: if the CUDA library cannot be loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

FKD_OK, FKD_E_ARG, FKD_E_CAPACITY, FKD_E_BUDGET, FKD_E_CUDA, FKD_E_TIMEOUT, FKD_E_STATE = (
    0, -1, -2, -3, -4, -5, -6)
FKD_MASK_FULL, FKD_MASK_ID, FKD_MASK_KB, FKD_MASK_IDP = 0, 1, 2, 3
FKD_VERSION = 3
FKD_KP_PROPAGATED = 1

KEYPOINT_DTYPE = np.dtype(
    [("x", "<u2"), ("y", "<u2"), ("layer", "u1"), ("score", "u1"), ("flags", "<u2")])

EXPORTS = [
    "fkd_last_error", "fkd_params_default", "fkd_create_stream", "fkd_destroy_stream",
    "fkd_num_layers", "fkd_layer_info", "fkd_push_frame", "fkd_get_keypoints", "fkd_get_mask",
    "fkd_push_frames", "fkd_synchronize", "fkd_frame_count", "fkd_device_keypoints",
    "fkd_reset_stream", "fkd_profile_enable", "fkd_profile_read", "fkd_id_mask_noalloc",
    "fkd_group_create", "fkd_group_destroy", "fkd_group_add_stream", "fkd_group_remove_stream",
    "fkd_group_tick", "fkd_group_use_graph", "fkd_group_synchronize", "fkd_group_get_keypoints",
    "fkd_group_get_mask", "fkd_group_device_keypoints", "fkd_group_profile_enable",
    "fkd_group_profile_read", "fkd_server_create", "fkd_server_destroy", "fkd_server_open_stream",
    "fkd_server_close_stream", "fkd_server_submit", "fkd_server_poll", "fkd_server_drain",
    "fkd_server_get_stats", "fkd_get_launch_config", "fkd_set_launch_config", "fkd_autotune",
    "fkd_group_get_launch_config", "fkd_group_set_launch_config", "fkd_group_autotune",
    "fkd_get_pixel_mask", "fkd_set_descriptor", "fkd_get_descriptors", "fkd_group_set_descriptor",
    "fkd_group_get_descriptors", "fkd_server_set_descriptor", "fkd_server_get_descriptors",
    "fkd_check_build", "fkd_check_guards", "fkd_group_check_guards",
    "fkd_server_submit_ref", "fkd_server_keep_results", "fkd_server_replay",
]
STAGES = ["pyramid", "mask", "worklist", "detect", "count", "emit", "describe"]


class fkd_params(ctypes.Structure):
    _fields_ = [("version", ctypes.c_uint32)] + [
        (n, ctypes.c_int32) for n in
        ("N_r", "N_c", "T_I", "T_H", "O", "intra", "t", "n", "mask_mode", "mask_layer",
         "K_max", "T_max", "nms_scale")]


class fkd_profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 7), ("launches", ctypes.c_uint64 * 7),
                ("batches", ctypes.c_uint64), ("frames", ctypes.c_uint64),
                ("tiles", ctypes.c_uint64), ("tile_pixels", ctypes.c_uint64)]


class fkd_server_stats(ctypes.Structure):
    _fields_ = [("frames_done", ctypes.c_uint64), ("ticks", ctypes.c_uint64),
                ("rejected_frames", ctypes.c_uint64), ("rejected_streams", ctypes.c_uint64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("fps", ctypes.c_double), ("mean_batch", ctypes.c_double),
                ("bytes_in_use", ctypes.c_size_t), ("budget_bytes", ctypes.c_size_t)]


class fkd_launch_config(ctypes.Structure):
    _fields_ = [("tile_h", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32)]


def _lc_dict(c: fkd_launch_config) -> dict:
    return {"tile_w": 128, "tile_h": c.tile_h, "warps_per_cta": c.warps_per_cta,
            "ctas_per_sm": c.ctas_per_sm}


def _lc(cfg: dict) -> fkd_launch_config:
    return fkd_launch_config(cfg["tile_h"], cfg["warps_per_cta"], cfg["ctas_per_sm"])


class FkdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fkd error {code}: {msg}")
        self.code = code


_lib = None


def check_build_requested() -> bool:
    """FKD_CHECK=1 in the environment selects the debug library
    libfkd_check.so (index checks in the kernels, guard-banded allocations)."""
    return os.environ.get("FKD_CHECK", "0") not in ("", "0")


def load(build: bool = True) -> ctypes.CDLL:
    """Load libfkd.so, or libfkd_check.so when FKD_CHECK=1 (building it first
    if asked). Raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    check = check_build_requested()
    path = _build.build(check=check) if build else (_build.LIB_CHECK if check else _build.LIB)
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run build() first")
    lib = ctypes.CDLL(path)
    vp, c_int, c_size = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    P = ctypes.POINTER
    lib.fkd_last_error.restype = ctypes.c_char_p
    lib.fkd_params_default.argtypes = [P(fkd_params)]
    lib.fkd_create_stream.argtypes = [P(fkd_params), c_int, c_int, vp, P(vp)]
    lib.fkd_destroy_stream.argtypes = [vp]
    lib.fkd_num_layers.argtypes = [vp, P(c_int)]
    lib.fkd_layer_info.argtypes = [vp, c_int, P(c_int), P(c_int), P(c_int)]
    lib.fkd_push_frame.argtypes = [vp, vp, c_size, c_int]
    lib.fkd_get_keypoints.argtypes = [vp, vp, c_size, P(c_size)]
    lib.fkd_get_mask.argtypes = [vp, vp]
    lib.fkd_push_frames.argtypes = [vp, vp, c_size, c_size, c_int, c_int, vp, c_size, vp, vp, c_int]
    lib.fkd_synchronize.argtypes = [vp]
    lib.fkd_frame_count.argtypes = [vp, P(ctypes.c_int64)]
    lib.fkd_device_keypoints.argtypes = [vp, P(vp), P(vp)]
    lib.fkd_reset_stream.argtypes = [vp]
    lib.fkd_profile_enable.argtypes = [vp, c_int]
    lib.fkd_profile_read.argtypes = [vp, P(fkd_profile), c_int]
    lib.fkd_id_mask_noalloc.argtypes = [vp, vp, c_int, c_int, c_size, c_int, c_int, c_int, vp, vp]
    lib.fkd_group_create.argtypes = [c_int, c_int, vp, P(vp)]
    lib.fkd_group_destroy.argtypes = [vp]
    lib.fkd_group_add_stream.argtypes = [vp, P(fkd_params), c_int, c_int, P(c_int), P(c_size)]
    lib.fkd_group_remove_stream.argtypes = [vp, c_int]
    lib.fkd_group_tick.argtypes = [vp, c_int, P(c_int), P(vp), P(c_size)]
    lib.fkd_group_use_graph.argtypes = [vp, c_int]
    lib.fkd_group_synchronize.argtypes = [vp]
    lib.fkd_group_get_keypoints.argtypes = [vp, c_int, vp, c_size, P(c_size)]
    lib.fkd_group_get_mask.argtypes = [vp, c_int, vp]
    lib.fkd_group_device_keypoints.argtypes = [vp, c_int, P(vp), P(vp)]
    lib.fkd_group_profile_enable.argtypes = [vp, c_int]
    lib.fkd_group_profile_read.argtypes = [vp, P(fkd_profile), c_int]
    lib.fkd_server_create.argtypes = [c_int, c_int, c_size, c_size, P(vp)]
    lib.fkd_server_destroy.argtypes = [vp]
    lib.fkd_server_open_stream.argtypes = [vp, P(fkd_params), c_int, c_int, P(c_int)]
    lib.fkd_server_close_stream.argtypes = [vp, c_int]
    lib.fkd_server_submit.argtypes = [vp, c_int, vp, c_size, ctypes.c_int64]
    lib.fkd_server_poll.argtypes = [vp, c_int, P(ctypes.c_int64), vp, c_size, P(c_size)]
    lib.fkd_server_drain.argtypes = [vp, c_int]
    lib.fkd_server_get_stats.argtypes = [vp, P(fkd_server_stats), c_int]
    lib.fkd_get_pixel_mask.argtypes = [vp, c_int, vp]
    lib.fkd_set_descriptor.argtypes = [vp, vp, c_int]
    lib.fkd_get_descriptors.argtypes = [vp, vp, c_size, P(c_size), c_int]
    lib.fkd_group_set_descriptor.argtypes = [vp, c_int, vp, c_int]
    lib.fkd_group_get_descriptors.argtypes = [vp, c_int, vp, c_size, P(c_size), c_int]
    lib.fkd_server_set_descriptor.argtypes = [vp, c_int, vp, c_int]
    lib.fkd_server_get_descriptors.argtypes = [vp, c_int, vp, c_size, P(c_size)]
    lib.fkd_get_launch_config.argtypes = [vp, P(fkd_launch_config)]
    lib.fkd_set_launch_config.argtypes = [vp, P(fkd_launch_config)]
    lib.fkd_server_submit_ref.argtypes = [vp, c_int, vp, c_size, ctypes.c_int64]
    lib.fkd_server_keep_results.argtypes = [vp, c_int]
    lib.fkd_server_replay.argtypes = [vp, c_int, P(c_int), P(vp), P(c_size), P(ctypes.c_int64),
                                      P(ctypes.c_uint64)]
    lib.fkd_check_build.argtypes = []
    lib.fkd_check_guards.argtypes = [vp]
    lib.fkd_group_check_guards.argtypes = [vp]
    lib.fkd_autotune.argtypes = [vp, vp, c_size, c_size, c_int, c_int, P(fkd_launch_config),
                                 P(ctypes.c_float)]
    lib.fkd_group_get_launch_config.argtypes = [vp, P(fkd_launch_config)]
    lib.fkd_group_set_launch_config.argtypes = [vp, P(fkd_launch_config)]
    lib.fkd_group_autotune.argtypes = [vp, c_int, P(c_int), c_int, P(vp), P(c_size), c_int,
                                       P(fkd_launch_config), P(ctypes.c_float)]
    for name in EXPORTS:
        if name != "fkd_last_error":
            getattr(lib, name).restype = c_int
    _lib = lib
    return lib


def _check(rc: int):
    if rc != FKD_OK:
        raise FkdError(rc, _lib.fkd_last_error().decode())


def _is_torch_cuda(a) -> bool:
    return type(a).__module__.startswith("torch") and getattr(a, "is_cuda", False)


def _ptr(a):
    if a is None:
        return None
    if _is_torch_cuda(a):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


def params_default() -> fkd_params:
    lib = load()
    p = fkd_params()
    _check(lib.fkd_params_default(ctypes.byref(p)))
    return p


class Stream:
    """One video stream: fkd_create_stream ... fkd_destroy_stream.

    Keyword arguments are the fields of fkd_params (paper names); `pattern`
    (D x 4 int8 pairs) turns on masked description (fkd_set_descriptor)."""

    def __init__(self, W: int, H: int, *, N_r: int = 8, N_c: int = 8, T_I: int = 4, T_H: int = 1,
                 O: int = 1, intra: int = 0, t: int = 20, n: int = 9,
                 mask_mode: int = FKD_MASK_ID, mask_layer: int = 0, K_max: int = 65536,
                 T_max: int = 1, cuda_stream: int | None = None, nms_scale: int = 0,
                 pattern=None):
        lib = load()
        p = params_default()
        p.N_r, p.N_c, p.T_I, p.T_H, p.O, p.intra, p.t, p.n = N_r, N_c, T_I, T_H, O, intra, t, n
        p.mask_mode, p.mask_layer, p.K_max, p.T_max = mask_mode, mask_layer, K_max, T_max
        p.nms_scale = nms_scale
        self.params = p
        self.W, self.H, self.N_r, self.N_c = W, H, N_r, N_c
        h = ctypes.c_void_p()
        _check(lib.fkd_create_stream(ctypes.byref(p), W, H, ctypes.c_void_p(cuda_stream or 0),
                                     ctypes.byref(h)))
        self._h = h
        self._D = 0
        if pattern is not None:
            self.set_descriptor(pattern)

    # -- geometry
    def num_layers(self) -> int:
        L = ctypes.c_int()
        _check(_lib.fkd_num_layers(self._h, ctypes.byref(L)))
        return L.value

    def layer_info(self, layer: int):
        w, h, S = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(_lib.fkd_layer_info(self._h, layer, ctypes.byref(w), ctypes.byref(h), ctypes.byref(S)))
        return w.value, h.value, S.value

    # -- one frame at a time
    def push_frame(self, frame):
        on_device = 1 if _is_torch_cuda(frame) else 0
        if not on_device:
            frame = np.ascontiguousarray(frame, dtype=np.uint8)
            pitch = frame.strides[0]
        else:
            assert frame.dtype.itemsize == 1 and frame.stride(1) == 1
            pitch = frame.stride(0)
        assert tuple(frame.shape) == (self.H, self.W)
        _check(_lib.fkd_push_frame(self._h, _ptr(frame), pitch, on_device))

    def get_keypoints(self, cap: int | None = None) -> np.ndarray:
        cap = self.params.K_max if cap is None else cap
        out = np.zeros(cap, KEYPOINT_DTYPE)
        n = ctypes.c_size_t()
        _check(_lib.fkd_get_keypoints(self._h, _ptr(out), cap, ctypes.byref(n)))
        return out[:n.value].copy()

    def get_pixel_mask(self, layer: int) -> np.ndarray:
        """FKD_MASK_IDP: the last frame's per-pixel mask of a layer (h x w, 0/1)."""
        w, h, _ = self.layer_info(layer)
        out = np.zeros((h, w), np.uint8)
        _check(_lib.fkd_get_pixel_mask(self._h, layer, _ptr(out)))
        return out

    def get_mask(self) -> np.ndarray:
        out = np.zeros(self.N_r * self.N_c, np.uint8)
        _check(_lib.fkd_get_mask(self._h, _ptr(out)))
        return out.reshape(self.N_r, self.N_c)

    # -- batches
    def push_frames(self, frames, *, out=None, offsets=None, masks=None, cap: int | None = None,
                    want_masks: bool = True):
        """T consecutive frames in one call.

        Host frames (numpy, T x H x W): returns (records, offsets, masks) as numpy.
        Device frames (torch CUDA uint8, T x H x W): writes into the given
        device tensors ``out`` (records as int64 / 8-byte rows), ``offsets``
        (int32, T+1) and ``masks`` (uint8, T x N_r x N_c, optional) and
        returns immediately (asynchronous)."""
        T = frames.shape[0]
        if _is_torch_cuda(frames):
            assert frames.stride(2) == 1
            pitch, stride = frames.stride(1), frames.stride(0)
            on_device = 1
        else:
            frames = np.asarray(frames)
            if frames.dtype != np.uint8 or frames.strides[2] != 1 or min(frames.strides[:2]) <= 0:
                frames = np.ascontiguousarray(frames, dtype=np.uint8)
            pitch, stride = frames.strides[1], frames.strides[0]  # row pitch and frame stride kept
            on_device = 0
        if out is not None and _is_torch_cuda(out):
            cap = out.numel() * out.element_size() // 8 if cap is None else cap
            _check(_lib.fkd_push_frames(self._h, _ptr(frames), pitch, stride, T, on_device,
                                        _ptr(out), cap, _ptr(offsets), _ptr(masks), 1))
            return out, offsets, masks
        if out is not None:
            # caller-owned host buffers (e.g. pinned): out must be KEYPOINT_DTYPE
            # or 8-byte rows, offsets uint32 (T+1), masks uint8 or None
            cap = out.nbytes // 8 if cap is None else cap
            _check(_lib.fkd_push_frames(self._h, _ptr(frames), pitch, stride, T, on_device,
                                        _ptr(out), cap, _ptr(offsets), _ptr(masks), 0))
            return out, offsets, masks
        cap = T * self.params.K_max if cap is None else cap
        rec = np.zeros(cap, KEYPOINT_DTYPE)
        off = np.zeros(T + 1, np.uint32)
        msk = np.zeros((T, self.N_r, self.N_c), np.uint8) if want_masks else None
        _check(_lib.fkd_push_frames(self._h, _ptr(frames), pitch, stride, T, on_device,
                                    _ptr(rec), cap, _ptr(off), _ptr(msk), 0))
        return rec[:off[T]].copy(), off, msk

    def synchronize(self):
        _check(_lib.fkd_synchronize(self._h))

    # -- masked description
    def set_descriptor(self, pattern):
        """Describe keypoints with a D x 4 int8 pattern of pairs (ax, ay, bx, by);
        None turns description off. Resets the stream."""
        if pattern is None:
            _check(_lib.fkd_set_descriptor(self._h, None, 0))
            self._D = 0
            return
        pat = np.ascontiguousarray(pattern, dtype=np.int8)
        assert pat.ndim == 2 and pat.shape[1] == 4
        _check(_lib.fkd_set_descriptor(self._h, _ptr(pat), pat.shape[0]))
        self._D = pat.shape[0]

    def get_descriptors(self, out=None):
        """Descriptors of the records of the last push (n x D/8 uint8, in record
        order). With a torch CUDA ``out`` (uint8, rows of D/8 bytes) they are
        copied there on the device and ``out[:n]`` is returned."""
        n = ctypes.c_size_t()
        if out is not None and _is_torch_cuda(out):
            _check(_lib.fkd_get_descriptors(self._h, _ptr(out), out.shape[0], ctypes.byref(n), 1))
            return out[:n.value]
        _check(_lib.fkd_get_descriptors(self._h, None, 0, ctypes.byref(n), 0))
        res = np.zeros((n.value, self._D // 8), np.uint8)
        if n.value:
            _check(_lib.fkd_get_descriptors(self._h, _ptr(res), n.value, ctypes.byref(n), 0))
        return res

    def check_guards(self):
        """fkd_check_guards: raises if a guard band of the stream's device
        allocations changed (debug library; a no-op in the release one)."""
        _check(_lib.fkd_check_guards(self._h))

    def frame_count(self) -> int:
        n = ctypes.c_int64()
        _check(_lib.fkd_frame_count(self._h, ctypes.byref(n)))
        return n.value

    def reset(self):
        _check(_lib.fkd_reset_stream(self._h))

    # -- detection launch shape
    def launch_config(self) -> dict:
        c = fkd_launch_config()
        _check(_lib.fkd_get_launch_config(self._h, ctypes.byref(c)))
        return _lc_dict(c)

    def set_launch_config(self, cfg: dict):
        c = _lc(cfg)
        _check(_lib.fkd_set_launch_config(self._h, ctypes.byref(c)))

    def autotune(self, frames, reps: int = 2) -> tuple[dict, float]:
        """Time every launch shape on T device frames (torch CUDA uint8,
        T x H x W), keep the fastest; resets the stream. Returns (shape, ms)."""
        assert _is_torch_cuda(frames) and frames.stride(2) == 1
        c, ms = fkd_launch_config(), ctypes.c_float()
        _check(_lib.fkd_autotune(self._h, _ptr(frames), frames.stride(1), frames.stride(0),
                                 frames.shape[0], reps, ctypes.byref(c), ctypes.byref(ms)))
        return _lc_dict(c), ms.value

    def profile_enable(self, on: bool = True):
        _check(_lib.fkd_profile_enable(self._h, int(on)))

    def profile_read(self, reset: bool = True) -> dict:
        p = fkd_profile()
        _check(_lib.fkd_profile_read(self._h, ctypes.byref(p), int(reset)))
        return {"ms": {STAGES[i]: p.ms[i] for i in range(len(STAGES))},
                "launches": {STAGES[i]: int(p.launches[i]) for i in range(len(STAGES))},
                "batches": int(p.batches), "frames": int(p.frames), "tiles": int(p.tiles),
                "tile_pixels": int(p.tile_pixels)}

    def close(self):
        if getattr(self, "_h", None):
            _lib.fkd_destroy_stream(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """Many streams, one frame of each per tick (fkd_group_*)."""

    def __init__(self, O: int, intra: int, cuda_stream: int | None = None):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.fkd_group_create(O, intra, ctypes.c_void_p(cuda_stream or 0), ctypes.byref(h)))
        self._h = h
        self.O, self.intra = O, intra
        self.streams = {}
        self._desc_bits = {}

    def add_stream(self, W: int, H: int, *, N_r: int = 8, N_c: int = 8, T_I: int = 4,
                   T_H: int = 1, t: int = 20, mask_mode: int = FKD_MASK_ID, mask_layer: int = 0,
                   K_max: int = 65536, nms_scale: int = 0) -> tuple[int, int]:
        p = params_default()
        p.N_r, p.N_c, p.T_I, p.T_H, p.O, p.intra, p.t = N_r, N_c, T_I, T_H, self.O, self.intra, t
        p.mask_mode, p.mask_layer, p.K_max, p.nms_scale = mask_mode, mask_layer, K_max, nms_scale
        sid, nbytes = ctypes.c_int(), ctypes.c_size_t()
        _check(_lib.fkd_group_add_stream(self._h, ctypes.byref(p), W, H, ctypes.byref(sid),
                                         ctypes.byref(nbytes)))
        self.streams[sid.value] = (W, H, N_r, N_c, K_max)
        return sid.value, nbytes.value

    def remove_stream(self, sid: int):
        _check(_lib.fkd_group_remove_stream(self._h, sid))
        self.streams.pop(sid, None)

    def tick(self, ids, frames):
        """frames: torch CUDA uint8 (H x W) tensors, one per id."""
        n = len(ids)
        ia = (ctypes.c_int * n)(*ids)
        fa = (ctypes.c_void_p * n)(*[f.data_ptr() for f in frames])
        pa = (ctypes.c_size_t * n)(*[f.stride(0) for f in frames])
        _check(_lib.fkd_group_tick(self._h, n, ia, fa, pa))

    def check_guards(self):
        """fkd_group_check_guards over every stream of the group."""
        _check(_lib.fkd_group_check_guards(self._h))

    def use_graph(self, on: bool):
        _check(_lib.fkd_group_use_graph(self._h, int(on)))

    def launch_config(self) -> dict:
        c = fkd_launch_config()
        _check(_lib.fkd_group_get_launch_config(self._h, ctypes.byref(c)))
        return _lc_dict(c)

    def set_launch_config(self, cfg: dict):
        c = _lc(cfg)
        _check(_lib.fkd_group_set_launch_config(self._h, ctypes.byref(c)))

    def autotune(self, ids, ticks, reps: int = 2) -> tuple[dict, float]:
        """ticks: list of m lists, each holding one torch CUDA uint8 (H x W)
        frame per id. Times every launch shape over the m ticks, keeps the
        fastest and resets every stream of the group. Returns (shape, ms)."""
        n, m = len(ids), len(ticks)
        ia = (ctypes.c_int * n)(*ids)
        flat = [f for tick in ticks for f in tick]
        assert len(flat) == n * m
        fa = (ctypes.c_void_p * (n * m))(*[f.data_ptr() for f in flat])
        pa = (ctypes.c_size_t * n)(*[f.stride(0) for f in ticks[0]])
        c, ms = fkd_launch_config(), ctypes.c_float()
        _check(_lib.fkd_group_autotune(self._h, n, ia, m, fa, pa, reps, ctypes.byref(c),
                                       ctypes.byref(ms)))
        return _lc_dict(c), ms.value

    def synchronize(self):
        _check(_lib.fkd_group_synchronize(self._h))

    def get_keypoints(self, sid: int, cap: int | None = None) -> np.ndarray:
        if cap is None:
            cap = self.streams[sid][4] if sid in self.streams else 1
        out = np.zeros(cap, KEYPOINT_DTYPE)
        n = ctypes.c_size_t()
        _check(_lib.fkd_group_get_keypoints(self._h, sid, _ptr(out), cap, ctypes.byref(n)))
        return out[:n.value].copy()

    def set_descriptor(self, sid: int, pattern):
        """Masked description for stream `sid` (before its first tick): a D x 4
        int8 pattern of pairs (ax, ay, bx, by); None turns it off."""
        if pattern is None:
            _check(_lib.fkd_group_set_descriptor(self._h, sid, None, 0))
            self._desc_bits.pop(sid, None)
            return
        pat = np.ascontiguousarray(pattern, dtype=np.int8)
        assert pat.ndim == 2 and pat.shape[1] == 4
        _check(_lib.fkd_group_set_descriptor(self._h, sid, _ptr(pat), pat.shape[0]))
        self._desc_bits[sid] = pat.shape[0]

    def get_descriptors(self, sid: int) -> np.ndarray:
        """Descriptors of the stream's last frame (n x D/8 uint8, record order)."""
        n = ctypes.c_size_t()
        _check(_lib.fkd_group_get_descriptors(self._h, sid, None, 0, ctypes.byref(n), 0))
        res = np.zeros((n.value, self._desc_bits.get(sid, 0) // 8), np.uint8)
        if n.value:
            _check(_lib.fkd_group_get_descriptors(self._h, sid, _ptr(res), n.value, ctypes.byref(n), 0))
        return res

    def get_mask(self, sid: int) -> np.ndarray:
        W, H, N_r, N_c, _ = self.streams[sid]
        out = np.zeros(N_r * N_c, np.uint8)
        _check(_lib.fkd_group_get_mask(self._h, sid, _ptr(out)))
        return out.reshape(N_r, N_c)

    def profile_enable(self, on: bool = True):
        _check(_lib.fkd_group_profile_enable(self._h, int(on)))

    def profile_read(self, reset: bool = True) -> dict:
        p = fkd_profile()
        _check(_lib.fkd_group_profile_read(self._h, ctypes.byref(p), int(reset)))
        return {"ms": {STAGES[i]: p.ms[i] for i in range(len(STAGES))},
                "launches": {STAGES[i]: int(p.launches[i]) for i in range(len(STAGES))},
                "batches": int(p.batches), "frames": int(p.frames), "tiles": int(p.tiles),
                "tile_pixels": int(p.tile_pixels)}

    def close(self):
        if getattr(self, "_h", None):
            _lib.fkd_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving loop over many streams (fkd_server_*): submit host frames as
    they arrive, poll keypoints as they finish."""

    def __init__(self, O: int, intra: int, budget_bytes: int, max_tick_keypoints: int = 1 << 22):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.fkd_server_create(O, intra, budget_bytes, max_tick_keypoints, ctypes.byref(h)))
        self._h = h
        self.O, self.intra = O, intra
        self.streams = {}
        self._desc_bits = {}

    def open_stream(self, W: int, H: int, *, N_r: int = 8, N_c: int = 8, T_I: int = 4,
                    T_H: int = 1, t: int = 20, mask_mode: int = FKD_MASK_ID, mask_layer: int = 0,
                    K_max: int = 16384, nms_scale: int = 0) -> int:
        p = params_default()
        p.N_r, p.N_c, p.T_I, p.T_H, p.O, p.intra, p.t = N_r, N_c, T_I, T_H, self.O, self.intra, t
        p.mask_mode, p.mask_layer, p.K_max, p.nms_scale = mask_mode, mask_layer, K_max, nms_scale
        sid = ctypes.c_int()
        _check(_lib.fkd_server_open_stream(self._h, ctypes.byref(p), W, H, ctypes.byref(sid)))
        self.streams[sid.value] = (W, H, K_max)
        return sid.value

    def close_stream(self, sid: int):
        _check(_lib.fkd_server_close_stream(self._h, sid))
        self.streams.pop(sid, None)

    def submit(self, sid: int, frame: np.ndarray, arrival_ns: int = 0):
        frame = np.ascontiguousarray(frame, dtype=np.uint8)
        _check(_lib.fkd_server_submit(self._h, sid, _ptr(frame), frame.strides[0], arrival_ns))

    def submit_ref(self, sid: int, frame, arrival_ns: int = 0):
        """fkd_server_submit_ref: queue a host frame (numpy or pinned torch
        CPU tensor) by reference; it must stay alive until drained."""
        ptr = frame.data_ptr() if hasattr(frame, "data_ptr") else frame.ctypes.data
        pitch = frame.stride(0) if hasattr(frame, "data_ptr") else frame.strides[0]
        _check(_lib.fkd_server_submit_ref(self._h, sid, ctypes.c_void_p(ptr), pitch, arrival_ns))

    def keep_results(self, keep: bool):
        _check(_lib.fkd_server_keep_results(self._h, int(keep)))

    def replay(self, ids, frame_ptrs, pitches, arrival_ns) -> int:
        """fkd_server_replay: submit frame_ptrs[i] (host addresses, kept alive
        by the caller until drain) to ids[i] at arrival_ns[i] (steady clock),
        in C; returns the number of frames dropped for a full queue."""
        n = len(ids)
        ia = np.ascontiguousarray(ids, dtype=np.int32)
        fa = np.ascontiguousarray(frame_ptrs, dtype=np.uint64)
        pa = np.ascontiguousarray(pitches, dtype=np.uint64)
        ta = np.ascontiguousarray(arrival_ns, dtype=np.int64)
        refused = ctypes.c_uint64()
        _check(_lib.fkd_server_replay(self._h, n, ia.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                      fa.ctypes.data_as(ctypes.POINTER(ctypes.c_void_p)),
                                      pa.ctypes.data_as(ctypes.POINTER(ctypes.c_size_t)),
                                      ta.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ctypes.byref(refused)))
        return refused.value

    def poll(self, sid: int):
        """(frame index, keypoints) of the oldest finished frame, or None."""
        cap = self.streams.get(sid, (0, 0, 1))[2]
        out = np.zeros(cap, KEYPOINT_DTYPE)
        idx, n = ctypes.c_int64(), ctypes.c_size_t()
        rc = _lib.fkd_server_poll(self._h, sid, ctypes.byref(idx), _ptr(out), cap, ctypes.byref(n))
        if rc == FKD_E_STATE:
            return None
        _check(rc)
        return idx.value, out[:n.value].copy()

    def set_descriptor(self, sid: int, pattern):
        """Masked description for stream `sid` (before its first frame): a
        D x 4 int8 pattern of pairs (ax, ay, bx, by); None turns it off."""
        if pattern is None:
            _check(_lib.fkd_server_set_descriptor(self._h, sid, None, 0))
            self._desc_bits.pop(sid, None)
            return
        pat = np.ascontiguousarray(pattern, dtype=np.int8)
        assert pat.ndim == 2 and pat.shape[1] == 4
        _check(_lib.fkd_server_set_descriptor(self._h, sid, _ptr(pat), pat.shape[0]))
        self._desc_bits[sid] = pat.shape[0]

    def get_descriptors(self, sid: int) -> np.ndarray:
        """Descriptors of the result the last poll of `sid` returned (n x D/8)."""
        n = ctypes.c_size_t()
        _check(_lib.fkd_server_get_descriptors(self._h, sid, None, 0, ctypes.byref(n)))
        res = np.zeros((n.value, self._desc_bits.get(sid, 0) // 8), np.uint8)
        if n.value:
            _check(_lib.fkd_server_get_descriptors(self._h, sid, _ptr(res), n.value, ctypes.byref(n)))
        return res

    def drain(self, timeout_ms: int = 60000):
        _check(_lib.fkd_server_drain(self._h, timeout_ms))

    def stats(self, reset: bool = False) -> dict:
        st = fkd_server_stats()
        _check(_lib.fkd_server_get_stats(self._h, ctypes.byref(st), int(reset)))
        return {f: getattr(st, f) for f, _ in fkd_server_stats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            _lib.fkd_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def check_build() -> bool:
    """True when the loaded library is the debug build (fkd_check_build)."""
    return bool(load().fkd_check_build())


def id_mask_noalloc(cur, prev, N_r: int, N_c: int, T_I: int, mask_out, cuda_stream: int | None = None):
    """fkd_id_mask_noalloc: the intensity-difference mask of one frame pair
    computed without any device allocation (for callers that manage all
    device memory themselves). cur, prev: torch CUDA uint8 H x W frames with
    the same row stride; mask_out: torch CUDA uint8 tensor of N_r*N_c bytes.
    Asynchronous on `cuda_stream` (default: the legacy default stream)."""
    import torch
    lib = load()
    dev = torch.cuda.current_device()
    for name, t in (("cur", cur), ("prev", prev), ("mask_out", mask_out)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.uint8):
            raise TypeError(f"{name} must be a torch CUDA uint8 tensor")
        if t.device.index != dev:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{dev}")
    H, W = cur.shape
    if tuple(prev.shape) != (H, W) or cur.stride(0) != prev.stride(0):
        raise ValueError("cur and prev must have the same shape and row stride")
    if cur.stride(1) != 1 or prev.stride(1) != 1:
        raise ValueError("frame rows must be contiguous")
    if not mask_out.is_contiguous() or mask_out.numel() != N_r * N_c:
        raise ValueError("mask_out must be a contiguous tensor of N_r * N_c bytes")
    _check(lib.fkd_id_mask_noalloc(_ptr(cur), _ptr(prev), W, H, cur.stride(0), N_r, N_c, T_I,
                                   _ptr(mask_out), ctypes.c_void_p(cuda_stream or 0)))


def split_frames(records: np.ndarray, offsets: np.ndarray):
    """Per-frame keypoint arrays from a batch's concatenated records."""
    base = int(offsets[0])
    return [records[int(offsets[k]) - base:int(offsets[k + 1]) - base]
            for k in range(len(offsets) - 1)]
