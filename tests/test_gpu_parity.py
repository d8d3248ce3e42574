"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Keypoints (x, y, layer, score, flags), their order and the masks are
integer results: the bar is bit-exact equality, element by element.
"""
import numpy as np
import pytest

import oracle
from paper_1503_06959_gb300 import fkd, synth

pytestmark = pytest.mark.gpu

MODES = {"full": (fkd.FKD_MASK_FULL, oracle.MASK_FULL), "id": (fkd.FKD_MASK_ID, oracle.MASK_ID),
         "kb": (fkd.FKD_MASK_KB, oracle.MASK_KB)}


def run_oracle(frames, **kw):
    s = oracle.Stream(frames.shape[2], frames.shape[1], **kw)
    kps, masks = [], []
    for f in frames:
        s.push(f)
        kps.append(s.keypoints())
        masks.append(s.mask())
    return kps, masks


def assert_same_kp(got, exp, where=""):
    assert len(got) == len(exp), f"{where}: {len(got)} vs {len(exp)} keypoints"
    for field in ("layer", "y", "x", "score", "flags"):
        np.testing.assert_array_equal(got[field], exp[field], err_msg=f"{where}: field {field}")


def params(cfg, mode="id", **over):
    p = dict(N_r=cfg.N_r, N_c=cfg.N_c, T_I=cfg.T_I, O=cfg.O, intra=cfg.intra, t=cfg.t)
    p.update(over)
    return p


def both(p, mode):
    g = dict(p, mask_mode=MODES[mode][0])
    o = dict(p, mask_mode=MODES[mode][1])
    o.pop("K_max", None)
    o.pop("T_max", None)
    return g, o


@pytest.fixture(scope="module")
def clip1():
    cfg = synth.config1()
    return cfg, synth.source_for(cfg, 1).frames(cfg.frames)


@pytest.fixture(scope="module")
def clip2():
    cfg = synth.config2()
    return cfg, synth.source_for(cfg, 2).frames(36)  # includes the camera step at frame 30


@pytest.mark.parametrize("mode", ["id", "full", "kb"])
def test_config1_frame_by_frame(clip1, mode):
    cfg, frames = clip1
    g, o = both(params(cfg), mode)
    exp_kp, exp_m = run_oracle(frames, **o)
    s = fkd.Stream(cfg.W, cfg.H, **g)
    for n, f in enumerate(frames):
        s.push_frame(f)
        assert_same_kp(s.get_keypoints(), exp_kp[n], f"frame {n}")
        np.testing.assert_array_equal(s.get_mask(), exp_m[n])
    if mode == "id":
        assert any(m.sum() < m.size for m in exp_m[1:]), "the clip must have inactive bins"
        assert any((k["flags"] == 1).any() for k in exp_kp), "some keypoints must be carried over"


@pytest.mark.parametrize("mode", ["id", "kb"])
def test_config1_one_batch(clip1, mode):
    cfg, frames = clip1
    g, o = both(params(cfg), mode)
    exp_kp, exp_m = run_oracle(frames, **o)
    s = fkd.Stream(cfg.W, cfg.H, T_max=len(frames), **g)
    rec, off, masks = s.push_frames(frames)
    for n, kp in enumerate(fkd.split_frames(rec, off)):
        assert_same_kp(kp, exp_kp[n], f"frame {n}")
        np.testing.assert_array_equal(masks[n], exp_m[n])


def test_config2_batches_and_frames(clip2):
    """640x480, 4 octaves + intra-octaves: a batch of 13, a batch of 20 and
    3 single frames give the oracle's keypoints on every frame."""
    cfg, frames = clip2
    g, o = both(params(cfg), "id")
    exp_kp, exp_m = run_oracle(frames, **o)
    s = fkd.Stream(cfg.W, cfg.H, T_max=20, **g)
    n = 0
    for T in (13, 20):
        rec, off, masks = s.push_frames(frames[n:n + T])
        for k, kp in enumerate(fkd.split_frames(rec, off)):
            assert_same_kp(kp, exp_kp[n + k], f"frame {n + k}")
            np.testing.assert_array_equal(masks[k], exp_m[n + k])
        n += T
    for f in frames[n:]:
        s.push_frame(f)
        assert_same_kp(s.get_keypoints(), exp_kp[n], f"frame {n}")
        n += 1
    assert sum(len(k) for k in exp_kp) > 1000


def test_config2_full_detection(clip2):
    cfg, frames = clip2
    g, o = both(params(cfg), "full")
    exp_kp, _ = run_oracle(frames[:6], **o)
    s = fkd.Stream(cfg.W, cfg.H, T_max=6, **g)
    rec, off, _ = s.push_frames(frames[:6])
    for k, kp in enumerate(fkd.split_frames(rec, off)):
        assert_same_kp(kp, exp_kp[k], f"frame {k}")
    assert {int(l) for l in rec["layer"]} == set(range(8)), "every layer must yield keypoints"


def push_in_pieces(s, frames, pieces, exp_kp, exp_m):
    """Feed frames as batches of the given sizes (1 = fkd_push_frame) and
    compare every frame with the oracle."""
    n = 0
    for T in pieces:
        if T == 1:
            s.push_frame(frames[n])
            assert_same_kp(s.get_keypoints(), exp_kp[n], f"frame {n}")
            np.testing.assert_array_equal(s.get_mask(), exp_m[n])
        else:
            rec, off, masks = s.push_frames(frames[n:n + T])
            for k, kp in enumerate(fkd.split_frames(rec, off)):
                assert_same_kp(kp, exp_kp[n + k], f"frame {n + k}")
                np.testing.assert_array_equal(masks[k], exp_m[n + k])
        n += T
    assert n == len(frames)


@pytest.mark.parametrize("mask_layer", [-1, 3, 1])
def test_mask_on_coarser_layer(clip2, mask_layer):
    # the change sums of a coarser layer carry the previous batch's last
    # frame across batches, single pushes and the camera step at frame 30
    cfg, frames = clip2
    g, o = both(params(cfg, mask_layer=mask_layer), "id")
    exp_kp, exp_m = run_oracle(frames, **o)
    s = fkd.Stream(cfg.W, cfg.H, T_max=14, **g)
    push_in_pieces(s, frames, [8, 12, 1, 1, 14], exp_kp, exp_m)
    assert any(m.sum() < m.size for m in exp_m[1:]), "the clip must have inactive bins"


@pytest.mark.parametrize("W,H,O,intra,mask_layer", [
    (333, 207, 3, 1, -1), (333, 207, 3, 1, 1), (97, 61, 2, 0, -1), (200, 150, 6, 1, -1)])
def test_coarse_mask_layer_ragged(W, H, O, intra, mask_layer):
    src = synth.VideoSource(W, H, seed=W + H + O, n_rect=10, n_movers=2, mover_size=min(W, H) // 3,
                            speed=(1, 3))
    frames = src.frames(9)
    g, o = both(dict(N_r=5, N_c=7, T_I=2, O=O, intra=intra, t=10, mask_layer=mask_layer), "id")
    exp_kp, exp_m = run_oracle(frames, **o)
    s = fkd.Stream(W, H, T_max=4, **g)
    push_in_pieces(s, frames, [3, 1, 4, 1], exp_kp, exp_m)
    s.reset()
    push_in_pieces(s, frames[:5], [2, 3], exp_kp[:5], exp_m[:5])


@pytest.mark.parametrize("W,H,O,intra,N_r,N_c", [
    (333, 207, 3, 1, 7, 9),     # ragged everywhere: tiles, bins, words, layers
    (97, 61, 2, 1, 30, 97),     # one-pixel-wide bins on c0
    (7, 7, 1, 0, 1, 1),         # a single scorable pixel
    (16, 12, 3, 1, 2, 2),       # layers smaller than the ring
    (1, 1, 1, 1, 1, 1),         # empty layers
    (200, 150, 6, 1, 3, 5),     # six octaves on a small frame
])
def test_ragged_and_degenerate_sizes(W, H, O, intra, N_r, N_c):
    if min(W, H) >= 10:
        src = synth.VideoSource(W, H, seed=W * 7 + H, n_rect=10, n_movers=1,
                                mover_size=min(W, H) // 3, speed=(1, 3))
        frames = src.frames(5)
    else:
        frames = np.random.default_rng(W * 7 + H).integers(0, 256, (5, H, W), dtype=np.uint8)
    p = dict(N_r=N_r, N_c=N_c, T_I=2, O=O, intra=intra, t=10)
    g, o = both(p, "id")
    exp_kp, exp_m = run_oracle(frames, **o)
    s = fkd.Stream(W, H, T_max=3, **g)
    rec, off, masks = s.push_frames(frames[:3])
    for k, kp in enumerate(fkd.split_frames(rec, off)):
        assert_same_kp(kp, exp_kp[k], f"frame {k}")
        np.testing.assert_array_equal(masks[k], exp_m[k])
    for k in (3, 4):
        s.push_frame(frames[k])
        assert_same_kp(s.get_keypoints(), exp_kp[k], f"frame {k}")


@pytest.mark.parametrize("t", [1, 2, 127, 128, 200, 254, 255])
def test_thresholds_extremes(t):
    rng = np.random.default_rng(t)
    frames = np.stack([rng.integers(0, 256, (70, 90), dtype=np.uint8) for _ in range(2)])
    frames[1, :35] = frames[0, :35]  # top half unchanged
    g, o = both(dict(N_r=2, N_c=3, T_I=1, O=2, intra=1, t=t), "id")
    exp_kp, _ = run_oracle(frames, **o)
    s = fkd.Stream(90, 70, T_max=2, **g)
    rec, off, _ = s.push_frames(frames)
    for k, kp in enumerate(fkd.split_frames(rec, off)):
        assert_same_kp(kp, exp_kp[k], f"t={t} frame {k}")


def test_saturated_and_constant_frames():
    frames = np.zeros((4, 64, 80), np.uint8)
    frames[1] = 255
    frames[2, ::2, ::2] = 255  # checkerboard-like extremes
    frames[3, 20:30, 20:30] = 255
    g, o = both(dict(N_r=2, N_c=2, T_I=0, O=2, intra=1, t=1), "id")
    exp_kp, exp_m = run_oracle(frames, **o)
    s = fkd.Stream(80, 64, T_max=4, **g)
    rec, off, masks = s.push_frames(frames)
    for k, kp in enumerate(fkd.split_frames(rec, off)):
        assert_same_kp(kp, exp_kp[k], f"frame {k}")
        np.testing.assert_array_equal(masks[k], exp_m[k])


def test_device_frames_and_unaligned_pitch(clip1):
    """torch CUDA frames, including a view with an odd base and pitch, give
    the same keypoints as host frames."""
    torch = pytest.importorskip("torch")
    cfg, frames = clip1
    g, o = both(params(cfg), "id")
    exp_kp, _ = run_oracle(frames[:6], **o)
    big = torch.zeros((6, cfg.H, cfg.W + 13), dtype=torch.uint8, device="cuda")
    big[:, :, 3:3 + cfg.W] = torch.from_numpy(frames[:6]).cuda()
    view = big[:, :, 3:3 + cfg.W]
    s = fkd.Stream(cfg.W, cfg.H, **g)
    for n in range(3):
        s.push_frame(view[n])
        assert_same_kp(s.get_keypoints(), exp_kp[n], f"frame {n}")
    s2 = fkd.Stream(cfg.W, cfg.H, T_max=3, **g)
    rec, off, _ = s2.push_frames(frames[:3])
    out = torch.zeros(65536, dtype=torch.int64, device="cuda")
    offs = torch.zeros(4, dtype=torch.int32, device="cuda")
    masks = torch.zeros((3, cfg.N_r, cfg.N_c), dtype=torch.uint8, device="cuda")
    s2.push_frames(view[3:6], out=out, offsets=offs, masks=masks)
    s2.synchronize()
    off2 = offs.cpu().numpy().astype(np.int64)
    rec2 = out.cpu().numpy().view(fkd.KEYPOINT_DTYPE)[off2[0]:off2[3]]
    for k, kp in enumerate(fkd.split_frames(rec2, off2)):
        assert_same_kp(kp, exp_kp[3 + k], f"frame {3 + k}")


def test_capacity_errors(clip1):
    cfg, frames = clip1
    g, _ = both(params(cfg), "id")
    s = fkd.Stream(cfg.W, cfg.H, K_max=5, **g)
    s.push_frame(frames[0])
    with pytest.raises(fkd.FkdError) as e:
        s.get_keypoints()
    assert e.value.code == fkd.FKD_E_CAPACITY
    s2 = fkd.Stream(cfg.W, cfg.H, T_max=2, **g)
    with pytest.raises(fkd.FkdError) as e:
        s2.push_frames(frames[:2], cap=10)
    assert e.value.code == fkd.FKD_E_CAPACITY
    # the kept set is whole even when the output was cut: the next frames agree
    _, o = both(params(cfg), "id")
    exp_kp, _ = run_oracle(frames[:4], **o)
    s2.push_frame(frames[2])
    assert_same_kp(s2.get_keypoints(), exp_kp[2], "frame 2 after overflow")


@pytest.mark.parametrize("mode,mask_layer", [("full", 0), ("id", -1), ("id", 0), ("kb", 0)])
def test_scale_space_suppression(clip2, mode, mask_layer):
    # nms_scale = 1: detections must also beat the adjacent layers' windows
    cfg, frames = clip2
    frames = frames[:12]
    g, o = both(params(cfg, mask_layer=mask_layer, nms_scale=1), mode)
    exp_kp, exp_m = run_oracle(frames, **o)
    s = fkd.Stream(cfg.W, cfg.H, T_max=6, **g)
    pieces = [1] * 12 if mode == "kb" else [5, 1, 6]
    push_in_pieces(s, frames, pieces, exp_kp, exp_m)
    # the suppression removes keypoints on every layer pair
    g0, o0 = both(params(cfg, mask_layer=mask_layer), mode)
    plain, _ = run_oracle(frames[:1], **o0)
    assert len(exp_kp[0]) < len(plain[0])


@pytest.mark.parametrize("W,H,O,intra", [(333, 207, 3, 1), (200, 150, 6, 1), (97, 61, 2, 0), (16, 12, 3, 1)])
def test_scale_space_suppression_ragged(W, H, O, intra):
    src = synth.VideoSource(W, H, seed=3 * W + H, n_rect=12, n_movers=2, mover_size=max(4, min(W, H) // 3),
                            speed=(1, 3))
    frames = src.frames(6)
    g, o = both(dict(N_r=3, N_c=4, T_I=2, O=O, intra=intra, t=8, nms_scale=1, mask_layer=-1), "id")
    exp_kp, exp_m = run_oracle(frames, **o)
    s = fkd.Stream(W, H, T_max=3, **g)
    push_in_pieces(s, frames, [3, 1, 2], exp_kp, exp_m)


def pixel_masks_equal(s, ref, L):
    for l in range(L):
        np.testing.assert_array_equal(s.get_pixel_mask(l), ref.pixel_mask(l), err_msg=f"layer {l}")


@pytest.mark.parametrize("T_I,mask_nms", [(8, 0), (4, 1), (20, 0)])
def test_per_pixel_mask(clip2, T_I, mask_nms):
    # Eq. 2 per pixel of every layer; batches, single pushes, the camera step
    cfg, frames = clip2
    frames = frames[:34]
    kw = dict(N_r=cfg.N_r, N_c=cfg.N_c, T_I=T_I, O=cfg.O, intra=cfg.intra, t=cfg.t, nms_scale=mask_nms)
    ref = oracle.Stream(cfg.W, cfg.H, mask_mode=oracle.MASK_IDP, **kw)
    exp = []
    for f in frames:
        ref.push(f)
        exp.append(ref.keypoints())
    s = fkd.Stream(cfg.W, cfg.H, mask_mode=fkd.FKD_MASK_IDP, T_max=12, **kw)
    n = 0
    for T in [10, 1, 1, 12, 10]:
        if T == 1:
            s.push_frame(frames[n])
            assert_same_kp(s.get_keypoints(), exp[n], f"frame {n}")
        else:
            rec, off, _ = s.push_frames(frames[n:n + T], want_masks=False)
            for k, kp in enumerate(fkd.split_frames(rec, off)):
                assert_same_kp(kp, exp[n + k], f"frame {n + k}")
        n += T
    pixel_masks_equal(s, ref, 8)
    assert any((k["flags"] == 1).any() for k in exp[1:]) and any((k["flags"] == 0).any() for k in exp[1:])


@pytest.mark.parametrize("W,H,O,intra", [(333, 207, 3, 1), (97, 61, 2, 0), (16, 12, 3, 1), (200, 150, 6, 1)])
def test_per_pixel_mask_ragged(W, H, O, intra):
    src = synth.VideoSource(W, H, seed=5 * W + H, n_rect=12, n_movers=2, mover_size=max(4, min(W, H) // 3),
                            speed=(1, 3))
    frames = src.frames(7)
    kw = dict(N_r=3, N_c=4, T_I=5, O=O, intra=intra, t=8)
    ref = oracle.Stream(W, H, mask_mode=oracle.MASK_IDP, **kw)
    exp = []
    for f in frames:
        ref.push(f)
        exp.append(ref.keypoints())
    s = fkd.Stream(W, H, mask_mode=fkd.FKD_MASK_IDP, T_max=3, **kw)
    n = 0
    for T in [3, 1, 3]:
        rec, off, _ = s.push_frames(frames[n:n + T], want_masks=False)
        for k, kp in enumerate(fkd.split_frames(rec, off)):
            assert_same_kp(kp, exp[n + k], f"frame {n + k}")
        n += T
    pixel_masks_equal(s, ref, oracle.num_layers(O, intra))


def test_per_pixel_mask_rejected_in_groups():
    g = fkd.Group(2, 1)
    with pytest.raises(fkd.FkdError):
        g.add_stream(64, 48, mask_mode=fkd.FKD_MASK_IDP)


@pytest.mark.parametrize("mode,T", [("id", 36), ("kb", 33), ("full", 32)])
def test_host_batch_layouts(clip2, mode, T):
    # host frames of a batch are uploaded with one copy when back to back,
    # else frame by frame; the records must not change, nor must later
    # single pushes
    cfg, frames = clip2
    g, o = both(params(cfg, mask_layer=-1), mode)
    exp_kp, exp_m = run_oracle(frames[:T], **o)
    s = fkd.Stream(cfg.W, cfg.H, T_max=T, **g)
    push_in_pieces(s, frames[:T], [T - 2, 1, 1] if T > 33 else [T], exp_kp, exp_m)
    # rows of pitch W + 8 (frames still back to back), then frames with gaps
    # between them (frame by frame copies)
    wide = np.zeros((T, cfg.H, cfg.W + 8), np.uint8)
    wide[:, :, :cfg.W] = frames[:T]
    gaps = np.zeros((T, cfg.H + 3, cfg.W), np.uint8)
    gaps[:, :cfg.H] = frames[:T]
    for view in (wide[:, :, :cfg.W], gaps[:, :cfg.H]):
        s.reset()
        rec, off, _ = s.push_frames(view)
        for k, kp in enumerate(fkd.split_frames(rec, off)):
            assert_same_kp(kp, exp_kp[k], f"strided frame {k}")


@pytest.mark.parametrize("mode", ["id", "kb"])
def test_host_batch_into_pinned_output(clip2, mode):
    """Host frames with caller-owned pinned outputs: a batch of 32 or more
    back-to-back frames is uploaded in parts, each part its own batch whose
    kernels start while the later parts are still arriving. Records, offsets
    and masks must equal the oracle's; a cap below the total keeps the
    records up to it and reports the overflow."""
    torch = pytest.importorskip("torch")
    cfg, frames = clip2
    T = len(frames)
    g, o = both(params(cfg, mask_layer=-1), mode)
    exp_kp, exp_m = run_oracle(frames, **o)
    s = fkd.Stream(cfg.W, cfg.H, T_max=T, **g)
    total = sum(len(k) for k in exp_kp)
    out = torch.zeros(total + 1000, dtype=torch.int64).pin_memory().numpy().view(fkd.KEYPOINT_DTYPE)
    off = torch.zeros(T + 1, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
    msk = torch.zeros((T, cfg.N_r, cfg.N_c), dtype=torch.uint8).pin_memory().numpy()
    for rep in range(2):  # the second call reuses the staging and the parts
        s.reset()
        s.push_frames(frames, out=out, offsets=off, masks=msk)
        assert off[T] == total
        for k, kp in enumerate(fkd.split_frames(out[:off[T]], off)):
            assert_same_kp(kp, exp_kp[k], f"call {rep} frame {k}")
            np.testing.assert_array_equal(msk[k], exp_m[k], err_msg=f"mask of frame {k}")
    # a capacity below the total: the records up to it, then FKD_E_CAPACITY
    cap = total // 2
    out[:] = 0
    s.reset()
    with pytest.raises(fkd.FkdError):
        s.push_frames(frames, out=out, offsets=off, masks=msk, cap=cap)
    flat = np.concatenate(exp_kp)
    got = out[:cap]
    for field in ("layer", "y", "x", "score", "flags"):
        np.testing.assert_array_equal(got[field], flat[:cap][field], err_msg=f"capped records: {field}")
    assert not out[cap:].view(np.int64).any(), "nothing past the capacity"


@pytest.mark.parametrize("T_H,nms_scale", [(0, 0), (1, 0), (2, 0), (4, 0), (1, 1)])
def test_keypoint_binning_spans(clip2, T_H, nms_scale):
    """Keypoint binning (Eqs. 3-4) in batches: spans of 16 frames are detected
    on the bins active at each span's start and the masks resolved after;
    every frame must equal the oracle's frame-by-frame result, across span
    and batch boundaries, with bins going inactive inside spans."""
    cfg, frames = clip2
    g, o = both(params(cfg, T_H=T_H, nms_scale=nms_scale), "kb")
    exp_kp, exp_m = run_oracle(frames, **o)
    s = fkd.Stream(cfg.W, cfg.H, T_max=20, **g)
    push_in_pieces(s, frames, [20, 1, 15], exp_kp, exp_m)
    if T_H > 0:
        # some bin turns inactive at a frame that is not the first of a span
        starts = {0, 16, 20, 21}  # first frames of the spans of the batches above
        drops = [n for n in range(1, len(exp_m)) if n not in starts and (exp_m[n - 1] & ~exp_m[n]).any()]
        assert drops, "the clip must switch bins off inside a span"
