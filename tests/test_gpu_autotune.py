"""Detection launch shapes and the autotuner.

The tile height, warps per CTA and CTAs per SM only change how the work is
cut: every shape must give keypoints and masks bit-identical to the oracle,
on layers whose sizes leave ragged tiles at every height.
"""
import numpy as np
import pytest

import oracle
from paper_1503_06959_gb300 import fkd, synth

pytestmark = pytest.mark.gpu

W, H = 333, 250  # layers of 333x250 .. 41x31: ragged at tile heights 8, 16 and 24
P = dict(N_r=7, N_c=9, T_I=3, O=3, intra=1, t=18)
T = 10


def check(got, exp, where):
    assert len(got) == len(exp), f"{where}: {len(got)} vs {len(exp)}"
    for f in ("layer", "y", "x", "score", "flags"):
        np.testing.assert_array_equal(got[f], exp[f], err_msg=f"{where}: {f}")


@pytest.fixture(scope="module")
def clip():
    src = synth.VideoSource(W, H, seed=77, n_movers=3, mover_size=60, speed=(2, 4))
    frames = src.frames(T)
    ref = oracle.Stream(W, H, mask_mode=oracle.MASK_ID, mask_layer=-1, **P)
    kps, masks = [], []
    for f in frames:
        ref.push(f)
        kps.append(ref.keypoints())
        masks.append(ref.mask())
    assert any(m.sum() < m.size for m in masks[1:]), "the clip must have inactive bins"
    return frames, kps, masks


def max_ctas(s, tile_h, warps):
    for c in range(16, 0, -1):
        try:
            s.set_launch_config(dict(tile_h=tile_h, warps_per_cta=warps, ctas_per_sm=c))
            return c
        except fkd.FkdError:
            pass
    raise AssertionError(f"no CTA count fits tile_h {tile_h}, {warps} warps")


def shapes(s):
    out = []
    for th in (8, 16, 24):
        for w in (4, 8):
            m = max_ctas(s, th, w)
            out += [dict(tile_h=th, warps_per_cta=w, ctas_per_sm=c) for c in sorted({1, m})]
    return out


def test_every_shape_matches_oracle(clip):
    torch = pytest.importorskip("torch")
    frames, kps, masks = clip
    s = fkd.Stream(W, H, mask_mode=fkd.FKD_MASK_ID, mask_layer=-1, T_max=T, **P)
    dev = torch.from_numpy(frames).cuda()
    for shape in shapes(s):
        s.set_launch_config(shape)
        assert s.launch_config() == dict(shape, tile_w=128)
        s.reset()
        rec, off, msk = s.push_frames(frames)
        for n in range(T):
            check(rec[off[n]:off[n + 1]], kps[n], f"{shape} frame {n}")
            np.testing.assert_array_equal(msk[n], masks[n])
        # device input, frame by frame
        s.reset()
        for n in range(T):
            s.push_frame(dev[n])
            check(s.get_keypoints(), kps[n], f"{shape} single frame {n}")


def test_bad_shapes_rejected():
    s = fkd.Stream(W, H, **P)
    default = s.launch_config()
    assert default["tile_h"] == 16 and default["warps_per_cta"] == 8 and default["ctas_per_sm"] >= 1
    for bad in (dict(tile_h=12, warps_per_cta=8, ctas_per_sm=1),
                dict(tile_h=16, warps_per_cta=6, ctas_per_sm=1),
                dict(tile_h=16, warps_per_cta=8, ctas_per_sm=0),
                dict(tile_h=16, warps_per_cta=8, ctas_per_sm=64)):
        with pytest.raises(fkd.FkdError):
            s.set_launch_config(bad)
        assert s.launch_config() == default


def test_autotune_then_parity(clip):
    torch = pytest.importorskip("torch")
    frames, kps, masks = clip
    s = fkd.Stream(W, H, mask_mode=fkd.FKD_MASK_ID, mask_layer=-1, T_max=T, **P)
    dev = torch.from_numpy(frames).cuda()
    s.push_frames(frames[:3])
    best, ms = s.autotune(dev, reps=1)
    assert ms > 0
    assert best["tile_w"] == 128 and best["tile_h"] in (8, 16, 24) and best["warps_per_cta"] in (4, 8)
    assert 1 <= best["ctas_per_sm"] <= max_ctas(s, best["tile_h"], best["warps_per_cta"])
    s.set_launch_config(best)
    assert s.frame_count() == 0, "tuning resets the stream"
    rec, off, msk = s.push_frames(frames)
    for n in range(T):
        check(rec[off[n]:off[n + 1]], kps[n], f"tuned {best} frame {n}")


SPECS = [(320, 240, dict(N_r=8, N_c=8, T_I=4, t=20)),
         (333, 207, dict(N_r=7, N_c=9, T_I=3, t=15, mask_layer=-1)),
         (200, 150, dict(N_r=3, N_c=5, T_H=2, t=12, mask_mode=fkd.FKD_MASK_KB))]


def test_group_shapes_and_autotune():
    torch = pytest.importorskip("torch")
    O, intra, m = 2, 1, 5
    orc_mode = {fkd.FKD_MASK_ID: oracle.MASK_ID, fkd.FKD_MASK_KB: oracle.MASK_KB}
    clips, exp = [], []
    for i, (w, h, p) in enumerate(SPECS):
        clips.append(synth.VideoSource(w, h, seed=90 + i, n_movers=2, mover_size=min(w, h) // 4,
                                       speed=(2, 4)).frames(m))
        q = dict(p)
        mode = q.pop("mask_mode", fkd.FKD_MASK_ID)
        ref = oracle.Stream(w, h, O=O, intra=intra, mask_mode=orc_mode[mode], **q)
        e = []
        for f in clips[-1]:
            ref.push(f)
            e.append(ref.keypoints())
        exp.append(e)
    dev = [[torch.from_numpy(np.ascontiguousarray(c[j])).cuda() for c in clips] for j in range(m)]
    stream = torch.cuda.Stream()
    g = fkd.Group(O, intra, cuda_stream=stream.cuda_stream)
    ids = [g.add_stream(w, h, **p)[0] for w, h, p in SPECS]

    def run(tag):
        for j in range(m):
            g.tick(ids, dev[j])
            for i, sid in enumerate(ids):
                check(g.get_keypoints(sid), exp[i][j], f"{tag} stream {i} frame {j}")

    for th in (8, 24, 16):
        g.set_launch_config(dict(tile_h=th, warps_per_cta=4, ctas_per_sm=1))
        for sid in ids:  # restart every stream
            g.remove_stream(sid)
        ids = [g.add_stream(w, h, **p)[0] for w, h, p in SPECS]
        assert g.launch_config()["tile_h"] == th
        run(f"tile_h {th}")
    best, ms = g.autotune(ids, dev, reps=1)
    assert ms > 0 and g.launch_config() == best
    run(f"tuned {best}")
