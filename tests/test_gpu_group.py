"""Groups: one frame of each of many streams per tick, one launch sequence.

Each stream's keypoints and masks must be bit-identical to the oracle run
frame by frame on that stream alone, whatever the mix of sizes and
parameters in a tick and whichever streams sit a tick out.
"""
import numpy as np
import pytest

import oracle
from paper_1503_06959_gb300 import fkd, synth

pytestmark = pytest.mark.gpu

ORC = {fkd.FKD_MASK_FULL: oracle.MASK_FULL, fkd.FKD_MASK_ID: oracle.MASK_ID,
       fkd.FKD_MASK_KB: oracle.MASK_KB}


def check(got, exp, where):
    assert len(got) == len(exp), f"{where}: {len(got)} vs {len(exp)}"
    for f in ("layer", "y", "x", "score", "flags"):
        np.testing.assert_array_equal(got[f], exp[f], err_msg=f"{where}: {f}")


SPECS = [  # W, H, params
    (320, 240, dict(N_r=8, N_c=8, T_I=4, t=20, mask_mode=fkd.FKD_MASK_ID)),
    (333, 207, dict(N_r=7, N_c=9, T_I=3, t=15, mask_mode=fkd.FKD_MASK_ID, mask_layer=-1)),
    (640, 480, dict(N_r=12, N_c=16, T_I=4, t=30, mask_mode=fkd.FKD_MASK_ID)),
    (200, 150, dict(N_r=3, N_c=5, T_H=2, t=12, mask_mode=fkd.FKD_MASK_KB)),
    (128, 96, dict(N_r=2, N_c=2, t=25, mask_mode=fkd.FKD_MASK_FULL)),
]
# which streams take part in each tick (some sit ticks out)
TICKS = [[0, 1, 2, 3, 4], [0, 2, 4], [1, 2, 3], [0, 1, 2, 3, 4], [3], [0, 1, 4], [0, 1, 2, 3, 4]]


@pytest.mark.parametrize("graph", [True, False])
def test_group_ticks_match_oracle_per_stream(graph):
    torch = pytest.importorskip("torch")
    O, intra = 2, 1
    stream = torch.cuda.Stream()
    g = fkd.Group(O, intra, cuda_stream=stream.cuda_stream)
    g.use_graph(graph)
    n_frames = [sum(i in t for t in TICKS) for i in range(len(SPECS))]
    clips, refs, ids = [], [], []
    for i, (W, H, p) in enumerate(SPECS):
        src = synth.VideoSource(W, H, seed=50 + i, n_movers=2, mover_size=min(W, H) // 4,
                                speed=(2, 4))
        clips.append(src.frames(n_frames[i]))
        q = dict(p)
        mode = q.pop("mask_mode")
        refs.append(oracle.Stream(W, H, O=O, intra=intra, mask_mode=ORC[mode],
                                  **{k: v for k, v in q.items()}))
        sid, nbytes = g.add_stream(W, H, mask_mode=mode, **q)
        assert nbytes > W * H
        ids.append(sid)
    pos = [0] * len(SPECS)
    for tick, members in enumerate(TICKS):
        frames = []
        for i in members:
            # a fresh device buffer per frame: the group keeps its own copies
            frames.append(torch.from_numpy(clips[i][pos[i]]).cuda())
        torch.cuda.synchronize()
        g.tick([ids[i] for i in members], frames)
        for i in members:
            refs[i].push(clips[i][pos[i]])
            check(g.get_keypoints(ids[i]), refs[i].keypoints(), f"tick {tick} stream {i}")
            np.testing.assert_array_equal(g.get_mask(ids[i]), refs[i].mask())
            pos[i] += 1
        del frames
    g.close()


def test_group_equals_solo_streams_and_removal():
    torch = pytest.importorskip("torch")
    cfg = synth.config2()
    g = fkd.Group(cfg.O, cfg.intra, cuda_stream=torch.cuda.Stream().cuda_stream)
    kw = dict(N_r=cfg.N_r, N_c=cfg.N_c, T_I=cfg.T_I, t=cfg.t)
    a, _ = g.add_stream(cfg.W, cfg.H, **kw)
    b, _ = g.add_stream(cfg.W, cfg.H, **kw)
    fa = synth.source_for(cfg, 2, 0).frames(5)
    fb = synth.source_for(cfg, 2, 1).frames(5)
    solo = fkd.Stream(cfg.W, cfg.H, O=cfg.O, intra=cfg.intra, T_max=5, **kw)
    rec, off, _ = solo.push_frames(fa)
    expect = fkd.split_frames(rec, off)
    for n in range(5):
        if n == 3:
            g.remove_stream(b)
        ids = [a] if n >= 3 else [a, b]
        frames = [torch.from_numpy(fa[n]).cuda()] + ([] if n >= 3 else [torch.from_numpy(fb[n]).cuda()])
        g.tick(ids, frames)
        check(g.get_keypoints(a), expect[n], f"frame {n}")
    with pytest.raises(fkd.FkdError):
        g.get_keypoints(b)
    g.close()


def test_group_mixed_scale_space_suppression():
    # streams with and without the scale-space suppression in one tick
    torch = pytest.importorskip("torch")
    O, intra, m = 3, 1, 5
    specs = [(320, 240, dict(N_r=8, N_c=8, T_I=4, t=20, nms_scale=1, mask_layer=-1)),
             (333, 207, dict(N_r=7, N_c=9, T_I=3, t=15, nms_scale=0)),
             (200, 150, dict(N_r=3, N_c=5, t=12, nms_scale=1, mask_mode=fkd.FKD_MASK_FULL))]
    stream = torch.cuda.Stream()
    g = fkd.Group(O, intra, cuda_stream=stream.cuda_stream)
    refs, clips, ids = [], [], []
    for i, (W, H, p) in enumerate(specs):
        clips.append(synth.VideoSource(W, H, seed=70 + i, n_movers=2, mover_size=min(W, H) // 4,
                                       speed=(2, 4)).frames(m))
        q = dict(p)
        mode = q.pop("mask_mode", fkd.FKD_MASK_ID)
        refs.append(oracle.Stream(W, H, O=O, intra=intra, mask_mode=ORC[mode], **q))
        ids.append(g.add_stream(W, H, mask_mode=mode, **q)[0])
    for j in range(m):
        frames = [torch.from_numpy(np.ascontiguousarray(c[j])).cuda() for c in clips]
        g.tick(ids, frames)
        for i, sid in enumerate(ids):
            refs[i].push(clips[i][j])
            check(g.get_keypoints(sid), refs[i].keypoints(), f"stream {i} frame {j}")
