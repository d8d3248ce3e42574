"""Parity at the benchmark workloads' full sizes, in the launch shapes the
bench uses (tuned by the autotuner on the same frames).

* config 2: the whole 640x480 clip, 300 frames in one batch, every frame's
  keypoints and mask against the oracle;
* config 5: 3840x2160 frames with 5 octaves + intra-octaves (ten layers), the
  first frames of a moving segment;
* config 3: the 64-stream group, one stream of each resolution checked
  against the oracle (the others run in the same ticks).
"""
import numpy as np
import pytest

import oracle
from paper_1503_06959_gb300 import fkd, synth

pytestmark = pytest.mark.gpu


def check(got, exp, where):
    assert len(got) == len(exp), f"{where}: {len(got)} vs {len(exp)} keypoints"
    for f in ("layer", "y", "x", "score", "flags"):
        np.testing.assert_array_equal(got[f], exp[f], err_msg=f"{where}: {f}")


def oracle_run(cfg, frames):
    ref = oracle.Stream(cfg.W, cfg.H, N_r=cfg.N_r, N_c=cfg.N_c, T_I=cfg.T_I, O=cfg.O, intra=cfg.intra,
                        t=cfg.t, mask_mode=oracle.MASK_ID, mask_layer=cfg.mask_layer)
    kps, masks = [], []
    for f in frames:
        ref.push(f)
        kps.append(ref.keypoints())
        masks.append(ref.mask())
    return kps, masks


def test_config2_whole_clip_one_batch():
    torch = pytest.importorskip("torch")
    cfg = synth.config2()
    frames = synth.source_for(cfg, 2).frames(cfg.frames)
    s = fkd.Stream(cfg.W, cfg.H, N_r=cfg.N_r, N_c=cfg.N_c, T_I=cfg.T_I, O=cfg.O, intra=cfg.intra, t=cfg.t,
                   mask_mode=fkd.FKD_MASK_ID, mask_layer=cfg.mask_layer, T_max=cfg.frames)
    shape, _ = s.autotune(torch.from_numpy(frames).cuda(), reps=1)
    s.set_launch_config(shape)
    rec, off, masks = s.push_frames(frames)
    exp_kp, exp_m = oracle_run(cfg, frames)
    for k, kp in enumerate(fkd.split_frames(rec, off)):
        check(kp, exp_kp[k], f"{shape} frame {k}")
        np.testing.assert_array_equal(masks[k], exp_m[k], err_msg=f"mask of frame {k}")
    assert sum(len(k) for k in exp_kp) > 100000


def test_config5_4k_frames():
    cfg = synth.config5()
    frames = synth.source_for(cfg, 5).frames(3)
    s = fkd.Stream(cfg.W, cfg.H, N_r=cfg.N_r, N_c=cfg.N_c, T_I=cfg.T_I, O=cfg.O, intra=cfg.intra, t=cfg.t,
                   mask_mode=fkd.FKD_MASK_ID, mask_layer=cfg.mask_layer, T_max=3, K_max=1 << 20)
    assert s.num_layers() == 10
    rec, off, masks = s.push_frames(frames)
    exp_kp, exp_m = oracle_run(cfg, frames)
    for k, kp in enumerate(fkd.split_frames(rec, off)):
        check(kp, exp_kp[k], f"4K frame {k}")
        np.testing.assert_array_equal(masks[k], exp_m[k])


def test_config3_group_sampled_streams():
    torch = pytest.importorskip("torch")
    streams = synth.config3_streams(16)
    m = 2
    clips = [synth.source_for(c, 3, j).frames(m) for j, c in enumerate(streams)]
    dev = [[torch.from_numpy(np.ascontiguousarray(c[n])).cuda() for c in clips] for n in range(m)]
    torch.cuda.synchronize()
    st = torch.cuda.Stream()
    g = fkd.Group(streams[0].O, streams[0].intra, cuda_stream=st.cuda_stream)
    ids = [g.add_stream(c.W, c.H, N_r=c.N_r, N_c=c.N_c, T_I=c.T_I, t=c.t, mask_mode=fkd.FKD_MASK_ID,
                        mask_layer=c.mask_layer, K_max=1 << 17)[0] for c in streams]
    shape, _ = g.autotune(ids, dev, reps=1)  # resets every stream
    checked = [j for j in range(len(streams)) if j % 16 == 0]  # one stream per resolution
    exp = {j: oracle_run(streams[j], clips[j])[0] for j in checked}
    for n in range(m):
        g.tick(ids, dev[n])
        for j in checked:
            check(g.get_keypoints(ids[j]), exp[j][n], f"{shape} stream {j} ({streams[j].W}x{streams[j].H}) frame {n}")
    g.close()
