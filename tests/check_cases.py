"""Small parity cases run on the debug library (FKD_CHECK=1): every kernel
checks the indices of its shared- and global-memory accesses and the stream
allocations carry guard bands. A failed index check surfaces as an FkdError
from the call that launched the work; the guard bands are checked after each
case. Every result is also compared with the CPU oracle.

Run by tests/test_gpu_check.py in a process of its own (the binding loads
one library per process): python tests/check_cases.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
os.environ["FKD_CHECK"] = "1"

import oracle  # noqa: E402
from paper_1503_06959_gb300 import fkd, synth  # noqa: E402

MODES = {"full": (fkd.FKD_MASK_FULL, oracle.MASK_FULL), "id": (fkd.FKD_MASK_ID, oracle.MASK_ID),
         "kb": (fkd.FKD_MASK_KB, oracle.MASK_KB), "idp": (fkd.FKD_MASK_IDP, oracle.MASK_IDP)}


def oracle_run(frames, mode, **kw):
    s = oracle.Stream(frames.shape[2], frames.shape[1], mask_mode=MODES[mode][1], **kw)
    out = []
    for f in frames:
        s.push(f)
        out.append(s.keypoints())
    return out


def same(got, exp, where):
    assert len(got) == len(exp), f"{where}: {len(got)} vs {len(exp)} keypoints"
    for f in ("layer", "y", "x", "score", "flags"):
        assert np.array_equal(got[f], exp[f]), f"{where}: {f}"


def stream_case(name, frames, mode, pieces, T_max, **kw):
    H, W = frames.shape[1:]
    exp = oracle_run(frames, mode, **kw)
    s = fkd.Stream(W, H, mask_mode=MODES[mode][0], T_max=T_max, **kw)
    n = 0
    for T in pieces:
        if T == 1:
            s.push_frame(frames[n])
            same(s.get_keypoints(), exp[n], f"{name} frame {n}")
        else:
            rec, off, _ = s.push_frames(frames[n:n + T])
            for k, kp in enumerate(fkd.split_frames(rec, off)):
                same(kp, exp[n + k], f"{name} frame {n + k}")
        n += T
    s.check_guards()
    s.close()
    print(f"{name}: {n} frames ok", flush=True)


def main():
    assert fkd.check_build(), "the debug library must be loaded"
    cfg = synth.config1()
    clip1 = synth.source_for(cfg, 1).frames(cfg.frames)
    base1 = dict(N_r=cfg.N_r, N_c=cfg.N_c, T_I=cfg.T_I, O=cfg.O, intra=cfg.intra, t=cfg.t)
    for mode in ("id", "full", "kb"):
        stream_case(f"320x240 {mode}", clip1, mode, [12, 1, 7], 12, **base1)
    cfg2 = synth.config2()
    clip2 = synth.source_for(cfg2, 2).frames(36)
    base2 = dict(N_r=cfg2.N_r, N_c=cfg2.N_c, T_I=cfg2.T_I, O=cfg2.O, intra=cfg2.intra, t=cfg2.t)
    stream_case("640x480 id coarsest", clip2, "id", [20, 1, 15], 20, mask_layer=-1, **base2)
    stream_case("640x480 kb spans", clip2, "kb", [20, 1, 15], 20, T_H=2, **base2)
    stream_case("640x480 id scale-space", clip2[:12], "id", [6, 1, 5], 6, mask_layer=-1, nms_scale=1, **base2)
    rag = synth.VideoSource(333, 207, seed=11, n_rect=12, n_movers=2, mover_size=60, speed=(1, 3)).frames(8)
    stream_case("333x207 id", rag, "id", [3, 1, 4], 4, N_r=7, N_c=9, T_I=3, O=3, intra=1, t=15, mask_layer=-1)
    stream_case("333x207 idp", rag, "idp", [3, 1, 4], 4, N_r=7, N_c=9, T_I=4, O=2, intra=1, t=15)
    tiny = synth.VideoSource(7, 7, seed=5, n_rect=3, n_movers=1, mover_size=3, speed=(1, 1)).frames(4)
    stream_case("7x7 full", tiny, "full", [2, 1, 1], 2, N_r=1, N_c=1, T_I=1, O=1, intra=0, t=5)
    # description
    pattern = synth.descriptor_pattern(256)
    exp_o = oracle.Stream(cfg.W, cfg.H, mask_mode=oracle.MASK_ID, pattern=pattern, **base1)
    exp_d = []
    for f in clip1[:6]:
        exp_o.push(f)
        exp_d.append(exp_o.descriptors())
    s = fkd.Stream(cfg.W, cfg.H, mask_mode=fkd.FKD_MASK_ID, T_max=6, pattern=pattern, **base1)
    rec, off, _ = s.push_frames(clip1[:6])
    desc = s.get_descriptors()
    for k in range(6):
        assert np.array_equal(desc[off[k]:off[k + 1]], exp_d[k]), f"descriptors of frame {k}"
    s.check_guards()
    s.close()
    print("describe: 6 frames ok", flush=True)
    # a group tick mix, replayed from the captured graphs
    import torch
    specs = [(clip1, "id", base1), (rag, "kb", dict(N_r=7, N_c=9, T_I=3, O=1, intra=0, t=15)),
             (clip1[:, :120, :200].copy(), "full", dict(N_r=3, N_c=5, T_I=4, O=1, intra=0, t=20))]
    g = fkd.Group(1, 0, cuda_stream=torch.cuda.Stream().cuda_stream)
    ids, exps, devs = [], [], []
    for frames, mode, kw in specs:
        kw = dict(kw)
        kw.pop("O"), kw.pop("intra")
        ids.append(g.add_stream(frames.shape[2], frames.shape[1], mask_mode=MODES[mode][0], **kw)[0])
        exps.append(oracle_run(frames[:4], mode, O=1, intra=0, **kw))
        devs.append(torch.from_numpy(np.ascontiguousarray(frames[:4])).cuda())
    for n in range(4):
        g.tick(ids, [d[n] for d in devs])
        for i, e in zip(ids, exps):
            same(g.get_keypoints(i), e[n], f"group stream {i} frame {n}")
    g.check_guards()
    g.close()
    print("group: 4 ticks ok", flush=True)
    print("check cases ok")


if __name__ == "__main__":
    main()
