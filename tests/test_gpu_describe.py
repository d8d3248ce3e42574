"""Masked description on the GPU against the oracle (through the C ABI).

Descriptors are integer results (bits of comparisons of integer box sums):
the bar is bit-exact equality for every record, new and carried, on top of
bit-exact keypoints.
"""
import numpy as np
import pytest

import oracle
from paper_1503_06959_gb300 import fkd, synth

pytestmark = pytest.mark.gpu

MODES = {"full": (fkd.FKD_MASK_FULL, oracle.MASK_FULL), "id": (fkd.FKD_MASK_ID, oracle.MASK_ID),
         "kb": (fkd.FKD_MASK_KB, oracle.MASK_KB), "idp": (fkd.FKD_MASK_IDP, oracle.MASK_IDP)}


def run_oracle(frames, pattern, **kw):
    s = oracle.Stream(frames.shape[2], frames.shape[1], pattern=pattern, **kw)
    kps, descs = [], []
    for f in frames:
        s.push(f)
        kps.append(s.keypoints())
        descs.append(s.descriptors())
    return kps, descs


def check(rec, desc, exp_kp, exp_desc, where):
    assert len(rec) == len(exp_kp), f"{where}: {len(rec)} vs {len(exp_kp)} keypoints"
    for f in ("layer", "y", "x", "score", "flags"):
        np.testing.assert_array_equal(rec[f], exp_kp[f], err_msg=f"{where}: {f}")
    assert desc.shape == exp_desc.shape, where
    bad = np.flatnonzero((desc != exp_desc).any(axis=1))
    assert bad.size == 0, (f"{where}: {bad.size} of {len(desc)} descriptors differ, first at record "
                           f"{bad[0]} {rec[bad[0]]}")


def streams(W, H, mode, pattern, T_max, **p):
    g = fkd.Stream(W, H, mask_mode=MODES[mode][0], T_max=T_max, pattern=pattern, **p)
    o = dict(p, mask_mode=MODES[mode][1])
    return g, o


@pytest.mark.parametrize("mode,mask_layer,D", [("id", -1, 256), ("id", 0, 32), ("kb", 0, 128),
                                               ("idp", 0, 512), ("full", 0, 64)])
def test_batches_match_oracle(mode, mask_layer, D):
    W, H = 333, 250
    src = synth.VideoSource(W, H, seed=41, n_movers=3, mover_size=60, speed=(2, 4), jitter_every=7)
    frames = src.frames(17)
    pattern = synth.descriptor_pattern(D, seed=D)
    p = dict(N_r=7, N_c=9, T_I=4, T_H=2, O=3, intra=1, t=18, mask_layer=mask_layer)
    g, o = streams(W, H, mode, pattern, 8, **p)
    exp_kp, exp_d = run_oracle(frames, pattern, **o)
    carried = sum(int((k["flags"] == 1).sum()) for k in exp_kp)
    if mode != "full":
        assert carried > 0, "the clip must carry keypoints"
    # batches of 8, 1 and 8: carried descriptors cross batch boundaries
    n0 = 0
    for T in (8, 1, 8):
        rec, off, _ = g.push_frames(frames[n0:n0 + T])
        desc = g.get_descriptors()
        assert len(desc) == off[T]
        for k in range(T):
            check(rec[off[k]:off[k + 1]], desc[off[k]:off[k + 1]], exp_kp[n0 + k], exp_d[n0 + k],
                  f"{mode} frame {n0 + k}")
        n0 += T


@pytest.mark.parametrize("mode", ["id", "idp"])
def test_frame_by_frame_and_device_output(mode):
    torch = pytest.importorskip("torch")
    W, H = 200, 150
    frames = synth.VideoSource(W, H, seed=5, n_movers=2, mover_size=40, speed=(2, 3)).frames(9)
    pattern = synth.descriptor_pattern(256, seed=9)
    p = dict(N_r=5, N_c=6, T_I=4, O=2, intra=1, t=15, mask_layer=0)
    g, o = streams(W, H, mode, pattern, 4, **p)
    exp_kp, exp_d = run_oracle(frames, pattern, **o)
    dev = torch.from_numpy(frames).cuda()
    for n in range(5):  # single frames, host then device input
        g.push_frame(frames[n] if n % 2 else dev[n])
        check(g.get_keypoints(), g.get_descriptors(), exp_kp[n], exp_d[n], f"frame {n}")
    # then a device batch with device outputs
    cap = 4 * 20000
    out = torch.zeros(cap, dtype=torch.int64, device="cuda")
    offs = torch.zeros(5, dtype=torch.int32, device="cuda")
    g.push_frames(dev[5:9], out=out, offsets=offs)
    g.synchronize()
    dbuf = torch.zeros((cap, 32), dtype=torch.uint8, device="cuda")
    d = g.get_descriptors(out=dbuf).cpu().numpy()
    off = offs.cpu().numpy()
    rec = out[:int(off[4])].cpu().numpy().view(fkd.KEYPOINT_DTYPE)
    assert len(d) == off[4]
    for k in range(4):
        check(rec[off[k]:off[k + 1]], d[off[k]:off[k + 1]], exp_kp[5 + k], exp_d[5 + k], f"frame {5 + k}")


def test_config2_batch_matches_oracle():
    """640x480, four octaves with intra-octaves, coarse-layer mask: 32 frames
    in one batch (including the camera step at frame 30), every descriptor."""
    cfg = synth.config2()
    frames = synth.source_for(cfg, 2).frames(32)
    pattern = synth.descriptor_pattern(256)
    p = dict(N_r=cfg.N_r, N_c=cfg.N_c, T_I=cfg.T_I, O=cfg.O, intra=cfg.intra, t=cfg.t,
             mask_layer=cfg.mask_layer)
    g, o = streams(cfg.W, cfg.H, "id", pattern, 32, **p)
    exp_kp, exp_d = run_oracle(frames, pattern, **o)
    rec, off, _ = g.push_frames(frames)
    desc = g.get_descriptors()
    for k in range(32):
        check(rec[off[k]:off[k + 1]], desc[off[k]:off[k + 1]], exp_kp[k], exp_d[k], f"config 2 frame {k}")


def test_pattern_validation_and_state():
    W, H = 64, 48
    s = fkd.Stream(W, H, N_r=2, N_c=2, O=1, t=15)
    frame = synth.VideoSource(W, H, seed=2).frame(0)
    with pytest.raises(fkd.FkdError):
        s.get_descriptors()  # description off
    for bad in (np.zeros((31, 4), np.int8), np.zeros((544, 4), np.int8), np.full((32, 4), 14, np.int8),
                np.full((32, 4), -14, np.int8)):
        with pytest.raises(fkd.FkdError):
            s.set_descriptor(bad)
    s.set_descriptor(np.full((32, 4), 13, np.int8))
    with pytest.raises(fkd.FkdError):
        s.get_descriptors()  # nothing pushed since
    s.push_frame(frame)
    d = s.get_descriptors()
    assert d.shape == (len(s.get_keypoints()), 4)
    assert not d.any()  # every pair compares a box with itself
    s.set_descriptor(None)
    with pytest.raises(fkd.FkdError):
        s.get_descriptors()


def test_described_detection_equals_undescribed():
    """Description adds kernels after the emission; keypoints stay the same."""
    cfg = synth.config1()
    frames = synth.source_for(cfg, 1).frames(12)
    p = dict(N_r=cfg.N_r, N_c=cfg.N_c, T_I=cfg.T_I, O=2, intra=1, t=cfg.t, T_max=12)
    a = fkd.Stream(cfg.W, cfg.H, pattern=synth.descriptor_pattern(128), **p)
    b = fkd.Stream(cfg.W, cfg.H, **p)
    ra, oa, ma = a.push_frames(frames)
    rb, ob, mb = b.push_frames(frames)
    np.testing.assert_array_equal(oa, ob)
    np.testing.assert_array_equal(ra, rb)
    np.testing.assert_array_equal(ma, mb)


def test_capacity_overflow_then_reset():
    """Records past `cap` are dropped and reported; the descriptors of the
    records that fit are still right, and after a reset the stream describes
    bit-exactly again."""
    cfg = synth.config1()
    frames = synth.source_for(cfg, 1).frames(8)
    pattern = synth.descriptor_pattern(64, seed=4)
    p = dict(N_r=cfg.N_r, N_c=cfg.N_c, T_I=cfg.T_I, O=2, intra=1, t=cfg.t)
    g, o = streams(cfg.W, cfg.H, "id", pattern, 4, **p)
    exp_kp, exp_d = run_oracle(frames, pattern, **o)
    total = sum(len(k) for k in exp_kp[:4])
    cap = total // 2
    out = np.zeros(cap, fkd.KEYPOINT_DTYPE)
    off = np.zeros(5, np.uint32)
    with pytest.raises(fkd.FkdError):
        g.push_frames(frames[:4], out=out, offsets=off)
    d = g.get_descriptors()
    assert len(d) == cap
    n0 = len(exp_kp[0])
    np.testing.assert_array_equal(d[:min(n0, cap)], exp_d[0][:min(n0, cap)])
    g.reset()
    for n0 in (0, 4):
        rec, off2, _ = g.push_frames(frames[n0:n0 + 4])
        desc = g.get_descriptors()
        for k in range(4):
            check(rec[off2[k]:off2[k + 1]], desc[off2[k]:off2[k + 1]], exp_kp[n0 + k], exp_d[n0 + k],
                  f"after reset, frame {n0 + k}")


def test_group_description_matches_oracle():
    """Streams of a group describe in their ticks (with and without the
    captured graphs), each bit-exact with the oracle; a stream that does not
    describe is unaffected."""
    torch = pytest.importorskip("torch")
    O, intra, m = 2, 1, 7
    specs = [(320, 240, dict(N_r=8, N_c=8, T_I=4, t=20), "id", 256),
             (333, 207, dict(N_r=7, N_c=9, T_I=4, t=15, mask_layer=-1), "id", 128),
             (200, 150, dict(N_r=3, N_c=5, T_H=2, t=12), "kb", 64),
             (256, 192, dict(N_r=4, N_c=4, T_I=4, t=18), "id", 0)]
    clips, exp_kp, exp_d = [], [], []
    for i, (w, h, p, mode, D) in enumerate(specs):
        clips.append(synth.VideoSource(w, h, seed=60 + i, n_movers=2, mover_size=min(w, h) // 4,
                                       speed=(2, 4)).frames(m))
        pat = synth.descriptor_pattern(D, seed=D) if D else None
        ref = oracle.Stream(w, h, O=O, intra=intra, mask_mode=MODES[mode][1], pattern=pat, **p)
        ek, ed = [], []
        for f in clips[-1]:
            ref.push(f)
            ek.append(ref.keypoints())
            ed.append(ref.descriptors() if D else None)
        exp_kp.append(ek)
        exp_d.append(ed)
    dev = [[torch.from_numpy(np.ascontiguousarray(c[j])).cuda() for c in clips] for j in range(m)]
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()  # graphs need a stream of their own
    for graph in (True, False):
        g = fkd.Group(O, intra, cuda_stream=stream.cuda_stream)
        g.use_graph(graph)
        ids = []
        for (w, h, p, mode, D) in specs:
            sid = g.add_stream(w, h, mask_mode=MODES[mode][0], **p)[0]
            if D:
                g.set_descriptor(sid, synth.descriptor_pattern(D, seed=D))
            ids.append(sid)
        for j in range(m):
            g.tick(ids, dev[j])
            for i, sid in enumerate(ids):
                kp = g.get_keypoints(sid)
                if specs[i][4]:
                    check(kp, g.get_descriptors(sid), exp_kp[i][j], exp_d[i][j], f"graph {graph} stream {i} frame {j}")
                else:
                    assert len(kp) == len(exp_kp[i][j])
                    with pytest.raises(fkd.FkdError):
                        g.get_descriptors(sid)
        with pytest.raises(fkd.FkdError):  # after the first tick
            g.set_descriptor(ids[3], synth.descriptor_pattern(64))
        g.close()


def test_server_description_matches_oracle():
    """A served stream that describes hands out each polled frame's
    descriptors, bit-exact with the oracle; a stream beside it that does not
    describe is unaffected."""
    O, intra, m = 2, 1, 8
    specs = [(320, 240, dict(N_r=8, N_c=8, T_I=4, t=20), 256), (200, 150, dict(N_r=3, N_c=5, T_I=4, t=12), 0)]
    clips, exp_kp, exp_d = [], [], []
    for i, (w, h, p, D) in enumerate(specs):
        clips.append(synth.VideoSource(w, h, seed=70 + i, n_movers=2, mover_size=min(w, h) // 4,
                                       speed=(2, 4)).frames(m))
        pat = synth.descriptor_pattern(D, seed=11) if D else None
        ref = oracle.Stream(w, h, O=O, intra=intra, mask_mode=oracle.MASK_ID, pattern=pat, **p)
        ek, ed = [], []
        for f in clips[-1]:
            ref.push(f)
            ek.append(ref.keypoints())
            ed.append(ref.descriptors() if D else None)
        exp_kp.append(ek)
        exp_d.append(ed)
    srv = fkd.Server(O, intra, budget_bytes=2 << 30)
    ids = [srv.open_stream(w, h, **p) for (w, h, p, D) in specs]
    srv.set_descriptor(ids[0], synth.descriptor_pattern(256, seed=11))
    got = {sid: [] for sid in ids}
    for j in range(m):
        for i, sid in enumerate(ids):
            srv.submit(sid, clips[i][j])
        srv.drain()
        for i, sid in enumerate(ids):
            while True:
                r = srv.poll(sid)
                if r is None:
                    break
                idx, kp = r
                got[sid].append((idx, kp, srv.get_descriptors(sid) if specs[i][3] else None))
    with pytest.raises(fkd.FkdError):  # frames were submitted already
        srv.set_descriptor(ids[1], synth.descriptor_pattern(64))
    for i, sid in enumerate(ids):
        assert [g[0] for g in got[sid]] == list(range(m))
        for idx, kp, d in got[sid]:
            if specs[i][3]:
                check(kp, d, exp_kp[i][idx], exp_d[i][idx], f"served stream {i} frame {idx}")
            else:
                assert len(kp) == len(exp_kp[i][idx])
    srv.close()
