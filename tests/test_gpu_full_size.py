"""Parity at the benchmark workloads' full sizes, in the launch shapes the
bench uses (tuned by the autotuner on the same frames). Every keypoint field
and every mask is compared with the CPU oracle (run in a pool of spawned
processes while the GPU works).

* config 2: the whole 640x480 clip, 300 frames in one batch;
* config 3: the 64-stream group of mixed resolutions, every stream checked
  on every one of five ticks, one tick with half the streams sitting out;
* config 4: the 256-stream serving mix (64 streams of each resolution)
  submitted through the serving loop, two streams of each resolution checked
  frame by frame, every stream's results accounted for;
* config 5: 3840x2160 frames with ten layers across the boundary between the
  moving and the static segment (frames 96-103 of the 200-frame clip), as a
  batch of one stream and through a group; in the static frames every bin is
  inactive and D_n is D_{n-1} carried over whole (Eq. 1).
"""
import time

import numpy as np
import pytest

import oracle
import oracle_jobs
from paper_1503_06959_gb300 import fkd, synth

pytestmark = pytest.mark.gpu


def check(got, exp, where):
    assert len(got) == len(exp), f"{where}: {len(got)} vs {len(exp)} keypoints"
    for f in ("layer", "y", "x", "score", "flags"):
        np.testing.assert_array_equal(got[f], exp[f], err_msg=f"{where}: {f}")


def test_config2_whole_clip_one_batch():
    torch = pytest.importorskip("torch")
    cfg = synth.config2()
    frames = synth.source_for(cfg, 2).frames(cfg.frames)
    with oracle_jobs.pool(1) as ex:
        fut = ex.submit(oracle_jobs.run_frames, cfg.W, cfg.H, oracle_jobs.params_of(cfg, oracle.MASK_ID), frames)
        s = fkd.Stream(cfg.W, cfg.H, N_r=cfg.N_r, N_c=cfg.N_c, T_I=cfg.T_I, O=cfg.O, intra=cfg.intra, t=cfg.t,
                       mask_mode=fkd.FKD_MASK_ID, mask_layer=cfg.mask_layer, T_max=cfg.frames)
        shape, _ = s.autotune(torch.from_numpy(frames).cuda(), reps=1)
        s.set_launch_config(shape)
        rec, off, masks = s.push_frames(frames)
        exp_kp, exp_m = fut.result()
    for k, kp in enumerate(fkd.split_frames(rec, off)):
        check(kp, exp_kp[k], f"{shape} frame {k}")
        np.testing.assert_array_equal(masks[k], exp_m[k], err_msg=f"mask of frame {k}")
    assert sum(len(k) for k in exp_kp) > 100000


def test_config3_group_every_stream():
    """All 64 streams, five ticks; on tick 2 only the even streams take a
    frame (the odd ones sit it out and resume with their next frame)."""
    torch = pytest.importorskip("torch")
    streams = synth.config3_streams(16)
    ticks = 5
    sits_out = {2: {j for j in range(len(streams)) if j % 2}}
    frames_of = [ticks - len([1 for n in range(ticks) if j in sits_out.get(n, ())]) for j in range(len(streams))]
    clips = [synth.source_for(c, 3, j).frames(frames_of[j]) for j, c in enumerate(streams)]
    with oracle_jobs.pool() as ex:
        futs = [ex.submit(oracle_jobs.run_frames, c.W, c.H, oracle_jobs.params_of(c, oracle.MASK_ID), clips[j])
                for j, c in enumerate(streams)]
        dev = [torch.from_numpy(c).cuda() for c in clips]
        torch.cuda.synchronize()
        st = torch.cuda.Stream()
        g = fkd.Group(streams[0].O, streams[0].intra, cuda_stream=st.cuda_stream)
        ids = [g.add_stream(c.W, c.H, N_r=c.N_r, N_c=c.N_c, T_I=c.T_I, t=c.t, mask_mode=fkd.FKD_MASK_ID,
                            mask_layer=c.mask_layer, K_max=1 << 17)[0] for c in streams]
        shape, _ = g.autotune(ids, [[d[n] for d in dev] for n in range(2)], reps=1)  # resets every stream
        got = [[] for _ in streams]
        pos = [0] * len(streams)
        for n in range(ticks):
            members = [j for j in range(len(streams)) if j not in sits_out.get(n, ())]
            g.tick([ids[j] for j in members], [dev[j][pos[j]] for j in members])
            for j in members:
                got[j].append((g.get_keypoints(ids[j]), g.get_mask(ids[j])))
                pos[j] += 1
        g.close()
        exp = [f.result() for f in futs]
    for j, c in enumerate(streams):
        assert len(got[j]) == frames_of[j]
        for n, (kp, m) in enumerate(got[j]):
            where = f"{shape} stream {j} ({c.W}x{c.H}) frame {n}"
            check(kp, exp[j][0][n], where)
            np.testing.assert_array_equal(m, exp[j][1][n], err_msg=f"{where}: mask")
    assert any((e[1][n] == 0).any() for e in exp for n in range(1, len(e[1]))), "some bins must be inactive"


def test_config4_serving_mix():
    """The 256-stream serving mix (64 of each resolution, O=4 + intra, mask on
    the coarsest octave, 8 GB budget), frames submitted round robin so that
    every round mixes resolutions; each stream's n-th frame is frame
    (7 j + n) mod 12 of its resolution's pool, as in the serving bench."""
    res_list = [(320, 240), (640, 480), (1280, 720), (1920, 1080)]
    per_res, F, pool_n = 64, 6, 12
    pools = {}
    for k, (W, H) in enumerate(res_list):
        src = synth.VideoSource(W, H, seed=1000 + 400 + k, n_movers=4,
                                mover_size=int(np.sqrt(0.3 * W * H / 4)), speed=(1, 4))
        pools[(W, H)] = src.frames(pool_n)
    streams = [(W, H, k * per_res + j) for k, (W, H) in enumerate(res_list) for j in range(per_res)]
    frames_of = lambda W, H, j: np.stack([pools[(W, H)][(j * 7 + n) % pool_n] for n in range(F)])
    sampled = [i for i, (W, H, j) in enumerate(streams) if j % per_res in (0, 37)]
    prm = dict(N_r=12, N_c=16, T_I=4, t=30, mask_mode=fkd.FKD_MASK_ID, mask_layer=-1)
    oprm = dict(prm, O=4, intra=1, mask_mode=oracle.MASK_ID)
    with oracle_jobs.pool() as ex:
        futs = {i: ex.submit(oracle_jobs.run_frames, streams[i][0], streams[i][1], oprm, frames_of(*streams[i]))
                for i in sampled}
        srv = fkd.Server(4, 1, budget_bytes=8 << 30, max_tick_keypoints=1 << 23)
        ids = [srv.open_stream(W, H, K_max=1 << 17, **prm) for W, H, _ in streams]
        got = {i: [] for i in range(len(streams))}

        def collect():
            for i, sid in enumerate(ids):
                while (r := srv.poll(sid)) is not None:
                    got[i].append(r)

        for n in range(F):
            for i, (W, H, j) in enumerate(streams):
                f = pools[(W, H)][(j * 7 + n) % pool_n]
                while True:
                    try:
                        srv.submit(ids[i], f)
                        break
                    except fkd.FkdError as e:  # the stream's queue is full: collect and retry
                        if e.code != fkd.FKD_E_CAPACITY:
                            raise
                        collect()
                        time.sleep(0.001)
        srv.drain(120000)
        collect()
        stats = srv.stats()
        srv.close()
        exp = {i: f.result() for i, f in futs.items()}
    assert stats["rejected_streams"] == 0 and stats["frames_done"] == len(streams) * F
    assert stats["mean_batch"] > 1.0, "rounds must batch several streams"
    for i in range(len(streams)):
        assert [r[0] for r in got[i]] == list(range(F)), f"stream {i}: frames {[r[0] for r in got[i]]}"
    for i in sampled:
        W, H, j = streams[i]
        for n in range(F):
            check(got[i][n][1], exp[i][0][n], f"served stream {j} ({W}x{H}) frame {n}")


def test_config5_moving_to_static_boundary():
    torch = pytest.importorskip("torch")
    cfg = synth.config5()
    first, last = 96, 104  # frames 96..103; the static segment starts at frame 100
    frames = synth.source_for(cfg, 5).frames(last)[first:]
    oprm = oracle_jobs.params_of(cfg, oracle.MASK_ID)
    with oracle_jobs.pool(2) as ex:
        fut_a = ex.submit(oracle_jobs.run_frames, cfg.W, cfg.H, oprm, frames)
        fut_b = ex.submit(oracle_jobs.run_frames, cfg.W, cfg.H, oprm, frames[2:])
        kw = dict(N_r=cfg.N_r, N_c=cfg.N_c, T_I=cfg.T_I, t=cfg.t, mask_mode=fkd.FKD_MASK_ID,
                  mask_layer=cfg.mask_layer, K_max=1 << 20)
        # one stream, the eight frames as one batch
        s = fkd.Stream(cfg.W, cfg.H, O=cfg.O, intra=cfg.intra, T_max=len(frames), **kw)
        assert s.num_layers() == 10
        rec, off, masks = s.push_frames(frames)
        batch = fkd.split_frames(rec, off)
        s.close()
        # a group of two streams fed the same clip, the second joining two frames later
        dev = torch.from_numpy(frames).cuda()
        st = torch.cuda.Stream()
        g = fkd.Group(cfg.O, cfg.intra, cuda_stream=st.cuda_stream)
        a, b = g.add_stream(cfg.W, cfg.H, **kw)[0], g.add_stream(cfg.W, cfg.H, **kw)[0]
        shape, _ = g.autotune([a, b], [[dev[n], dev[n + 2]] for n in range(2)], reps=1)
        grp_a, grp_b = [], []
        for n in range(len(frames)):
            ids, fr = ([a, b], [dev[n], dev[n]]) if n >= 2 else ([a], [dev[n]])
            g.tick(ids, fr)
            grp_a.append((g.get_keypoints(a), g.get_mask(a)))
            if n >= 2:
                grp_b.append((g.get_keypoints(b), g.get_mask(b)))
        g.close()
        exp_a, exp_b = fut_a.result(), fut_b.result()
    for n in range(len(frames)):
        fi = first + n
        check(batch[n], exp_a[0][n], f"4K batch frame {fi}")
        np.testing.assert_array_equal(masks[n], exp_a[1][n], err_msg=f"4K batch mask {fi}")
        check(grp_a[n][0], exp_a[0][n], f"4K group {shape} frame {fi}")
        np.testing.assert_array_equal(grp_a[n][1], exp_a[1][n], err_msg=f"4K group mask {fi}")
    for n in range(len(frames) - 2):
        check(grp_b[n][0], exp_b[0][n], f"4K group (late stream) frame {first + 2 + n}")
        np.testing.assert_array_equal(grp_b[n][1], exp_b[1][n])
    # the moving frames detect; the static ones carry the last moving frame's set whole
    k99 = 99 - first
    assert masks[k99].sum() > 0, "frame 99 moves"
    assert len(batch[k99]) > 10000
    for n in range(100 - first, len(frames)):
        assert masks[n].sum() == 0, f"static frame {first + n} has active bins"
        assert len(batch[n]) == len(batch[k99])
        for f in ("layer", "y", "x", "score"):
            np.testing.assert_array_equal(batch[n][f], batch[k99][f])
        assert (batch[n]["flags"] == fkd.FKD_KP_PROPAGATED).all()
