"""Serving loop: frames of several streams submitted as they arrive,
continuously batched into group ticks. Each stream's results must be the
same alone and in the mix, and equal to the oracle frame by frame."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_1503_06959_gb300 import fkd, synth

pytestmark = pytest.mark.gpu

SPECS = [
    (320, 240, dict(N_r=8, N_c=8, T_I=4, t=20)),
    (333, 207, dict(N_r=7, N_c=9, T_I=3, t=15)),
    (640, 480, dict(N_r=12, N_c=16, T_I=4, t=30)),
]
O, INTRA, FRAMES = 2, 1, 8


def clip(i):
    W, H, _ = SPECS[i]
    return synth.VideoSource(W, H, seed=70 + i, n_movers=2, mover_size=min(W, H) // 4,
                             speed=(2, 4)).frames(FRAMES)


def oracle_run(i, frames):
    W, H, p = SPECS[i]
    s = oracle.Stream(W, H, O=O, intra=INTRA, mask_mode=oracle.MASK_ID, **p)
    out = []
    for f in frames:
        s.push(f)
        out.append(s.keypoints())
    return out


def serve(members, clips, jitter_seed):
    """Submit every frame of the member streams from one thread per stream,
    with random gaps, then drain and collect."""
    srv = fkd.Server(O, INTRA, budget_bytes=2 << 30, max_tick_keypoints=1 << 20)
    ids = {i: srv.open_stream(SPECS[i][0], SPECS[i][1], **SPECS[i][2]) for i in members}
    errors = []

    def feed(i):
        rng = np.random.default_rng(jitter_seed + i)
        for f in clips[i]:
            while True:
                try:
                    srv.submit(ids[i], f)
                    break
                except fkd.FkdError as e:  # queue full: wait for the worker
                    if e.code != fkd.FKD_E_CAPACITY:
                        errors.append(e)
                        return
                    time.sleep(0.001)
            time.sleep(float(rng.uniform(0, 0.004)))

    threads = [threading.Thread(target=feed, args=(i,)) for i in members]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    srv.drain(60000)
    assert not errors, errors
    got = {}
    for i in members:
        res = []
        while (r := srv.poll(ids[i])) is not None:
            res.append(r)
        got[i] = res
    stats = srv.stats()
    srv.close()
    return got, stats


def same(a, b, where):
    assert len(a) == len(b), f"{where}: {len(a)} vs {len(b)}"
    for f in ("layer", "y", "x", "score", "flags"):
        np.testing.assert_array_equal(a[f], b[f], err_msg=f"{where}: {f}")


def test_served_results_equal_alone_in_mix_and_oracle():
    clips = {i: clip(i) for i in range(len(SPECS))}
    expect = {i: oracle_run(i, clips[i]) for i in range(len(SPECS))}
    alone, _ = serve([2], clips, 1)
    mixed, stats = serve([0, 1, 2], clips, 2)
    assert [r[0] for r in alone[2]] == list(range(FRAMES))
    for n in range(FRAMES):
        same(alone[2][n][1], mixed[2][n][1], f"stream 2 frame {n}: alone vs mixed")
    for i in range(len(SPECS)):
        assert [r[0] for r in mixed[i]] == list(range(FRAMES))
        for n in range(FRAMES):
            same(mixed[i][n][1], expect[i][n], f"stream {i} frame {n}")
    assert stats["frames_done"] == 3 * FRAMES and stats["ticks"] >= FRAMES
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    assert stats["mean_batch"] >= 1


def test_admission_by_memory_budget():
    probe = fkd.Server(O, INTRA, budget_bytes=2 << 30, max_tick_keypoints=1 << 16)
    a = probe.open_stream(640, 480, N_r=12, N_c=16)
    need = probe.stats()["bytes_in_use"]
    probe.close()
    # room for the server's own buffers and about one such stream
    srv = fkd.Server(O, INTRA, budget_bytes=int(need * 1.5), max_tick_keypoints=1 << 16)
    a = srv.open_stream(640, 480, N_r=12, N_c=16)
    with pytest.raises(fkd.FkdError) as e:
        srv.open_stream(640, 480, N_r=12, N_c=16)
    assert e.value.code == fkd.FKD_E_BUDGET
    assert srv.stats()["rejected_streams"] == 1
    srv.close_stream(a)
    b = srv.open_stream(640, 480, N_r=12, N_c=16)  # memory came back
    f = clip(2)
    srv.submit(b, f[0])
    srv.drain(10000)
    idx, kp = srv.poll(b)
    assert idx == 0 and len(kp) > 0
    srv.close()


def test_replay_by_reference_equals_oracle_and_drops_when_overloaded():
    """fkd_server_replay submits pinned frames by reference at their arrival
    times from C: the served results equal the oracle's; then an offered load
    far beyond four queued frames per stream drops the surplus (counted) and
    every frame it kept is still served, with results dropped on request."""
    torch = pytest.importorskip("torch")
    clips = {i: clip(i) for i in range(len(SPECS))}
    expect = {i: oracle_run(i, clips[i]) for i in range(len(SPECS))}
    pinned = {i: torch.from_numpy(clips[i]).pin_memory() for i in clips}
    srv = fkd.Server(O, INTRA, budget_bytes=2 << 30, max_tick_keypoints=1 << 20)
    ids = {i: srv.open_stream(SPECS[i][0], SPECS[i][1], **SPECS[i][2]) for i in clips}
    t0 = time.monotonic_ns() + 50_000_000
    ev = sorted((t0 + n * 3_000_000 + i * 500_000, i, n) for i in clips for n in range(FRAMES))
    refused = srv.replay([ids[i] for _, i, _ in ev], [pinned[i][n].data_ptr() for _, i, n in ev],
                         [pinned[i].stride(1) for _, i, _ in ev], [t for t, _, _ in ev])
    srv.drain(60000)
    assert refused == 0
    for i in clips:
        got = []
        while (r := srv.poll(ids[i])) is not None:
            got.append(r)
        assert [r[0] for r in got] == list(range(FRAMES))
        for n in range(FRAMES):
            same(got[n][1], expect[i][n], f"replayed stream {i} frame {n}")
    # overload: every frame of stream 2 offered at the same instant, 4 times over
    srv.stats(reset=True)
    srv.keep_results(False)
    t1 = time.monotonic_ns() + 10_000_000
    refused = srv.replay([ids[2]] * (4 * FRAMES), [pinned[2][n % FRAMES].data_ptr() for n in range(4 * FRAMES)],
                         [pinned[2].stride(1)] * (4 * FRAMES), [t1] * (4 * FRAMES))
    srv.drain(60000)
    st = srv.stats()
    assert refused > 0 and st["frames_done"] == 4 * FRAMES - refused
    assert st["rejected_frames"] == refused
    assert srv.poll(ids[2]) is None  # results were not kept
    srv.close()
