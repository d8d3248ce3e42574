"""The N > 1 path of bench.py on CPU: two gloo ranks.

Streams are independent (Eq. 1 only links frames of one stream), so the
path shards by stream: each rank runs its own seeded stream, nothing is
exchanged in the data path, and the only collective is the max-reduction of
the timings. These tests run that host logic with world size 2 on the gloo
backend; the per-rank detection itself is checked against the oracle, as a
rank would run it alone.
"""
import hashlib
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import oracle
    from paper_1503_06959_gb300 import synth
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    w, r, lr = bench.rank_env()
    # timings: rank r is slower on the first value, faster on the second
    ms = bench.max_over_ranks([10.0 + r, 20.0 - r], dist)
    # each rank's own clip, small enough for the oracle
    cfg = synth.config1()
    clip = bench.rank_clip(cfg, r, 4)
    s = oracle.Stream(cfg.W, cfg.H, N_r=cfg.N_r, N_c=cfg.N_c, T_I=cfg.T_I, O=cfg.O,
                      intra=cfg.intra, t=cfg.t, mask_mode=oracle.MASK_ID)
    counts = []
    for f in clip:
        s.push(f)
        counts.append(len(s.keypoints()))
    digest = hashlib.sha256(clip.tobytes()).hexdigest()
    gathered = [None] * world
    dist.all_gather_object(gathered, {"rank": r, "digest": digest, "counts": counts})
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
        json.dump({"env": [w, r, lr], "ms": ms, "gathered": gathered,
                   "value": bench.whole_job_fps(w, 300, 10, ms[0])}, fh)


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r, x in enumerate(res):
        assert x["env"] == [2, r, r]
        # the slowest rank decides each timing, on every rank
        assert x["ms"] == [11.0, 20.0]
        # whole-job value: frames of both ranks over the slowest time
        assert x["value"] == pytest.approx(2 * 300 * 10 / 0.011)
    g = res[0]["gathered"]
    assert g == res[1]["gathered"]
    # independent streams: different clips, each with its own keypoints
    assert g[0]["digest"] != g[1]["digest"]
    assert all(c > 0 for x in g for c in x["counts"])


def test_rank_clips_are_the_single_stream_clips():
    sys.path.insert(0, ROOT)
    import bench
    from paper_1503_06959_gb300 import synth
    cfg = synth.config1()
    np.testing.assert_array_equal(bench.rank_clip(cfg, 0, 3), synth.source_for(cfg, 2).frames(3))
    assert not np.array_equal(bench.rank_clip(cfg, 1, 3), bench.rank_clip(cfg, 0, 3))


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
