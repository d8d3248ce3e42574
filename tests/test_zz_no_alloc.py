"""The allocation-free entry point fkd_id_mask_noalloc, through the C ABI.

It serves callers that cannot let the library allocate device memory: an
application whose allocator or memory budget owns every byte of the GPU, a
plugin running inside a host program that owns the device memory, a real-time
loop that must not pay for cudaMalloc / cudaFree and their synchronisation.
Its masks must equal, bit for bit, the intensity-difference masks on c_0 of
the CPU oracle and of fkd_push_frames for the same frame pairs, call after
call, although every call reuses the same fixed scratch array.
This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
from paper_1503_06959_gb300 import fkd, synth

pytestmark = pytest.mark.gpu


def oracle_masks(frames, N_r, N_c, T_I):
    """Masks of Eq. 2 on c_0 (bin mean of |I_n - I_{n-1}| above T_I) of
    frames 1.. of a clip, from the CPU oracle."""
    H, W = frames.shape[1:]
    ref = oracle.Stream(W, H, N_r=N_r, N_c=N_c, T_I=T_I, O=1, intra=0, mask_mode=oracle.MASK_ID, mask_layer=0)
    out = []
    for f in frames:
        ref.push(f)
        out.append(ref.mask())
    return out


def test_noalloc_mask_equals_oracle_and_stream_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    cfg = synth.config2()  # 640 x 480, 16 columns x 12 rows of 40 x 40 bins
    frames = synth.source_for(cfg, 2).frames(3)
    exp = oracle_masks(frames, cfg.N_r, cfg.N_c, cfg.T_I)
    s = fkd.Stream(cfg.W, cfg.H, N_r=cfg.N_r, N_c=cfg.N_c, T_I=cfg.T_I, O=1, intra=0, t=cfg.t,
                   mask_mode=fkd.FKD_MASK_ID, T_max=3)
    _, _, masks = s.push_frames(frames)  # masks[n]: frame n against frame n-1
    dev = torch.from_numpy(frames).cuda()
    out = torch.full((cfg.N_r, cfg.N_c), 7, dtype=torch.uint8, device="cuda")
    for n in (1, 2):  # two calls in a row share the scratch array
        fkd.id_mask_noalloc(dev[n], dev[n - 1], cfg.N_r, cfg.N_c, cfg.T_I, out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), exp[n], err_msg=f"pair {n} vs oracle")
        np.testing.assert_array_equal(out.cpu().numpy(), masks[n], err_msg=f"pair {n} vs stream")
    assert 0 < int(exp[1].sum()) < exp[1].size, "the pair must have both kinds of bins"


def test_noalloc_uneven_bins_pitched_frames_side_stream():
    """333 x 251 frames in 7 columns x 5 rows of bins (no bin size divides the
    frame), read from a column slice of a wider buffer (row pitch 400 > W), on
    a non-default CUDA stream, over several consecutive pairs."""
    torch = pytest.importorskip("torch")
    W, H, N_r, N_c, T_I = 333, 251, 5, 7, 4
    frames = synth.VideoSource(W, H, seed=91, n_movers=2, mover_size=60, speed=(3, 5)).frames(5)
    exp = oracle_masks(frames, N_r, N_c, T_I)
    wide = torch.zeros((len(frames), H, 400), dtype=torch.uint8)
    wide[:, :, 40:40 + W] = torch.from_numpy(frames)
    wide = wide.cuda()
    view = wide[:, :, 40:40 + W]  # pitch 400, base offset 40 bytes
    side = torch.cuda.Stream()
    out = torch.full((N_r * N_c,), 9, dtype=torch.uint8, device="cuda")
    seen = set()
    with torch.cuda.stream(side):
        for n in range(1, len(frames)):
            fkd.id_mask_noalloc(view[n], view[n - 1], N_r, N_c, T_I, out, cuda_stream=side.cuda_stream)
            side.synchronize()
            got = out.cpu().numpy().reshape(N_r, N_c)
            np.testing.assert_array_equal(got, exp[n], err_msg=f"pair {n}")
            seen.update(int(v) for v in got.ravel())
    assert seen == {0, 1}, "the pairs must have active and inactive bins"


def test_noalloc_rejects_grids_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    frame = torch.zeros((480, 640), dtype=torch.uint8, device="cuda")
    out = torch.zeros(65 * 64, dtype=torch.uint8, device="cuda")
    with pytest.raises(fkd.FkdError) as e:
        fkd.id_mask_noalloc(frame, frame, 65, 64, 4, out)  # 4160 bins > 4096
    assert e.value.code == fkd.FKD_E_ARG
