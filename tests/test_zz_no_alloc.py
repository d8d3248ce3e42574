"""The allocation-free entry point fkd_id_mask_noalloc, through the C ABI.

It serves callers that cannot let the library allocate device memory (a
host program or allocator that owns all GPU memory, a real-time loop that
must not allocate). Its masks must equal, bit for bit, the intensity-
difference masks fkd_push_frames computes for the same frame pairs, call
after call, although every call reuses the same fixed scratch array.
This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1503_06959_gb300 import fkd, synth

pytestmark = pytest.mark.gpu


def test_noalloc_mask_equals_stream_mask_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    cfg = synth.config2()  # 640 x 480, 16 columns x 12 rows of bins
    frames = synth.source_for(cfg, 2).frames(3)
    s = fkd.Stream(cfg.W, cfg.H, N_r=cfg.N_r, N_c=cfg.N_c, T_I=cfg.T_I, O=1, intra=0, t=cfg.t,
                   mask_mode=fkd.FKD_MASK_ID, T_max=3)
    _, _, masks = s.push_frames(frames)  # masks[n]: frame n against frame n-1
    dev = torch.from_numpy(frames).cuda()
    out = torch.full((cfg.N_r, cfg.N_c), 7, dtype=torch.uint8, device="cuda")
    for n in (1, 2):  # two calls in a row share the scratch array
        fkd.id_mask_noalloc(dev[n], dev[n - 1], cfg.N_r, cfg.N_c, cfg.T_I, out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), masks[n])
    assert 0 < int(masks[1].sum()) < masks[1].size, "the pair must have both kinds of bins"


def test_noalloc_rejects_grids_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    frame = torch.zeros((480, 640), dtype=torch.uint8, device="cuda")
    out = torch.zeros(65 * 64, dtype=torch.uint8, device="cuda")
    with pytest.raises(fkd.FkdError) as e:
        fkd.id_mask_noalloc(frame, frame, 65, 64, 4, out)  # 4160 bins > 4096
    assert e.value.code == fkd.FKD_E_ARG
