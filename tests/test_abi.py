"""The C-ABI library builds, loads without a GPU, exports every entry point
that include/fkd.h declares, and rejects bad arguments on the host."""
import ctypes
import os
import re

import pytest

from paper_1503_06959_gb300 import fkd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "fkd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fkd_\w+)\s*\(", text)))


def test_header_declares_the_binding_exports():
    assert declared_functions() == sorted(fkd.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = fkd.load()
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_debug_library_loads_and_exports_every_declared_symbol():
    """libfkd_check.so (FKD_CHECK=1: index checks, guard bands) builds, loads
    without a GPU, exports the same entry points and says it is the debug
    build; the release library says it is not."""
    from paper_1503_06959_gb300 import build
    dbg = ctypes.CDLL(build.build(check=True))
    for name in declared_functions():
        assert hasattr(dbg, name), name
    assert dbg.fkd_check_build() == 1
    assert fkd.load().fkd_check_build() == 0


def test_params_default_and_validation_without_gpu():
    lib = fkd.load()
    p = fkd.params_default()
    assert (p.version, p.N_r, p.N_c, p.t, p.n, p.O, p.mask_mode, p.T_max) == (3, 8, 8, 20, 9, 1, 1, 1)
    h = ctypes.c_void_p()
    bad = [dict(n=8), dict(t=0), dict(t=256), dict(O=7), dict(N_r=0), dict(N_c=700),
           dict(mask_mode=4), dict(mask_layer=1), dict(K_max=0), dict(T_max=0), dict(intra=2),
           dict(version=1), dict(version=2), dict(T_I=-1), dict(nms_scale=2)]
    for over in bad:
        q = fkd.params_default()
        for k, v in over.items():
            setattr(q, k, v)
        rc = lib.fkd_create_stream(ctypes.byref(q), 640, 480, None, ctypes.byref(h))
        assert rc == fkd.FKD_E_ARG, over
        assert lib.fkd_last_error()
    q = fkd.params_default()
    for W, H in [(0, 10), (10, 0), (16385, 10)]:
        assert lib.fkd_create_stream(ctypes.byref(q), W, H, None, ctypes.byref(h)) == fkd.FKD_E_ARG
    assert lib.fkd_create_stream(None, 64, 64, None, ctypes.byref(h)) == fkd.FKD_E_ARG
    assert lib.fkd_destroy_stream(None) == fkd.FKD_OK
    assert lib.fkd_push_frame(None, None, 0, 0) == fkd.FKD_E_ARG
    assert lib.fkd_synchronize(None) == fkd.FKD_E_ARG


def test_descriptor_entry_points_reject_bad_arguments_without_gpu():
    """Argument checks that run before any device work."""
    lib = fkd.load()
    n = ctypes.c_size_t()
    assert lib.fkd_set_descriptor(None, None, 0) == fkd.FKD_E_ARG
    assert lib.fkd_get_descriptors(None, None, 0, ctypes.byref(n), 0) == fkd.FKD_E_ARG
    assert lib.fkd_group_set_descriptor(None, 0, None, 0) == fkd.FKD_E_ARG
    assert lib.fkd_group_get_descriptors(None, 0, None, 0, None, 0) == fkd.FKD_E_ARG
    assert lib.fkd_server_set_descriptor(None, 0, None, 0) == fkd.FKD_E_ARG
    assert lib.fkd_server_get_descriptors(None, 0, None, 0, ctypes.byref(n)) == fkd.FKD_E_ARG


def test_descriptor_pattern_generator():
    """The seeded pattern: deterministic, D x 4 int8 within the library's
    offset bound, not degenerate."""
    import numpy as np

    from paper_1503_06959_gb300 import synth
    a, b = synth.descriptor_pattern(256, seed=3), synth.descriptor_pattern(256, seed=3)
    np.testing.assert_array_equal(a, b)
    assert a.shape == (256, 4) and a.dtype == np.int8
    assert np.abs(a).max() <= synth.DESC_RADIUS == 13
    assert not np.array_equal(a, synth.descriptor_pattern(256, seed=4))
    assert (a[:, :2] != a[:, 2:]).any(axis=1).mean() > 0.95  # pairs of two distinct points


def test_bench_reads_profile_counters_per_launch_shape(tmp_path, monkeypatch):
    """The bench takes the dominant kernel's traffic and ALU counts from a
    profile summary only for the launch shape in use and while the kernel's
    sources match the hash the summary records."""
    import hashlib
    import sys
    sys.path.insert(0, ROOT)
    import bench
    csrc = tmp_path / "paper_1503_06959_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    h = hashlib.sha256()
    for f in bench.KERNEL_SOURCES["detect"]:
        data = open(os.path.join(ROOT, "paper_1503_06959_gb300", "csrc", f), "rb").read()
        (csrc / f).write_bytes(data)
        h.update(data)
    summary = (f"source_sha256: {h.hexdigest()[:16]}\n"
               "counters 16,8,2: traffic_bytes_per_launch 1000 alu_warp_inst_per_launch 2000 "
               "alu_peak_warp_inst_per_sm_cycle 2\n")
    (tmp_path / "profiles" / "k_detect_masked_clip_640x480x300.md").write_text(summary)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    got = bench.profile_counters("detect", dict(tile_h=16, warps_per_cta=8, ctas_per_sm=2))
    assert got == {"traffic_bytes_per_launch": 1000.0, "alu_warp_inst_per_launch": 2000.0,
                   "alu_peak_warp_inst_per_sm_cycle": 2.0}
    assert bench.profile_counters("detect", dict(tile_h=8, warps_per_cta=4, ctas_per_sm=1)) is None
    # a changed source no longer matches the recorded hash
    (csrc / bench.KERNEL_SOURCES["detect"][0]).write_bytes(data + b"\n")
    assert bench.profile_counters("detect", dict(tile_h=16, warps_per_cta=8, ctas_per_sm=2)) is None
