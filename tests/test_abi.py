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
