"""Host-side checks of libstda that need no GPU: the library loads, exports
every entry point its header declares, and its host logic (parameter
initialisation, status strings, argument validation) is right."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2307_09063_gb300 import build as B
from paper_2307_09063_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    from paper_2307_09063_gb300 import stda

    return stda


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(stda_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(L):
    lib = L.lib()
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_counts(L):
    assert L.num_params() == I.NUM_PARAMS == 137915
    assert L.num_buffers() == I.NUM_BUFFERS == 1360


def test_init_params_bit_exact_with_shared_input_module(L):
    for seed in (0, 7):
        p, b = L.init_params(seed)
        pr, br = I.init_params(seed)
        assert np.array_equal(p.view(np.uint32), pr.view(np.uint32))
        assert np.array_equal(b.view(np.uint32), br.view(np.uint32))


def test_status_strings(L):
    lib = L.lib()
    for s in range(9):
        assert len(lib.stda_status_string(s)) > 0
    assert lib.stda_status_string(0) == b"ok"


def test_null_arguments_rejected_without_gpu(L):
    lib = L.lib()
    assert lib.stda_create(None, None) == L.ERR_INVALID_ARG
    assert lib.stda_destroy(None) == L.ERR_INVALID_ARG
    assert lib.stda_forward(None, None, None, 1, 8, 8, None) == L.ERR_INVALID_ARG
    assert lib.stda_forward_host(None, None, None, 1, 8, 8, None) == L.ERR_INVALID_ARG
    assert lib.stda_init_params(0, None, None) == L.ERR_INVALID_ARG
    cfg = L.Config(12, 16, 1, 0, 0, 0)  # H not a multiple of 8
    h = ctypes.c_void_p()
    assert lib.stda_create(ctypes.byref(cfg), ctypes.byref(h)) == L.ERR_SHAPE
    g = L.GenConfig(64, 16, 60, 64, 1, 1, 1, 1, 0, 0, 0, 0, 1, 1)  # P not a power of two
    assert lib.stda_generate(ctypes.byref(g), 0, 0, 0, 1, 0, None, None, None, None, None) != L.OK
