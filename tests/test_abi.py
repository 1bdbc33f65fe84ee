"""The C-ABI library builds, loads and exports every function include/gpe.h declares
(no compute calls; runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2310_03636_gb300", "libgpe.so")


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            if m.group(1) not in ("if", "while", "sizeof", "defined"):
                names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2310_03636_gb300 import build
        build.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("tw_init_noise", "gpe_step_batch", "observables_accumulate", "gpe_batch_create",
              "gpe_batch_destroy", "gpe_sync_status", "gpe_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_argument_errors_without_gpu(lib):
    """Argument checks return GPE_EINVAL before any device work."""
    lib.gpe_batch_create.restype = ctypes.c_int
    out = ctypes.c_void_p()
    assert lib.gpe_batch_create(None, 0, 0, None, ctypes.byref(out)) == 1
    lib.gpe_last_error.restype = ctypes.c_char_p
    assert lib.gpe_last_error()
    lib.gpe_step_batch.restype = ctypes.c_int
    assert lib.gpe_step_batch(None, ctypes.c_int64(1), None) == 1
    lib.gpe_fma_rate.restype = ctypes.c_int
    rate = ctypes.c_double(0.0)
    assert lib.gpe_fma_rate(ctypes.c_int32(3), ctypes.c_int64(16), ctypes.byref(rate), None) == 1
    assert lib.gpe_fma_rate(ctypes.c_int32(0), ctypes.c_int64(0), ctypes.byref(rate), None) == 1
    assert lib.gpe_fma_rate(ctypes.c_int32(0), ctypes.c_int64(16), None, None) == 1
    lib.gpe_batch_set_tiles.restype = ctypes.c_int
    assert lib.gpe_batch_set_tiles(None, 0, 4, 0) == 1
    lib.gpe_batch_set_lanes.restype = ctypes.c_int
    assert lib.gpe_batch_set_lanes(None, 2) == 1
    lib.gpe_debug_table_memory.restype = ctypes.c_int
    assert lib.gpe_debug_table_memory(ctypes.c_int32(2)) == 1
    assert lib.gpe_debug_table_memory(ctypes.c_int32(-1)) == 1
    assert lib.gpe_debug_table_memory(ctypes.c_int32(1)) == 0
