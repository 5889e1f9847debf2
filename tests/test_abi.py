"""CPU-side checks of the C ABI library: it builds, loads, exports exactly the
entry points include/se.h declares, and rejects bad calls without a GPU."""
import ctypes as C
import os
import re

import pytest

from paper_2204_14194_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "se.h")).read()
    return set(re.findall(r"^(?:se_status|const char \*)\s*(se_\w+)\s*\(", text, re.M))


def test_header_declares_binding_exports():
    assert _declared() == set(binding.EXPORTS)


def test_library_loads_and_exports_every_declared_symbol():
    lib = binding.load()
    for name in _declared():
        assert hasattr(lib, name), name
    assert os.path.dirname(binding.lib_path()).startswith(ROOT)


def test_ctx_create_without_device_is_an_error_not_a_crash():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = binding.load()
    h = C.c_void_p()
    st = lib.se_ctx_create(0, 0, C.byref(h))
    assert st in (-1, -3)
    assert not h.value
    assert lib.se_last_error()


def test_null_arguments_rejected():
    lib = binding.load()
    assert lib.se_ctx_destroy(None) == 0
    assert lib.se_plan(None, None, None) == -1
    assert lib.se_extrapolate_batch(None, None, 0, None, None) == -1
    assert lib.se_poll(None, 1, 0, None) == -1
    assert lib.se_plan_reset_tables(None) == -1
    t = C.c_uint64(7)
    assert lib.se_extrapolate_host_async(None, None, 4, None, None, None, None, 0, C.byref(t)) == -1
    assert lib.se_host_wait(None, 1) == -1
    assert b"NULL" in lib.se_last_error()
