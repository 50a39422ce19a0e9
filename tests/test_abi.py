"""The C-ABI library builds, loads without a GPU, and exports every declared entry point."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2310_03920_gb300", "libb2.so")


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(b2_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        import __graft_entry__
        __graft_entry__.build()
    return ctypes.CDLL(LIB)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_binds_every_symbol(lib):
    from paper_2310_03920_gb300 import b2
    assert set(b2.EXPORTED) == _declared()


def test_create_without_gpu_fails_cleanly(lib):
    """On a machine without a GPU b2_create returns an error code and a message; it must
    not abort the process."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    lib.b2_create.restype = ctypes.c_int
    lib.b2_last_error.restype = ctypes.c_char_p
    h = ctypes.c_void_p()
    rc = lib.b2_create(ctypes.byref(h), 0, None, None, None, None)
    assert rc in (-1, -3)
    assert lib.b2_last_error(None)
