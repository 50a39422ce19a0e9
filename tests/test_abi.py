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


def _header_structs():
    """{typedef name: [(type, field), ...]} of the typedef'd structs in include/b2.h, and the
    integer #defines."""
    src = open(os.path.join(ROOT, "include", "b2.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    defines = {m.group(1): eval(m.group(2)) for m in
               re.finditer(r"#define\s+(B2_[A-Z0-9_]+)\s+\(?([0-9]+(?:\s*<<\s*[0-9]+)?)\)?", src)}
    structs = {}
    for m in re.finditer(r"typedef struct\s*\{(.*?)\}\s*(b2_[a-z0-9_]+)\s*;", src, flags=re.S):
        fields = []
        for decl in m.group(1).split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            fm = re.match(r"(.*?)\s*(\**)\s*([a-z0-9_]+)\s*(\[[A-Z0-9_]+\])?$", decl)
            fields.append((fm.group(1) + fm.group(2) + (fm.group(4) or ""), fm.group(3)))
        structs[m.group(2)] = fields
    return structs, defines


def _ctype_of(c_type, defines):
    c_type = c_type.replace("const ", "")
    arr = re.search(r"\[([A-Z0-9_]+)\]$", c_type)
    base = re.sub(r"\[.*\]$", "", c_type)
    table = {"int": ctypes.c_int, "double": ctypes.c_double, "b2_prec": ctypes.c_int,
             "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64, "size_t": ctypes.c_size_t}
    if base.endswith("*"):
        t = ctypes.c_void_p
    else:
        t = table[base]
    if arr:
        n = int(arr.group(1)) if arr.group(1).isdigit() else defines[arr.group(1)]
        t = t * n
    return t


def test_binding_structs_match_the_header(lib):
    """The ctypes mirrors in the binding have the header's fields, in order, with the same
    sizes and offsets (a reordered or missing field would corrupt every call)."""
    from paper_2310_03920_gb300 import b2
    structs, defines = _header_structs()
    mirrors = {"b2_dav_opts": b2.DavOpts, "b2_sweep_opts": b2.SweepOpts,
               "b2_sweep_result": b2.SweepResult, "b2_tdvp_opts": b2.TdvpOpts,
               "b2_tdvp_result": b2.TdvpResult}
    for name, cls in mirrors.items():
        fields = structs[name]
        assert [f for _, f in fields] == [f for f, _ in cls._fields_], name

        class Ref(ctypes.Structure):
            _fields_ = [(f, _ctype_of(t, defines)) for t, f in fields]
        assert ctypes.sizeof(Ref) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert getattr(Ref, f).offset == getattr(cls, f).offset, (name, f)
            assert getattr(Ref, f).size == getattr(cls, f).size, (name, f)


def test_binding_constants_match_the_header():
    from paper_2310_03920_gb300 import b2
    _, defines = _header_structs()
    assert defines["B2_ONE_SITE"] == b2.B2_ONE_SITE
    assert b2.SweepResult.root_energy.size == 8 * defines["B2_MAX_ROOTS"]
