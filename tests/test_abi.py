"""The C library loads without a GPU and exports every entry point include/lq.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "lq.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(lq_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1207_2223_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_functions():
    names = declared_functions()
    assert "lq_create" in names and "lq_solve_MdagM" in names
    assert len(names) >= 10


def test_every_declared_symbol_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declaration():
    from paper_1207_2223_gb300 import lq
    assert set(declared_functions()) == set(lq.SIGNATURES)


def test_version_without_gpu(lib):
    lib.lq_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.lq_version()


def test_create_rejects_bad_shape_without_gpu(lib):
    out = ctypes.c_void_p()
    dims = (ctypes.c_int * 4)(1, 4, 4, 4)
    assert lib.lq_create(ctypes.byref(out), dims, 1, None) == 2      # LQ_ERR_SHAPE
    assert not out.value
    # extents whose product would overflow are refused before it is formed
    for bad in ((65536, 65536, 65536, 65536), (2, 2, 2, 2 ** 30), (2 ** 31 - 1, 2, 2, 2)):
        dims = (ctypes.c_int * 4)(*bad)
        assert lib.lq_create(ctypes.byref(out), dims, 1, None) == 2, bad
        assert not out.value


def declared_constants():
    """Every `NAME = value` of the header's enums (options, precisions, status codes)."""
    txt = open(os.path.join(ROOT, "include", "lq.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    out = {}
    for body in re.findall(r"enum\s*\{([^}]*)\}", txt):
        nxt = 0
        for item in body.split(","):
            item = item.strip()
            if not item:
                continue
            m = re.match(r"(LQ_\w+)\s*(?:=\s*(-?\d+))?$", item)
            assert m, item
            nxt = int(m.group(2)) if m.group(2) is not None else nxt
            out[m.group(1)] = nxt
            nxt += 1
    return out


def test_binding_constants_match_the_header():
    """The binding's precision, status and option constants equal the header's enums."""
    from paper_1207_2223_gb300 import lq
    consts = declared_constants()
    assert "LQ_OPT_HOST_DIRECT" in consts and "LQ_F16_12" in consts and "LQ_ERR_TIMEOUT" in consts
    for name, value in consts.items():
        assert getattr(lq, name) == value, name
