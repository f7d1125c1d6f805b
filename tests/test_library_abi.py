"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every symbol include/qmcdu.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_1708_00744_b300 import build as qbuild
from paper_1708_00744_b300 import qmcdu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "qmcdu.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qmcdu_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    qbuild.build()
    return ctypes.CDLL(qbuild.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    assert set(declared_functions()) == set(qmcdu.SIGNATURES)


def test_version_and_argument_errors_without_gpu(lib):
    lib.qmcdu_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.qmcdu_version()
    h = ctypes.c_void_p()
    # invalid arguments are rejected before any CUDA call
    assert lib.qmcdu_create(0, 1, 0, 1, None, ctypes.byref(h)) == 1
    assert lib.qmcdu_create(64, 65, 0, 1, None, ctypes.byref(h)) == 1
    assert lib.qmcdu_create(64, 8, 7, 1, None, ctypes.byref(h)) == 1
    assert lib.qmcdu_create(64, 300, 0, 1, None, ctypes.byref(h)) == 1
    assert lib.qmcdu_create(9000, 8, 0, 1, None, ctypes.byref(h)) == 1
    assert lib.qmcdu_destroy(None) == 1
    assert lib.qmcdu_flush(None) == 1


def test_library_is_built_for_sm_103a():
    assert "arch=compute_103a,code=sm_103a" in qbuild.ARCH


def header_enums():
    text = open(os.path.join(ROOT, "include", "qmcdu.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(QMCDU_\w+)\s*=\s*(\d+)", text)}


def test_binding_constants_match_the_header():
    enums = header_enums()
    opts = {k[len("QMCDU_OPT_"):].lower(): v for k, v in enums.items() if k.startswith("QMCDU_OPT_")}
    assert opts == qmcdu.OPTIONS
    assert {"QMCDU_FP64": qmcdu.PRECISIONS["fp64"], "QMCDU_FP32": qmcdu.PRECISIONS["fp32"],
            "QMCDU_FP32_BF16X3": qmcdu.PRECISIONS["bf16x3"]} == {
        k: enums[k] for k in ("QMCDU_FP64", "QMCDU_FP32", "QMCDU_FP32_BF16X3")}
    status = {v: k[len("QMCDU_"):] for k, v in enums.items()
              if k == "QMCDU_OK" or k.startswith("QMCDU_ERR_")}
    assert status == qmcdu.STATUS
