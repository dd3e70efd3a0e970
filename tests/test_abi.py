"""The C ABI library builds, loads and exports every entry point declared in include/relnn.h
(CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "relnn.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(relnn_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2605_24207_b300 import build_lib
    return build_lib.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["relnn_join_build", "relnn_join_probe", "relnn_rule_forward", "relnn_rule_backward",
                     "relnn_rule_plan"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_status_strings_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.relnn_status_string.restype = ctypes.c_char_p
    lib.relnn_version.restype = ctypes.c_int32
    assert lib.relnn_version() >= 100
    assert lib.relnn_status_string(0) == b"ok"
    assert lib.relnn_status_string(3) == b"output capacity too small"


def test_binding_lists_exports(libpath):
    from paper_2605_24207_b300 import relnn
    L = relnn.lib()
    for n in relnn.EXPORTS:
        assert hasattr(L, n)


def test_null_arguments_rejected_on_host(libpath):
    """Argument checks run on the host before any CUDA call."""
    from paper_2605_24207_b300 import relnn
    L = relnn.lib()
    assert L.relnn_join_build(None, 10, 0, None, None) == 1          # null out -> EINVAL
    assert L.relnn_rule_plan(None, None, None) == 1
    assert L.relnn_rule_forward(None, None, None, None, None, None) == 1
    assert L.relnn_plan_info(None, None, None, None) == 1
