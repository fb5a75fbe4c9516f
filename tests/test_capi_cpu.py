"""The C-ABI library builds for sm_103a, loads without a GPU and exports every declared symbol;
its reading constants equal the oracle's independently declared ones."""
import ctypes
import os
import re

import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tpc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tpc_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1712_09434_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name


def test_constants_match_oracle(lib_path):
    lib = ctypes.CDLL(lib_path)
    buf = (ctypes.c_int64 * 32)()
    n = lib.tpc_constants(buf, 32)
    mine = [buf[i] for i in range(n)]
    assert mine == list(O.constants().values())


def test_rule_constants_match_oracle(lib_path):
    lib = ctypes.CDLL(lib_path)
    buf = (ctypes.c_int64 * 8)()
    n = lib.tpc_rule_constants(buf, 8)
    assert [buf[i] for i in range(n)] == list(O.rule_constants().values())


def test_match_constants_match_oracle(lib_path):
    lib = ctypes.CDLL(lib_path)
    buf = (ctypes.c_double * 16)()
    n = lib.tpc_match_constants(buf, 16)
    assert n == 11
    assert [buf[i] for i in range(n)] == list(O.its_constants().values()) + list(O.loop_constants().values())


def test_strerror_covers_codes(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.tpc_strerror.restype = ctypes.c_char_p
    seen = {lib.tpc_strerror(c) for c in range(0, -7, -1)}
    assert len(seen) == 7 and b"unknown error" not in seen
