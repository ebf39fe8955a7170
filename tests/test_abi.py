"""The C ABI (CPU only): the library loads, exports every symbol that
include/hc.h declares, sizes its workspaces, and rejects bad arguments on the
host before any CUDA call (fake device addresses are never dereferenced)."""
import os
import re

import pytest

from paper_1608_00206_gb300 import _lib
from paper_1608_00206_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build()
    return _lib.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "hc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hc_[a-z0-9_]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert _declared() == sorted(_lib.SIGNATURES)


def test_every_declared_symbol_exported(L):
    assert _lib.missing_symbols() == []


def test_status_strings(L):
    for s in range(8):
        assert L.hc_status_string(s).decode().startswith("HC_")
    assert L.hc_version() > 0


def test_workspace_sizes(L):
    assert L.hc_workspace_size(-1, 0) == 0
    assert L.hc_workspace_size(_lib.HC_MAX_D + 1, 0) == 0
    assert L.hc_workspace_size(5, 9) == 0
    # D <= tile axes: a header only
    assert L.hc_workspace_size(8, _lib.HC_INT64) == 256
    # D = 20 int64: two evaluated operands of 3^12 * 2^8 int64 and ping-pong buffers
    ws = L.hc_workspace_size(20, _lib.HC_INT64)
    assert ws >= 2 * 3 ** 12 * 2 ** 8 * 8
    # mixed precision keeps a float-float copy of the 3^D intermediate
    assert L.hc_workspace_size(16, _lib.HC_FP32_MIXED) >= 3 ** 16 * 8


FAKE = 1 << 40  # a 16-byte aligned fake device address, never dereferenced


def test_argument_errors_caught_on_host(L):
    n2 = 1 << 10
    x, y, z = FAKE, FAKE + 8 * n2, FAKE + 64 * n2
    ws = FAKE + (1 << 30)
    size = L.hc_workspace_size(10, _lib.HC_INT64)
    conv = L.hc_convolve
    assert conv(x, y, z, -1, _lib.HC_INT64, ws, size, None) == _lib.HC_ERR_ARG
    assert conv(x, y, z, _lib.HC_MAX_D + 1, _lib.HC_INT64, ws, size, None) == _lib.HC_ERR_ARG
    assert conv(x, y, z, 10, 7, ws, size, None) == _lib.HC_ERR_DTYPE
    assert conv(None, y, z, 10, _lib.HC_INT64, ws, size, None) == _lib.HC_ERR_ARG
    assert conv(x + 8, y, z, 10, _lib.HC_INT64, ws, size, None) == _lib.HC_ERR_ALIGN
    # z overlapping x or y
    assert conv(x, y, x + 16, 10, _lib.HC_INT64, ws, size, None) == _lib.HC_ERR_ALIAS
    assert conv(x, y, y, 10, _lib.HC_INT64, ws, size, None) == _lib.HC_ERR_ALIAS
    # workspace too small / missing / misaligned
    big = L.hc_workspace_size(20, _lib.HC_INT64)
    zz = FAKE + (1 << 36)
    assert conv(x, y, zz, 20, _lib.HC_INT64, ws, big - 1, None) == _lib.HC_ERR_WORKSPACE
    assert conv(x, y, zz, 20, _lib.HC_INT64, None, big, None) == _lib.HC_ERR_ARG
    assert conv(x, y, zz, 20, _lib.HC_INT64, ws + 16, big, None) == _lib.HC_ERR_ALIGN
    # workspace overlapping the output
    assert conv(x, y, zz, 20, _lib.HC_INT64, zz, big, None) == _lib.HC_ERR_ALIAS
    # explicit schedules out of range
    cfg = L.hc_convolve_config
    assert cfg(x, y, z, 10, _lib.HC_INT64, 9, 0, ws, size, None) == _lib.HC_ERR_ARG
    assert cfg(x, y, z, 10, _lib.HC_INT64, 0, 7, ws, size, None) == _lib.HC_ERR_ARG
    assert L.hc_device_status(None, None) == _lib.HC_ERR_ARG
