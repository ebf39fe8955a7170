"""The C ABI (CPU only): the library loads, exports every symbol that
include/hc.h declares, sizes its workspaces, and rejects bad arguments on the
host before any CUDA call (fake device addresses are never dereferenced)."""
import ctypes
import os
import re

import pytest

from paper_1608_00206_gb300 import _lib
from paper_1608_00206_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    """The library with the built-in default schedules for the duration of
    the module (a tuned table installed by an earlier test in the same
    process is put back afterwards)."""
    build()
    lib = _lib.lib()
    saved = {}
    for D in range(_lib.HC_MAX_D + 1):
        for dt in range(4):
            s = _lib.hc_schedule()
            assert lib.hc_get_default_schedule(D, dt, ctypes.byref(s)) == 0
            saved[D, dt] = s
            assert lib.hc_set_default_schedule(D, dt, None) == 0
    yield lib
    for (D, dt), s in saved.items():
        builtin = _lib.hc_schedule()
        lib.hc_get_default_schedule(D, dt, ctypes.byref(builtin))
        if s.as_dict() != builtin.as_dict():
            assert lib.hc_set_default_schedule(D, dt, ctypes.byref(s)) == 0


def _declared():
    src = open(os.path.join(ROOT, "include", "hc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hc_[a-z0-9_]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert _declared() == sorted(_lib.SIGNATURES)


def test_every_declared_symbol_exported(L):
    assert _lib.missing_symbols() == []


def test_default_schedule_table(L):
    """hc_set_default_schedule changes what hc_convolve and hc_workspace_size
    use for one (D, dtype); NULL restores the built-in choice."""
    got = _lib.hc_schedule()
    assert L.hc_get_default_schedule(20, _lib.HC_INT64, ctypes.byref(got)) == 0
    assert got.kind == _lib.HC_SCHED_CHUNKED
    builtin = L.hc_workspace_size(20, _lib.HC_INT64)
    s = _lib.hc_schedule(_lib.HC_SCHED_PASSES, 8, 6, 16)
    assert L.hc_set_default_schedule(20, _lib.HC_INT64, ctypes.byref(s)) == 0
    try:
        assert L.hc_get_default_schedule(20, _lib.HC_INT64, ctypes.byref(got)) == 0
        assert got.as_dict() == {"kind": 1, "c": 8, "k": 6, "cols": 16, "cols_outer": 0, "top": 0}
        assert L.hc_workspace_size(20, _lib.HC_INT64) == \
            L.hc_workspace_size_schedule(20, _lib.HC_INT64, ctypes.byref(s))
        assert L.hc_workspace_size(19, _lib.HC_INT64) != 0  # other entries untouched
    finally:
        assert L.hc_set_default_schedule(20, _lib.HC_INT64, None) == 0
    assert L.hc_workspace_size(20, _lib.HC_INT64) == builtin
    assert L.hc_autotune_workspace_size(20, _lib.HC_INT64) >= builtin


def test_status_strings(L):
    for s in range(8):
        assert L.hc_status_string(s).decode().startswith("HC_")
    # the float-float dtype: x, y, z are float32; plain form only
    assert L.hc_workspace_size(12, _lib.HC_FP32_FF) > 0
    assert L.hc_backward_workspace_size(12, _lib.HC_FP32_FF) == 0
    assert L.hc_workspace_size(5, 5) == 0
    assert L.hc_version() > 0


def test_workspace_sizes(L):
    assert L.hc_workspace_size(-1, 0) == 0
    assert L.hc_workspace_size(_lib.HC_MAX_D + 1, 0) == 0
    assert L.hc_workspace_size(5, 9) == 0
    # default (chunked) schedule: a single chunk with at most 3 middle axes
    # needs only the status header and two counters
    assert L.hc_workspace_size(8, _lib.HC_INT64) == 512
    assert L.hc_workspace_size(11, _lib.HC_INT64) == 512
    # D = 20 int64: 3^6 chunks of 14 axes; the operands evaluated on the 6
    # outer and the first 3 middle axes, [3^9][2^11] int64 each
    ws = L.hc_workspace_size(20, _lib.HC_INT64)
    assert ws >= 2 * 3 ** 9 * 2 ** 11 * 8
    # whole-array-pass schedule: operands evaluated on the 12 outer axes
    s = _lib.hc_schedule(_lib.HC_SCHED_PASSES, 8, 6, 0)
    assert L.hc_workspace_size_schedule(20, _lib.HC_INT64, ctypes.byref(s)) >= \
        2 * 3 ** 12 * 2 ** 8 * 8
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
    for bad in [(1, 9, 0, 0), (2, 0, 7, 0), (5, 0, 0, 0), (3, 0, 7, 0), (1, 0, 0, 12), (-1, 0, 0, 0),
                (4, 8, 6, 0, 0, 0), (4, 9, 6, 0, 0, 3), (4, 8, 6, 0, 0, 7), (1, 8, 6, 0, 0, 2),
                (1, 0, 0, -8), (2, 0, 0, -64), (1, 8, 6, 16, 12), (1, 8, 6, 16, -8)]:
        s = _lib.hc_schedule(*bad)
        assert L.hc_convolve_schedule(x, y, z, 10, _lib.HC_INT64, ctypes.byref(s), ws, size,
                                      None) == _lib.HC_ERR_ARG
        assert L.hc_set_default_schedule(10, _lib.HC_INT64, ctypes.byref(s)) == _lib.HC_ERR_ARG
    # 16-byte row copies are a valid tile width
    for good in [(1, 8, 6, -16), (2, 8, 6, -32), (1, 8, 6, 16, 32), (1, 8, 6, 32, -16)]:
        s = _lib.hc_schedule(*good)
        assert L.hc_set_default_schedule(10, _lib.HC_INT64, ctypes.byref(s)) == _lib.HC_OK
    assert L.hc_set_default_schedule(10, _lib.HC_INT64, None) == _lib.HC_OK
    assert L.hc_convolve_schedule(x, y, z, 10, _lib.HC_INT64, None, ws, size, None) == \
        _lib.HC_ERR_ARG
    assert L.hc_device_status(None, None) == _lib.HC_ERR_ARG
    # the hybrid schedule: fewer than 4 axes below the direct ones, or a
    # float-float dtype
    s = _lib.hc_schedule(_lib.HC_SCHED_HYBRID, 8, 6, 0, 0, 7)
    assert L.hc_convolve_schedule(x, y, z, 10, _lib.HC_INT64, ctypes.byref(s), ws, size,
                                  None) == _lib.HC_ERR_ARG
    s = _lib.hc_schedule(_lib.HC_SCHED_HYBRID, 8, 6, 0, 0, 2)
    assert L.hc_convolve_schedule(x, y, z, 10, _lib.HC_FP32_MIXED, ctypes.byref(s), ws, size,
                                  None) == _lib.HC_ERR_ARG
    assert L.hc_workspace_size_schedule(10, _lib.HC_INT64, ctypes.byref(s)) > 0
    # a default schedule keeps the recurrence's rounding: hybrid for int64 only
    assert L.hc_set_default_schedule(10, _lib.HC_FP32, ctypes.byref(s)) == _lib.HC_ERR_ARG
    assert L.hc_set_default_schedule(10, _lib.HC_INT64, ctypes.byref(s)) == _lib.HC_OK
    assert L.hc_set_default_schedule(10, _lib.HC_INT64, None) == _lib.HC_OK


# Largest D that hc_convolve_noalloc accepts per dtype, as include/hc.h states
# it (16 MiB array, built-in chunked schedule).
NOALLOC_LIMITS = {_lib.HC_INT64: 16, _lib.HC_FP64: 16, _lib.HC_FP32: 17, _lib.HC_FP32_MIXED: 13,
                  _lib.HC_FP32_FF: 13}


@pytest.mark.parametrize("code,limit", sorted(NOALLOC_LIMITS.items()))
def test_noalloc_limits_per_dtype(L, code, limit):
    """The documented per-dtype limits of the no-allocation entry point hold:
    the built-in chunked schedule's workspace fits the fixed array at the
    limit and not one axis beyond, and a call one axis beyond is refused on
    the host (fake addresses, no CUDA call)."""
    cap = 16 << 20
    builtin = _lib.hc_schedule(_lib.HC_SCHED_CHUNKED, 0, 0, 0, 0)
    assert L.hc_workspace_size_schedule(limit, code, ctypes.byref(builtin)) <= cap
    assert L.hc_workspace_size_schedule(limit + 1, code, ctypes.byref(builtin)) > cap
    D = limit + 1
    x, y, z = FAKE, FAKE + (1 << 32), FAKE + (1 << 36)
    assert L.hc_convolve_noalloc(x, y, z, D, code, None) == _lib.HC_ERR_WORKSPACE


def test_carryfree_arguments_caught_on_host(L):
    """hc_carryfree sizes its workspace (padded copies of both vectors plus
    the plain form's workspace) and rejects bad arguments before any CUDA
    call."""
    es = 8
    for N, D in [(1, 0), (2, 1), (5, 3), (8, 3), (9, 4), (3001, 12)]:
        nb = L.hc_carryfree_workspace_size(N, _lib.HC_INT64)
        conv = L.hc_workspace_size(D, _lib.HC_INT64)
        if N == 1 << D:
            assert nb == conv
        else:
            assert nb >= 2 * (es << D) + conv
    assert L.hc_carryfree_workspace_size(0, _lib.HC_INT64) == 0
    assert L.hc_carryfree_workspace_size((1 << _lib.HC_MAX_D) + 1, _lib.HC_INT64) == 0
    assert L.hc_carryfree_workspace_size(5, 9) == 0
    x, y, z, ws = FAKE, FAKE + (1 << 20), FAKE + (1 << 24), FAKE + (1 << 30)
    N = 3001
    nb = L.hc_carryfree_workspace_size(N, _lib.HC_INT64)
    cf = L.hc_carryfree
    assert cf(x, y, z, 0, _lib.HC_INT64, ws, nb, None) == _lib.HC_ERR_ARG
    assert cf(x, y, z, N, 9, ws, nb, None) == _lib.HC_ERR_DTYPE
    assert cf(None, y, z, N, _lib.HC_INT64, ws, nb, None) == _lib.HC_ERR_ARG
    assert cf(x + 8, y, z, N, _lib.HC_INT64, ws, nb, None) == _lib.HC_ERR_ALIGN
    assert cf(x, y, z, N, _lib.HC_INT64, ws, nb - 1, None) == _lib.HC_ERR_WORKSPACE
    assert cf(x, y, z, N, _lib.HC_INT64, None, nb, None) == _lib.HC_ERR_ARG
    assert cf(x, y, z, N, _lib.HC_INT64, ws + 16, nb, None) == _lib.HC_ERR_ALIGN
    assert cf(x, y, x + 16, N, _lib.HC_INT64, ws, nb, None) == _lib.HC_ERR_ALIAS
    assert cf(x, y, z, N, _lib.HC_INT64, z, nb, None) == _lib.HC_ERR_ALIAS
    assert cf(x, y, z, N, _lib.HC_INT64, y - 256, nb, None) == _lib.HC_ERR_ALIAS


def test_lowmem_workspace_is_small(L):
    """The low-workspace schedule needs the two leaf inputs and one leaf's
    workspace: at D = 20 int64 with 6 top axes, inputs of 2^14 elements and a
    14-axis leaf's operands -- a few MB against the 2.2 GB of the whole-array
    passes."""
    s = _lib.hc_schedule(_lib.HC_SCHED_LOWMEM, 8, 6, 16, 32, 6)
    low = L.hc_workspace_size_schedule(20, _lib.HC_INT64, ctypes.byref(s))
    p = _lib.hc_schedule(_lib.HC_SCHED_PASSES, 8, 6, 16, 32, 0)
    passes = L.hc_workspace_size_schedule(20, _lib.HC_INT64, ctypes.byref(p))
    assert 0 < low < 8 << 20 and passes > 2 * 3 ** 12 * 2 ** 8 * 8
    # D = 22: leaves of 16 axes, still a small fraction of the passes' need
    assert L.hc_workspace_size_schedule(22, _lib.HC_INT64, ctypes.byref(s)) * 50 < \
        L.hc_workspace_size_schedule(22, _lib.HC_INT64, ctypes.byref(p))
    # not for the float-float dtypes, and not when no axis is left below
    assert L.hc_workspace_size_schedule(20, _lib.HC_FP32_MIXED, ctypes.byref(s)) == 0
    x, y, z, ws = FAKE, FAKE + (1 << 20), FAKE + (1 << 24), FAKE + (1 << 30)
    bad = _lib.hc_schedule(_lib.HC_SCHED_LOWMEM, 8, 6, 16, 32, 6)
    assert L.hc_convolve_schedule(x, y, z, 6, _lib.HC_INT64, ctypes.byref(bad), ws, 1 << 20,
                                  None) == _lib.HC_ERR_ARG


def test_maxconv_plan_matches_the_oracle(L, oracle):
    """hc_maxconv_plan's p is the oracle's exact choice (the smallest p with
    M (2^(D/p) - 1) < 7/16, decided in integers), and its limbs hold vmax^p
    with every convolution entry below 2^63."""
    for D in range(0, 17):
        for vmax in (0, 1, 2, 3, 5, 7, 15, 40):
            p, b, e, n = (ctypes.c_int() for _ in range(4))
            st = L.hc_maxconv_plan(D, vmax, ctypes.byref(p), ctypes.byref(b), ctypes.byref(e),
                                   ctypes.byref(n))
            if st != _lib.HC_OK:
                assert st == _lib.HC_ERR_ARG
                assert L.hc_maxconv_workspace_size(D, vmax) == 0
                # refused only where the oracle's own plan needs more than 12
                # limb axes or more than HC_MAX_D axes in all
                try:
                    _, _, eo, _ = oracle.maxconv_limb_plan(D, vmax)
                    assert eo > 12 or D + eo > _lib.HC_MAX_D
                except ValueError:
                    pass
                continue
            assert p.value == oracle.maxconv_p(D, vmax), (D, vmax)
            bits = max(1, (vmax ** p.value).bit_length()) if vmax > 1 else 1
            assert n.value * b.value >= bits and n.value <= (1 << e.value)
            assert D + e.value + 2 * b.value <= 63 and 1 <= b.value <= 31
            De = D + e.value
            nb = L.hc_maxconv_workspace_size(D, vmax)
            assert nb >= 2 * (8 << De) + 8 * 3 ** De + L.hc_workspace_size(De, _lib.HC_INT64)


def test_maxconv_arguments_caught_on_host(L):
    """hc_maxconv rejects bad arguments before any CUDA call."""
    D, vmax = 6, 3
    nb = L.hc_maxconv_workspace_size(D, vmax)
    assert nb > 0
    x, y, z, ws = FAKE, FAKE + (1 << 20), FAKE + (1 << 24), FAKE + (1 << 30)
    mc = L.hc_maxconv
    assert mc(x, y, z, -1, vmax, ws, nb, None) == _lib.HC_ERR_ARG
    assert mc(x, y, z, D, -1, ws, nb, None) == _lib.HC_ERR_ARG
    assert mc(x, y, z, D, 1 << 40, ws, nb, None) == _lib.HC_ERR_ARG
    assert mc(x, y, z, 20, 1000, ws, nb, None) == _lib.HC_ERR_ARG   # no plan
    assert mc(None, y, z, D, vmax, ws, nb, None) == _lib.HC_ERR_ARG
    assert mc(x, y, z, D, vmax, None, nb, None) == _lib.HC_ERR_ARG
    assert mc(x + 8, y, z, D, vmax, ws, nb, None) == _lib.HC_ERR_ALIGN
    assert mc(x, y, z, D, vmax, ws + 16, nb, None) == _lib.HC_ERR_ALIGN
    assert mc(x, y, z, D, vmax, ws, nb - 1, None) == _lib.HC_ERR_WORKSPACE
    assert mc(x, y, x + 16, D, vmax, ws, nb, None) == _lib.HC_ERR_ALIAS
    assert mc(x, y, z, D, vmax, z, nb, None) == _lib.HC_ERR_ALIAS
