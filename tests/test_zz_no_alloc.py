"""hc_convolve_noalloc, the entry point for callers that must not allocate
device memory when they call the library (another framework owns the memory
pool, allocation's device-wide synchronisation is unaffordable, or the host
application forbids it after set-up).  It works in a fixed array inside the
library instead of a caller workspace.  Its output must equal hc_convolve's
(bit for bit, the tolerance used throughout these tests) on two calls in a
row, the second of which finds the first call's leftovers in the shared
array; the first call of each pair is also checked against the CPU oracle.
This file is collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1608_00206_gb300 import _lib, inputs  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def L():
    from paper_1608_00206_gb300.build import build
    build()
    assert torch.cuda.is_available()
    torch.cuda.init()
    return _lib.lib()


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _with_workspace(L, x, y, D, code, tdtype):
    """The existing entry point, hc_convolve, with a caller-owned workspace."""
    z = torch.empty(3 ** D, dtype=tdtype, device=DEV)
    nb = L.hc_workspace_size(D, code)
    ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=DEV)
    _lib.check(L.hc_convolve(x.data_ptr(), y.data_ptr(), z.data_ptr(), D, code, ws.data_ptr(),
                             nb, _stream()), "hc_convolve")
    return z


def _no_alloc(L, x, y, D, code, tdtype):
    z = torch.empty(3 ** D, dtype=tdtype, device=DEV)
    _lib.check(L.hc_convolve_noalloc(x.data_ptr(), y.data_ptr(), z.data_ptr(), D, code,
                                     _stream()), "hc_convolve_noalloc")
    return z


CASES = [
    # (code, torch dtype, D of the first call, D of the second call)
    (_lib.HC_INT64, torch.int64, 16, 12),
    (_lib.HC_FP64, torch.float64, 13, 15),
    (_lib.HC_FP32, torch.float32, 17, 11),
    (_lib.HC_FP32_MIXED, torch.float32, 13, 12),
    (_lib.HC_FP32_FF, torch.float32, 12, 13),
]


@pytest.mark.parametrize("code,tdtype,D1,D2", CASES)
def test_no_alloc_matches_hc_convolve_on_two_calls_in_a_row(L, oracle, code, tdtype, D1, D2):
    outs, hosts = [], []
    for call, D in enumerate((D1, D2)):
        if tdtype == torch.int64:
            x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=10 * D + call)
        elif tdtype == torch.float64:
            x, y = inputs.prob_exponential_pair(D, seed=10 * D + call)
        else:
            x, y = inputs.uniform01_pair(D, seed=10 * D + call)
        xt = torch.from_numpy(x).to(DEV)
        yt = torch.from_numpy(y).to(DEV)
        outs.append((_no_alloc(L, xt, yt, D, code, tdtype),
                     _with_workspace(L, xt, yt, D, code, tdtype)))
        hosts.append((x, y))
    torch.cuda.synchronize()
    for got, want in outs:
        g = got.cpu().numpy()
        w = want.cpu().numpy()
        view = np.uint64 if g.itemsize == 8 else np.uint32
        assert np.array_equal(g.view(view), w.view(view))
    # the first call against the oracle in the same arithmetic
    x, y = hosts[0]
    if code == _lib.HC_FP32_MIXED:
        ref = oracle.convolve_mixed(x, y)
    elif code == _lib.HC_FP32_FF:
        ref = oracle.convolve_ff(x, y)
    else:
        ref = oracle.convolve(x, y)
    g = outs[0][0].cpu().numpy()
    view = np.uint64 if g.itemsize == 8 else np.uint32
    assert np.array_equal(g.view(view), ref.view(view))


def test_no_alloc_refuses_problems_beyond_its_array(L):
    D = 18  # int64 needs about 114 MiB of workspace, more than the 16 MiB array
    import ctypes
    builtin = _lib.hc_schedule(_lib.HC_SCHED_CHUNKED, 0, 0, 0)
    assert L.hc_workspace_size_schedule(D, _lib.HC_INT64, ctypes.byref(builtin)) > 16 << 20
    x = torch.zeros(1 << D, dtype=torch.int64, device=DEV)
    z = torch.empty(3 ** D, dtype=torch.int64, device=DEV)
    s = L.hc_convolve_noalloc(x.data_ptr(), x.data_ptr(), z.data_ptr(), D, _lib.HC_INT64,
                              _stream())
    assert s == _lib.HC_ERR_WORKSPACE
