"""GPU parity of the max-convolution (hc_maxconv through the C ABI; paper,
Discussion: exact max-convolution of bounded non-negative integers through a
p-norm ring) against the oracle's max-convolution from its definition.
Results are integers and must be bit-exact."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1608_00206_gb300 import _lib, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def hc():
    from paper_1608_00206_gb300.build import build
    build()
    import paper_1608_00206_gb300 as hc
    assert torch.cuda.is_available()
    return hc


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def gpu_max(hc, x, y, vmax, **kw):
    z = hc.maxconv(T(x), T(y), vmax, **kw)
    torch.cuda.synchronize()
    return z.cpu().numpy().reshape(-1)


def assert_equal(got, want):
    assert got.shape == want.shape
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, f"{bad.size} mismatches, first at {bad[:5]}: {got[bad[:5]]} vs {want[bad[:5]]}"


# (D, vmax): the limb embedding spans 0 to 6 extra axes, D + e up to 18
CASES = [(0, 5), (0, 2 ** 31 - 1), (1, 3), (2, 15), (3, 0), (3, 31), (4, 1), (4, 7), (5, 2),
         (6, 3), (6, 7), (8, 3), (9, 2), (10, 3), (11, 1), (12, 3), (13, 2)]


@pytest.mark.parametrize("D,vmax", CASES)
def test_maxconv_bit_exact(hc, D, vmax):
    x, y = inputs.uniform_int_pair(D, 0, vmax, seed=1000 + 37 * D + vmax % 1000)
    assert_equal(gpu_max(hc, x, y, vmax), oracle.maxconv_brute(x, y))


@pytest.mark.parametrize("D,vmax", [(4, 3), (6, 2), (8, 3), (5, 7), (12, 1)])
def test_maxconv_tightest_case(hc, D, vmax):
    """Every entry vmax: the all-ones output has 2^D equal products M, where
    the p-norm estimate sits furthest above the maximum."""
    x = np.full(1 << D, vmax, dtype=np.int64)
    got = gpu_max(hc, x, x, vmax)
    assert_equal(got, oracle.maxconv_brute(x, x))
    assert got[(3 ** D - 1) // 2] == vmax * vmax


@pytest.mark.parametrize("D,vmax", [(6, 3), (10, 2)])
def test_maxconv_sparse_inputs(hc, D, vmax):
    """Mostly zero entries: outputs whose pairs are all zero are 0, and small
    maxima next to large ones survive the p-th powers."""
    g = np.random.default_rng(D)
    x = np.where(g.random(1 << D) < 0.2, g.integers(1, vmax + 1, 1 << D), 0).astype(np.int64)
    y = np.where(g.random(1 << D) < 0.2, g.integers(1, vmax + 1, 1 << D), 0).astype(np.int64)
    assert_equal(gpu_max(hc, x, y, vmax), oracle.maxconv_brute(x, y))


def test_maxconv_bound_larger_than_the_entries(hc):
    """vmax only bounds the entries: a larger bound gives the same maxima."""
    D = 7
    x, y = inputs.uniform_int_pair(D, 0, 3, seed=5)
    want = oracle.maxconv_brute(x, y)
    for vmax in (3, 4, 9):
        assert_equal(gpu_max(hc, x, y, vmax), want)


def test_maxconv_out_of_range_entry_is_reported(hc):
    """An entry outside [0, vmax] is recorded as HC_ERR_ARG in the workspace
    status word; the next call with valid entries clears it."""
    D, vmax = 5, 3
    x, y = inputs.uniform_int_pair(D, 0, vmax, seed=6)
    nb = hc.maxconv_workspace_size(D, vmax)
    ws = torch.empty(nb, dtype=torch.uint8, device=DEV)
    bad = x.copy()
    bad[3] = vmax + 1
    hc.maxconv(T(bad), T(y), vmax, workspace=ws)
    assert hc.device_status(ws) == _lib.HC_ERR_ARG
    bad[3] = -1
    hc.maxconv(T(x), T(bad), vmax, workspace=ws)
    assert hc.device_status(ws) == _lib.HC_ERR_ARG
    z = hc.maxconv(T(x), T(y), vmax, workspace=ws)
    assert hc.device_status(ws) == _lib.HC_OK
    assert_equal(z.cpu().numpy(), oracle.maxconv_brute(x, y))


def test_maxconv_shaped_output(hc):
    D, vmax = 3, 2
    x, y = inputs.uniform_int_pair(D, 0, vmax, seed=8)
    z = hc.maxconv(T(x.reshape((2,) * D)), T(y.reshape((2,) * D)), vmax)
    assert tuple(z.shape) == (3,) * D
    assert_equal(z.cpu().numpy().reshape(-1), oracle.maxconv_brute(x, y))


@pytest.mark.slow
def test_maxconv_bench_workload(hc):
    """The benchmark's max-convolution workload at full size: D = 14, entries
    iid in [0, 3] (a 4-axis limb embedding, an 18-axis int64 convolution),
    every output against the oracle's definition."""
    D, vmax = 14, 3
    x, y = inputs.uniform_int_pair(D, 0, vmax, seed=14)
    plan = hc.maxconv_plan(D, vmax)
    assert plan["e"] == 4
    assert_equal(gpu_max(hc, x, y, vmax), oracle.maxconv_brute(x, y))


@pytest.mark.slow
@pytest.mark.parametrize("D,vmax,e", [(17, 2, 3), (20, 1, 0)])
def test_maxconv_largest_embeddings(hc, D, vmax, e):
    """The largest convolutions the limb embedding reaches at these bounds:
    D + e = 20 axes (a 28 GB int64 convolution in the workspace), sampled
    outputs against the oracle's definition one output at a time, plus the
    outputs with every digit equal."""
    x, y = inputs.uniform_int_pair(D, 0, vmax, seed=500 + D)
    assert hc.maxconv_plan(D, vmax)["e"] == e
    z = hc.maxconv(T(x), T(y), vmax)
    torch.cuda.synchronize()
    n3 = 3 ** D
    ks = np.unique(np.concatenate([
        np.random.default_rng(D).integers(0, n3, size=20000),
        [0, (n3 - 1) // 2, n3 - 1]]))
    got = z[torch.from_numpy(ks.astype(np.int64)).to(DEV)].cpu().numpy()
    assert_equal(got, oracle.maxconv_points(x, y, ks))
    del z
    torch.cuda.empty_cache()
