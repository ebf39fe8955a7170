"""GPU parity of the adjoint (hc_convolve_backward through the C ABI) and the
autograd Function, against the oracle's transposed recurrence (bitwise, same
per-element order), brute force, the adjoint identity and finite
differences."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1608_00206_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def hc():
    from paper_1608_00206_gb300.build import build
    build()
    import paper_1608_00206_gb300 as hc
    return hc


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def bits(a):
    return a.view(np.uint64) if a.dtype.itemsize == 8 else a.view(np.uint32)


def gpu_adj(hc, dz, x, y, **kw):
    dx, dy = hc.convolve_backward(T(dz), T(x), T(y), **kw)
    torch.cuda.synchronize()
    return (None if dx is None else dx.cpu().numpy()), (None if dy is None else dy.cpu().numpy())


@pytest.mark.parametrize("D", list(range(0, 13)))
def test_int64_adjoint_bit_exact(hc, D):
    x, y = inputs.uniform_int_pair(D, -100, 100, seed=D)
    dz = np.random.default_rng(D).integers(-100, 101, size=3 ** D, dtype=np.int64)
    dx, dy = gpu_adj(hc, dz, x, y)
    wx, wy = oracle.adjoint_brute(dz, x, y) if D <= 9 else oracle.adjoint(dz, x, y)
    assert np.array_equal(dx, wx) and np.array_equal(dy, wy)


@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("D", [0, 1, 2, 3, 5, 8, 9, 11, 13])
def test_fp_adjoint_bit_exact(hc, dt, D):
    x, y = inputs.normal_pair(D, seed=D, dtype=dt)
    dz = inputs.normal(3 ** D, seed=100 + D, dtype=dt)
    dx, dy = gpu_adj(hc, dz, x, y)
    wx, wy = oracle.adjoint(dz, x, y)
    assert np.array_equal(bits(dx), bits(wx)) and np.array_equal(bits(dy), bits(wy))


@pytest.mark.parametrize("cols", [8, 16, 32, -16, -32])
@pytest.mark.parametrize("dt", [np.int64, np.float64, np.float32])
def test_adjoint_every_tile_width(hc, dt, cols):
    """The adjoint's I^T passes take the tile width of the forward default
    schedule for (D, dtype): installed here through the library's default
    table, every width (per-element and 16-byte row copies) gives the
    oracle's bits.  D = 14: six outer axes in one transposed pass, ragged
    column tiles, rows at every 16-byte offset."""
    import ctypes

    from paper_1608_00206_gb300 import _lib
    D = 14
    code = {np.int64: _lib.HC_INT64, np.float64: _lib.HC_FP64, np.float32: _lib.HC_FP32}[dt]
    if dt == np.int64:
        x, y = inputs.uniform_int_pair(D, -100, 100, seed=7)
        dz = np.random.default_rng(7).integers(-100, 101, size=3 ** D, dtype=np.int64)
    else:
        x, y = inputs.normal_pair(D, seed=7, dtype=dt)
        dz = inputs.normal(3 ** D, seed=8, dtype=dt)
    hc.convolve(T(x), T(y))  # installs the shipped table, as any first call does
    lib = _lib.lib()
    saved = _lib.hc_schedule()
    assert lib.hc_get_default_schedule(D, code, ctypes.byref(saved)) == 0
    s = _lib.hc_schedule(_lib.HC_SCHED_PASSES, 8, 6, cols, -cols if cols in (16, 32) else 0)
    assert lib.hc_set_default_schedule(D, code, ctypes.byref(s)) == 0
    try:
        dx, dy = gpu_adj(hc, dz, x, y)
    finally:
        assert lib.hc_set_default_schedule(D, code, ctypes.byref(saved)) == 0
    wx, wy = oracle.adjoint(dz, x, y)
    assert np.array_equal(bits(dx), bits(wx)) and np.array_equal(bits(dy), bits(wy))


@pytest.mark.parametrize("cols,cols_outer", [(16, -32), (32, 8)])
def test_adjoint_outermost_pass_width(hc, cols, cols_outer):
    """D = 16: eight outer axes, two transposed passes; the one over the
    outermost axes takes the default schedule's cols_outer."""
    import ctypes

    from paper_1608_00206_gb300 import _lib
    D = 16
    x, y = inputs.uniform_int_pair(D, -100, 100, seed=9)
    dz = np.random.default_rng(9).integers(-100, 101, size=3 ** D, dtype=np.int64)
    hc.convolve(T(x), T(y))
    lib = _lib.lib()
    saved = _lib.hc_schedule()
    assert lib.hc_get_default_schedule(D, _lib.HC_INT64, ctypes.byref(saved)) == 0
    s = _lib.hc_schedule(_lib.HC_SCHED_PASSES, 8, 4, cols, cols_outer)
    assert lib.hc_set_default_schedule(D, _lib.HC_INT64, ctypes.byref(s)) == 0
    try:
        dx, dy = gpu_adj(hc, dz, x, y)
    finally:
        assert lib.hc_set_default_schedule(D, _lib.HC_INT64, ctypes.byref(saved)) == 0
    wx, wy = oracle.adjoint(dz, x, y)
    assert np.array_equal(dx, wx) and np.array_equal(dy, wy)


def test_one_sided(hc):
    D = 11
    x, y = inputs.normal_pair(D, seed=1, dtype=np.float64)
    dz = inputs.normal(3 ** D, seed=2, dtype=np.float64)
    wx, wy = oracle.adjoint(dz, x, y)
    dx, dy = gpu_adj(hc, dz, x, y, need_dy=False)
    assert dy is None and np.array_equal(dx, wx)
    dx, dy = gpu_adj(hc, dz, x, y, need_dx=False)
    assert dx is None and np.array_equal(dy, wy)


def test_adjoint_identity_int64(hc):
    """<dz, x*y> = <dx, x> = <dy, y>, exact in Z/2^64 (D = 14)."""
    D = 14
    x, y = inputs.uniform_int_pair(D, -100, 100, seed=3)
    dz = np.random.default_rng(4).integers(-100, 101, size=3 ** D, dtype=np.int64)
    z = hc.convolve(T(x), T(y)).cpu().numpy()
    dx, dy = gpu_adj(hc, dz, x, y)
    with np.errstate(over="ignore"):
        lhs = int((dz * z).sum())
        assert lhs == int((dx * x).sum()) == int((dy * y).sum())


def test_autograd_matches_adjoint_and_gradcheck(hc):
    """loss = sum(w * (x*y)) through torch.autograd; gradcheck (finite
    differences, float64, D = 8) on the scalar loss."""
    D = 8
    x = T(inputs.normal(1 << D, seed=1, dtype=np.float64)).requires_grad_()
    y = T(inputs.normal(1 << D, seed=2, dtype=np.float64)).requires_grad_()
    w = T(inputs.normal(3 ** D, seed=3, dtype=np.float64))
    loss = (w * hc.hypercube_conv(x, y)).sum()
    loss.backward()
    wx, wy = oracle.adjoint(w.cpu().numpy(), x.detach().cpu().numpy(), y.detach().cpu().numpy())
    assert np.array_equal(x.grad.cpu().numpy(), wx) and np.array_equal(y.grad.cpu().numpy(), wy)
    f = lambda a, b: (w * hc.hypercube_conv(a, b)).sum()  # noqa: E731
    assert torch.autograd.gradcheck(f, (x.detach().requires_grad_(), y.detach().requires_grad_()),
                                    eps=1e-6, atol=1e-7, rtol=1e-6)


def test_d18_fp32_fwd_bwd_full_size(hc):
    """The differentiation workload: D = 18 float32, x, y, w iid N(0,1),
    loss = sum(w * z).  Gradients bitwise equal to the oracle's adjoint."""
    D = 18
    x = inputs.normal(1 << D, seed=18, dtype=np.float32)
    y = inputs.normal(1 << D, seed=19, dtype=np.float32)
    w = inputs.normal(3 ** D, seed=20, dtype=np.float32)
    xt, yt = T(x).requires_grad_(), T(y).requires_grad_()
    loss = (T(w) * hc.hypercube_conv(xt, yt)).sum()
    loss.backward()
    wx, wy = oracle.adjoint(w, x, y)
    assert np.array_equal(bits(xt.grad.cpu().numpy()), bits(wx))
    assert np.array_equal(bits(yt.grad.cpu().numpy()), bits(wy))
