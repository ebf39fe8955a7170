"""GPU parity of the forward convolution (hc_convolve through the C ABI)
against the CPU oracle.  Floating-point results must be bitwise identical to
the oracle's recurrence in the same precision (same per-element operation
order, no FMA); int64 results bitwise identical to Algorithm 1."""
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


def gpu_conv(hc, x, y, **kw):
    xt = torch.from_numpy(np.ascontiguousarray(x)).to(DEV)
    yt = torch.from_numpy(np.ascontiguousarray(y)).to(DEV)
    z = hc.convolve(xt, yt, **kw)
    torch.cuda.synchronize()
    return z.cpu().numpy().reshape(-1)


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def bits(a):
    return a.view(np.uint64) if a.dtype.itemsize == 8 else a.view(np.uint32)


def assert_bit_equal(got, want):
    assert got.shape == want.shape and got.dtype == want.dtype
    bad = np.flatnonzero(bits(got) != bits(want))
    assert bad.size == 0, f"{bad.size} mismatches, first at {bad[:5]}: {got[bad[:5]]} vs {want[bad[:5]]}"


# ----------------------------------------------------------------- int64


@pytest.mark.parametrize("D", list(range(0, 13)))
def test_int64_bit_exact(hc, D):
    x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=100 + D)
    want = oracle.brute_force(x, y) if D <= 10 else oracle.convolve(x, y, threads=8)
    assert_bit_equal(gpu_conv(hc, x, y), want)


@pytest.mark.parametrize("D", [13, 14, 15, 16])
def test_int64_sweep_sizes_bit_exact(hc, D):
    """The benchmark sweep's smaller points with their tuned schedules (the
    hybrid direct form on two top axes at D = 13, 15 and 16, whole-array
    passes at 14; values in [-1000, 1000] as the D = 20 workload): every
    output bitwise the oracle's recurrence."""
    x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=4000 + D)
    assert_bit_equal(gpu_conv(hc, x, y), oracle.convolve(x, y, threads=16))


@pytest.mark.parametrize("c", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("kmax", [1, 3, 4, 6])
def test_int64_every_schedule(hc, c, kmax):
    """Every (tile axes, axes per pass) schedule gives the same bits: D = 11
    spans several tiles, K1/K3 passes of every width and ragged column tiles."""
    D = 11
    x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=c * 10 + kmax)
    assert_bit_equal(gpu_conv(hc, x, y, c=c, kmax=kmax), oracle.convolve(x, y))


def test_int64_wraps(hc):
    g = np.random.default_rng(3)
    x = g.integers(-(1 << 62), 1 << 62, size=1 << 12, dtype=np.int64)
    y = g.integers(-(1 << 62), 1 << 62, size=1 << 12, dtype=np.int64)
    with np.errstate(over="ignore"):
        assert_bit_equal(gpu_conv(hc, x, y), oracle.convolve(x, y))


# --------------------------------------------------------- floating point


@pytest.mark.parametrize("D", list(range(0, 14)))
def test_fp64_bit_exact(hc, D):
    x, y = inputs.prob_exponential_pair(D, seed=200 + D)
    assert_bit_equal(gpu_conv(hc, x, y), oracle.convolve(x, y, threads=8))


@pytest.mark.parametrize("D", list(range(0, 14)))
def test_fp32_bit_exact(hc, D):
    x, y = inputs.normal_pair(D, seed=300 + D)
    assert_bit_equal(gpu_conv(hc, x, y), oracle.convolve(x, y, threads=8))


@pytest.mark.parametrize("D", list(range(0, 14)))
def test_mixed_bit_exact(hc, D):
    x, y = inputs.uniform01_pair(D, seed=400 + D)
    assert_bit_equal(gpu_conv(hc, x, y, mixed=True), oracle.convolve_mixed(x, y))


@pytest.mark.slow
@pytest.mark.parametrize("mixed", [True, "ff"])
def test_float_float_forms_full_size(hc, mixed):
    """The benchmark's D = 16 precision forms (float32 probability
    hypercubes; binary32 evaluation and products with float-float
    interpolation, and every value in float-float) with their tuned
    schedules: every output bitwise the oracle's recurrence in the same
    arithmetic."""
    D = 16
    x, y = inputs.prob_exponential_pair(D, seed=1000)
    x, y = x.astype(np.float32), y.astype(np.float32)
    want = oracle.convolve_mixed(x, y) if mixed is True else oracle.convolve_ff(x, y)
    assert_bit_equal(gpu_conv(hc, x, y, mixed=mixed), want)


@pytest.mark.parametrize("D", list(range(0, 14)))
def test_ff_bit_exact(hc, D):
    """Every value in float-float (HC_FP32_FF): bitwise the oracle's
    float-float recurrence (same two-sum, FMA two-product and quick-two-sum
    steps in the same order)."""
    x, y = inputs.uniform01_pair(D, seed=500 + D)
    assert_bit_equal(gpu_conv(hc, x, y, mixed="ff"), oracle.convolve_ff(x, y))


@pytest.mark.parametrize("sched", [dict(c=3, kmax=2), dict(c=8, kmax=6), dict(c=7, kmax=4, cols=-32),
                                   dict(c=8, m=3), dict(c=5, m=6), dict(c=8, m=6, bulk=True),
                                   dict(c=7, m=4, bulk=True)])
def test_ff_every_schedule(hc, sched):
    """The float-float form through whole-array passes, the chunked engine and
    the slab kernel (D = 15: outer passes after the chunks)."""
    D = 15
    x, y = inputs.normal_pair(D, seed=600 + int(sched["c"]), dtype=np.float32)
    assert_bit_equal(gpu_conv(hc, x, y, mixed="ff", **sched), oracle.convolve_ff(x, y))


def test_ff_final_stores_into_host_memory(hc):
    """hc_convolve_out with the float-float dtype: the intermediate stays in
    the workspace (w must be NULL) and the last pass rounds straight into a
    page-locked host z; bitwise the oracle."""
    import ctypes

    from paper_1608_00206_gb300 import _lib as L
    D = 14
    x, y = inputs.uniform01_pair(D, seed=1414)
    lib = L.lib()
    nb = int(lib.hc_workspace_size(D, L.HC_FP32_FF))
    ws = torch.empty(nb, dtype=torch.uint8, device=DEV)
    zh = torch.empty(3 ** D, dtype=torch.float32, pin_memory=True)
    xd, yd = T(x), T(y)
    st = torch.cuda.current_stream().cuda_stream
    assert lib.hc_convolve_out(xd.data_ptr(), yd.data_ptr(), xd.data_ptr(), zh.data_ptr(), D,
                               L.HC_FP32_FF, ws.data_ptr(), nb, st) == L.HC_ERR_ARG
    assert lib.hc_convolve_out(xd.data_ptr(), yd.data_ptr(), None, zh.data_ptr(), D,
                               L.HC_FP32_FF, ws.data_ptr(), nb, st) == L.HC_OK
    torch.cuda.synchronize()
    assert_bit_equal(zh.numpy(), oracle.convolve_ff(x, y))


def test_ff_integer_inputs_rounded_exact(hc):
    """Integer inputs (values in [-2000, 2000], D = 12): the float-float form
    returns the exact result rounded once to binary32 at every output."""
    xi, yi = inputs.uniform_int_pair(12, -2000, 2000, seed=12)
    got = gpu_conv(hc, xi.astype(np.float32), yi.astype(np.float32), mixed="ff")
    assert_bit_equal(got, oracle.convolve(xi, yi).astype(np.float32))


@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("c,kmax", [(1, 1), (4, 2), (7, 5), (8, 6), (9, 6)])
def test_fp_every_schedule(hc, dt, c, kmax):
    if c == 9 and dt != np.float32:
        pytest.skip("9-axis tiles are float32 only")
    D = 12
    x, y = inputs.normal_pair(D, seed=c + kmax, dtype=dt)
    assert_bit_equal(gpu_conv(hc, x, y, c=c, kmax=kmax), oracle.convolve(x, y, threads=8))


@pytest.mark.parametrize("c", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("m", [1, 3, 4, 6])
def test_int64_chunked_every_schedule(hc, c, m):
    """Chunked schedule: chunks of c + m axes in one persistent launch, the
    D - c - m outer axes by whole-array passes (D = 13 gives up to 9 outer
    axes: two evaluation and two interpolation passes)."""
    D = 13
    x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=100 * c + m)
    assert_bit_equal(gpu_conv(hc, x, y, c=c, m=m), oracle.convolve(x, y))


@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("c,m", [(2, 1), (4, 5), (8, 6), (9, 6), (9, 2)])
def test_fp_chunked_schedules(hc, dt, c, m):
    if c == 9 and dt != np.float32:
        pytest.skip("9-axis tiles are float32 only")
    D = 14
    x, y = inputs.normal_pair(D, seed=c + 10 * m, dtype=dt)
    assert_bit_equal(gpu_conv(hc, x, y, c=c, m=m), oracle.convolve(x, y, threads=8))


@pytest.mark.parametrize("c,m", [(3, 2), (8, 4), (8, 6)])
def test_mixed_chunked_schedules(hc, c, m):
    D = 13
    x, y = inputs.uniform01_pair(D, seed=c + m)
    assert_bit_equal(gpu_conv(hc, x, y, mixed=True, c=c, m=m), oracle.convolve_mixed(x, y))


@pytest.mark.parametrize("c", [7, 8, 5])
@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6])
def test_int64_chunked_bulk_every_middle_depth(hc, c, m):
    """Chunked-bulk schedule (every middle axis evaluated by the passes; the
    slab kernel for c = 7, 8, the generic engine on the same plan for c = 5):
    D = 15 gives 3^(15-c-m) units of 3^m tiles, up to 3 outer passes, ragged
    column tickets (3^c columns in tickets of cpt * 8)."""
    D = 15
    x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=300 + 10 * c + m)
    assert_bit_equal(gpu_conv(hc, x, y, c=c, m=m, bulk=True), oracle.convolve(x, y, threads=16))


@pytest.mark.parametrize("kind,c,m", [("float64", 8, 6), ("float64", 7, 3), ("float32", 9, 6),
                                      ("float32", 8, 4), ("float32", 9, 1), ("mixed", 8, 6),
                                      ("mixed", 7, 5), ("mixed", 8, 2)])
def test_fp_chunked_bulk_schedules(hc, kind, c, m):
    """The slab kernel in every floating-point mode: same per-element order
    as the recurrence, so bitwise the oracle (mixed: float-float
    intermediates in the workspace, the columns or the last pass round)."""
    D = 15
    if kind == "mixed":
        x, y = inputs.uniform01_pair(D, seed=c + 10 * m)
        want = oracle.convolve_mixed(x, y)
    else:
        x, y = inputs.normal_pair(D, seed=c + 10 * m,
                                  dtype=np.float64 if kind == "float64" else np.float32)
        want = oracle.convolve(x, y, threads=16)
    assert_bit_equal(gpu_conv(hc, x, y, mixed=(kind == "mixed"), c=c, m=m, bulk=True), want)


@pytest.mark.parametrize("D,m", [(14, 6), (12, 4), (9, 1)])
def test_chunked_bulk_single_unit(hc, D, m):
    """D = c + m: one unit, the columns write the final result (no outer
    pass); int64 and float32."""
    x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=D)
    assert_bit_equal(gpu_conv(hc, x, y, c=D - m, m=m, bulk=True), oracle.convolve(x, y, threads=8))
    xf, yf = inputs.normal_pair(D, seed=D, dtype=np.float32)
    assert_bit_equal(gpu_conv(hc, xf, yf, c=D - m, m=m, bulk=True),
                     oracle.convolve(xf, yf, threads=8))


def test_chunked_bulk_managed_output_falls_back(hc):
    """A managed output takes the generic engine on the chunked-bulk plan
    (no bulk copies into managed memory): same bits."""
    import ctypes

    from paper_1608_00206_gb300 import _lib
    rt = _cudart()
    D = 14
    x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=77)
    lib = _lib.lib()
    s = _lib.hc_schedule(_lib.HC_SCHED_CHUNKED_BULK, 8, 4, 0, 0)
    nb = int(lib.hc_workspace_size_schedule(D, _lib.HC_INT64, ctypes.byref(s)))
    ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=DEV)
    xd, yd = T(x), T(y)
    ptr = ctypes.c_void_p()
    assert rt.cudaMallocManaged(ctypes.byref(ptr), ctypes.c_size_t(8 * 3 ** D), 1) == 0
    try:
        st = torch.cuda.current_stream().cuda_stream
        assert lib.hc_convolve_schedule(xd.data_ptr(), yd.data_ptr(), ptr.value, D, _lib.HC_INT64,
                                        ctypes.byref(s), ws.data_ptr(), nb, st) == 0
        torch.cuda.synchronize()
        got = np.ctypeslib.as_array((ctypes.c_byte * (8 * 3 ** D)).from_address(ptr.value))
        assert_bit_equal(got.view(np.int64).copy(), oracle.convolve(x, y, threads=8))
    finally:
        torch.cuda.synchronize()
        rt.cudaFree(ptr)


@pytest.mark.parametrize("dt", [np.int64, np.float64, np.float32])
@pytest.mark.parametrize("D,top,c,kmax", [(9, 1, 8, 6), (10, 2, 8, 6), (12, 3, 5, 4),
                                          (13, 4, 8, 2), (14, 6, 4, 3), (15, 3, 8, 6),
                                          (16, 2, 7, 5)])
def test_hybrid_bit_exact(hc, dt, D, top, c, kmax):
    """Hybrid schedule (direct form on the top axes): bitwise the oracle's
    hybrid form in every dtype, and Algorithm 1 in int64.  Covers a final
    tile with no middle axes (D = top + c), ragged pairs (up to 2^6 per
    tile) and one to three middle passes."""
    if dt is np.int64:
        x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=700 + D + top)
    else:
        x, y = inputs.normal_pair(D, seed=700 + D + top, dtype=dt)
    want = oracle.convolve_direct_top(x, y, top)
    got = gpu_conv(hc, x, y, top=top, c=c, kmax=kmax, cols=-32 if D % 2 else 32)
    assert_bit_equal(got, want)
    if dt is np.int64:
        assert_bit_equal(got, oracle.convolve(x, y, threads=8))


@pytest.mark.parametrize("kind", ["int64", "float64", "float32", "mixed", "ff"])
@pytest.mark.parametrize("D,c,kmax,cols,cols_outer", [(9, 8, 6, 16, 0), (11, 8, 3, 32, 0),
                                                      (14, 8, 6, 16, 32), (15, 7, 4, -16, 16),
                                                      (16, 5, 6, -32, 32), (13, 4, 5, 8, -16),
                                                      (12, 6, 2, 32, 0)])
def test_padded_every_dtype(hc, kind, D, c, kmax, cols, cols_outer):
    """Padded schedule (the intermediate with 128-byte-aligned tile pitch in
    the workspace, the last pass writing z's layout): the recurrence's bits in
    every dtype -- last passes of 1 to 6 axes (register-only and shared-memory
    forms, 16 and 32 columns), inner passes with every tile width, tiles
    whose 3^c outputs are padded by 1 to 31 elements."""
    if kind == "int64":
        x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=900 + D + c)
        want = oracle.convolve(x, y, threads=8)
    elif kind in ("mixed", "ff"):
        x, y = inputs.uniform01_pair(D, seed=900 + D + c)
        want = oracle.convolve_mixed(x, y) if kind == "mixed" else oracle.convolve_ff(x, y)
    else:
        x, y = inputs.normal_pair(D, seed=900 + D + c,
                                  dtype=np.float64 if kind == "float64" else np.float32)
        want = oracle.convolve(x, y, threads=8)
    mixed = {"mixed": True, "ff": "ff"}.get(kind, False)
    got = gpu_conv(hc, x, y, mixed=mixed, padded=True, c=c, kmax=kmax, cols=cols,
                   cols_outer=cols_outer)
    assert_bit_equal(got, want)


@pytest.mark.parametrize("dt", [np.int64, np.float64, np.float32])
@pytest.mark.parametrize("D,top,c,kmax,cols", [(7, 1, 8, 6, 32), (10, 3, 5, 2, 16),
                                               (13, 6, 4, 3, -32), (15, 2, 8, 6, 8),
                                               (14, 6, 8, 6, 32), (12, 6, 6, 0, 0)])
def test_lowmem_bit_exact(hc, dt, D, top, c, kmax, cols):
    """Low-workspace schedule (the top axes split leaf by leaf): the same bits
    as the recurrence in every dtype -- leaves of one tile (D - top <= c),
    of several passes, up to 2^6 sub-cubes summed per leaf element, and a
    16-byte row-copy width, which the leaves' unaligned slices replace by
    per-element copies."""
    if dt is np.int64:
        x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=800 + D + top)
    else:
        x, y = inputs.normal_pair(D, seed=800 + D + top, dtype=dt)
    got = gpu_conv(hc, x, y, top=top, lowmem=True, c=c, kmax=kmax, cols=cols)
    assert_bit_equal(got, oracle.convolve(x, y, threads=8))


def test_hybrid_d18_float32_workload(hc):
    """The D = 18 float32 workload with 3 direct axes (one 6-axis middle
    pass).  A slice whose top digits hold no 1 has a single sub-cube pair, so
    it is the plain recurrence on that pair: bitwise the oracle's.  Slices
    with digit-1 axes sum 2, 4 or 8 pairs' products: within the float32
    forward bound of the exact slice (the pairs' float64 recurrences)."""
    D, top = 18, 3
    x, y = inputs.uniform01_pair(D, seed=1818)
    z = hc.convolve(T(x), T(y), top=top, c=8, kmax=6, cols=32).cpu().numpy()
    n, h = 3 ** (D - top), 1 << (D - top)
    for a in (0, 26, 8, 18, 13, 5):
        digits = [a // 9 % 3, a // 3 % 3, a % 3]
        ones = [i for i, d in enumerate(digits) if d == 1]
        parts, pairs = [], []
        for sidx in range(1 << len(ones)):
            bx = [d // 2 for d in digits]
            by = [d // 2 for d in digits]
            for q, i in enumerate(ones):
                if (sidx >> (len(ones) - 1 - q)) & 1:
                    bx[i] = 1
                else:
                    by[i] = 1
            ox = sum(b << (top - 1 - i) for i, b in enumerate(bx)) * h
            oy = sum(b << (top - 1 - i) for i, b in enumerate(by)) * h
            parts.append(oracle.convolve(x[ox:ox + h], y[oy:oy + h], threads=16) if not ones
                         else None)
            pairs.append((ox, oy))
        got = z[a * n:(a + 1) * n]
        if not ones:
            assert_bit_equal(got, parts[0])
        else:
            # float64 pair recurrences summed (error far below float32's);
            # the bound: gamma_{3D+1}(2^-24) times the pairs' magnitudes
            want = np.zeros(n)
            za = np.zeros(n)
            for (ox, oy) in pairs:
                xs, ys = x[ox:ox + h].astype(np.float64), y[oy:oy + h].astype(np.float64)
                want += oracle.convolve(xs, ys, threads=16)
                za += oracle.zabs(xs, ys)
            err = np.abs(got.astype(np.float64) - want)
            assert np.all(err <= oracle.gamma(3 * D + 1, 2.0 ** -24) * za), a


@pytest.mark.parametrize("cols", [8, 16, 32, -16, -32])
@pytest.mark.parametrize("kind", ["int64", "float64", "float32", "mixed"])
def test_every_interpolation_tile_width(hc, kind, cols):
    """Whole-array interpolation passes of 4, 5 and 6 axes at every tile
    width, with per-element copies (cols > 0) and with 16-byte row copies of
    widened rows (cols < 0); lo = 3^c gives ragged column tiles and rows at
    every 16-byte offset."""
    D = 12
    if kind == "int64":
        x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=abs(cols))
        want = oracle.convolve(x, y)
    elif kind == "mixed":
        x, y = inputs.uniform01_pair(D, seed=abs(cols))
        want = oracle.convolve_mixed(x, y)
    else:
        x, y = inputs.normal_pair(D, seed=abs(cols), dtype=np.float64 if kind == "float64" else np.float32)
        want = oracle.convolve(x, y, threads=8)
    for c, kmax in [(6, 6), (7, 5), (8, 4)]:
        assert_bit_equal(gpu_conv(hc, x, y, mixed=(kind == "mixed"), c=c, kmax=kmax, cols=cols), want)


@pytest.mark.parametrize("cols,cols_outer", [(16, 32), (32, 16), (16, -32), (-32, 8), (8, -16)])
@pytest.mark.parametrize("kind", ["int64", "float32", "mixed"])
def test_outermost_pass_width(hc, kind, cols, cols_outer):
    """A separate width for the pass over the outermost axes: D = 14, c = 6
    leaves 8 outer axes, two passes of 4; the second one takes cols_outer."""
    D = 14
    if kind == "int64":
        x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=cols + 100)
        want = oracle.convolve(x, y, threads=8)
    elif kind == "mixed":
        x, y = inputs.uniform01_pair(D, seed=cols + 100)
        want = oracle.convolve_mixed(x, y)
    else:
        x, y = inputs.normal_pair(D, seed=cols + 100, dtype=np.float32)
        want = oracle.convolve(x, y, threads=8)
    got = gpu_conv(hc, x, y, mixed=(kind == "mixed"), c=6, kmax=4, cols=cols, cols_outer=cols_outer)
    assert_bit_equal(got, want)


@pytest.mark.parametrize("cols", [-16, -32, 8])
def test_chunked_outer_passes_tile_width(hc, cols):
    """The chunked schedule's whole-array passes (7 outer axes: 4 + 3) at a
    forced tile width."""
    D = 15
    x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=15)
    assert_bit_equal(gpu_conv(hc, x, y, c=4, m=4, cols=cols), oracle.convolve(x, y, threads=16))


def test_mixed_every_schedule(hc):
    D = 12
    x, y = inputs.uniform01_pair(D, seed=5)
    want = oracle.convolve_mixed(x, y)
    for c, kmax in [(2, 1), (5, 4), (8, 6)]:
        assert_bit_equal(gpu_conv(hc, x, y, mixed=True, c=c, kmax=kmax), want)


def test_paper_accuracy_workload(hc):
    """Table 1 input x = y = [1..2^D]: z[0...0] = 1 exactly, z[2...2] = 4^D."""
    for D in (11, 14, 16):
        x = inputs.paper_accuracy(D)
        z = gpu_conv(hc, x, x)
        assert z[0] == 1.0 and z[-1] == float(4 ** D)


# ------------------------------------------------------------ full sizes


def test_d16_fp64_probability_full(hc):
    """D = 16 float64 PMFs (Exponential(1) normalised): all 3^16 outputs bitwise
    equal to the oracle recurrence; the sum is 1."""
    x, y = inputs.prob_exponential_pair(16, seed=16)
    z = gpu_conv(hc, x, y)
    assert_bit_equal(z, oracle.convolve(x, y, threads=16))
    assert abs(z.sum() - 1.0) < 1e-12


def test_d16_fp64_separable_closed_form(hc):
    D = 16
    x, y, a, b = inputs.prob_separable_pair(D, seed=7)
    c = np.stack([a[:, 0] * b[:, 0], a[:, 0] * b[:, 1] + a[:, 1] * b[:, 0], a[:, 1] * b[:, 1]], 1)
    z_closed = inputs.outer_product_cube(c)
    z = gpu_conv(hc, x, y)
    za = oracle.zabs(x, y)
    u = 2.0 ** -53
    bound = oracle.gamma(3 * D + 1, u) * za + oracle.gamma(3 * D, u) * np.abs(z_closed)
    assert np.all(np.abs(z - z_closed) <= bound)


@pytest.mark.parametrize("D,sched", [(17, None), (18, None), (19, None), (20, None),
                                     (18, "bulk"), (20, "bulk"), (20, "lowmem"),
                                     (19, "padded"), (20, "padded")])
def test_int64_full_size(hc, D, sched):
    """D = 17..20 int64, values in [-1000, 1000] (the benchmark workload and
    its sweep, with the tuned schedule of each D, the launch configuration
    the benchmark times): 3^D outputs, 27.9 GB at D = 20.  Checked on whole
    slices (four prefix digits fixed, the oracle's (D-4)-D recurrence on the
    matching sub-cube pairs, summed over the pairs of the digit-1 axes), on
    random single outputs (the definition), and on the sum invariant over all
    outputs.  sched "bulk": the chunked-bulk schedule (8-axis tiles, 6 middle
    axes per L2-resident unit, one outer pass); "lowmem": the low-workspace
    schedule (6 top axes leaf by leaf, leaves of 14 axes); None: the tuned
    default."""
    x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=2000 + D)
    xt, yt = torch.from_numpy(x).to(DEV), torch.from_numpy(y).to(DEV)
    kw = {"bulk": dict(c=8, m=6, bulk=True, cols=32),
          "lowmem": dict(top=6, lowmem=True, c=8, kmax=6, cols=16, cols_outer=32),
          "padded": dict(padded=True, c=8, kmax=6, cols=16, cols_outer=16)}.get(sched, {})
    z = hc.convolve(xt, yt, **kw)
    torch.cuda.synchronize()
    # sum invariant (no overflow: |sum z| <= (2^20 * 1000)^2)
    assert int(z.sum().item()) == int(x.sum()) * int(y.sum())
    # slices with 4 leading digits fixed, by the direct form on those axes:
    # digit 0 -> sub-cube pair (0, 0), 2 -> (1, 1), 1 -> (0, 1) + (1, 0); the
    # slice is the sum over the pairs of the oracle's 16-D recurrence
    r = D - 4  # axes of each slice
    n16 = 3 ** r
    for digits in [(0, 0, 0, 0), (2, 2, 2, 2), (0, 2, 2, 0), (1, 0, 2, 1)]:
        off_z = sum(d * 3 ** (3 - i) for i, d in enumerate(digits)) * n16
        want = np.zeros(n16, np.int64)
        ones = [i for i, d in enumerate(digits) if d == 1]
        for choice in range(1 << len(ones)):
            bx = [d // 2 for d in digits]
            for q, i in enumerate(ones):
                bx[i] = (choice >> q) & 1
            by = [d - b for d, b in zip(digits, bx)]
            sx = sum(b << (3 - i) for i, b in enumerate(bx)) << r
            sy = sum(b << (3 - i) for i, b in enumerate(by)) << r
            with np.errstate(over="ignore"):
                want += oracle.convolve(x[sx:sx + (1 << r)], y[sy:sy + (1 << r)], threads=16)
        got = z[off_z:off_z + n16].cpu().numpy()
        assert np.array_equal(got, want), digits
    g = np.random.default_rng(0)
    ks = np.sort(g.integers(0, 3 ** D, size=20000, dtype=np.int64))
    got = z[torch.from_numpy(ks).to(DEV)].cpu().numpy()
    assert np.array_equal(got, oracle.points(x, y, ks))
    del z


@pytest.mark.slow
@pytest.mark.parametrize("kind,D,dist", [("float32", 18, "u01"), ("float32", 18, "normal"),
                                         ("float32", 19, "u01"), ("float32", 20, "u01"),
                                         ("float64", 18, "u01")])
def test_float_full_size_sampled(hc, kind, D, dist):
    """Floating-point convolutions at full size with the tuned default
    schedules (the benchmark's D = 18 float32 form and the forward of the
    D = 18 differentiation form, the D = 19 and 20 float32 plans, D = 18
    float64): 20 000 sampled outputs and the all-0 and all-2 outputs (and,
    up to D = 18, the all-1 output, which takes the oracle 3^D products)
    against the recurrence evaluated at those outputs (oracle.points_rec),
    bit for bit."""
    dt = np.float32 if kind == "float32" else np.float64
    if dist == "u01":
        x, y = inputs.uniform01_pair(D, seed=3000 + D, dtype=dt)
    else:
        x = inputs.normal(1 << D, 3100 + D, dt)
        y = inputs.normal(1 << D, 3200 + D, dt)
    z = hc.convolve(torch.from_numpy(x).to(DEV), torch.from_numpy(y).to(DEV))
    torch.cuda.synchronize()
    n3 = 3 ** D
    special = [0, n3 - 1] + ([(n3 - 1) // 2] if D <= 18 else [])  # all-1: 3^D oracle products
    ks = np.unique(np.concatenate([np.random.default_rng(D).integers(0, n3, size=20000),
                                   special]))
    got = z[torch.from_numpy(ks.astype(np.int64)).to(DEV)].cpu().numpy()
    assert_bit_equal(got, oracle.points_rec(x, y, ks))
    del z
    torch.cuda.empty_cache()


def test_d20_int64_separable_points(hc):
    D = 20
    a = inputs.separable_factors(D, 1, "int")
    b = inputs.separable_factors(D, 2, "int")
    x, y = inputs.outer_product_cube(a), inputs.outer_product_cube(b)
    z = hc.convolve(torch.from_numpy(x).to(DEV), torch.from_numpy(y).to(DEV))
    g = np.random.default_rng(1)
    ks = g.integers(0, 3 ** D, size=5000, dtype=np.int64)
    got = z[torch.from_numpy(ks).to(DEV)].cpu().numpy()
    c = np.stack([a[:, 0] * b[:, 0], a[:, 0] * b[:, 1] + a[:, 1] * b[:, 0], a[:, 1] * b[:, 1]], 1)
    want = np.ones(ks.size, np.int64)
    kk = ks.copy()
    with np.errstate(over="ignore"):
        for d in range(D - 1, -1, -1):
            want = want * c[d][kk % 3]
            kk //= 3
    assert np.array_equal(got, want)
    del z


# ------------------------------------------------------------ host buffers


def test_host_buffers_end_to_end(hc):
    D = 13
    x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=13)
    xt = torch.from_numpy(x).pin_memory()
    yt = torch.from_numpy(y).pin_memory()
    z = hc.convolve(xt, yt)
    assert not z.is_cuda and z.is_pinned()
    assert np.array_equal(z.numpy(), oracle.convolve(x, y))


@pytest.mark.parametrize("kind,D,sched", [
    ("int64", 13, None), ("int64", 14, (2, 8, 6, 0)), ("int64", 15, (2, 4, 4, -32)),
    ("int64", 14, (1, 7, 6, 16)), ("float64", 12, None), ("float32", 16, None),
    ("float32", 13, (2, 8, 3, 0)), ("mixed", 12, None), ("mixed", 13, (2, 8, 5, 0))])
def test_final_stores_into_pinned_host_memory(hc, kind, D, sched):
    """hc_convolve_out: the intermediate in a device array, the final stores
    (last whole-array pass, or the chunk's column tickets when no outer pass
    follows, or the tile when there is neither) straight into page-locked
    host memory; bitwise the oracle's result, for the default and for forced
    schedules (installed as the default, since hc_convolve_out takes it)."""
    import ctypes

    from paper_1608_00206_gb300 import _lib
    if kind == "int64":
        x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=D)
        want = oracle.convolve(x, y, threads=8)
    elif kind == "mixed":
        x, y = inputs.uniform01_pair(D, seed=D)
        want = oracle.convolve_mixed(x, y)
    else:
        x, y = inputs.normal_pair(D, seed=D, dtype=np.float64 if kind == "float64" else np.float32)
        want = oracle.convolve(x, y, threads=8)
    code = {"int64": _lib.HC_INT64, "float64": _lib.HC_FP64, "float32": _lib.HC_FP32,
            "mixed": _lib.HC_FP32_MIXED}[kind]
    xt = torch.from_numpy(x).pin_memory()
    yt = torch.from_numpy(y).pin_memory()
    hc.convolve(xt.to(DEV), yt.to(DEV))  # installs the shipped table, as any first call does
    lib = _lib.lib()
    saved = _lib.hc_schedule()
    assert lib.hc_get_default_schedule(D, code, ctypes.byref(saved)) == 0
    if sched is not None:
        s = _lib.hc_schedule(*sched)
        assert lib.hc_set_default_schedule(D, code, ctypes.byref(s)) == 0
    from paper_1608_00206_gb300 import api
    threshold = api._DIRECT_HOST_BYTES
    api._DIRECT_HOST_BYTES = 0  # this size goes through the final-store path too
    try:
        z = hc.convolve(xt, yt, mixed=(kind == "mixed"))
    finally:
        api._DIRECT_HOST_BYTES = threshold
        assert lib.hc_set_default_schedule(D, code, ctypes.byref(saved)) == 0
    assert not z.is_cuda and z.is_pinned()
    assert_bit_equal(z.numpy().reshape(-1), want)


def test_convolve_out_device_arrays_and_argument_checks(hc):
    """hc_convolve_out with device z and w gives hc_convolve's bits; a null or
    misplaced intermediate, an output the device cannot store to (pageable
    host memory) and overlapping arrays are rejected on the host, before any
    launch."""
    from paper_1608_00206_gb300 import _lib
    lib = _lib.lib()
    D = 12
    x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=3)
    xd, yd = T(x), T(y)
    z = torch.empty(3 ** D, dtype=torch.int64, device=DEV)
    w = torch.empty(3 ** D, dtype=torch.int64, device=DEV)
    nb = int(lib.hc_workspace_size(D, _lib.HC_INT64))
    ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=DEV)
    st = torch.cuda.current_stream().cuda_stream
    args = (D, _lib.HC_INT64, ws.data_ptr(), nb, st)
    assert lib.hc_convolve_out(xd.data_ptr(), yd.data_ptr(), w.data_ptr(), z.data_ptr(), *args) == 0
    torch.cuda.synchronize()
    assert_bit_equal(z.cpu().numpy(), oracle.convolve(x, y))
    assert lib.hc_convolve_out(xd.data_ptr(), yd.data_ptr(), None, z.data_ptr(), *args) == \
        _lib.HC_ERR_ARG
    assert lib.hc_convolve_out(xd.data_ptr(), yd.data_ptr(), z.data_ptr(), z.data_ptr(), *args) == \
        _lib.HC_ERR_ALIAS
    pageable = np.empty(3 ** D, np.int64)  # not known to the CUDA runtime
    assert lib.hc_convolve_out(xd.data_ptr(), yd.data_ptr(), w.data_ptr(),
                               pageable.ctypes.data, *args) == _lib.HC_ERR_ARG
    pinned_w = torch.empty(3 ** D, dtype=torch.int64).pin_memory()  # w must be device memory
    assert lib.hc_convolve_out(xd.data_ptr(), yd.data_ptr(), pinned_w.data_ptr(), z.data_ptr(),
                               *args) == _lib.HC_ERR_ARG
    zf = torch.empty(3 ** D, dtype=torch.float32, device=DEV)
    xf, yf = T(x.astype(np.float32)), T(y.astype(np.float32))
    nbm = int(lib.hc_workspace_size(D, _lib.HC_FP32_MIXED))
    wsm = torch.empty(max(nbm, 256), dtype=torch.uint8, device=DEV)
    assert lib.hc_convolve_out(xf.data_ptr(), yf.data_ptr(), w.data_ptr(), zf.data_ptr(), D,
                               _lib.HC_FP32_MIXED, wsm.data_ptr(), nbm, st) == _lib.HC_ERR_ARG
    torch.cuda.synchronize()


@pytest.mark.parametrize("kind,top", [("hybrid", 3), ("lowmem", 4), ("bulk", 0), ("padded", 0)])
def test_convolve_out_with_each_int64_default(hc, kind, top):
    """hc_convolve_out runs the default schedule: with each of the hybrid,
    low-workspace and chunked-bulk schedules installed as the int64 default,
    the intermediate goes to w and only the final stores reach a page-locked
    host z; the oracle's bits, and the default is put back afterwards."""
    import ctypes

    from paper_1608_00206_gb300 import _lib
    lib = _lib.lib()
    D = 13
    x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=31 + top)
    hc.convolve(T(x[:2]), T(y[:2]))  # the tuned table is installed first
    saved = _lib.hc_schedule()
    assert lib.hc_get_default_schedule(D, _lib.HC_INT64, ctypes.byref(saved)) == 0
    s = {"hybrid": _lib.hc_schedule(_lib.HC_SCHED_HYBRID, 6, 6, 16, 0, top),
         "lowmem": _lib.hc_schedule(_lib.HC_SCHED_LOWMEM, 5, 2, 16, 32, top),
         "bulk": _lib.hc_schedule(_lib.HC_SCHED_CHUNKED_BULK, 7, 4, 16, 0, 0),
         "padded": _lib.hc_schedule(_lib.HC_SCHED_PADDED, 7, 3, 16, 32, 0)}[kind]
    assert lib.hc_set_default_schedule(D, _lib.HC_INT64, ctypes.byref(s)) == 0
    try:
        nb = int(lib.hc_workspace_size(D, _lib.HC_INT64))
        ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=DEV)
        w = torch.empty(3 ** D, dtype=torch.int64, device=DEV)
        zh = torch.empty(3 ** D, dtype=torch.int64, pin_memory=True)
        st = torch.cuda.current_stream().cuda_stream
        assert lib.hc_convolve_out(T(x).data_ptr(), T(y).data_ptr(), w.data_ptr(),
                                   zh.data_ptr(), D, _lib.HC_INT64, ws.data_ptr(), nb, st) == 0
        torch.cuda.synchronize()
        assert_bit_equal(zh.numpy(), oracle.convolve(x, y, threads=8))
    finally:
        assert lib.hc_set_default_schedule(D, _lib.HC_INT64, ctypes.byref(saved)) == 0


def _cudart():
    import ctypes
    import glob
    import os
    cands = [os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64", "libcudart.so")]
    cands += sorted(glob.glob("/usr/local/cuda*/lib64/libcudart.so*"))
    for c in cands:
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    pytest.skip("no shared CUDA runtime to allocate managed memory with")


@pytest.mark.parametrize("kind", ["int64", "float32"])
def test_managed_output_takes_per_thread_tile_stores(hc, kind):
    """Intermediate tiles go out with bulk (TMA engine) copies only into plain
    device allocations; a managed z takes the per-thread stores.  Both give
    the oracle's bits."""
    import ctypes

    from paper_1608_00206_gb300 import _lib
    rt = _cudart()
    D = 12
    if kind == "int64":
        x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=41)
        code, es, dt = _lib.HC_INT64, 8, np.int64
    else:
        x, y = inputs.normal_pair(D, seed=41, dtype=np.float32)
        code, es, dt = _lib.HC_FP32, 4, np.float32
    want = oracle.convolve(x, y)
    lib = _lib.lib()
    s = _lib.hc_schedule(1, 8, 4, 16, 0)
    nb = int(lib.hc_workspace_size_schedule(D, code, ctypes.byref(s)))
    ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=DEV)
    xd, yd = T(x), T(y)
    ptr = ctypes.c_void_p()
    assert rt.cudaMallocManaged(ctypes.byref(ptr), ctypes.c_size_t(es * 3 ** D), 1) == 0
    try:
        st = torch.cuda.current_stream().cuda_stream
        assert lib.hc_convolve_schedule(xd.data_ptr(), yd.data_ptr(), ptr.value, D, code,
                                        ctypes.byref(s), ws.data_ptr(), nb, st) == 0
        torch.cuda.synchronize()
        got = np.ctypeslib.as_array((ctypes.c_byte * (es * 3 ** D)).from_address(ptr.value))
        assert_bit_equal(got.view(dt).copy(), want)
        zd = torch.empty(3 ** D, dtype=torch.int64 if kind == "int64" else torch.float32,
                         device=DEV)
        assert lib.hc_convolve_schedule(xd.data_ptr(), yd.data_ptr(), zd.data_ptr(), D, code,
                                        ctypes.byref(s), ws.data_ptr(), nb, st) == 0
        torch.cuda.synchronize()
        assert_bit_equal(zd.cpu().numpy(), want)
    finally:
        torch.cuda.synchronize()
        rt.cudaFree(ptr)


def test_shaped_input_gives_shaped_output(hc):
    x = torch.arange(1, 9, dtype=torch.float64, device=DEV).reshape(2, 2, 2)
    z = hc.convolve(x, x)
    assert z.shape == (3, 3, 3)
    assert z[2, 1, 2].item() == float(oracle.convolve(x.cpu().numpy(), x.cpu().numpy())[23])


def test_stream_ordering(hc):
    """The call is asynchronous on the given stream."""
    D = 14
    x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=1)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        xt, yt = torch.from_numpy(x).to(DEV), torch.from_numpy(y).to(DEV)
        z = hc.convolve(xt, yt)
        zc = z.cpu()
    assert np.array_equal(zc.numpy(), oracle.convolve(x, y))


def test_carry_free_1d_convolution(hc, oracle):
    """Discussion section: carry-free 1D convolution through hc_carryfree;
    7 (+) 5 lands in (2,1,2) = 23, and random vectors of power-of-two and
    other lengths match the oracle's definition bit for bit."""
    x = torch.zeros(8, dtype=torch.int64, device=DEV)
    y = torch.zeros(8, dtype=torch.int64, device=DEV)
    x[7], y[5] = 3, 4
    z = hc.carry_free_convolve(x, y).cpu().numpy()
    assert z.size == 27 and z[23] == 12 and np.count_nonzero(z) == 1
    g = np.random.default_rng(5)
    for N in (1, 2, 7, 1 << 11, 1000, 1500, 3001):
        xs = g.integers(-9, 10, size=N, dtype=np.int64)
        ys = g.integers(-9, 10, size=N, dtype=np.int64)
        z = hc.carry_free_convolve(torch.from_numpy(xs).to(DEV), torch.from_numpy(ys).to(DEV))
        assert np.array_equal(z.cpu().numpy(), oracle.carry_free(xs, ys)), N


@pytest.mark.parametrize("code,dt", [(_lib.HC_INT64, np.int64), (_lib.HC_FP64, np.float64),
                                     (_lib.HC_FP32, np.float32),
                                     (_lib.HC_FP32_MIXED, np.float32)])
def test_carry_free_c_abi_every_dtype(oracle, code, dt):
    """hc_carryfree called through the C ABI on a length that is not a power
    of two (2^11 < N < 2^12, so the device pads to 2^12): bit for bit the
    oracle's carry-free definition (int64) or the oracle's recurrence on the
    zero-padded vectors in the same arithmetic (floats, whose rounding
    follows the recurrence)."""
    L = _lib.lib()
    N = 3001
    D = (N - 1).bit_length()
    g = np.random.default_rng(7)
    if dt is np.int64:
        x = g.integers(-1000, 1001, size=N, dtype=np.int64)
        y = g.integers(-1000, 1001, size=N, dtype=np.int64)
    else:
        x = g.random(N).astype(dt)
        y = g.random(N).astype(dt)
    xt, yt = torch.from_numpy(x).to(DEV), torch.from_numpy(y).to(DEV)
    z = torch.empty(3 ** D, dtype=xt.dtype, device=DEV)
    nb = int(L.hc_carryfree_workspace_size(N, code))
    assert nb >= 2 * x.itemsize << D
    ws = torch.empty(nb, dtype=torch.uint8, device=DEV)
    st = torch.cuda.current_stream().cuda_stream
    _lib.check(L.hc_carryfree(xt.data_ptr(), yt.data_ptr(), z.data_ptr(), N, code, ws.data_ptr(),
                              nb, st), "hc_carryfree")
    got = z.cpu().numpy()
    xp = np.zeros(1 << D, dt)
    yp = np.zeros(1 << D, dt)
    xp[:N], yp[:N] = x, y
    if dt is np.int64:
        want = oracle.carry_free(x, y)
    elif code == _lib.HC_FP32_MIXED:
        want = oracle.convolve_mixed(xp, yp)
    else:
        want = oracle.convolve(xp, yp)
    view = np.uint64 if got.itemsize == 8 else np.uint32
    assert np.array_equal(got.view(view), want.view(view))
