"""Pins for the CPU oracle: every function is checked against something other
than itself -- a library routine that reduces to the definition, the paper's
worked examples, closed forms, invariants, and exact results within the
floating-point error bound.  A set of deliberately broken recurrences
(planted mistakes) shows that the pins catch dropped terms, wrong signs,
wrong indices and transposed operands.  CPU only."""
import os

import numpy as np
import pytest
import scipy.signal

from paper_1608_00206_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U64 = 2.0 ** -53
U32 = 2.0 ** -24


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _scipy_conv(x, y, D):
    if D == 0:
        return (x * y).reshape(-1)
    z = scipy.signal.convolve(x.reshape((2,) * D), y.reshape((2,) * D), method="direct")
    assert z.shape == (3,) * D
    return z.reshape(-1)


# ----------------------------------------------------------------- definition


@pytest.mark.parametrize("D", list(range(0, 9)))
def test_brute_force_matches_scipy_nd_convolution(oracle, D):
    """Algorithm 1 equals scipy's direct N-d convolution of (2,)*D arrays."""
    x, y = inputs.uniform_int_pair(D, -100, 100, seed=D)
    assert np.array_equal(oracle.brute_force(x, y), _scipy_conv(x, y, D))
    xf, yf = x.astype(np.float64), y.astype(np.float64)
    assert np.array_equal(oracle.brute_force(xf, yf), _scipy_conv(xf, yf, D))


def test_base_cases_closed_form(oracle):
    """D = 0 returns the product; D = 1 is (x0 y0, x0 y1 + x1 y0, x1 y1)."""
    for dt in (np.int64, np.float64, np.float32):
        x = np.array([3], dtype=dt)
        y = np.array([-5], dtype=dt)
        for f in (oracle.brute_force, oracle.convolve):
            assert f(x, y).tolist() == [-15]
        x = np.array([2, 7], dtype=dt)
        y = np.array([-3, 5], dtype=dt)
        expect = [2 * -3, 2 * 5 + 7 * -3, 7 * 5]
        for f in (oracle.brute_force, oracle.convolve,
                  lambda a, b: oracle.convolve(a, b, direct_last_axis=True)):
            assert f(x, y).tolist() == expect


def test_carry_free_worked_example(oracle):
    """Discussion section: bits (1,1,1) + (1,0,1) -> digits (2,1,2) = flat 23."""
    (D, i, j, digits, k), = _golden("carry_free_example.txt")
    D, i, j, k = int(D), int(i), int(j), int(k)
    assert oracle.tmap(D)[i] + oracle.tmap(D)[j] == k
    assert [int(c) for c in digits.split(",")] == [k // 9 % 3, k // 3 % 3, k % 3]
    x = np.zeros(1 << D, np.int64)
    y = np.zeros(1 << D, np.int64)
    x[i], y[j] = 3, 4
    for f in (oracle.brute_force, oracle.convolve):
        z = f(x, y)
        assert z[k] == 12 and np.count_nonzero(z) == 1


def test_carry_free_oracle_worked_example(oracle):
    """The 1D carry-free oracle puts x[7] * y[5] at (2,1,2) = 23 (Discussion),
    not at the carried sum 12."""
    (D, i, j, digits, k), = _golden("carry_free_example.txt")
    x = np.zeros(8, np.int64)
    y = np.zeros(8, np.int64)
    x[int(i)], y[int(j)] = 3, 4
    z = oracle.carry_free(x, y)
    assert z.size == 27 and z[int(k)] == 12 and np.count_nonzero(z) == 1


@pytest.mark.parametrize("N", [1, 2, 3, 5, 8, 13, 100, 256, 777])
def test_carry_free_oracle_folds_to_ordinary_convolution(oracle, N):
    """Applying the carries turns the carry-free convolution back into the
    ordinary one: summing z[k] over the outputs whose base-3 digits, read as
    base-2 weights, give m yields (x conv y)[m] (numpy's direct 1D
    convolution), exactly in int64."""
    g = np.random.default_rng(N)
    x = g.integers(-50, 51, size=N, dtype=np.int64)
    y = g.integers(-50, 51, size=N, dtype=np.int64)
    z = oracle.carry_free(x, y)
    D = (N - 1).bit_length()
    assert z.size == 3 ** D
    k = np.arange(3 ** D)
    val2 = np.zeros_like(k)
    for d in range(D):
        val2 += (k // 3 ** d % 3) << d
    folded = np.zeros(2 * N - 1 if N > 1 else 1, np.int64)
    if D == 0:
        folded[0] = z[0]
    else:
        reach = val2 < folded.size
        assert not np.any(z[~reach])  # no pair of indices < N lands beyond 2N - 2
        np.add.at(folded, val2[reach], z[reach])
    assert np.array_equal(folded, np.convolve(x, y))


@pytest.mark.parametrize("N", [2, 8, 64, 3, 6, 45, 200])
def test_carry_free_oracle_is_padded_hypercube_convolution(oracle, N):
    """For N = 2^D the carry-free convolution is Algorithm 1 on the vectors as
    hypercubes; otherwise on the vectors zero-padded to 2^D (float64 too)."""
    g = np.random.default_rng(100 + N)
    D = (N - 1).bit_length()
    for dt in (np.int64, np.float64):
        x = g.integers(-9, 10, size=N).astype(dt)
        y = g.integers(-9, 10, size=N).astype(dt)
        xp = np.zeros(1 << D, dt)
        yp = np.zeros(1 << D, dt)
        xp[:N], yp[:N] = x, y
        assert np.array_equal(oracle.carry_free(x, y), oracle.brute_force(xp, yp))


@pytest.mark.parametrize("D", [1, 4, 9])
def test_delta_inputs(oracle, D):
    """x = e_i, y = e_j gives z = e_{t(i)+t(j)} (single product, no carries)."""
    g = np.random.default_rng(100 + D)
    t = oracle.tmap(D)
    for _ in range(6):
        i, j = (int(v) for v in g.integers(0, 1 << D, size=2))
        x = np.zeros(1 << D, np.int64)
        y = np.zeros(1 << D, np.int64)
        x[i], y[j] = 1, 1
        z = oracle.convolve(x, y)
        e = np.zeros(3 ** D, np.int64)
        e[t[i] + t[j]] = 1
        assert np.array_equal(z, e)


# ------------------------------------------------------ recurrence vs brute


@pytest.mark.parametrize("D", list(range(0, 13)))
def test_recurrence_bit_exact_vs_brute_int64(oracle, D):
    x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=7 + D)
    zb = oracle.brute_force(x, y)
    assert np.array_equal(oracle.convolve(x, y), zb)
    assert np.array_equal(oracle.convolve(x, y, direct_last_axis=True), zb)
    assert np.array_equal(oracle.convolve(x, y, threads=4), zb)


def test_recurrence_int64_wraps_mod_2_64(oracle):
    """Values near 2^62 overflow; the ring map to Z/2^64 makes every order agree."""
    g = np.random.default_rng(5)
    D = 7
    x = g.integers(-(1 << 62), 1 << 62, size=1 << D, dtype=np.int64)
    y = g.integers(-(1 << 62), 1 << 62, size=1 << D, dtype=np.int64)
    with np.errstate(over="ignore"):
        assert np.array_equal(oracle.convolve(x, y), oracle.brute_force(x, y))


@pytest.mark.parametrize("D", [10, 13, 16])
def test_sum_invariant_int64(oracle, D):
    """sum(z) = sum(x) * sum(y), exact in Z/2^64."""
    x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=D)
    z = oracle.convolve(x, y, threads=4)
    with np.errstate(over="ignore"):
        assert int(z.sum()) == int(x.sum()) * int(y.sum())


@pytest.mark.parametrize("D", [8, 14])
def test_separable_closed_form_int64(oracle, D):
    """x = kron(a_1..a_D), y = kron(b_1..b_D) gives z = kron(a_d * b_d), the
    per-axis 3-point convolutions (np.kron, exact in Z/2^64)."""
    a = inputs.separable_factors(D, 1, "int")
    b = inputs.separable_factors(D, 2, "int")
    x, y = inputs.outer_product_cube(a), inputs.outer_product_cube(b)
    c = np.stack([a[:, 0] * b[:, 0], a[:, 0] * b[:, 1] + a[:, 1] * b[:, 0], a[:, 1] * b[:, 1]], 1)
    with np.errstate(over="ignore"):
        z_closed = inputs.outer_product_cube(c)
        assert np.array_equal(oracle.convolve(x, y), z_closed)


def test_linearity_int64(oracle):
    D = 9
    x1, y = inputs.uniform_int_pair(D, -50, 50, seed=3)
    x2, _ = inputs.uniform_int_pair(D, -50, 50, seed=4)
    lhs = oracle.convolve(5 * x1 + x2, y)
    rhs = 5 * oracle.convolve(x1, y) + oracle.convolve(x2, y)
    assert np.array_equal(lhs, rhs)
    assert np.array_equal(oracle.convolve(x1, y), oracle.convolve(y, x1))


@pytest.mark.parametrize("D", [0, 3, 10])
def test_points_match_brute(oracle, D):
    x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=11)
    zb = oracle.brute_force(x, y)
    ks = np.arange(3 ** D)
    assert np.array_equal(oracle.points(x, y, ks), zb)


# ----------------------------------------------------------- floating point


def test_paper_accuracy_workload(oracle):
    """Table 1 workload x = y = [1..2^D]: z[0...0] = 1 with no error, and for
    D <= 11 every magnitude stays below 2^53 so float64 equals int64 exactly."""
    for D, z_first, z_last in _golden("paper_accuracy.txt"):
        D = int(D)
        if D > 14:
            continue
        x = inputs.paper_accuracy(D)
        z = oracle.convolve(x, x, threads=4)
        assert z[0] == float(z_first) and z[-1] == float(z_last)
        if D <= 11:
            zi = oracle.convolve(x.astype(np.int64), x.astype(np.int64))
            assert np.array_equal(z, zi.astype(np.float64))
            assert oracle.zabs(x, x).max() < 2.0 ** 53


@pytest.mark.parametrize("D", [4, 8, 12])
@pytest.mark.parametrize("dt,bits,u", [(np.float64, 24, U64), (np.float32, 10, U32)])
def test_forward_error_bound_vs_exact(oracle, D, dt, bits, u):
    """Dyadic inputs are exact in the float type, so the int64 oracle gives the
    exact real result; the recurrence must stay within gamma_{3D+1} * zabs."""
    g = np.random.default_rng(D)
    xi = inputs.dyadic(g.random(1 << D), bits)
    yi = inputs.dyadic(g.random(1 << D), bits)
    scale = float(1 << bits) ** 2
    z_exact = oracle.convolve(xi, yi).astype(np.float64) / scale
    x, y = (xi / float(1 << bits)).astype(dt), (yi / float(1 << bits)).astype(dt)
    zh = oracle.convolve(x, y).astype(np.float64)
    za = oracle.zabs(x, y)
    err = np.abs(zh - z_exact)
    assert np.all(err <= oracle.gamma(3 * D + 1, u) * za * 1.0000001)
    # the bound is not vacuous: the observed error stays far below zabs
    assert err.max() <= 64 * u * za.max()


def test_zabs_separable_closed_form(oracle):
    """For separable non-negative inputs the magnitude recurrence factorises
    into per-axis (p0, p0 + p1 + p2, p2) maps of the evaluated products."""
    D = 10
    a = np.abs(inputs.separable_factors(D, 7, "int")).astype(np.float64) + 1
    b = np.abs(inputs.separable_factors(D, 8, "int")).astype(np.float64) + 1
    x, y = inputs.outer_product_cube(a), inputs.outer_product_cube(b)
    p0, p2 = a[:, 0] * b[:, 0], a[:, 1] * b[:, 1]
    p1 = (a[:, 0] + a[:, 1]) * (b[:, 0] + b[:, 1])
    c = np.stack([p0, p0 + p1 + p2, p2], 1)
    assert np.array_equal(oracle.zabs(x, y), inputs.outer_product_cube(c))


@pytest.mark.parametrize("D", [6, 10])
def test_separable_probability_fp64(oracle, D):
    """Dirichlet-separable PMFs: recurrence within its bound of the closed form."""
    x, y, a, b = inputs.prob_separable_pair(D, seed=D)
    c = np.stack([a[:, 0] * b[:, 0], a[:, 0] * b[:, 1] + a[:, 1] * b[:, 0], a[:, 1] * b[:, 1]], 1)
    z_closed = inputs.outer_product_cube(c)
    z = oracle.convolve(x, y)
    za = oracle.zabs(x, y)
    bound = oracle.gamma(3 * D + 1, U64) * za + oracle.gamma(3 * D, U64) * np.abs(z_closed)
    assert np.all(np.abs(z - z_closed) <= bound)
    assert abs(z.sum() - 1.0) < 1e-12


# ------------------------------------------- in-place schedule (Methods)


@pytest.mark.parametrize("D", list(range(0, 10)))
def test_inplace_schedule_int64_vs_brute(oracle, D):
    """The corrected in-place schedule (sums in the first halves of x and y,
    put back before each call returns) equals brute force in Z/2^64 with
    either way of putting back, and hands x and y back unchanged."""
    x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=50 + D)
    want = oracle.brute_force(x, y)
    for save in (True, False):
        z, xa, ya = oracle.convolve_inplace(x, y, save=save)
        assert np.array_equal(z, want), save
        assert np.array_equal(xa, x) and np.array_equal(ya, y), save


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_inplace_schedule_with_saved_halves_is_the_recurrence(oracle, dt):
    """With the first halves copied aside, every element sees the
    recurrence's operations in its order: the result is bitwise the fresh-
    temporary recurrence's, exact on dyadic inputs within the forward bound,
    and x, y come back bitwise."""
    D = 10
    x, y = inputs.normal_pair(D, seed=5, dtype=dt)
    z, xa, ya = oracle.convolve_inplace(x, y, save=True)
    assert np.array_equal(z.view(np.uint8), oracle.convolve(x, y).view(np.uint8))
    assert np.array_equal(xa.view(np.uint8), x.view(np.uint8))
    assert np.array_equal(ya.view(np.uint8), y.view(np.uint8))


def test_inplace_schedule_subtracting_back_needs_exact_sums(oracle):
    """Putting the first halves back by subtraction is exact only when
    (a + b) - b = a (the paper's exactness condition): with a half that the
    sum absorbs (0.1 next to 1e17) x comes back changed, and the result
    departs from the recurrence; with integer-valued inputs, whose sums are
    all exact, it is the recurrence bit for bit."""
    D = 3
    x = np.array([0.1, 0.2, 0.3, 0.4, 1e17, 1e17, 1e17, 1e17])
    y = np.arange(1.0, 9.0)
    z, xa, _ = oracle.convolve_inplace(x, y, save=False)
    assert not np.array_equal(xa, x)
    assert xa[0] == 0.0  # (0.1 + 1e17) - 1e17
    zr, _, _ = oracle.convolve_inplace(x, y, save=True)
    assert not np.array_equal(z, zr)
    xi, yi = inputs.uniform_int_pair(10, -1000, 1000, seed=4)
    xs, ys = xi.astype(np.float64), yi.astype(np.float64)  # every sum exact
    z, xa, ya = oracle.convolve_inplace(xs, ys, save=False)
    assert np.array_equal(z, oracle.convolve(xs, ys)) and np.array_equal(xa, xs)


def test_direct_last_axis_is_a_different_rounding(oracle):
    """Integers: identical; floats: the D = 1 base case rounds differently but
    stays within the same bound."""
    D = 10
    x, y = inputs.prob_exponential_pair(D, seed=1)
    z0 = oracle.convolve(x, y)
    z1 = oracle.convolve(x, y, direct_last_axis=True)
    za = oracle.zabs(x, y)
    assert not np.array_equal(z0, z1)
    assert np.all(np.abs(z0 - z1) <= 2 * oracle.gamma(3 * D + 1, U64) * za)


def test_threads_bitwise_identical(oracle):
    x, y = inputs.prob_exponential_pair(12, seed=2)
    assert np.array_equal(oracle.convolve(x, y).view(np.uint64),
                          oracle.convolve(x, y, threads=8).view(np.uint64))


# ------------------------------------------------------------ mixed precision


def test_mixed_exact_when_every_product_is_exact(oracle):
    """x = (2795, -6686), y = (-3436, 3): every value and product is an integer
    below 2^24, so exact in binary32.  P0 = -9603620, P1 = 13357803,
    P2 = -20058, and z[1] = (P1 - P0) - P2 = 22981481 exactly, which rounds to
    22981480 in binary32 (ties to even).  Plain binary32 rounds P1 - P0 =
    22961423 to 22961424 first and ends at 22981482; the float-float
    interpolation keeps 22961423 exactly and rounds once.  Embedding the pair
    along the last axis of a D = 3 cube with (1, 0) factors on the other axes
    repeats the same operations."""
    for D in (1, 3):
        lead = inputs.outer_product_cube(np.array([[1, 0]] * (D - 1), np.int64))
        xi = np.kron(lead, np.array([2795, -6686], np.int64))
        yi = np.kron(lead, np.array([-3436, 3], np.int64))
        z_exact = oracle.convolve(xi, yi)
        k = 1  # flat index of digits (0, ..., 0, 1)
        assert z_exact[k] == 22981481
        x, y = xi.astype(np.float32), yi.astype(np.float32)
        zm = oracle.convolve_mixed(x, y)
        z32 = oracle.convolve(x, y)
        assert zm[k] == np.float32(22981480.0) and z32[k] == np.float32(22981482.0)
        assert np.array_equal(zm, z_exact.astype(np.float32))


@pytest.mark.parametrize("D", [6, 10])
def test_mixed_within_fp32_bound(oracle, D):
    g = np.random.default_rng(D)
    xi = inputs.dyadic(g.random(1 << D), 10)
    yi = inputs.dyadic(g.random(1 << D), 10)
    z_exact = oracle.convolve(xi, yi).astype(np.float64) / float(1 << 20)
    x, y = (xi / 1024.0).astype(np.float32), (yi / 1024.0).astype(np.float32)
    zm = oracle.convolve_mixed(x, y).astype(np.float64)
    za = oracle.zabs(x, y)
    assert np.all(np.abs(zm - z_exact) <= oracle.gamma(3 * D + 1, U32) * za + U32 * np.abs(z_exact))


# ------------------------------------------------------------------ adjoint


@pytest.mark.parametrize("D", list(range(0, 10)))
def test_adjoint_recurrence_vs_brute_int64(oracle, D):
    x, y = inputs.uniform_int_pair(D, -100, 100, seed=D)
    g = inputs.uniform_int(D, -100, 100, seed=50 + D)
    dz = np.random.default_rng(D).integers(-100, 101, size=3 ** D, dtype=np.int64)
    dx, dy = oracle.adjoint(dz, x, y)
    bx, by = oracle.adjoint_brute(dz, x, y)
    assert np.array_equal(dx, bx) and np.array_equal(dy, by)
    del g


@pytest.mark.parametrize("D", [3, 8, 11])
def test_adjoint_identity_int64(oracle, D):
    """<dz, x*y> = <dx, x> = <dy, y>: the adjoint is the transpose (exact in Z/2^64)."""
    x, y = inputs.uniform_int_pair(D, -100, 100, seed=D)
    dz = np.random.default_rng(D).integers(-100, 101, size=3 ** D, dtype=np.int64)
    z = oracle.brute_force(x, y) if D <= 8 else oracle.convolve(x, y)
    dx, dy = oracle.adjoint(dz, x, y)
    with np.errstate(over="ignore"):
        lhs = int((dz * z).sum())
        assert lhs == int((dx * x).sum()) == int((dy * y).sum())


def test_adjoint_all_ones_upstream(oracle):
    """dz = 1 everywhere gives dx = sum(y), dy = sum(x) in every entry."""
    D = 9
    x, y = inputs.uniform_int_pair(D, -100, 100, seed=1)
    dx, dy = oracle.adjoint(np.ones(3 ** D, np.int64), x, y)
    assert np.all(dx == y.sum()) and np.all(dy == x.sum())


def test_adjoint_finite_differences_fp64(oracle):
    """L = sum(w * (x*y)) is linear in x, so central differences are exact up to
    rounding; they match the float64 adjoint at D = 8."""
    D = 8
    x, y = inputs.normal_pair(D, seed=3, dtype=np.float64)
    w = inputs.normal(3 ** D, seed=4, dtype=np.float64)
    dx, dy = oracle.adjoint(w, x, y)
    g = np.random.default_rng(0)
    h = 1e-3
    for i in g.integers(0, 1 << D, size=12):
        e = np.zeros(1 << D)
        e[i] = h
        fd_x = (np.dot(w, oracle.convolve(x + e, y)) - np.dot(w, oracle.convolve(x - e, y))) / (2 * h)
        fd_y = (np.dot(w, oracle.convolve(x, y + e)) - np.dot(w, oracle.convolve(x, y - e))) / (2 * h)
        assert abs(fd_x - dx[i]) <= 1e-9 * (1 + abs(dx[i]))
        assert abs(fd_y - dy[i]) <= 1e-9 * (1 + abs(dy[i]))


# --------------------------------------------------------- planted mistakes


def _py_rec(x, y, mutation=None):
    """Small pure-Python copy of the recurrence with an optional planted mistake."""
    D = len(x).bit_length() - 1
    if D == 0:
        return [x[0] * y[0]]
    h, n = 1 << (D - 1), 3 ** (D - 1)
    z0 = _py_rec(x[:h], y[:h], mutation)
    z2 = _py_rec(x[h:], y[h:], mutation)
    if mutation == "drop_y1":
        t = _py_rec([x[k] + x[h + k] for k in range(h)], y[:h], mutation)
    elif mutation == "swap_operand_halves":
        t = _py_rec([x[k] + x[h + k] for k in range(h)], [y[k] + y[h + k] for k in range(h)],
                    mutation)
        z0, z2 = _py_rec(x[:h], y[h:], mutation), _py_rec(x[h:], y[:h], mutation)
    else:
        t = _py_rec([x[k] + x[h + k] for k in range(h)], [y[k] + y[h + k] for k in range(h)],
                    mutation)
    if mutation == "sign":
        z1 = [t[k] - z0[k] + z2[k] for k in range(n)]
    else:
        z1 = [t[k] - z0[k] - z2[k] for k in range(n)]
    if mutation == "order":
        return z2 + z1 + z0
    if mutation == "interleave":
        return [v for trip in zip(z0, z1, z2) for v in trip]
    return z0 + z1 + z2


@pytest.mark.parametrize("mutation", ["sign", "drop_y1", "swap_operand_halves", "order",
                                      "interleave"])
def test_pins_catch_planted_mistakes(oracle, mutation):
    D = 4
    x, y = inputs.uniform_int_pair(D, -9, 9, seed=12)
    good = np.array(_py_rec(list(x), list(y)))
    assert np.array_equal(good, _scipy_conv(x, y, D))
    bad = np.array(_py_rec(list(x), list(y), mutation))
    assert not np.array_equal(bad, _scipy_conv(x, y, D))
    # index and layout mistakes are also caught by a single delta pair:
    # bits (1,0,0) + (1,1,0) -> digits (2,1,0) = flat 21 (not a palindrome)
    e4, e6 = np.zeros(8, np.int64), np.zeros(8, np.int64)
    e4[4], e6[6] = 1, 1
    if mutation in ("order", "interleave"):
        assert np.array(_py_rec(list(e4), list(e6), mutation)).argmax() != 21
    assert np.array(_py_rec(list(e4), list(e6))).argmax() == 21


# ------------------------------------------------------- float-float form


def test_ff_hand_example(oracle):
    """x = y = (4097, 1): z = (4097^2, 2 * 4097, 1) = (16785409, 8194, 1).  In
    binary32 the product 4097^2 = 2^24 + 8193 rounds (ties to even) to
    16785408, so plain binary32 and the float-float-interpolation form both
    end at z[1] = (4098^2 - 16785408) - 1 = 8195.  The float-float form keeps
    the product's low part (4097^2 - 16785408 = 1, from the FMA two-product)
    and gets z[1] = 8194 exactly; z[0] rounds once, to 16785408."""
    x = np.array([4097, 1], np.float32)
    zf = oracle.convolve_ff(x, x)
    assert zf.tolist() == [16785408.0, 8194.0, 1.0]
    assert oracle.convolve(x, x)[1] == 8195.0
    assert oracle.convolve_mixed(x, x)[1] == 8195.0


@pytest.mark.parametrize("D,r", [(4, 4000), (8, 4000), (10, 2000), (12, 1000)])
def test_ff_is_the_rounded_exact_result_on_integer_inputs(oracle, D, r):
    """Integer inputs: every sum, product and difference of the recurrence is
    an integer that a float-float pair holds exactly here, so the form returns
    the exact result (the int64 oracle) rounded once to binary32, at every
    output -- while binary32 products lose bits (plain binary32 and the
    mixed form miss outputs)."""
    xi, yi = inputs.uniform_int_pair(D, -r, r, seed=D)
    want = oracle.convolve(xi, yi).astype(np.float32)
    x, y = xi.astype(np.float32), yi.astype(np.float32)
    assert np.array_equal(oracle.convolve_ff(x, y), want)
    assert np.count_nonzero(oracle.convolve(x, y) != want) > 0
    assert np.count_nonzero(oracle.convolve_mixed(x, y) != want) > 0


@pytest.mark.parametrize("D", [6, 10, 12])
def test_ff_within_float_float_bound(oracle, D):
    """Dyadic U[0,1) inputs (exact result from the int64 oracle): the error is
    one final binary32 rounding plus the float-float rounding of the 3D + 1
    operations on the longest path, bounded with u = 2^-44 (the float-float
    operations' unit roundoff is about 2^-47)."""
    g = np.random.default_rng(D)
    xi = inputs.dyadic(g.random(1 << D), 10)
    yi = inputs.dyadic(g.random(1 << D), 10)
    z_exact = oracle.convolve(xi, yi).astype(np.float64) / float(1 << 20)
    x, y = (xi / 1024.0).astype(np.float32), (yi / 1024.0).astype(np.float32)
    zf = oracle.convolve_ff(x, y).astype(np.float64)
    za = oracle.zabs(x, y)
    assert np.all(np.abs(zf - z_exact) <= oracle.gamma(3 * D + 1, 2.0 ** -44) * za
                  + U32 * np.abs(z_exact))
    # and far inside the binary32 bound the other forms need
    z32 = oracle.convolve(x, y).astype(np.float64)
    assert np.max(np.abs(zf - z_exact)) < np.max(np.abs(z32 - z_exact))


# ---------------------------------------------------------------- hybrid form


@pytest.mark.parametrize("D", [1, 4, 7, 9])
def test_direct_top_int64_equals_brute_force_for_every_split(oracle, D):
    """The hybrid form (4-way direct form on the top mt axes, Karatsuba on
    the rest) is exact in Z/2^64 for every mt: Algorithm 1's result."""
    x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=900 + D)
    want = oracle.brute_force(x, y)
    for mt in range(D + 1):
        assert np.array_equal(oracle.convolve_direct_top(x, y, mt), want), mt


@pytest.mark.parametrize("D", [3, 6, 8])
def test_direct_top_float_end_points(oracle, D):
    """Floating point: with no direct axes it is the recurrence bit for bit,
    with every axis direct it is Algorithm 1's summation bit for bit (pairs
    summed in increasing x index, as the brute force visits them)."""
    for dt in (np.float64, np.float32):
        x, y = inputs.normal_pair(D, seed=910 + D, dtype=dt)
        assert np.array_equal(oracle.convolve_direct_top(x, y, 0).view(np.uint8),
                              oracle.convolve(x, y).view(np.uint8))
        assert np.array_equal(oracle.convolve_direct_top(x, y, D).view(np.uint8),
                              oracle.brute_force(x, y).view(np.uint8))


@pytest.mark.parametrize("D,mt", [(8, 3), (10, 4), (10, 2)])
def test_direct_top_within_forward_bound(oracle, D, mt):
    """Dyadic inputs (exact result from the int64 oracle): float32 hybrid
    results stay within gamma_{3D+1}(2^-24) * zabs (the direct axes replace
    the Karatsuba ones' sums and differences by at most as many additions of
    terms no larger in magnitude)."""
    g = np.random.default_rng(D + mt)
    xi = inputs.dyadic(g.random(1 << D), 10)
    yi = inputs.dyadic(g.random(1 << D), 10)
    z_exact = oracle.convolve(xi, yi).astype(np.float64) / float(1 << 20)
    x, y = (xi / 1024.0).astype(np.float32), (yi / 1024.0).astype(np.float32)
    zh = oracle.convolve_direct_top(x, y, mt).astype(np.float64)
    za = oracle.zabs(x, y)
    assert np.all(np.abs(zh - z_exact) <= oracle.gamma(3 * D + 1, U32) * za)


@pytest.mark.parametrize("D", [0, 1, 5, 9, 12])
@pytest.mark.parametrize("dt", [np.int64, np.float64, np.float32])
def test_points_rec_is_the_recurrence_at_each_output(oracle, D, dt):
    """The recurrence at single outputs (only the entries each output depends
    on, every digit 1) gives the full recurrence's bits, in every dtype."""
    if dt == np.int64:
        x, y = inputs.uniform_int_pair(D, -1000, 1000, seed=40 + D)
    else:
        x, y = inputs.uniform01_pair(D, seed=40 + D, dtype=dt)
        x = x - dt(0.5)
    full = oracle.convolve(x, y)
    ks = np.arange(3 ** D) if D <= 9 else np.random.default_rng(D).integers(0, 3 ** D, 4000)
    got = oracle.points_rec(x, y, ks)
    bits = np.uint64 if np.dtype(dt).itemsize == 8 else np.uint32
    assert np.array_equal(got.view(bits), full[ks].view(bits))
    if dt == np.int64:
        assert np.array_equal(got, oracle.points(x, y, ks))
