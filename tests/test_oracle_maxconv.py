"""Pins for the max-convolution oracle (Discussion: exact max-convolution of
bounded non-negative integers through p-norm rings).

The brute-force max-convolution is pinned by hand examples, the separable
closed form, delta inputs, the 0/1 special case (an OR of pair indicators,
i.e. the sum-convolution's support) and the max <= sum <= count * max
sandwich.  The p-norm route is pinned to the brute force, its choice of p
to the tightness of the bound, and the limb embedding to the exact sums of
p-th powers in Python integers.  CPU only."""

import numpy as np
import pytest

from paper_1608_00206_gb300 import inputs


def _digits(k, D):
    out = []
    for _ in range(D):
        out.append(k % 3)
        k //= 3
    return out[::-1]          # axis 1 first


def test_maxconv_hand_examples(oracle):
    """D = 1: (x0 y0, max(x0 y1, x1 y0), x1 y1); D = 2 worked by hand."""
    x = np.array([2, 5], dtype=np.int64)
    y = np.array([3, 1], dtype=np.int64)
    assert oracle.maxconv_brute(x, y).tolist() == [6, 15, 5]
    # x[i1, i2] = [[1, 4], [2, 0]], y = [[3, 1], [0, 2]]
    x = np.array([1, 4, 2, 0], dtype=np.int64)
    y = np.array([3, 1, 0, 2], dtype=np.int64)
    # k = (k1, k2): pairs per axis (0,0) | (0,1),(1,0) | (1,1)
    expect = [
        1 * 3,                      # (0,0): x00 y00
        max(1 * 1, 4 * 3),          # (0,1): x00 y01, x01 y00
        4 * 1,                      # (0,2): x01 y01
        max(1 * 0, 2 * 3),          # (1,0): x00 y10, x10 y00
        max(1 * 2, 4 * 0, 2 * 1, 0 * 3),  # (1,1)
        max(4 * 2, 0 * 1),          # (1,2): x01 y11, x11 y01
        2 * 0,                      # (2,0): x10 y10
        max(2 * 2, 0 * 0),          # (2,1): x10 y11, x11 y10
        0 * 2,                      # (2,2)
    ]
    assert oracle.maxconv_brute(x, y).tolist() == expect
    assert oracle.maxconv_brute(np.array([7]), np.array([6])).tolist() == [42]


@pytest.mark.parametrize("D", [1, 3, 6, 9])
def test_maxconv_separable_closed_form(oracle, D):
    """x = (x) a_d, y = (x) b_d with non-negative factors: the maximum over a
    product of independent per-axis choices is the product of per-axis maxima,
    m_d = (a0 b0, max(a0 b1, a1 b0), a1 b1)."""
    g = np.random.default_rng(100 + D)
    a = g.integers(0, 4, size=(D, 2), dtype=np.int64)
    b = g.integers(0, 4, size=(D, 2), dtype=np.int64)
    x = inputs.outer_product_cube(a)
    y = inputs.outer_product_cube(b)
    m = [(a[d, 0] * b[d, 0], max(a[d, 0] * b[d, 1], a[d, 1] * b[d, 0]), a[d, 1] * b[d, 1])
         for d in range(D)]
    z = oracle.maxconv_brute(x, y)
    for k in range(3 ** D):
        want = 1
        for d, q in enumerate(_digits(k, D)):
            want *= int(m[d][q])
        assert int(z[k]) == want, k


@pytest.mark.parametrize("D", [2, 5])
def test_maxconv_delta_inputs(oracle, D):
    """x = u e_i, y = v e_j: u v at t(i) + t(j), zero elsewhere."""
    t = oracle.tmap(D)
    for i, j in [(0, 0), (1, (1 << D) - 1), ((1 << D) - 1, (1 << D) - 1), (2 % (1 << D), 1)]:
        x = np.zeros(1 << D, dtype=np.int64)
        y = np.zeros(1 << D, dtype=np.int64)
        x[i], y[j] = 3, 11
        z = oracle.maxconv_brute(x, y)
        want = np.zeros(3 ** D, dtype=np.int64)
        want[t[i] + t[j]] = 33
        assert np.array_equal(z, want)


@pytest.mark.parametrize("D", [4, 8])
def test_maxconv_of_0_1_inputs_is_the_support(oracle, D):
    """For 0/1 entries the maximum is 1 exactly where some pair has x = y = 1,
    i.e. where the (sum) convolution is non-zero."""
    x, y = inputs.uniform_int_pair(D, 0, 1, seed=D)
    assert np.array_equal(oracle.maxconv_brute(x, y), (oracle.brute_force(x, y) > 0).astype(np.int64))


@pytest.mark.parametrize("D", [3, 7, 10])
def test_maxconv_sandwich(oracle, D):
    """Non-negative inputs: max <= sum <= (number of pairs) * max, with
    2^{#ones(k)} pairs at output k."""
    x, y = inputs.uniform_int_pair(D, 0, 9, seed=7 * D)
    zm = oracle.maxconv_brute(x, y)
    zs = oracle.brute_force(x, y)
    ones = np.zeros(3 ** D, dtype=np.int64)
    k = np.arange(3 ** D)
    for _ in range(D):
        ones += (k % 3 == 1)
        k //= 3
    assert np.all(zm <= zs)
    assert np.all(zs <= (np.int64(1) << ones) * zm)


@pytest.mark.parametrize("D,vmax", [(0, 5), (1, 3), (2, 15), (3, 3), (4, 7), (5, 2), (6, 1),
                                    (6, 3), (3, 0)])
def test_pnorm_route_equals_maximum(oracle, D, vmax):
    """The integer nearest the p-norm estimate is the maximum (Discussion)."""
    x, y = inputs.uniform_int_pair(D, 0, vmax, seed=31 * D + vmax)
    assert np.array_equal(oracle.maxconv_pnorm(x, y, vmax), oracle.maxconv_brute(x, y))


@pytest.mark.parametrize("D,vmax", [(1, 1), (3, 2), (4, 3), (6, 2), (2, 7)])
def test_p_is_the_smallest_that_keeps_the_bound(oracle, D, vmax):
    """p satisfies M (2^(D/p) - 1) < 7/16 and p - 1 does not; with the paper's
    own 1/2, p - 1 already rounds the all-vmax input's all-ones output (2^D
    equal products M) to M + 1: the bound is what makes the rounding exact."""
    p = oracle.maxconv_p(D, vmax)
    M = vmax * vmax
    assert oracle.maxconv_bound_holds(D, vmax, p)
    assert p == 1 or not oracle.maxconv_bound_holds(D, vmax, p - 1)
    assert abs(M * (2.0 ** (D / p) - 1.0)) < 7 / 16
    ph = oracle.maxconv_p(D, vmax, num=1, den=2)
    assert ph <= p
    if ph > 1:
        x = np.full(1 << D, vmax, dtype=np.int64)
        z_bad = oracle.maxconv_pnorm(x, x, vmax, p=ph - 1)
        assert int(z_bad[(3 ** D - 1) // 2]) == M + 1
        z_ok = oracle.maxconv_pnorm(x, x, vmax, p=ph)
        assert np.array_equal(z_ok, oracle.maxconv_brute(x, x))


def test_nearest_root_exact():
    """nearest_root against hand values and a brute search."""
    import oracle as o
    assert o.nearest_root(0, 5) == 0
    assert o.nearest_root(1, 9) == 1
    assert o.nearest_root(3 ** 40, 40) == 3
    assert o.nearest_root(2 * 3 ** 40, 40) == 3
    for p in (1, 2, 3, 7):
        for s in range(0, 3000, 7):
            best = min(range(0, s + 2), key=lambda r: abs(r - s ** (1.0 / p)))
            assert o.nearest_root(s, p) == best


@pytest.mark.parametrize("D,vmax", [(1, 2), (3, 3), (4, 7), (2, 15), (5, 1), (0, 4)])
def test_limb_embedding_gives_the_sums_of_powers(oracle, D, vmax):
    """One int64 convolution of D + e axes, the limb index on the top e axes,
    gives slices whose limb-weighted sum is exactly sum (x[i] y[j])^p."""
    x, y = inputs.uniform_int_pair(D, 0, vmax, seed=5 + D)
    w, b, p = oracle.maxconv_limb_sums(x, y, vmax)
    exact = oracle._pow_sums(x, y, p)
    for k in range(3 ** D):
        s = sum(int(w[c, k]) << (c * b) for c in range(w.shape[0]))
        assert s == exact[k], k
    pp, bb, e, L = oracle.maxconv_limb_plan(D, vmax)
    assert pp == p and bb == b and L <= (1 << e) and D + e + 2 * b <= 63
    assert L * b >= max(1, (vmax ** p).bit_length())


def test_limb_embedding_catches_a_carry(oracle):
    """Reading the limb digits with carries (base 3 instead of the carry-free
    base-2 value) breaks the sums: the embedding's index reading matters."""
    D, vmax = 2, 15
    x, y = inputs.uniform_int_pair(D, 0, vmax, seed=9)
    w, b, p = oracle.maxconv_limb_sums(x, y, vmax)
    _, _, e, _ = oracle.maxconv_limb_plan(D, vmax)
    assert e >= 2
    exact = oracle._pow_sums(x, y, p)
    # Rebuild with the digit string read in base 3 (a wrong reading).
    n = 1 << D
    mask = (1 << b) - 1
    L = oracle.maxconv_limb_plan(D, vmax)[3]

    def limbs(v):
        U = np.zeros(((1 << e), n), dtype=np.int64)
        for i, val in enumerate(v.tolist()):
            for a in range(L):
                U[a, i] = ((int(val) ** p) >> (a * b)) & mask
        return U.reshape(-1)

    W = oracle.convolve(limbs(x), limbs(y)).reshape(3 ** e, 3 ** D)
    wrong = [sum(int(W[d, k]) << (d * b) for d in range(3 ** e)) for k in range(3 ** D)]
    assert wrong != exact


@pytest.mark.parametrize("D,vmax", [(0, 7), (3, 3), (8, 5)])
def test_maxconv_points_equal_brute(oracle, D, vmax):
    """The one-output-at-a-time definition agrees with the pair loop."""
    x, y = inputs.uniform_int_pair(D, 0, vmax, seed=70 + D)
    ks = np.arange(3 ** D)
    assert np.array_equal(oracle.maxconv_points(x, y, ks), oracle.maxconv_brute(x, y))
