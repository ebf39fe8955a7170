"""CPU oracle for hypercube convolution (arXiv 1608.00206) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package.  The product (``paper_1608_00206_gb300``)
never does: it has no CPU fallback.

Everything numeric lives in ``hc_oracle.cpp`` (plain C++, built with
``-O2 -ffp-contract=off``); this module only builds it, loads it with ctypes
and marshals numpy arrays.  Functions and the passages they follow:

* :func:`brute_force` -- Algorithm 1 (naive convolution), hypercube case.
* :func:`points`      -- the definition (Introduction) evaluated at chosen outputs.
* :func:`points_rec`  -- the Methods recurrence evaluated at chosen outputs,
  with its own rounding (full-size float checks on sampled outputs).
* :func:`carry_free`  -- the carry-free 1D convolution (Discussion), from its
  definition, for vectors of any length.
* :func:`convolve`    -- the Methods recurrence (3-way split, base case D = 0;
  ``direct_last_axis=True`` uses the 3-product D = 1 base case instead).
* :func:`convolve_mixed` -- the same recurrence with binary32 evaluation and
  products and float-float interpolation.
* :func:`convolve_direct_top` -- the hybrid form: 4-way direct form on the
  top ``mt`` axes, Karatsuba recurrence (Kronecker form) on the others.
* :func:`convolve_ff` -- the same recurrence with every value in float-float
  (two-sum evaluation, FMA two-product, two-sum interpolation), binary32 in
  and out.
* :func:`adjoint`, :func:`adjoint_brute` -- gradient of the convolution with
  respect to x and y (transpose of the recurrence; brute-force correlation).
* :func:`zabs` -- magnitude companion for the forward-error bound
  ``|z_hat - z| <= gamma_{3D+1} * zabs``.
* :func:`maxconv_brute`, :func:`maxconv_points` -- max-convolution
  (Discussion, the (x, max) semiring) from its definition, in C++: every
  output, or chosen outputs one at a time.
* :func:`maxconv_p`, :func:`maxconv_pnorm`, :func:`maxconv_limb_plan`,
  :func:`maxconv_limb_sums` -- the Discussion's p-norm route to exact
  max-convolution of bounded non-negative integers, in Python integers
  (arbitrary size, exact; small D only): the choice of p, the p-norm
  estimate rounded to the nearest integer, and the sums of p-th powers
  recovered from one int64 hypercube convolution whose extra axes are the
  bits of a limb index (the carry-free embedding of the same Discussion).

Dtype handling: int64 arrays are computed in Z/2^64 (two's complement wrap),
float64 and float32 in their own precision.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hc_oracle.cpp")
_SO = os.path.join(_HERE, "liboracle.so")
_LOCK = threading.Lock()
_LIB = None

_DTYPE_CODE = {np.dtype(np.int64): 0, np.dtype(np.float64): 1, np.dtype(np.float32): 2}


def build(force: bool = False) -> str:
    """Compile hc_oracle.cpp into liboracle.so next to it (no -Ofast, no FMA contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            build()
            lib = ctypes.CDLL(_SO)
            vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
            lib.oracle_brute.argtypes = [vp, vp, vp, i, i]
            lib.oracle_points.argtypes = [vp, vp, i, i, vp, sz, vp]
            lib.oracle_carryfree.argtypes = [vp, vp, vp, sz, i, i]
            lib.oracle_recurrence.argtypes = [vp, vp, vp, i, i, i, i]
            lib.oracle_recurrence_mixed.argtypes = [vp, vp, vp, i]
            lib.oracle_recurrence_ff.argtypes = [vp, vp, vp, i]
            lib.oracle_direct_top.argtypes = [vp, vp, vp, i, i, i]
            lib.oracle_recurrence_inplace.argtypes = [vp, vp, vp, i, i, i]
            lib.oracle_adjoint.argtypes = [vp, vp, vp, vp, vp, i, i]
            lib.oracle_adjoint_brute.argtypes = [vp, vp, vp, vp, vp, i, i]
            lib.oracle_zabs.argtypes = [vp, vp, vp, i]
            lib.oracle_points_rec.argtypes = [vp, vp, i, i, vp, sz, vp]
            lib.oracle_maxconv_brute.argtypes = [vp, vp, vp, i]
            lib.oracle_maxconv_points.argtypes = [vp, vp, i, vp, sz, vp]
            lib.oracle_max_threads.restype = i
            _LIB = lib
    return _LIB


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def dim_of(x: np.ndarray) -> int:
    """D such that x has 2^D elements."""
    n = int(x.size)
    D = n.bit_length() - 1
    if n < 1 or (1 << D) != n:
        raise ValueError(f"hypercube length {n} is not a power of two")
    return D


def _prep(x, y):
    x = np.ascontiguousarray(x).reshape(-1)
    y = np.ascontiguousarray(y).reshape(-1)
    if x.dtype != y.dtype or x.dtype not in _DTYPE_CODE:
        raise TypeError(f"unsupported dtypes {x.dtype}, {y.dtype}")
    if x.size != y.size:
        raise ValueError("x and y differ in length")
    return x, y, dim_of(x), _DTYPE_CODE[x.dtype]


def tmap(D: int) -> np.ndarray:
    """t(i) for every i in [0, 2^D): the bits of i read as base-3 digits."""
    t = np.zeros(1 << D, dtype=np.int64)
    i = np.arange(1 << D, dtype=np.int64)
    for d in range(D - 1, -1, -1):
        t = t * 3 + ((i >> d) & 1)
    return t


def brute_force(x, y) -> np.ndarray:
    """Algorithm 1 on hypercubes: z[t(i)+t(j)] += x[i]*y[j] for all pairs (O(4^D))."""
    x, y, D, code = _prep(x, y)
    z = np.empty(3 ** D, dtype=x.dtype)
    if _lib().oracle_brute(_ptr(x), _ptr(y), _ptr(z), D, code):
        raise RuntimeError("oracle_brute failed")
    return z


def points(x, y, ks) -> np.ndarray:
    """z[k] for each flat index k, summed over the 2^{#ones(k)} pairs i+j=k."""
    x, y, D, code = _prep(x, y)
    ks = np.ascontiguousarray(ks, dtype=np.uint64).reshape(-1)
    if ks.size and int(ks.max()) >= 3 ** D:
        raise ValueError("output index out of range")
    out = np.empty(ks.size, dtype=x.dtype)
    if _lib().oracle_points(_ptr(x), _ptr(y), D, code, _ptr(ks), ks.size, _ptr(out)):
        raise RuntimeError("oracle_points failed")
    return out


def points_rec(x, y, ks) -> np.ndarray:
    """z[k] at chosen flat indices k as the Methods recurrence computes it,
    with its rounding (the 2^{#ones(k)} entries that z[k] depends on, run
    through the recurrence with every output digit 1); bitwise equal to
    convolve(x, y)[ks] in every dtype.  OpenMP over the outputs."""
    x, y, D, code = _prep(x, y)
    ks = np.ascontiguousarray(ks, dtype=np.uint64).reshape(-1)
    if ks.size and int(ks.max()) >= 3 ** D:
        raise ValueError("output index out of range")
    out = np.empty(ks.size, dtype=x.dtype)
    if _lib().oracle_points_rec(_ptr(x), _ptr(y), D, code, _ptr(ks), ks.size, _ptr(out)):
        raise RuntimeError("oracle_points_rec failed")
    return out


def carry_free(x, y) -> np.ndarray:
    """Carry-free 1D convolution of two length-N vectors (any N >= 1): the
    bits of i and j added position by position without carries give the D
    base-3 digits of the output index, D = (N - 1).bit_length()."""
    x = np.ascontiguousarray(x).reshape(-1)
    y = np.ascontiguousarray(y).reshape(-1)
    if x.dtype != y.dtype or x.dtype not in _DTYPE_CODE or x.size != y.size or x.size < 1:
        raise ValueError("x and y must be non-empty, of one supported dtype and one length")
    N = int(x.size)
    D = (N - 1).bit_length()
    z = np.empty(3 ** D, dtype=x.dtype)
    if _lib().oracle_carryfree(_ptr(x), _ptr(y), _ptr(z), N, D, _DTYPE_CODE[x.dtype]):
        raise RuntimeError("oracle_carryfree failed")
    return z


def convolve(x, y, direct_last_axis: bool = False, threads: int = 1) -> np.ndarray:
    """The Methods recurrence on fresh temporaries; threads > 1 runs the top
    sub-problems as OpenMP tasks (bitwise identical result)."""
    x, y, D, code = _prep(x, y)
    z = np.empty(3 ** D, dtype=x.dtype)
    if _lib().oracle_recurrence(_ptr(x), _ptr(y), _ptr(z), D, code, int(direct_last_axis),
                                int(threads)):
        raise RuntimeError("oracle_recurrence failed")
    return z


def convolve_inplace(x, y, save: bool = True):
    """The in-place schedule (sums formed in the first halves of x and y,
    put back before each call returns): returns (z, x_after, y_after).
    save=True copies the first halves aside (exact for every type);
    save=False subtracts again (exact for int64 only)."""
    x = np.array(x, copy=True).reshape(-1)
    y = np.array(y, copy=True).reshape(-1)
    x, y, D, code = _prep(x, y)
    x = np.array(x, copy=True)
    y = np.array(y, copy=True)
    z = np.empty(3 ** D, dtype=x.dtype)
    if _lib().oracle_recurrence_inplace(_ptr(x), _ptr(y), _ptr(z), D, code, int(save)):
        raise RuntimeError("oracle_recurrence_inplace failed")
    return z, x, y


def convolve_mixed(x, y) -> np.ndarray:
    """binary32 evaluation and products, float-float interpolation, binary32 result."""
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1)
    y = np.ascontiguousarray(y, dtype=np.float32).reshape(-1)
    D = dim_of(x)
    z = np.empty(3 ** D, dtype=np.float32)
    _lib().oracle_recurrence_mixed(_ptr(x), _ptr(y), _ptr(z), D)
    return z


def convolve_direct_top(x, y, mt: int) -> np.ndarray:
    """The hybrid form: on the top mt axes the 4-way direct form (products of
    sub-cube pairs summed, no interpolation), on the other D - mt axes the
    Karatsuba form; mt = 0 is the recurrence, mt = D Algorithm 1."""
    x, y, D, code = _prep(x, y)
    z = np.empty(3 ** D, dtype=x.dtype)
    if _lib().oracle_direct_top(_ptr(x), _ptr(y), _ptr(z), D, int(mt), code):
        raise RuntimeError("oracle_direct_top failed")
    return z


def convolve_ff(x, y) -> np.ndarray:
    """Float-float evaluation, products (FMA two-product) and interpolation,
    binary32 in and out: one rounding at the end."""
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1)
    y = np.ascontiguousarray(y, dtype=np.float32).reshape(-1)
    D = dim_of(x)
    z = np.empty(3 ** D, dtype=np.float32)
    _lib().oracle_recurrence_ff(_ptr(x), _ptr(y), _ptr(z), D)
    return z


def adjoint(dz, x, y):
    """(dx, dy) for z = x*y and upstream gradient dz, by the transposed recurrence."""
    x, y, D, code = _prep(x, y)
    dz = np.ascontiguousarray(dz, dtype=x.dtype).reshape(-1)
    if dz.size != 3 ** D:
        raise ValueError("dz must have 3^D elements")
    dx = np.empty_like(x)
    dy = np.empty_like(y)
    if _lib().oracle_adjoint(_ptr(dz), _ptr(x), _ptr(y), _ptr(dx), _ptr(dy), D, code):
        raise RuntimeError("oracle_adjoint failed")
    return dx, dy


def adjoint_brute(dz, x, y):
    """(dx, dy) straight from the definition: dx[i] = sum_j dz[t(i)+t(j)] y[j]."""
    x, y, D, code = _prep(x, y)
    dz = np.ascontiguousarray(dz, dtype=x.dtype).reshape(-1)
    if dz.size != 3 ** D:
        raise ValueError("dz must have 3^D elements")
    dx = np.empty_like(x)
    dy = np.empty_like(y)
    if _lib().oracle_adjoint_brute(_ptr(dz), _ptr(x), _ptr(y), _ptr(dx), _ptr(dy), D, code):
        raise RuntimeError("oracle_adjoint_brute failed")
    return dx, dy


def zabs(x, y) -> np.ndarray:
    """The recurrence on |x|, |y| with subtractions turned into additions (float64)."""
    ax = np.abs(np.ascontiguousarray(x, dtype=np.float64).reshape(-1))
    ay = np.abs(np.ascontiguousarray(y, dtype=np.float64).reshape(-1))
    D = dim_of(ax)
    z = np.empty(3 ** D, dtype=np.float64)
    _lib().oracle_zabs(_ptr(ax), _ptr(ay), _ptr(z), D)
    return z


def gamma(n: int, u: float) -> float:
    """Higham's gamma_n = n u / (1 - n u)."""
    return n * u / (1.0 - n * u)


def max_threads() -> int:
    return int(_lib().oracle_max_threads())


# --------------------------------------------------------------------------
# Max-convolution through p-norm rings (Discussion).
#
# For non-negative integers of bounded range, max over a set of N terms u of
# the products x[i]*y[j] with i + j = k is approximated by the p-norm
# ||u||_p = (sum u^p)^(1/p), and sum u^p over those pairs is the ordinary
# convolution of x^p and y^p.  Since max u <= ||u||_p <= N^(1/p) max u, the
# estimate exceeds the maximum by at most M (N^(1/p) - 1), M the largest
# possible product; once that is below 1/2, the integer nearest the estimate
# is the maximum.  Readings: N = 2^D (an output has 2^{#ones(k)} <= 2^D
# pairs); M = vmax^2 for entries in [0, vmax]; the half unit is kept with a
# margin of 1/16 (the bound is required to be below 7/16) so that a root
# extracted in floating point still rounds to the right integer.

def maxconv_brute(x, y) -> np.ndarray:
    """z[k] = max of x[i]*y[j] over the pairs i + j = k (O(4^D), int64)."""
    x = np.ascontiguousarray(x, dtype=np.int64).reshape(-1)
    y = np.ascontiguousarray(y, dtype=np.int64).reshape(-1)
    if x.size != y.size:
        raise ValueError("x and y differ in length")
    D = dim_of(x)
    z = np.empty(3 ** D, dtype=np.int64)
    if _lib().oracle_maxconv_brute(_ptr(x), _ptr(y), _ptr(z), D):
        raise RuntimeError("oracle_maxconv_brute failed")
    return z


def maxconv_points(x, y, ks) -> np.ndarray:
    """Max-convolution at chosen flat output indices k, each from its
    2^{#ones(k)} pairs (the definition, one output at a time)."""
    x = np.ascontiguousarray(x, dtype=np.int64).reshape(-1)
    y = np.ascontiguousarray(y, dtype=np.int64).reshape(-1)
    D = dim_of(x)
    ks = np.ascontiguousarray(ks, dtype=np.uint64).reshape(-1)
    if ks.size and int(ks.max()) >= 3 ** D:
        raise ValueError("output index out of range")
    out = np.empty(ks.size, dtype=np.int64)
    if _lib().oracle_maxconv_points(_ptr(x), _ptr(y), D, _ptr(ks), ks.size, _ptr(out)):
        raise RuntimeError("oracle_maxconv_points failed")
    return out


def maxconv_bound_holds(D: int, vmax: int, p: int, num: int = 7, den: int = 16) -> bool:
    """M (2^(D/p) - 1) < num/den with M = vmax^2, decided exactly:
    2^D (den M)^p < (den M + num)^p in integers."""
    M = vmax * vmax
    return (1 << D) * (den * M) ** p < (den * M + num) ** p


def maxconv_p(D: int, vmax: int, num: int = 7, den: int = 16) -> int:
    """The smallest integer p >= 1 for which the p-norm estimate of every
    output is within num/den of its maximum (default 7/16: the paper's 1/2
    with a margin of 1/16)."""
    if vmax < 0 or D < 0:
        raise ValueError("vmax and D must be non-negative")
    M = vmax * vmax
    if M == 0:
        return 1
    # Starting guess from logarithms, then exact steps down and up.
    p = max(1, int(math.ceil(D * math.log(2.0) / math.log1p(num / (den * M)))))
    while p > 1 and maxconv_bound_holds(D, vmax, p - 1, num, den):
        p -= 1
    while not maxconv_bound_holds(D, vmax, p, num, den):
        p += 1
    return p


def _iroot(s: int, p: int) -> int:
    """floor(s^(1/p)) for an integer s >= 0 (integer Newton from above)."""
    if s < 2 or p == 1:
        return s
    r = 1 << -(-s.bit_length() // p)
    while True:
        q = ((p - 1) * r + s // r ** (p - 1)) // p
        if q >= r:
            return r
        r = q


def nearest_root(s: int, p: int) -> int:
    """The integer nearest s^(1/p) (exact; a tie cannot occur for the sums here
    but would round up)."""
    r = _iroot(s, p)
    return r + 1 if (s << p) >= (2 * r + 1) ** p else r


def _pow_sums(x, y, p: int):
    """s[k] = sum over i + j = k of (x[i] y[j])^p in Python integers
    (Algorithm 1's pair loop)."""
    D = dim_of(np.asarray(x).reshape(-1))
    t = tmap(D).tolist()
    xp = [int(v) ** p for v in np.asarray(x).reshape(-1).tolist()]
    yp = [int(v) ** p for v in np.asarray(y).reshape(-1).tolist()]
    s = [0] * (3 ** D)
    for i, a in enumerate(xp):
        if a:
            ti = t[i]
            for j, b in enumerate(yp):
                if b:
                    s[ti + t[j]] += a * b
    return s


def maxconv_pnorm(x, y, vmax: int, p: int | None = None) -> np.ndarray:
    """The Discussion's route: the sums of p-th powers (an ordinary hypercube
    convolution of x^p and y^p), then the integer nearest each p-th root.
    Entries must lie in [0, vmax]; p defaults to maxconv_p(D, vmax)."""
    x = np.asarray(x, dtype=np.int64).reshape(-1)
    y = np.asarray(y, dtype=np.int64).reshape(-1)
    D = dim_of(x)
    if x.min(initial=0) < 0 or y.min(initial=0) < 0 or max(x.max(), y.max()) > vmax:
        raise ValueError("entries outside [0, vmax]")
    if p is None:
        p = maxconv_p(D, vmax)
    return np.array([nearest_root(sk, p) for sk in _pow_sums(x, y, p)], dtype=np.int64)


def maxconv_limb_plan(D: int, vmax: int):
    """(p, b, e, L) for the int64 evaluation of the sums of p-th powers: each
    vmax^p-sized value is written as L limbs of b bits, and the limb index a
    (0 <= a < 2^e, L <= 2^e) becomes e extra hypercube axes.  Every entry of
    the (D + e)-axis int64 convolution, and every sum of its limb-value
    slices, is below 2^(D + e + 2b) <= 2^63, so Z/2^64 holds it exactly."""
    p = maxconv_p(D, vmax)
    bits = max(1, (vmax ** p).bit_length()) if vmax > 1 else 1
    e = 0
    while True:
        b = min(31, (63 - D - e) // 2)
        if b < 1:
            raise ValueError("no limb width keeps the sums below 2^63")
        L = -(-bits // b)
        if L <= (1 << e):
            return p, b, e, L
        e += 1


def maxconv_limb_sums(x, y, vmax: int):
    """(w, b, p): w[c, k] = sum over limb pairs a + a' = c of the convolution of
    limb a of x^p with limb a' of y^p, so that sum_c w[c, k] 2^(c b) is the
    sum of p-th powers s[k].  Computed with one int64 recurrence of D + e
    axes (oracle.convolve) whose top e axes carry the limb index bits: the
    carry-free digit string of a + a' on those axes, read in base 2, is the
    value c = a + a'."""
    x = np.asarray(x, dtype=np.int64).reshape(-1)
    y = np.asarray(y, dtype=np.int64).reshape(-1)
    D = dim_of(x)
    p, b, e, L = maxconv_limb_plan(D, vmax)
    n = 1 << D
    mask = (1 << b) - 1

    def limbs(v):
        U = np.zeros(((1 << e), n), dtype=np.int64)
        for i, val in enumerate(v.tolist()):
            w = int(val) ** p
            for a in range(L):
                U[a, i] = (w >> (a * b)) & mask
        return U.reshape(-1)

    W = convolve(limbs(x), limbs(y)).reshape(3 ** e, 3 ** D)
    w = np.zeros(((2 << e) - 1, 3 ** D), dtype=np.int64)
    for d in range(3 ** e):
        c, q = 0, d
        for j in range(e):           # digit j of d (least significant first) weighs 2^j
            c += (q % 3) << j
            q //= 3
        w[c] += W[d]
    return w, b, p
