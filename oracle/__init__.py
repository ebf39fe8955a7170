"""CPU oracle for hypercube convolution (arXiv 1608.00206) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package.  The product (``paper_1608_00206_gb300``)
never does: it has no CPU fallback.

Everything numeric lives in ``hc_oracle.cpp`` (plain C++, built with
``-O2 -ffp-contract=off``); this module only builds it, loads it with ctypes
and marshals numpy arrays.  Functions and the passages they follow:

* :func:`brute_force` -- Algorithm 1 (naive convolution), hypercube case.
* :func:`points`      -- the definition (Introduction) evaluated at chosen outputs.
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

Dtype handling: int64 arrays are computed in Z/2^64 (two's complement wrap),
float64 and float32 in their own precision.
"""
from __future__ import annotations

import ctypes
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
