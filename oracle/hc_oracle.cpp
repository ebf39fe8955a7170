// Oracle for the exact convolution of two D-dimensional hypercubes
// (Serang, "An exact, cache-localized algorithm for the sub-quadratic
// convolution of hypercubes", arXiv 1608.00206).
//
// TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously correct
// CPU statement of what the GPU library computes.  It shares no code, header,
// table or helper with the CUDA path.  Only the test suite, the smoke check
// and the benchmark's CPU-baseline leg may load it.
//
// Conventions (Introduction and Methods of the paper):
//   x, y : hypercubes over {0,1}^D, row-major, flat length 2^D.  Axis 1 is the
//          slowest axis: x[i_1] is the first or second half of the flat array.
//   z    : the convolution over {0,1,2}^D, row-major, flat length 3^D.
//          (x*y)[k] = sum over i+j=k of x[i]*y[j]   (definition, Introduction).
// The int64 dtype computes in the ring Z/2^64 (uint64 arithmetic, wrap on
// overflow); the paper says nothing about overflow and this is the reading
// under which every order of operations gives the same bits.
//
// Build: g++ -O2 -ffp-contract=off -fopenmp -shared -fPIC (never -Ofast):
// floating-point results must follow the source's rounding order exactly.
//
// Parity pins for every function here live in tests/test_oracle_*.py.

#include <cstdint>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <vector>
#include <omp.h>

namespace {

typedef uint64_t u64;

size_t pow3(int d) {
  size_t r = 1;
  for (int i = 0; i < d; ++i) r *= 3;
  return r;
}

// t(i): the bits of i (axis 1 = most significant of D bits) read as base-3
// digits (axis 1 = most significant digit).  Because every digit of
// t(i)+t(j) is bit_d(i)+bit_d(j) <= 2, t(i)+t(j) is the flat index of the
// multi-index sum i+j with no carries (Discussion: the carry-free example).
size_t tmap(size_t i, int D) {
  size_t r = 0;
  for (int d = D - 1; d >= 0; --d) r = r * 3 + ((i >> d) & 1u);
  return r;
}

// ---------------------------------------------------------------------------
// Algorithm 1 (naive multidimensional convolution), specialised to hypercubes:
// every pair (i, j) adds x[i]*y[j] into z[i+j].  O(4^D).
template <class T>
void brute(const T* x, const T* y, T* z, int D) {
  const size_t n2 = (size_t)1 << D, n3 = pow3(D);
  for (size_t k = 0; k < n3; ++k) z[k] = T(0);
  std::vector<size_t> t(n2);
  for (size_t i = 0; i < n2; ++i) t[i] = tmap(i, D);
  for (size_t i = 0; i < n2; ++i)
    for (size_t j = 0; j < n2; ++j) z[t[i] + t[j]] += x[i] * y[j];
}

// Carry-free 1D convolution (Discussion): vectors of any length N >= 1 and
// D = number of bits needed for N - 1.  The bits of i and j are added
// position by position with no carry; the D resulting digits (each 0, 1 or 2,
// most significant first) are the base-3 output index.  Straight from that
// definition, O(N^2); entries no pair reaches stay zero.
template <class T>
void carryfree(const T* x, const T* y, T* z, size_t N, int D) {
  const size_t n3 = pow3(D);
  for (size_t k = 0; k < n3; ++k) z[k] = T(0);
  for (size_t i = 0; i < N; ++i)
    for (size_t j = 0; j < N; ++j) {
      size_t k = 0;
      for (int d = D - 1; d >= 0; --d) k = k * 3 + ((i >> d) & 1u) + ((j >> d) & 1u);
      z[k] += x[i] * y[j];
    }
}

// One output of the definition: z[k] = sum of x[i]*y[j] over the 2^{#ones(k)}
// pairs with i+j = k.  Per axis, digit 0 forces (0,0), digit 2 forces (1,1),
// digit 1 allows (0,1) and (1,0).  Pairs are visited in increasing i.
template <class T>
T point(const T* x, const T* y, int D, size_t k) {
  int dig[64];
  size_t kk = k;
  for (int d = D - 1; d >= 0; --d) { dig[d] = (int)(kk % 3); kk /= 3; }
  // dig[0] is axis 1 (most significant).
  int ones[64], m = 0;
  size_t ibase = 0;
  for (int d = 0; d < D; ++d) {
    size_t bit = (size_t)1 << (D - 1 - d);
    if (dig[d] == 2) ibase |= bit;
    if (dig[d] == 1) ones[m++] = d;
  }
  size_t jbase = ibase;
  T acc = T(0);
  for (size_t s = 0; s < ((size_t)1 << m); ++s) {
    size_t i = ibase, j = jbase;
    for (int q = 0; q < m; ++q) {
      size_t bit = (size_t)1 << (D - 1 - ones[q]);
      if ((s >> (m - 1 - q)) & 1u) i |= bit; else j |= bit;
    }
    acc += x[i] * y[j];
  }
  return acc;
}

// Max-convolution (Discussion: the (x, max) semiring that p-norm rings
// approximate): every pair (i, j) offers x[i]*y[j] to z[i+j] and z keeps the
// largest offer.  O(4^D), straight from the definition; every output index
// is reached (digit 0 by (0,0), 2 by (1,1), 1 by (0,1) and (1,0)), so no
// output keeps its starting value.  int64 products (the caller keeps
// |x|, |y| < 2^31).
void maxconv_brute(const int64_t* x, const int64_t* y, int64_t* z, int D) {
  const size_t n2 = (size_t)1 << D, n3 = pow3(D);
  for (size_t k = 0; k < n3; ++k) z[k] = INT64_MIN;
  std::vector<size_t> t(n2);
  for (size_t i = 0; i < n2; ++i) t[i] = tmap(i, D);
  for (size_t i = 0; i < n2; ++i)
    for (size_t j = 0; j < n2; ++j) {
      const int64_t v = x[i] * y[j];
      if (v > z[t[i] + t[j]]) z[t[i] + t[j]] = v;
    }
}

// One output of the max-convolution: the largest x[i]*y[j] over the
// 2^{#ones(k)} pairs with i+j = k (digit 0 forces (0,0), 2 forces (1,1), 1
// allows (0,1) and (1,0)), straight from the definition.
int64_t maxconv_point(const int64_t* x, const int64_t* y, int D, size_t k) {
  int dig[64];
  size_t kk = k;
  for (int d = D - 1; d >= 0; --d) { dig[d] = (int)(kk % 3); kk /= 3; }
  int ones[64], m = 0;
  size_t ibase = 0;
  for (int d = 0; d < D; ++d) {
    const size_t bit = (size_t)1 << (D - 1 - d);
    if (dig[d] == 2) ibase |= bit;
    if (dig[d] == 1) ones[m++] = d;
  }
  int64_t best = INT64_MIN;
  for (size_t s = 0; s < ((size_t)1 << m); ++s) {
    size_t i = ibase, j = ibase;
    for (int q = 0; q < m; ++q) {
      const size_t bit = (size_t)1 << (D - 1 - ones[q]);
      if ((s >> (m - 1 - q)) & 1u) i |= bit; else j |= bit;
    }
    const int64_t v = x[i] * y[j];
    if (v > best) best = v;
  }
  return best;
}

// One output of the Methods recurrence with the recurrence's own rounding.
// On an axis whose digit of k is 0 (or 2) the recurrence only descends into
// the first (second) halves of x and y, so z[k] depends on the 2^m entries
// whose bits agree with k on those axes (m = number of digits 1); gathered
// in axis order they form an m-axis problem whose output digits are all 1,
// and the recurrence on it performs, element by element, the same
// additions, products and subtractions as the full recurrence does for
// z[k].  rec_ones is that recurrence (z1 = (t - z0) - z2 on every axis).
template <class T>
T rec_ones(const T* x, const T* y, int m, T* scratch) {
  if (m == 0) return x[0] * y[0];
  const size_t h = (size_t)1 << (m - 1);
  T* xs = scratch;
  T* ys = scratch + h;
  for (size_t i = 0; i < h; ++i) {
    xs[i] = x[i] + x[h + i];
    ys[i] = y[i] + y[h + i];
  }
  const T t = rec_ones(xs, ys, m - 1, scratch + 2 * h);
  const T z0 = rec_ones(x, y, m - 1, scratch + 2 * h);
  const T z2 = rec_ones(x + h, y + h, m - 1, scratch + 2 * h);
  return (t - z0) - z2;
}

template <class T>
T point_rec(const T* x, const T* y, int D, size_t k, std::vector<T>& buf) {
  int dig[64];
  size_t kk = k;
  for (int d = D - 1; d >= 0; --d) { dig[d] = (int)(kk % 3); kk /= 3; }
  int ones[64], m = 0;
  size_t base = 0;
  for (int d = 0; d < D; ++d) {
    const size_t bit = (size_t)1 << (D - 1 - d);
    if (dig[d] == 2) base |= bit;
    if (dig[d] == 1) ones[m++] = d;
  }
  const size_t n = (size_t)1 << m;
  buf.assign(2 * n + 2 * n + 4, T(0));
  T* xc = buf.data();
  T* yc = xc + n;
  for (size_t s = 0; s < n; ++s) {  // s's bits, most significant first, on the digit-1 axes
    size_t i = base;
    for (int q = 0; q < m; ++q)
      if ((s >> (m - 1 - q)) & 1u) i |= (size_t)1 << (D - 1 - ones[q]);
    xc[s] = x[i];
    yc[s] = y[i];
  }
  return rec_ones(xc, yc, m, yc + n);
}

// ---------------------------------------------------------------------------
// The Methods recurrence (3-way split), on fresh temporaries:
//   z[0] = x[0]*y[0];  z[2] = x[1]*y[1];
//   t    = (x[0]+x[1]) * (y[0]+y[1]);
//   z[1] = (t - z[0]) - z[2];
// with base case D = 0: z = x*y (the product of two numbers).  With
// `direct` set, D = 1 is the base case instead, computed from the three
// products of the 4-way form (z[1] = x[1]*y[0] + x[0]*y[1]).
// The paper's in-place listing mutates x and y inside the first recursive
// call, which the later x[0]+x[1] then reads; here the sums go to scratch and
// x, y stay untouched.  `scratch` holds at least 2^(D+1) elements.
template <class T>
void rec(const T* x, const T* y, T* z, int D, bool direct, T* scratch) {
  if (D == 0) {
    z[0] = x[0] * y[0];
    return;
  }
  if (D == 1 && direct) {
    z[0] = x[0] * y[0];
    z[1] = x[1] * y[0] + x[0] * y[1];
    z[2] = x[1] * y[1];
    return;
  }
  const size_t h = (size_t)1 << (D - 1);
  const size_t n = pow3(D - 1);
  rec(x, y, z, D - 1, direct, scratch);                  // z[0] = x[0]*y[0]
  rec(x + h, y + h, z + 2 * n, D - 1, direct, scratch);  // z[2] = x[1]*y[1]
  T* xs = scratch;
  T* ys = scratch + h;
  for (size_t k = 0; k < h; ++k) {
    xs[k] = x[k] + x[h + k];
    ys[k] = y[k] + y[h + k];
  }
  rec(xs, ys, z + n, D - 1, direct, scratch + 2 * h);    // t
  for (size_t k = 0; k < n; ++k) z[n + k] = (z[n + k] - z[k]) - z[2 * n + k];
}

// The paper's in-place schedule done correctly (Methods; the memory pairing
// that Algorithm 2 is built on): z[0] and z[2] first, then the sums formed
// in place in the first halves of x and y (no fresh temporaries), the middle
// sub-problem on them, and the first halves put back before returning, so
// every call leaves its inputs as it found them (the listing forgets this,
// and its later sums read transformed data).  Putting back:
//   save = true : copy the first halves aside before summing (2^(D-1) each
//                 on the current path: O(2^D) in all) and copy them back --
//                 exact for every type, the same operations as rec();
//   save = false: subtract the second half again, x[k] = (x[k]+x[h+k]) -
//                 x[h+k] -- no scratch, exact in Z/2^64 only (in floating
//                 point the restored first halves are off by the rounding of
//                 the sum, which the paper's exactness condition (a+b)-a = b
//                 rules out).
// The output is formed in z exactly as in rec(); x and y are modified
// during the call.
template <class T>
void rec_inplace(T* x, T* y, T* z, int D, bool save, T* saved) {
  if (D == 0) {
    z[0] = x[0] * y[0];
    return;
  }
  const size_t h = (size_t)1 << (D - 1);
  const size_t n = pow3(D - 1);
  rec_inplace(x, y, z, D - 1, save, saved);                  // z[0] = x[0]*y[0]
  rec_inplace(x + h, y + h, z + 2 * n, D - 1, save, saved);  // z[2] = x[1]*y[1]
  if (save) {
    memcpy(saved, x, h * sizeof(T));
    memcpy(saved + h, y, h * sizeof(T));
  }
  for (size_t k = 0; k < h; ++k) {
    x[k] = x[k] + x[h + k];
    y[k] = y[k] + y[h + k];
  }
  rec_inplace(x, y, z + n, D - 1, save, saved + 2 * h);      // t
  if (save) {
    memcpy(x, saved, h * sizeof(T));
    memcpy(y, saved + h, h * sizeof(T));
  } else {
    for (size_t k = 0; k < h; ++k) {
      x[k] = x[k] - x[h + k];
      y[k] = y[k] - y[h + k];
    }
  }
  for (size_t k = 0; k < n; ++k) z[n + k] = (z[n + k] - z[k]) - z[2 * n + k];
}

// Same recurrence with the three sub-problems of the top `par_levels` levels
// run as OpenMP tasks.  Every element sees the same operations in the same
// order as rec(), so the result is bitwise identical.
template <class T>
void rec_par(const T* x, const T* y, T* z, int D, bool direct, int par_levels) {
  if (par_levels <= 0 || D <= 2) {
    std::vector<T> scratch(((size_t)2 << D) + 2);
    rec(x, y, z, D, direct, scratch.data());
    return;
  }
  const size_t h = (size_t)1 << (D - 1);
  const size_t n = pow3(D - 1);
  std::vector<T> xs(h), ys(h);
  for (size_t k = 0; k < h; ++k) {
    xs[k] = x[k] + x[h + k];
    ys[k] = y[k] + y[h + k];
  }
#pragma omp task shared(x, y, z)
  rec_par(x, y, z, D - 1, direct, par_levels - 1);
#pragma omp task shared(x, y, z)
  rec_par(x + h, y + h, z + 2 * n, D - 1, direct, par_levels - 1);
#pragma omp task shared(xs, ys, z)
  rec_par(xs.data(), ys.data(), z + n, D - 1, direct, par_levels - 1);
#pragma omp taskwait
  for (size_t k = 0; k < n; ++k) z[n + k] = (z[n + k] - z[k]) - z[2 * n + k];
}

template <class T>
void rec_top(const T* x, const T* y, T* z, int D, bool direct, int threads) {
  if (threads <= 1) {
    std::vector<T> scratch(((size_t)2 << D) + 2);
    rec(x, y, z, D, direct, scratch.data());
    return;
  }
  int levels = 0;
  for (size_t w = 1; w < (size_t)threads * 3 && levels < D; w *= 3) ++levels;
#pragma omp parallel num_threads(threads)
#pragma omp single
  rec_par(x, y, z, D, direct, levels);
}

// ---------------------------------------------------------------------------
// Mixed-precision form: evaluation (x[0]+x[1]) and the product in binary32;
// the cancelling interpolation (t - z[0]) - z[2] in float-float (a pair of
// binary32 values carried through error-free two-sum), rounded to binary32
// once at the end.  The float-float subtraction is
//   (s, e) = two_sum(a.h, -b.h);  e = e + (a.l - b.l);  (h, l) = quick_two_sum(s, e)
// with two_sum(a, b): s = a + b; v = s - a; e = (a - (s - v)) + (b - v)   (Knuth)
// and quick_two_sum(a, b): s = a + b; e = b - (s - a)                      (Dekker).
struct ff {
  float h, l;
};

inline ff ff_sub(ff a, ff b) {
  float s = a.h - b.h;
  float v = s - a.h;
  float e = (a.h - (s - v)) + (-b.h - v);
  e = e + (a.l - b.l);
  float h = s + e;
  float l = e - (h - s);
  return ff{h, l};
}

void rec_mixed(const float* x, const float* y, ff* z, int D, float* scratch) {
  if (D == 0) {
    z[0] = ff{x[0] * y[0], 0.0f};
    return;
  }
  const size_t h = (size_t)1 << (D - 1);
  const size_t n = pow3(D - 1);
  rec_mixed(x, y, z, D - 1, scratch);
  rec_mixed(x + h, y + h, z + 2 * n, D - 1, scratch);
  float* xs = scratch;
  float* ys = scratch + h;
  for (size_t k = 0; k < h; ++k) {
    xs[k] = x[k] + x[h + k];
    ys[k] = y[k] + y[h + k];
  }
  rec_mixed(xs, ys, z + n, D - 1, scratch + 2 * h);
  for (size_t k = 0; k < n; ++k) z[n + k] = ff_sub(ff_sub(z[n + k], z[k]), z[2 * n + k]);
}

// ---------------------------------------------------------------------------
// Hybrid form: the 4-way direct form on the top mt axes (Methods: z[1] =
// x[0]*y[1] + x[1]*y[0] needs no interpolation), the Karatsuba recurrence on
// the other n = D - mt axes, written as the Kronecker form the recurrence
// unrolls to.  For each top digit string a (axis 1 first):
//   P_a = sum over the pairs (b, c) of top bit strings with b + c = a of
//         (E^{(x)n} x_b) (.) (E^{(x)n} y_c),
//   z_a = I^{(x)n} P_a,
// where x_b is the sub-cube of x whose top bits are b.  Digit 0 takes bits
// (0, 0), digit 2 takes (1, 1), digit 1 takes (0, 1) or (1, 0); the pairs are
// summed in the order of increasing x index (the first pair of each digit-1
// axis gives x bit 0).  E is applied axis by axis outermost first and I
// innermost first, the recurrence's own per-element order, so mt = 0 is the
// recurrence bit for bit and mt = D is Algorithm 1's summation bit for bit.

// E^{(x)n} of one 2^n sub-cube into 3^n values, outermost axis first.
template <class T>
void kron_eval(const T* x, T* out, int n, T* scratch) {
  if (n == 0) {
    out[0] = x[0];
    return;
  }
  const size_t h = (size_t)1 << (n - 1), m = pow3(n - 1);
  T* s = scratch;
  for (size_t k = 0; k < h; ++k) s[k] = x[k] + x[h + k];
  kron_eval(x, out, n - 1, scratch + h);
  kron_eval(s, out + m, n - 1, scratch + h);
  kron_eval(x + h, out + 2 * m, n - 1, scratch + h);
}

// I^{(x)n} in place on 3^n values, innermost axis first.
template <class T>
void kron_interp(T* p, int n) {
  if (n == 0) return;
  const size_t m = pow3(n - 1);
  kron_interp(p, n - 1);
  kron_interp(p + m, n - 1);
  kron_interp(p + 2 * m, n - 1);
  for (size_t k = 0; k < m; ++k) p[m + k] = (p[m + k] - p[k]) - p[2 * m + k];
}

template <class T>
void direct_top(const T* x, const T* y, T* z, int D, int mt) {
  const int n = D - mt;
  const size_t n2 = (size_t)1 << n, n3 = pow3(n);
  std::vector<T> xe(n3), ye(n3), acc(n3), scratch(2 * n2 + 2);
  for (size_t a = 0; a < pow3(mt); ++a) {
    int dig[64];
    size_t aa = a;
    for (int d = mt - 1; d >= 0; --d) {
      dig[d] = (int)(aa % 3);
      aa /= 3;
    }
    int ones[64], m1 = 0;
    size_t base = 0;  // top bits fixed by digits 2
    for (int d = 0; d < mt; ++d) {
      const size_t bit = (size_t)1 << (mt - 1 - d);
      if (dig[d] == 2) base |= bit;
      if (dig[d] == 1) ones[m1++] = d;
    }
    for (size_t sidx = 0; sidx < ((size_t)1 << m1); ++sidx) {
      size_t bx = base, by = base;
      for (int q = 0; q < m1; ++q) {
        const size_t bit = (size_t)1 << (mt - 1 - ones[q]);
        if ((sidx >> (m1 - 1 - q)) & 1u) bx |= bit; else by |= bit;
      }
      kron_eval(x + bx * n2, xe.data(), n, scratch.data());
      kron_eval(y + by * n2, ye.data(), n, scratch.data());
      for (size_t j = 0; j < n3; ++j) {
        const T p = xe[j] * ye[j];
        acc[j] = sidx == 0 ? p : acc[j] + p;
      }
    }
    kron_interp(acc.data(), n);
    for (size_t j = 0; j < n3; ++j) z[a * n3 + j] = acc[j];
  }
}

// ---------------------------------------------------------------------------
// Float-float form: every value of the recurrence -- the inputs' sums
// (evaluation), the products and the interpolation -- is a float-float pair
// (h, l) of binary32 values, rounded to binary32 once at the end.  The
// operations, each from its published error-free building blocks:
//   add(a, b): (s, e) = two_sum(a.h, b.h);  e = e + (a.l + b.l);
//              (h, l) = quick_two_sum(s, e)
//   sub(a, b): as add with b negated (ff_sub above)
//   mul(a, b): p = a.h * b.h;  e = fma(a.h, b.h, -p)   (the exact error of the
//              binary32 product: TwoProduct with a fused multiply-add, Ogita,
//              Rump and Oishi 2005);  e = e + (a.h * b.l + a.l * b.h);
//              (h, l) = quick_two_sum(p, e)
// Inputs enter as (x, 0).  Same recursion and operation order as rec().
inline ff ff_add(ff a, ff b) {
  float s = a.h + b.h;
  float v = s - a.h;
  float e = (a.h - (s - v)) + (b.h - v);
  e = e + (a.l + b.l);
  float h = s + e;
  float l = e - (h - s);
  return ff{h, l};
}

inline ff ff_mul(ff a, ff b) {
  float p = a.h * b.h;
  float e = std::fma(a.h, b.h, -p);
  float c = a.h * b.l;
  float d = a.l * b.h;
  e = e + (c + d);
  float h = p + e;
  float l = e - (h - p);
  return ff{h, l};
}

void rec_ff(const ff* x, const ff* y, ff* z, int D, ff* scratch) {
  if (D == 0) {
    z[0] = ff_mul(x[0], y[0]);
    return;
  }
  const size_t h = (size_t)1 << (D - 1);
  const size_t n = pow3(D - 1);
  rec_ff(x, y, z, D - 1, scratch);
  rec_ff(x + h, y + h, z + 2 * n, D - 1, scratch);
  ff* xs = scratch;
  ff* ys = scratch + h;
  for (size_t k = 0; k < h; ++k) {
    xs[k] = ff_add(x[k], x[h + k]);
    ys[k] = ff_add(y[k], y[h + k]);
  }
  rec_ff(xs, ys, z + n, D - 1, scratch + 2 * h);
  for (size_t k = 0; k < n; ++k) z[n + k] = ff_sub(ff_sub(z[n + k], z[k]), z[2 * n + k]);
}

// ---------------------------------------------------------------------------
// Adjoint (differentiation form).  For z = x*y and an upstream gradient g =
// dL/dz, dL/dx[i] = sum_j g[i+j] * y[j] (a correlation).  Splitting axis 1 as
// in the Methods section gives four correlations of dimension D-1,
//   dx[0] = corr(g[0], y[0]) + corr(g[1], y[1])
//   dx[1] = corr(g[1], y[0]) + corr(g[2], y[1]),
// and bilinearity turns them into three:
//   A = corr(g[0] - g[1], y[0]);  B = corr(g[2] - g[1], y[1]);
//   C = corr(g[1], y[0] + y[1]);  dx[0] = A + C;  dx[1] = B + C.
// This is the transpose of the forward recurrence, factor by factor.
// `scratch` holds at least 3^D + 2^(D+1) elements.
template <class T>
void adj(const T* g, const T* w, T* out, int D, T* scratch) {
  if (D == 0) {
    out[0] = g[0] * w[0];
    return;
  }
  const size_t h = (size_t)1 << (D - 1);
  const size_t n = pow3(D - 1);
  T* ga = scratch;          // g[0] - g[1]
  T* gb = scratch + n;      // g[2] - g[1]
  T* ws = scratch + 2 * n;  // w[0] + w[1]
  T* c = ws + h;            // C
  T* rest = c + h;
  for (size_t k = 0; k < n; ++k) {
    ga[k] = g[k] - g[n + k];
    gb[k] = g[2 * n + k] - g[n + k];
  }
  for (size_t k = 0; k < h; ++k) ws[k] = w[k] + w[h + k];
  adj(ga, w, out, D - 1, rest);           // A -> out[0..h)
  adj(gb, w + h, out + h, D - 1, rest);   // B -> out[h..2h)
  adj(g + n, ws, c, D - 1, rest);         // C
  for (size_t k = 0; k < h; ++k) {
    out[k] = out[k] + c[k];
    out[h + k] = out[h + k] + c[k];
  }
}

template <class T>
size_t adj_scratch(int D) {
  return pow3(D) + ((size_t)2 << D) + 8;
}

// Brute-force adjoint straight from the definition: dx[i] = sum_j g[t(i)+t(j)] y[j],
// dy[j] = sum_i g[t(i)+t(j)] x[i].  O(4^D).
template <class T>
void adj_brute(const T* g, const T* x, const T* y, T* dx, T* dy, int D) {
  const size_t n2 = (size_t)1 << D;
  std::vector<size_t> t(n2);
  for (size_t i = 0; i < n2; ++i) t[i] = tmap(i, D);
  for (size_t i = 0; i < n2; ++i) {
    T acc = T(0);
    for (size_t j = 0; j < n2; ++j) acc += g[t[i] + t[j]] * y[j];
    dx[i] = acc;
  }
  for (size_t j = 0; j < n2; ++j) {
    T acc = T(0);
    for (size_t i = 0; i < n2; ++i) acc += g[t[i] + t[j]] * x[i];
    dy[j] = acc;
  }
}

// ---------------------------------------------------------------------------
// Companion magnitude for the floating-point forward-error bound: the same
// recurrence on |x|, |y| with every subtraction turned into an addition,
//   zabs[1] = t + zabs[0] + zabs[2].
// Each output of the recurrence is reached through at most D additions per
// operand, one product and 2D subtractions, so in precision u
// |z_computed - z_exact| <= gamma_{3D+1} * zabs with gamma_n = n u / (1 - n u).
void zabs_rec(const double* x, const double* y, double* z, int D, double* scratch) {
  if (D == 0) {
    z[0] = x[0] * y[0];
    return;
  }
  const size_t h = (size_t)1 << (D - 1);
  const size_t n = pow3(D - 1);
  zabs_rec(x, y, z, D - 1, scratch);
  zabs_rec(x + h, y + h, z + 2 * n, D - 1, scratch);
  double* xs = scratch;
  double* ys = scratch + h;
  for (size_t k = 0; k < h; ++k) {
    xs[k] = x[k] + x[h + k];
    ys[k] = y[k] + y[h + k];
  }
  zabs_rec(xs, ys, z + n, D - 1, scratch + 2 * h);
  for (size_t k = 0; k < n; ++k) z[n + k] = (z[n + k] + z[k]) + z[2 * n + k];
}

}  // namespace

// ---------------------------------------------------------------------------
// C entry points.  dtype codes: 0 = int64 (computed as uint64, wraps),
// 1 = float64, 2 = float32.  All buffers are host memory owned by the caller.

extern "C" {

int oracle_brute(const void* x, const void* y, void* z, int D, int dtype) {
  switch (dtype) {
    case 0: brute((const u64*)x, (const u64*)y, (u64*)z, D); return 0;
    case 1: brute((const double*)x, (const double*)y, (double*)z, D); return 0;
    case 2: brute((const float*)x, (const float*)y, (float*)z, D); return 0;
  }
  return 1;
}

int oracle_carryfree(const void* x, const void* y, void* z, size_t N, int D, int dtype) {
  switch (dtype) {
    case 0: carryfree((const u64*)x, (const u64*)y, (u64*)z, N, D); return 0;
    case 1: carryfree((const double*)x, (const double*)y, (double*)z, N, D); return 0;
    case 2: carryfree((const float*)x, (const float*)y, (float*)z, N, D); return 0;
  }
  return 1;
}

int oracle_points(const void* x, const void* y, int D, int dtype, const uint64_t* ks,
                  size_t nk, void* out) {
  for (size_t q = 0; q < nk; ++q) {
    switch (dtype) {
      case 0: ((u64*)out)[q] = point((const u64*)x, (const u64*)y, D, ks[q]); break;
      case 1: ((double*)out)[q] = point((const double*)x, (const double*)y, D, ks[q]); break;
      case 2: ((float*)out)[q] = point((const float*)x, (const float*)y, D, ks[q]); break;
      default: return 1;
    }
  }
  return 0;
}

int oracle_recurrence(const void* x, const void* y, void* z, int D, int dtype, int direct,
                      int threads) {
  switch (dtype) {
    case 0: rec_top((const u64*)x, (const u64*)y, (u64*)z, D, direct != 0, threads); return 0;
    case 1: rec_top((const double*)x, (const double*)y, (double*)z, D, direct != 0, threads); return 0;
    case 2: rec_top((const float*)x, (const float*)y, (float*)z, D, direct != 0, threads); return 0;
  }
  return 1;
}

// In-place schedule; x and y are modified during the call and handed back
// (exactly with save != 0, or for int64).
int oracle_recurrence_inplace(void* x, void* y, void* z, int D, int dtype, int save) {
  const size_t es = dtype == 0 || dtype == 1 ? 8 : 4;
  std::vector<unsigned char> saved(save ? es * ((size_t)2 << D) + 16 : 16);
  switch (dtype) {
    case 0: rec_inplace((u64*)x, (u64*)y, (u64*)z, D, save != 0, (u64*)saved.data()); return 0;
    case 1: rec_inplace((double*)x, (double*)y, (double*)z, D, save != 0, (double*)saved.data()); return 0;
    case 2: rec_inplace((float*)x, (float*)y, (float*)z, D, save != 0, (float*)saved.data()); return 0;
  }
  return 1;
}

int oracle_recurrence_mixed(const float* x, const float* y, float* z, int D) {
  std::vector<ff> w(pow3(D));
  std::vector<float> scratch(((size_t)2 << D) + 2);
  rec_mixed(x, y, w.data(), D, scratch.data());
  for (size_t k = 0; k < w.size(); ++k) z[k] = w[k].h + w[k].l;
  return 0;
}

int oracle_direct_top(const void* x, const void* y, void* z, int D, int mt, int dtype) {
  if (mt < 0 || mt > D) return 1;
  switch (dtype) {
    case 0: direct_top((const u64*)x, (const u64*)y, (u64*)z, D, mt); return 0;
    case 1: direct_top((const double*)x, (const double*)y, (double*)z, D, mt); return 0;
    case 2: direct_top((const float*)x, (const float*)y, (float*)z, D, mt); return 0;
  }
  return 1;
}

int oracle_recurrence_ff(const float* x, const float* y, float* z, int D) {
  const size_t n2 = (size_t)1 << D;
  std::vector<ff> xf(n2), yf(n2), w(pow3(D));
  for (size_t i = 0; i < n2; ++i) {
    xf[i] = ff{x[i], 0.0f};
    yf[i] = ff{y[i], 0.0f};
  }
  std::vector<ff> scratch(((size_t)2 << D) + 2);
  rec_ff(xf.data(), yf.data(), w.data(), D, scratch.data());
  for (size_t k = 0; k < w.size(); ++k) z[k] = w[k].h + w[k].l;
  return 0;
}

int oracle_adjoint(const void* g, const void* x, const void* y, void* dx, void* dy, int D,
                   int dtype) {
  switch (dtype) {
    case 0: {
      std::vector<u64> s(adj_scratch<u64>(D));
      if (dx) adj((const u64*)g, (const u64*)y, (u64*)dx, D, s.data());
      if (dy) adj((const u64*)g, (const u64*)x, (u64*)dy, D, s.data());
      return 0;
    }
    case 1: {
      std::vector<double> s(adj_scratch<double>(D));
      if (dx) adj((const double*)g, (const double*)y, (double*)dx, D, s.data());
      if (dy) adj((const double*)g, (const double*)x, (double*)dy, D, s.data());
      return 0;
    }
    case 2: {
      std::vector<float> s(adj_scratch<float>(D));
      if (dx) adj((const float*)g, (const float*)y, (float*)dx, D, s.data());
      if (dy) adj((const float*)g, (const float*)x, (float*)dy, D, s.data());
      return 0;
    }
  }
  return 1;
}

int oracle_adjoint_brute(const void* g, const void* x, const void* y, void* dx, void* dy, int D,
                         int dtype) {
  switch (dtype) {
    case 0: adj_brute((const u64*)g, (const u64*)x, (const u64*)y, (u64*)dx, (u64*)dy, D); return 0;
    case 1: adj_brute((const double*)g, (const double*)x, (const double*)y, (double*)dx, (double*)dy, D); return 0;
    case 2: adj_brute((const float*)g, (const float*)x, (const float*)y, (float*)dx, (float*)dy, D); return 0;
  }
  return 1;
}

int oracle_zabs(const double* absx, const double* absy, double* z, int D) {
  std::vector<double> scratch(((size_t)2 << D) + 2);
  zabs_rec(absx, absy, z, D, scratch.data());
  return 0;
}

int oracle_maxconv_brute(const int64_t* x, const int64_t* y, int64_t* z, int D) {
  if (D < 0 || D > 20) return 1;
  maxconv_brute(x, y, z, D);
  return 0;
}

int oracle_maxconv_points(const int64_t* x, const int64_t* y, int D, const uint64_t* ks,
                          size_t nk, int64_t* out) {
  if (D < 0 || D > 30) return 1;
  for (size_t q = 0; q < nk; ++q) out[q] = maxconv_point(x, y, D, ks[q]);
  return 0;
}

int oracle_points_rec(const void* x, const void* y, int D, int dtype, const uint64_t* ks,
                      size_t nk, void* out) {
  if (D < 0 || D > 40) return 1;
  int bad = 0;
#pragma omp parallel
  {
    std::vector<u64> bu;
    std::vector<double> bd;
    std::vector<float> bf;
#pragma omp for schedule(dynamic, 64)
    for (long long q = 0; q < (long long)nk; ++q) {
      switch (dtype) {
        case 0: ((u64*)out)[q] = point_rec((const u64*)x, (const u64*)y, D, ks[q], bu); break;
        case 1: ((double*)out)[q] = point_rec((const double*)x, (const double*)y, D, ks[q], bd); break;
        case 2: ((float*)out)[q] = point_rec((const float*)x, (const float*)y, D, ks[q], bf); break;
        default: bad = 1;
      }
    }
  }
  return bad;
}

int oracle_max_threads(void) { return omp_get_max_threads(); }

}  // extern "C"
