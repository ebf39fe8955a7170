// Shared device-side building blocks of libhc (hypercube convolution,
// arXiv 1608.00206) for sm_103a.
//
// The Methods-section recurrence is a Kronecker product of per-axis maps:
//   evaluation    E: (a0, a1)     -> (a0, a0 + a1, a1)          (x[0], x[0]+x[1], x[1])
//   product          P = (E^{xD} x) (.) (E^{xD} y)              (base case D = 0)
//   interpolation I: (p0, p1, p2) -> (p0, (p1 - p0) - p2, p2)   (z[1] = t - z[0] - z[2])
// The recursion evaluates axis 1 first and interpolates axis D first; every
// kernel here keeps that per-element order so that floating-point results are
// bitwise those of the sequential recurrence.  All floating-point arithmetic
// goes through explicit round-to-nearest intrinsics, so no multiply-add is
// ever contracted into an FMA.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hc.h"

namespace hc {

typedef unsigned long long u64;

__host__ __device__ constexpr int p3(int k) { return k <= 0 ? 1 : 3 * p3(k - 1); }
__host__ __device__ constexpr int p2(int k) { return 1 << k; }

__host__ __device__ inline long long pow3_dev(int k) {
  long long r = 1;
  for (int i = 0; i < k; ++i) r *= 3;
  return r;
}

// 3^k for small k (k <= 19), in 32-bit arithmetic.
__host__ __device__ inline int pow3i(int k) {
  int r = 1;
  for (int i = 0; i < k; ++i) r *= 3;
  return r;
}

inline size_t pow3z(int k) {
  size_t r = 1;
  for (int i = 0; i < k; ++i) r *= 3;
  return r;
}

// Columns per column tile in the persistent ticket engine (host and device).
constexpr int kPersistCols = 8;

// A float-float value h + l (|l| <= ulp(h)/2 after renormalisation).
struct __align__(8) ffv {
  float h, l;
};

// a - b in float-float: Knuth's two-sum on the high parts, the low parts added
// to the error, then Dekker's quick-two-sum renormalisation.
__device__ __forceinline__ ffv ff_sub(ffv a, ffv b) {
  float s = __fsub_rn(a.h, b.h);
  float v = __fsub_rn(s, a.h);
  float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, v)), __fsub_rn(-b.h, v));
  e = __fadd_rn(e, __fsub_rn(a.l, b.l));
  float h = __fadd_rn(s, e);
  float l = __fsub_rn(e, __fsub_rn(h, s));
  return ffv{h, l};
}

// a + b in float-float: Knuth's two-sum on the high parts, the low parts
// added to the error, then Dekker's quick-two-sum (ff_sub with b negated).
__device__ __forceinline__ ffv ff_add(ffv a, ffv b) {
  float s = __fadd_rn(a.h, b.h);
  float v = __fsub_rn(s, a.h);
  float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, v)), __fsub_rn(b.h, v));
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  float h = __fadd_rn(s, e);
  float l = __fsub_rn(e, __fsub_rn(h, s));
  return ffv{h, l};
}

// a * b in float-float: the binary32 product of the high parts and its exact
// error from one fused multiply-add (the FMA two-product of Ogita, Rump and
// Oishi), the cross terms added to the error, then quick-two-sum.  The FMA
// here is deliberate: its result is the exact residual a.h * b.h - p.
__device__ __forceinline__ ffv ff_mul(ffv a, ffv b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  const float c = __fmul_rn(a.h, b.l);
  const float d = __fmul_rn(a.l, b.h);
  e = __fadd_rn(e, __fadd_rn(c, d));
  const float h = __fadd_rn(p, e);
  const float l = __fsub_rn(e, __fsub_rn(h, p));
  return ffv{h, l};
}

// Arithmetic modes.  In: element of x and y (and of the evaluated operands);
// W: element of products and interpolation intermediates; Out: element of z.
struct ModeI64 {  // Z/2^64
  typedef u64 In;
  typedef u64 W;
  typedef u64 Out;
  static constexpr hc_dtype kDtype = HC_INT64;
  static __device__ __forceinline__ In add(In a, In b) { return a + b; }
  static __device__ __forceinline__ In sub(In a, In b) { return a - b; }
  static __device__ __forceinline__ W mul(In a, In b) { return a * b; }
  static __device__ __forceinline__ W mulw(W a, In b) { return a * b; }
  static __device__ __forceinline__ W mid(W p0, W p1, W p2) { return (p1 - p0) - p2; }
  static __device__ __forceinline__ W wadd(W a, W b) { return a + b; }
  static __device__ __forceinline__ W wsub(W a, W b) { return a - b; }
  static __device__ __forceinline__ Out out(W w) { return w; }
  static __device__ __forceinline__ W win(Out v) { return v; }
};

struct ModeF64 {
  typedef double In;
  typedef double W;
  typedef double Out;
  static constexpr hc_dtype kDtype = HC_FP64;
  static __device__ __forceinline__ In add(In a, In b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ In sub(In a, In b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ W mul(In a, In b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ W mulw(W a, In b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ W mid(W p0, W p1, W p2) {
    return __dsub_rn(__dsub_rn(p1, p0), p2);
  }
  static __device__ __forceinline__ W wadd(W a, W b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ W wsub(W a, W b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ Out out(W w) { return w; }
  static __device__ __forceinline__ W win(Out v) { return v; }
};

struct ModeF32 {
  typedef float In;
  typedef float W;
  typedef float Out;
  static constexpr hc_dtype kDtype = HC_FP32;
  static __device__ __forceinline__ In add(In a, In b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ In sub(In a, In b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ W mul(In a, In b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ W mulw(W a, In b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ W mid(W p0, W p1, W p2) {
    return __fsub_rn(__fsub_rn(p1, p0), p2);
  }
  static __device__ __forceinline__ W wadd(W a, W b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ W wsub(W a, W b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ Out out(W w) { return w; }
  static __device__ __forceinline__ W win(Out v) { return v; }
};

// binary32 evaluation and products, float-float interpolation.
struct ModeMixed {
  typedef float In;
  typedef ffv W;
  typedef float Out;
  static constexpr hc_dtype kDtype = HC_FP32_MIXED;
  static __device__ __forceinline__ In add(In a, In b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ W mul(In a, In b) { return ffv{__fmul_rn(a, b), 0.0f}; }
  static __device__ __forceinline__ W mid(W p0, W p1, W p2) {
    return ff_sub(ff_sub(p1, p0), p2);
  }
  static __device__ __forceinline__ Out out(W w) { return __fadd_rn(w.h, w.l); }
  static __device__ __forceinline__ W win(Out v) { return ffv{v, 0.0f}; }
};

// Every value in float-float: evaluation (ff_add), products (ff_mul, exact
// high product) and interpolation (ff_sub); binary32 in and out.  The
// binary32 inputs are widened to (x, 0) pairs before the first pass.
struct ModeFF {
  typedef ffv In;
  typedef ffv W;
  typedef float Out;
  static constexpr hc_dtype kDtype = HC_FP32_FF;
  static __device__ __forceinline__ In add(In a, In b) { return ff_add(a, b); }
  static __device__ __forceinline__ W mul(In a, In b) { return ff_mul(a, b); }
  static __device__ __forceinline__ W mid(W p0, W p1, W p2) {
    return ff_sub(ff_sub(p1, p0), p2);
  }
  static __device__ __forceinline__ Out out(W w) { return __fadd_rn(w.h, w.l); }
  static __device__ __forceinline__ W win(Out v) { return ffv{v, 0.0f}; }
};

// ---------------------------------------------------------------------------
// Register pencils.  A pencil holds the values of K consecutive axes for one
// fixed index of all other axes, the first of the K axes most significant.

// Evaluate a 2^K pencil into 3^K values, the first (outermost) axis first.
// After step d the first 3^d * 2^(K-d) entries hold shape [3^d][2^(K-d)].
template <class M, int K, int Dn>
struct EvalSteps {
  template <class T>
  static __device__ __forceinline__ void run(T (&v)[p3(K)]) {
    constexpr int R = p2(K - Dn - 1);
    constexpr int O = p3(Dn);
    T nv[O * 3 * R];
#pragma unroll
    for (int o = 0; o < O; ++o) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        T a0 = v[(o * 2 + 0) * R + r];
        T a1 = v[(o * 2 + 1) * R + r];
        nv[(o * 3 + 0) * R + r] = a0;
        nv[(o * 3 + 1) * R + r] = M::add(a0, a1);
        nv[(o * 3 + 2) * R + r] = a1;
      }
    }
#pragma unroll
    for (int i = 0; i < O * 3 * R; ++i) v[i] = nv[i];
    EvalSteps<M, K, Dn + 1>::run(v);
  }
};
template <class M, int K>
struct EvalSteps<M, K, K> {
  template <class T>
  static __device__ __forceinline__ void run(T (&)[p3(K)]) {}
};

// v[0 .. 2^K) holds the pencil on entry; v holds the 3^K evaluated values on exit.
template <class M, int K, class T>
__device__ __forceinline__ void eval_pencil(T (&v)[p3(K)]) {
  EvalSteps<M, K, 0>::run(v);
}

// Interpolate a 3^K pencil in place, the last (innermost) axis first.
template <class M, int K, class T>
__device__ __forceinline__ void interp_pencil(T (&v)[p3(K)]) {
#pragma unroll
  for (int s = 1; s < p3(K); s *= 3) {
#pragma unroll
    for (int b = 0; b < p3(K); ++b) {
      if ((b / s) % 3 == 0) v[b + s] = M::mid(v[b], v[b + s], v[b + 2 * s]);
    }
  }
}

// Transposed interpolation I^T: (g0, g1, g2) -> (g0 - g1, g1, g2 - g1), the
// first (outermost) axis first.
template <class M, int K, class T>
__device__ __forceinline__ void interp_t_pencil(T (&v)[p3(K)]) {
#pragma unroll
  for (int s = p3(K - 1); s >= 1; s /= 3) {
#pragma unroll
    for (int b = 0; b < p3(K); ++b) {
      if ((b / s) % 3 == 0) {
        T g1 = v[b + s];
        v[b] = M::wsub(v[b], g1);
        v[b + 2 * s] = M::wsub(v[b + 2 * s], g1);
      }
    }
  }
}

// Transposed evaluation E^T: (h0, h1, h2) -> (h0 + h1, h1 + h2) on a 3^K
// pencil, the last (innermost) axis first; v[0 .. 2^K) holds the result.
template <class M, int K, int Dn>
struct EvalTSteps {  // Dn axes (the innermost ones) already reduced to 2
  template <class T>
  static __device__ __forceinline__ void run(T (&v)[p3(K)]) {
    // current shape [3^(K-Dn)][2^Dn]; reduce axis K-Dn (0-based K-Dn-1).
    constexpr int R = p2(Dn);
    constexpr int O = p3(K - Dn - 1);
    T nv[O * 2 * R];
#pragma unroll
    for (int o = 0; o < O; ++o) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        T h0 = v[(o * 3 + 0) * R + r];
        T h1 = v[(o * 3 + 1) * R + r];
        T h2 = v[(o * 3 + 2) * R + r];
        nv[(o * 2 + 0) * R + r] = M::wadd(h0, h1);
        nv[(o * 2 + 1) * R + r] = M::wadd(h1, h2);
      }
    }
#pragma unroll
    for (int i = 0; i < O * 2 * R; ++i) v[i] = nv[i];
    EvalTSteps<M, K, Dn + 1>::run(v);
  }
};
template <class M, int K>
struct EvalTSteps<M, K, K> {
  template <class T>
  static __device__ __forceinline__ void run(T (&)[p3(K)]) {}
};

template <class M, int K, class T>
__device__ __forceinline__ void eval_t_pencil(T (&v)[p3(K)]) {
  EvalTSteps<M, K, 0>::run(v);
}

// ---------------------------------------------------------------------------
// Host helpers shared by the translation units.

struct LaunchCaps {
  int sms;
  size_t smem_optin;
};
LaunchCaps device_caps();  // cached per device

hc_status record_cuda_error(cudaError_t e);  // remembers CUDA's message; HC_OK on success

bool aligned(const void* p, size_t a);
bool overlaps(const void* a, size_t na, const void* b, size_t nb);
size_t elem_size(hc_dtype dt);  // bytes of one x/y/z element (0 for unknown)
size_t in_size(hc_dtype dt);    // bytes of one evaluated-operand element (M::In)
size_t w_size(hc_dtype dt);     // bytes of one intermediate element (M::W)
// Whether the 3^D intermediate is of another type than z (float-float
// intermediates, binary32 output): it then lives in the workspace.
inline bool wide_intermediate(hc_dtype dt) { return dt == HC_FP32_MIXED || dt == HC_FP32_FF; }
size_t align_up(size_t v, size_t a);

// Workspace header: the first 256 bytes of every workspace.
struct WsHeader {
  unsigned int status;   // hc_status recorded by kernels (0 = OK)
  unsigned int where;    // diagnostic: which wait gave up
  unsigned long long pad[31];
};
static_assert(sizeof(WsHeader) == 256, "workspace header is 256 bytes");
constexpr size_t kWsHeader = 256;

}  // namespace hc
