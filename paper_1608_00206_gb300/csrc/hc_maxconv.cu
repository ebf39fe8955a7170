// Max-convolution of bounded non-negative integer hypercubes through a p-norm
// ring (Discussion of arXiv 1608.00206).
//
// For entries in [0, vmax], the maximum m[k] of the products x[i] * y[j]
// over the pairs i + j = k satisfies m <= s^(1/p) <= N^(1/p) m, where
// s[k] = sum over those pairs of (x[i] y[j])^p -- the ordinary hypercube
// convolution of x^p and y^p -- and N = 2^D bounds the number of pairs.  The
// estimate therefore exceeds m by at most M (N^(1/p) - 1), M = vmax^2; with
// p large enough for that to stay below 7/16 (the paper's 1/2, less a
// margin for the floating-point root below), the integer nearest s^(1/p) is m.
//
// s is exact integer arithmetic far beyond 64 bits, computed here with the
// library's int64 convolution alone: write v^p as L limbs of b bits,
// v^p = sum_a limb_a(v) 2^(a b), and put the limb index a (0 <= a < 2^e)
// on e extra axes above the D axes of x.  The convolution of the two
// (D + e)-axis cubes adds limb indices without carries (the embedding of the
// Discussion's carry-free convolution): its slice at limb digit string d
// holds the sum of conv(limb_a(x^p), limb_a'(y^p)) over the pairs whose
// carry-free sum is d, and d read in base 2 is a + a'.  So
//     s[k] = sum over d of W[d, k] 2^(value(d) b),
// every W entry below 2^(D + e + 2b) <= 2^63: exact in Z/2^64.
//
// Steps (one stream, no host synchronisation):
//   1. maxconv_pow_kernel: the table of v^p in limbs for v = 0..vmax.
//   2. maxconv_spread_kernel: the (D + e)-axis limb cubes of x and y from the
//      table; entries outside [0, vmax] are recorded in the status word.
//   3. the int64 convolution of D + e axes (the default schedule).
//   4. maxconv_root_kernel: per output, s in floating point from the 3^e
//      slices (all terms non-negative, so no cancellation), then the nearest
//      integer to s^(1/p).
#include <cmath>

#include "hc_common.cuh"
#include "hc_forward.cuh"
#include "hc_profile.cuh"

namespace hc {

// At most 12 limb axes: the root kernel reads 3^e slices per output.
constexpr int kMaxLimbAxes = 12;

struct MaxPlan {
  int D, p, b, e, L;
  long long vmax;
  bool table;  // powers from a table of vmax + 1 rows (else per element)
  size_t off_tab, off_u, off_v, off_w, off_conv;
  size_t conv_bytes, ws_bytes;
  bool ok;
};

// Smallest p >= 1 with M (2^(D/p) - 1) < 7/16, i.e. D ln 2 < p ln(1 + 7/(16M)).
static long long pick_p(int D, long long vmax) {
  if (vmax <= 0 || D == 0) return 1;
  const long double M = (long double)vmax * (long double)vmax;
  const long double r = (long double)D * logl(2.0L) / log1pl(7.0L / (16.0L * M));
  if (!(r < 1e9L)) return -1;
  return (long long)floorl(r) + 1;
}

static MaxPlan make_max_plan(int D, long long vmax) {
  MaxPlan P{};
  P.ok = false;
  if (D < 0 || D > HC_MAX_D || vmax < 0 || vmax > 0x7fffffffLL) return P;
  const long long p = pick_p(D, vmax);
  if (p < 1 || p > (1 << 24)) return P;
  // the root is taken in double precision for p > 1: results up to 2^38
  if (p > 1 && vmax > (1LL << 19)) return P;
  // bit length of vmax^p, plus one for rounding in the logarithm
  long long bits = 1;
  if (vmax > 1) bits = (long long)floorl((long double)p * log2l((long double)vmax)) + 2;
  int e = 0, b = 0;
  long long L = 0;
  for (;; ++e) {
    if (D + e > HC_MAX_D || e > kMaxLimbAxes) return P;
    b = (63 - D - e) / 2;
    if (b > 31) b = 31;
    if (b < 1) return P;
    L = (bits + b - 1) / b;
    if (L <= (1LL << e)) break;
  }
  P.D = D;
  P.p = (int)p;
  P.b = b;
  P.e = e;
  P.L = (int)L;
  P.vmax = vmax;
  const int De = D + e;
  const size_t E = (size_t)1 << e;
  P.conv_bytes = hc_workspace_size(De, HC_INT64);
  // a table of powers only when it has no more rows than the two operands
  // have elements
  P.table = (unsigned long long)vmax + 1 <= ((unsigned long long)2 << D);
  size_t off = kWsHeader;
  P.off_tab = off;
  if (P.table) off = align_up(off + (size_t)(vmax + 1) * E * 8, 256);
  P.off_u = off;
  off = align_up(off + ((size_t)8 << De), 256);
  P.off_v = off;
  off = align_up(off + ((size_t)8 << De), 256);
  P.off_w = off;
  off = align_up(off + 8 * pow3z(De), 256);
  P.off_conv = off;
  P.ws_bytes = off + P.conv_bytes;
  P.ok = true;
  return P;
}

// Limb a (b bits) of v^p into out[a * stride] for a < E (zero for a >= L):
// the limbs multiplied by v in place p times (schoolbook, carry in 64-bit
// registers: limb < 2^31 and v < 2^31).
__device__ void pow_limbs(unsigned long long v, int p, int b, int L, int E,
                          unsigned long long* out, long long stride) {
  const unsigned long long mask = (1ull << b) - 1;
  for (int a = 0; a < E; ++a) out[(long long)a * stride] = 0;
  out[0] = 1;
  int len = 1;  // limbs in use
  for (int q = 0; q < p; ++q) {
    unsigned long long carry = 0;
    for (int a = 0; a < len; ++a) {
      const unsigned long long t = out[(long long)a * stride] * v + carry;
      out[(long long)a * stride] = t & mask;
      carry = t >> b;
    }
    while (carry && len < L) {
      out[(long long)(len++) * stride] = carry & mask;
      carry >>= b;
    }
    if (v == 0) break;  // 0^p = 0 for p >= 1
  }
}

// tab[v * E + a] = limb a of v^p for v = 0..vmax, one thread per v.
__global__ void __launch_bounds__(128) maxconv_pow_kernel(unsigned long long* __restrict__ tab,
                                                          long long vmax, int p, int b, int L,
                                                          int E) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v > vmax) return;
  pow_limbs((unsigned long long)v, p, b, L, E, tab + v * E, 1);
}

// U[a * n + i] = limb a of x[i]^p (blockIdx.y = 0), V likewise from y
// (blockIdx.y = 1): the limb index a on the top e axes of the (D + e)-axis
// cube.  Consecutive threads take consecutive i: coalesced for every a.
// With a table (tab != NULL, vmax + 1 rows) the limbs are copied from it;
// without one (more possible values than elements) each thread computes its
// element's power in place.  An entry outside [0, vmax] is recorded in
// *status and taken as 0.
__global__ void __launch_bounds__(256) maxconv_spread_kernel(
    const long long* __restrict__ x, const long long* __restrict__ y,
    const unsigned long long* __restrict__ tab, unsigned long long* __restrict__ U,
    unsigned long long* __restrict__ V, long long n, int p, int b, int L, int E, long long vmax,
    unsigned int* __restrict__ status) {
  const long long* src = blockIdx.y ? y : x;
  unsigned long long* dst = blockIdx.y ? V : U;
#pragma unroll 1
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    long long v = src[i];
    if (v < 0 || v > vmax) {
      atomicExch(status, (unsigned int)HC_ERR_ARG);
      v = 0;
    }
    if (tab) {
      const unsigned long long* row = tab + v * E;
#pragma unroll 4
      for (int a = 0; a < E; ++a) dst[(long long)a * n + i] = __ldg(row + a);
    } else {
      pow_limbs((unsigned long long)v, p, b, L, E, dst + i, n);
    }
  }
}

// z[k] = nearest integer to s^(1/p), s = sum over the 3^e limb digit strings d
// of W[d * n3 + k] 2^(value(d) b), value(d) = sum_j digit_j(d) 2^j (digit j
// the j-th least significant base-3 digit).
// p = 1 (D = 0, or vmax = 0): s is the single product itself, summed exactly
// in 64-bit integers.  p > 1: s is accumulated in integers as
// A 2^(top b - G), A unsigned 128-bit, top the largest value(d) with a
// non-zero entry so far: a new top shifts A down, a lower term is shifted
// down into A, dropping bits below A's unit.  With G = 62 - ceil(e log2 3)
// the at most 3^e terms below 2^(63 + G) each keep A below 2^126, and the
// dropped bits (below 1 per term against A >= 2^G) leave s with a relative
// error below 3^e 2^-G <= 2^-23.  The root divides that by p, and the choice
// of p makes M / p <= 7 / (16 D ln 2): the root is off by less than
// 2^-23 0.63 / D.  Then q = 2^(lg / p), lg = log2(A) + top b - G in double
// precision once per output (relative error a few 1e-14, i.e. below 0.01
// for results up to vmax^2 <= 2^38), and the nearest integer: both well
// inside the 1/16 margin the choice of p leaves.
__global__ void __launch_bounds__(256) maxconv_root_kernel(const long long* __restrict__ W,
                                                           long long* __restrict__ z,
                                                           long long n3, int e, int b, int p,
                                                           int G) {
  typedef unsigned __int128 u128;
  // digit strings in groups of 3^eg (the eg lowest digits), loaded together
  const int eg = e < 2 ? e : 2;
  const int gsz = eg == 0 ? 1 : (eg == 1 ? 3 : 9);
  const int eh = e - eg;  // digits counted by the group counter
  long long n_g = 1;
  for (int j = 0; j < eh; ++j) n_g *= 3;
  // value of the eg lowest digits of the r-th member of a group
  const int off9[9] = {0, 1, 2, 2, 3, 4, 4, 5, 6};
  const double inv_p = 1.0 / (double)p;
#pragma unroll 1
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n3;
       k += (long long)gridDim.x * blockDim.x) {
    u128 A = 0;
    unsigned long long exact = 0;  // p = 1: s in Z/2^64
    int top = -1;
    int vbase = 0;         // value of the group's upper digits
    unsigned int dig = 0;  // base-3 digits eg.. of d, two bits each (e <= 12)
#pragma unroll 1
    for (long long g = 0; g < n_g; ++g) {
      long long w[9];
      const long long* src = W + (g * gsz) * n3 + k;
#pragma unroll
      for (int r = 0; r < 9; ++r) w[r] = r < gsz ? __ldcs(src + r * n3) : 0;
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        if (r >= gsz || w[r] == 0) continue;
        const int val = vbase + (eg == 1 ? r : off9[r]);
        const unsigned long long t = (unsigned long long)w[r];
        if (p == 1) {
          exact += t << (val * b);
        } else if (top < 0) {
          top = val;
          A = (u128)t << G;
        } else if (val > top) {
          const int sh = (val - top) * b;
          A = sh >= 128 ? (u128)0 : (A >> sh);
          top = val;
          A += (u128)t << G;
        } else {
          const int sh = (top - val) * b - G;
          if (sh <= 0) A += (u128)t << (-sh);
          else if (sh < 64) A += (u128)(t >> sh);
        }
      }
      // next group: base-3 increment of the upper digits, value alongside
      for (int j = 0; j < eh; ++j) {
        const unsigned int q = (dig >> (2 * j)) & 3u;
        if (q < 2) {
          dig += 1u << (2 * j);
          vbase += 1 << (j + eg);
          break;
        }
        dig &= ~(3u << (2 * j));
        vbase -= 2 << (j + eg);
      }
    }
    long long out = (long long)exact;
    if (p > 1 && top >= 0) {
      const double a = (double)(unsigned long long)(A >> 64) * 18446744073709551616.0 +
                       (double)(unsigned long long)A;
      const double lg = log2(a) + (double)top * (double)b - (double)G;
      out = llrint(exp2(lg * inv_p));
    }
    z[k] = out;
  }
}

}  // namespace hc

extern "C" hc_status hc_maxconv_plan(int D, int64_t vmax, int* p, int* limb_bits, int* limb_axes,
                                     int* limbs) {
  const hc::MaxPlan P = hc::make_max_plan(D, (long long)vmax);
  if (!P.ok) return HC_ERR_ARG;
  if (p) *p = P.p;
  if (limb_bits) *limb_bits = P.b;
  if (limb_axes) *limb_axes = P.e;
  if (limbs) *limbs = P.L;
  return HC_OK;
}

extern "C" size_t hc_maxconv_workspace_size(int D, int64_t vmax) {
  const hc::MaxPlan P = hc::make_max_plan(D, (long long)vmax);
  return P.ok ? P.ws_bytes : 0;
}

extern "C" hc_status hc_maxconv(const int64_t* x, const int64_t* y, int64_t* z, int D,
                                int64_t vmax, void* workspace, size_t ws_bytes,
                                hc_stream_t stream) {
  using namespace hc;
  const MaxPlan P = make_max_plan(D, (long long)vmax);
  if (!P.ok) return HC_ERR_ARG;
  if (!x || !y || !z || !workspace) return HC_ERR_ARG;
  if (!aligned(x, 16) || !aligned(y, 16) || !aligned(z, 16)) return HC_ERR_ALIGN;
  if (!aligned(workspace, 256)) return HC_ERR_ALIGN;
  if (ws_bytes < P.ws_bytes) return HC_ERR_WORKSPACE;
  const size_t nx = (size_t)8 << D, nz = 8 * pow3z(D);
  if (overlaps(z, nz, x, nx) || overlaps(z, nz, y, nx)) return HC_ERR_ALIAS;
  if (overlaps(workspace, P.ws_bytes, z, nz) || overlaps(workspace, P.ws_bytes, x, nx) ||
      overlaps(workspace, P.ws_bytes, y, nx))
    return HC_ERR_ALIAS;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* ws = (unsigned char*)workspace;
  unsigned int* status = &((WsHeader*)ws)->status;
  unsigned long long* tab = (unsigned long long*)(ws + P.off_tab);
  unsigned long long* U = (unsigned long long*)(ws + P.off_u);
  unsigned long long* V = (unsigned long long*)(ws + P.off_v);
  long long* W = (long long*)(ws + P.off_w);
  const int E = 1 << P.e;
  const int De = D + P.e;
  const long long cap = (long long)device_caps().sms * 8;
  hc_status s = record_cuda_error(cudaMemsetAsync(status, 0, sizeof(unsigned int), st));
  if (s != HC_OK) return s;
  if (P.table) {
    ProfileScope prof(st, "maxconv_pow");
    const unsigned blocks = (unsigned)((P.vmax + 1 + 127) / 128);
    maxconv_pow_kernel<<<blocks, 128, 0, st>>>(tab, P.vmax, P.p, P.b, P.L, E);
    s = record_cuda_error(cudaGetLastError());
    if (s != HC_OK) return s;
  }
  {
    ProfileScope prof(st, "maxconv_spread");
    const long long n = 1LL << D;
    long long blocks = (n + 255) / 256;
    if (blocks > cap) blocks = cap;
    maxconv_spread_kernel<<<dim3((unsigned)blocks, 2), 256, 0, st>>>(
        (const long long*)x, (const long long*)y, P.table ? tab : nullptr, U, V, n, P.p, P.b,
        P.L, E, P.vmax, status);
    s = record_cuda_error(cudaGetLastError());
    if (s != HC_OK) return s;
  }
  s = convolve_checked(U, V, W, De, HC_INT64, P.conv_bytes ? ws + P.off_conv : nullptr,
                       P.conv_bytes, st, nullptr);
  if (s != HC_OK) return s;
  {
    ProfileScope prof(st, "maxconv_root");
    const long long n3 = (long long)pow3z(D);
    long long blocks = (n3 + 255) / 256;
    if (blocks > cap) blocks = cap;
    int lg3e = 0;  // ceil(e log2 3)
    while ((double)lg3e < P.e * 1.5849625007211562) ++lg3e;
    maxconv_root_kernel<<<(unsigned)blocks, 256, 0, st>>>(W, (long long*)z, n3, P.e, P.b, P.p,
                                                          62 - lg3e);
    s = record_cuda_error(cudaGetLastError());
  }
  return s;
}
