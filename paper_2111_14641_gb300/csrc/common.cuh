// Common device helpers for librbgs (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "../../include/rbgs.h"

namespace rbgs {

// --------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two
// 32x32->64-bit products on counter words 0 and 2, the high halves xor-ed
// with words 1 and 3 and the key; key bumped by the Weyl increments between
// rounds.
__host__ __device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
#ifdef __CUDA_ARCH__
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
#else
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__host__ __device__ __forceinline__ uint2 seed_key(uint64_t seed) {
  return make_uint2((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
}

// Stream purposes carried in counter word 2.
enum : uint32_t {
  kPurposeGauss = 0,
  kPurposeRademacher = 1,
  kPurposeSrhtSign = 2,
  kPurposeSrhtSample = 3,
  kPurposeSparse = 4
};

// ------------------------------------------------ double-FP32 arithmetic --
// A double-float is an unevaluated sum x.x + x.y of two floats (Dekker 1971;
// Knuth's TwoSum).  GB300's FP64 pipe is narrow, so the Gaussian generator
// below evaluates its logarithm, square root and sine/cosine this way on the
// FP32 pipe.

// IEEE round-to-nearest division and square root, count of leading zeros and
// a bit cast, for the device and for the host copy of the generator
// (rbgs_gaussian_entries), which must give the same floats.
__host__ __device__ __forceinline__ float dfx_div_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fdiv_rn(a, b);
#else
  return a / b;
#endif
}
__host__ __device__ __forceinline__ float dfx_sqrt_rn(float a) {
#ifdef __CUDA_ARCH__
  return __fsqrt_rn(a);
#else
  return sqrtf(a);
#endif
}
__host__ __device__ __forceinline__ int dfx_clz64(uint64_t v) {  // v != 0
#ifdef __CUDA_ARCH__
  return __clzll((long long)v);
#else
  return __builtin_clzll(v);
#endif
}
__host__ __device__ __forceinline__ float dfx_u2f(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, sizeof f);
  return f;
#endif
}

__host__ __device__ __forceinline__ float2 dfx_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return make_float2(s, b - (s - a));
}
__host__ __device__ __forceinline__ float2 dfx_two_sum(float a, float b) {
  const float s = a + b;
  const float bp = s - a;
  return make_float2(s, (a - (s - bp)) + (b - bp));
}
__host__ __device__ __forceinline__ float2 dfx_add(float2 x, float2 y) {
  const float2 s = dfx_two_sum(x.x, y.x);
  return dfx_fast_two_sum(s.x, s.y + (x.y + y.y));
}
__host__ __device__ __forceinline__ float2 dfx_mul(float2 x, float2 y) {
  const float p = x.x * y.x;
  float e = fmaf(x.x, y.x, -p);
  e = fmaf(x.x, y.y, e);
  e = fmaf(x.y, y.x, e);
  return dfx_fast_two_sum(p, e);
}
__host__ __device__ __forceinline__ float2 dfx_mul_f(float2 x, float f) {
  const float p = x.x * f;
  float e = fmaf(x.x, f, -p);
  e = fmaf(x.y, f, e);
  return dfx_fast_two_sum(p, e);
}
__host__ __device__ __forceinline__ float2 dfx_neg(float2 x) { return make_float2(-x.x, -x.y); }
__host__ __device__ __forceinline__ float2 dfx_div(float2 x, float2 y) {  // one correction step
  const float q1 = dfx_div_rn(x.x, y.x);
  const float2 r = dfx_add(x, dfx_neg(dfx_mul_f(y, q1)));
  return dfx_fast_two_sum(q1, dfx_div_rn(r.x, y.x));
}
__host__ __device__ __forceinline__ float2 dfx_sqrt(float2 x) {  // x >= 0
  if (!(x.x > 0.f)) return make_float2(0.f, 0.f);
  const float s = dfx_sqrt_rn(x.x);
  const float p = s * s;
  const float e = fmaf(s, s, -p);
  return dfx_fast_two_sum(s, dfx_div_rn(((x.x - p) - e) + x.y, 2.f * s));
}
// |v| < 2^56 exactly as three 23-bit pieces, summed as a double-float
__host__ __device__ __forceinline__ float2 dfx_from_i64(int64_t v) {
  const bool neg = v < 0;
  const uint64_t a = (uint64_t)(neg ? -v : v);
  auto f23 = [](uint32_t t) { return dfx_u2f(0x4B000000u | t) - 8388608.0f; };  // t < 2^23, exact
  const float fa = f23((uint32_t)(a >> 46)) * 0x1p46f, fb = f23((uint32_t)(a >> 23) & 0x7fffffu) * 0x1p23f;
  const float fc = f23((uint32_t)a & 0x7fffffu);
  const float2 s = dfx_two_sum(fa, fb);
  const float2 s2 = dfx_two_sum(s.x, fc);
  const float2 r = dfx_fast_two_sum(s2.x, s.y + s2.y);
  return neg ? dfx_neg(r) : r;
}
// sum_k c_k y^k, the terms k < 5 in double-float, the rest in float
template <int N>
__host__ __device__ __forceinline__ float2 dfx_poly(float2 y, const float2 (&c)[N]) {
  float p = c[N - 1].x;
#pragma unroll
  for (int k = N - 2; k >= 5; --k) p = fmaf(p, y.x, c[k].x);
  float2 q = make_float2(p, 0.f);
#pragma unroll
  for (int k = 4; k >= 0; --k) q = dfx_add(dfx_mul(q, y), c[k]);
  return q;
}

// Gaussian pair for column j, row pair rp of Theta: Box-Muller on the 53-bit
// uniforms u = (U + 1/2) 2^-53 (U from two Philox words, the sum rounded to
// FP64 as written), z0 = sqrt(-2 ln u1) cos(2 pi u2) serves row 2 rp and
// z1 = sqrt(-2 ln u1) sin(2 pi u2) row 2 rp + 1.
//
// Evaluated in double-float arithmetic from the exact integers W = u 2^54
// (about 2^-46 relative to the pair's radius; a CPU model of these steps
// against 40-digit references gave at most 1.2e-14):
//   ln u1 = 2 atanh(t) + (e - 54) ln 2 with t = (W1 - 2^e) / (W1 + 2^e),
//           W1 / 2^e in [sqrt(1/2), sqrt(2)), |t| <= 0.172, the series
//           atanh(t) = t sum_k t^(2k) / (2k + 1) to k = 10;
//   2 u2 = q / 2 + r (q an integer, |r| <= 1/4, exact), sin and cos of
//           theta = pi r by their Taylor series to theta^17 and theta^18,
//           then rotated by the quarter turns q.
__host__ __device__ __forceinline__ void gauss_pair(uint2 key, int64_t j, uint32_t rp, double& z0, double& z1) {
  const uint4 x = philox10(make_uint4((uint32_t)j, rp, kPurposeGauss, (uint32_t)(j >> 32)), key);
  auto w54 = [](uint32_t hi, uint32_t lo) -> int64_t {  // u 2^54 for U = (hi >> 5) 2^26 + (lo >> 6)
    const uint64_t U = ((uint64_t)(hi >> 5) << 26) | (uint64_t)(lo >> 6);
    if (U < (1ull << 52)) return (int64_t)(2 * U + 1);  // U + 1/2 is exact in FP64
    return (int64_t)(2 * (U + (U & 1)));                // rounded to even
  };
  const int64_t W1 = w54(x.x, x.y), W2 = w54(x.z, x.w);
  const float2 kLn2 = {0x1.62e43p-1f, -0x1.05c61p-29f};
  const float2 kPi = {0x1.921fb6p+1f, -0x1.777a5cp-24f};
  const float2 kAtanh[11] = {{1.0f, 0.0f},
                             {0x1.555556p-2f, -0x1.555556p-27f},
                             {0x1.99999ap-3f, -0x1.99999ap-29f},
                             {0x1.24924ap-3f, -0x1.b6db6ep-28f},
                             {0x1.c71c72p-4f, -0x1.c71c72p-31f},
                             {0x1.745d18p-4f, -0x1.745d18p-29f},
                             {0x1.3b13b2p-4f, -0x1.89d89ep-29f},
                             {0x1.111112p-4f, -0x1.dddddep-29f},
                             {0x1.e1e1e2p-5f, -0x1.e1e1e2p-33f},
                             {0x1.af286cp-5f, -0x1.af286cp-32f},
                             {0x1.861862p-5f, -0x1.e79e7ap-31f}};
  const float2 kSin[9] = {{1.0f, 0.0f},
                          {-0x1.555556p-3f, 0x1.555556p-28f},
                          {0x1.111112p-7f, -0x1.dddddep-32f},
                          {-0x1.a01a02p-13f, 0x1.7f97fap-39f},
                          {0x1.71de3ap-19f, 0x1.55b1ccp-45f},
                          {-0x1.ae6456p-26f, -0x1.fd5138p-52f},
                          {0x1.612462p-33f, -0x1.8af25ep-58f},
                          {-0x1.ae7f3ep-41f, -0x1.ccee08p-67f},
                          {0x1.952c78p-49f, -0x1.f9ea56p-74f}};
  const float2 kCos[10] = {{1.0f, 0.0f},
                           {-0.5f, 0.0f},
                           {0x1.555556p-5f, -0x1.555556p-30f},
                           {-0x1.6c16c2p-10f, 0x1.27d27ep-35f},
                           {0x1.a01a02p-16f, -0x1.7f97fap-42f},
                           {-0x1.27e4fcp-22f, 0x1.10ec14p-47f},
                           {0x1.1eed8ep-29f, 0x1.ff1b12p-54f},
                           {-0x1.93974ap-37f, -0x1.180f94p-62f},
                           {0x1.ae7f3ep-45f, 0x1.ccee08p-71f},
                           {-0x1.682786p-53f, -0x1.dcbeccp-80f}};
  // ln u1
  int e = 63 - dfx_clz64((uint64_t)W1);
  const uint64_t top = e >= 20 ? ((uint64_t)W1 >> (e - 20)) : ((uint64_t)W1 << (20 - e));
  if (top > 1482910ull) ++e;  // W1 / 2^e above sqrt(2) (floor(sqrt(2) 2^20) = 1482910)
  const float2 t = dfx_div(dfx_from_i64(W1 - (1ll << e)), dfx_from_i64(W1 + (1ll << e)));
  const float2 lm = dfx_mul(t, dfx_poly(dfx_mul(t, t), kAtanh));
  const float2 lnu = dfx_add(make_float2(2.f * lm.x, 2.f * lm.y), dfx_mul_f(kLn2, (float)(e - 54)));
  const float2 rad = dfx_sqrt(make_float2(-2.f * lnu.x, -2.f * lnu.y));
  // sin and cos of pi x, x = 2 u2 = W2 2^-53
  const int64_t q = (W2 + (1ll << 51)) >> 52;
  const float2 rr = dfx_from_i64(W2 - (q << 52));
  const float2 th = dfx_mul(kPi, make_float2(rr.x * 0x1p-53f, rr.y * 0x1p-53f));
  const float2 y = dfx_mul(th, th);
  const float2 sn = dfx_mul(th, dfx_poly(y, kSin));
  const float2 cs = dfx_poly(y, kCos);
  float2 sv, cv;
  switch ((int)(q & 3)) {
    case 0: sv = sn; cv = cs; break;
    case 1: sv = cs; cv = dfx_neg(sn); break;
    case 2: sv = dfx_neg(sn); cv = dfx_neg(cs); break;
    default: sv = dfx_neg(cs); cv = sn; break;
  }
  const float2 a = dfx_mul(rad, cv), b = dfx_mul(rad, sv);
  z0 = (double)a.x + (double)a.y;
  z1 = (double)b.x + (double)b.y;
}

// 128 Rademacher sign bits for column j, rows [128 g, 128 g + 128).
__device__ __forceinline__ uint4 rademacher_bits(uint2 key, int64_t j, uint32_t g) {
  return philox10(make_uint4((uint32_t)j, g, kPurposeRademacher, (uint32_t)(j >> 32)), key);
}

// 128 SRHT diagonal sign bits for padded rows [128 g, 128 g + 128).
__device__ __forceinline__ uint4 srht_sign_bits(uint2 key, uint32_t g) {
  return philox10(make_uint4(g, 0u, kPurposeSrhtSign, 0u), key);
}

// Sparse sign, the block construction of the sparse Johnson-Lindenstrauss
// transform (Kane and Nelson 2014): with z = min(8, k) the rows split into z
// segments [floor(s k / z), floor((s + 1) k / z)); column j has one nonzero
// +-1/sqrt(z) in each, at offset (x >> 1) mod (segment size), negative when
// bit 0 of x is set, x = word s & 3 of the block with counter
// (j_lo, s >> 2, 4, j_hi).  Fills rows[s], neg[s] for s < z; returns z.
__host__ __device__ __forceinline__ int sparse_zeta(int64_t k) { return k < 8 ? (int)k : 8; }
__host__ __device__ __forceinline__ int sparse_column(uint2 key, int64_t j, int64_t k, int64_t (&rows)[8],
                                                      bool (&neg)[8]) {
  const int z = sparse_zeta(k);
  uint4 x = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    if (s < z) {
      if ((s & 3) == 0)
        x = philox10(make_uint4((uint32_t)j, (uint32_t)(s >> 2), kPurposeSparse, (uint32_t)(j >> 32)), key);
      const uint32_t v = (s & 3) == 0 ? x.x : ((s & 3) == 1 ? x.y : ((s & 3) == 2 ? x.z : x.w));
      const int64_t lo = (int64_t)s * k / z, hi = (int64_t)(s + 1) * k / z;
      rows[s] = lo + (int64_t)((v >> 1) % (uint32_t)(hi - lo));
      neg[s] = (v & 1u) != 0u;
    }
  }
  return z;
}

__device__ __forceinline__ uint32_t word_of(const uint4& v, int w) {
  return w == 0 ? v.x : (w == 1 ? v.y : (w == 2 ? v.z : v.w));
}

// Double-FP32 ("double-float") helpers: a value is an unevaluated sum hi + lo
// of two floats.
//
// df_split: v = hi + lo + d with |d| < 2^-46 |v|, from integer operations on
// the bits of v (GB300's FP64 pipe, which also converts, is narrow).  hi is v
// with its 52-bit fraction truncated to 23 bits; lo holds the next 23 bits of
// the fraction, with the sign of v.  Zero gives (0, 0); other exponents outside
// [-80, 127] (subnormals, huge values, inf, NaN) take the FP64 conversion.
__device__ __forceinline__ float2 df_split(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  if ((b << 1) == 0ull) return make_float2(0.f, 0.f);  // +-0 (the padding of product tiles)
  const int ex = (int)((b >> 52) & 0x7ffu) - 1023;
  if (ex < -80 || ex > 127) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
  }
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const unsigned hi_bits = sign | ((unsigned)(ex + 127) << 23) | (unsigned)((b >> 29) & 0x7fffffu);
  const unsigned r1 = (unsigned)(b >> 6) & 0x7fffffu;  // fraction bits 28..6
  // r1 as a float (exact: 2^23 + r1 minus 2^23), scaled by 2^(ex - 46)
  const float lo_mag = (__uint_as_float(0x4B000000u | r1) - 8388608.0f) * __uint_as_float((unsigned)(ex + 81) << 23);
  return make_float2(__uint_as_float(hi_bits), __uint_as_float(__float_as_uint(lo_mag) | sign));
}

// TwoSum (Knuth): s + e == a + b exactly, s = fl(a + b).
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

// acc (hi, lo) += k x for a split coefficient k = (k.x, k.y) and a float x:
// k.x x exactly as a product and its FMA error, k.y x added to the error,
// the product's leading part added to hi by TwoSum.
__device__ __forceinline__ void df_fma(float2 k, float x, float& hi, float& lo) {
  const float p = k.x * x;
  float e = fmaf(k.x, x, -p);
  e = fmaf(k.y, x, e);
  float s, t;
  df_two_sum(hi, p, s, t);
  hi = s;
  lo += t + e;
}

}  // namespace rbgs

#define RBGS_CUDA_TRY(expr)                  \
  do {                                       \
    cudaError_t _e = (expr);                 \
    if (_e != cudaSuccess) return RBGS_ECUDA; \
  } while (0)

namespace rbgs {
void count_launch();
}

#define RBGS_LAUNCH_CHECK()                                   \
  do {                                                        \
    rbgs::count_launch();                                     \
    if (cudaGetLastError() != cudaSuccess) return RBGS_ECUDA; \
  } while (0)
