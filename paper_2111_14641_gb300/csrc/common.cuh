// Common device helpers for librbgs (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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

// Gaussian pair for column j, row pair rp of Theta (Box-Muller on 53-bit
// uniforms in (0,1)); z0 serves row 2 rp, z1 row 2 rp + 1.
__device__ __forceinline__ void gauss_pair(uint2 key, int64_t j, uint32_t rp, double& z0, double& z1) {
  const uint4 x = philox10(make_uint4((uint32_t)j, rp, kPurposeGauss, (uint32_t)(j >> 32)), key);
  const double u1 = ((double)(x.x >> 5) * 67108864.0 + (double)(x.y >> 6) + 0.5) * (1.0 / 9007199254740992.0);
  const double u2 = ((double)(x.z >> 5) * 67108864.0 + (double)(x.w >> 6) + 0.5) * (1.0 / 9007199254740992.0);
  const double rad = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  z0 = rad * c;
  z1 = rad * s;
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
