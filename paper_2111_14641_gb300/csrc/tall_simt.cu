// SIMT tall update: Qout = [A1 | A2] * G  (step 3 of Alg. 2 fused with the
// multiplication by R_ii^{-1} of Alg. 5, through G = [-R_{1:i-1,i}; I] R_ii^{-1}).
//
// One CTA owns 128 rows and all mb <= 64 output columns; the K loop walks the
// c columns of A1 and then the mb columns of A2 in chunks of 16, staged in
// shared memory.  Each thread accumulates an 8 x 4 register tile.  This is
// the FP64 path (DFMA) and the FP32 reference path (FFMA); the tensor-core
// path lives in tall_tc.cu.
#include "common.cuh"
#include "internal.h"

namespace rbgs {
namespace {

constexpr int BM = 128;
constexpr int BN = 64;
constexpr int KC = 16;
constexpr int NT = 256;

template <class T>
__global__ void __launch_bounds__(NT) tall_simt_kernel(int64_t n, int64_t c, int mb, const T* __restrict__ A1,
                                                       int64_t lda1, const T* A2, int64_t lda2,
                                                       const T* __restrict__ G, int64_t ldg, T* Qout, int64_t ldo,
                                                       const int* active) {
  if (active && *active == 0) return;
  __shared__ T As[KC][BM + 1];
  __shared__ T Gs[KC][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15;   // columns tx + 16 q
  const int ty = tid >> 4;   // rows ty + 16 i
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int64_t K = c + mb;
  T acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[i][q] = 0;

  for (int64_t k0 = 0; k0 < K; k0 += KC) {
    // A chunk: KC columns x BM rows, column-major source
#pragma unroll
    for (int e = 0; e < (KC * BM) / NT; ++e) {
      const int idx = tid + e * NT;
      const int r = idx % BM, kk = idx / BM;
      const int64_t gk = k0 + kk, gr = row0 + r;
      T v = 0;
      if (gk < K && gr < n) v = (gk < c) ? A1[gr + gk * lda1] : A2[gr + (gk - c) * lda2];
      As[kk][r] = v;
    }
    // G chunk: KC rows x BN columns
#pragma unroll
    for (int e = 0; e < (KC * BN) / NT; ++e) {
      const int idx = tid + e * NT;
      const int kk = idx / BN, q = idx % BN;
      const int64_t gk = k0 + kk;
      Gs[kk][q] = (gk < K && q < mb) ? G[gk + (int64_t)q * ldg] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      T a[8], b[4];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = Gs[kk][tx + 16 * q];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] += a[i] * b[q];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t gr = row0 + ty + 16 * i;
    if (gr >= n) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int col = tx + 16 * q;
      if (col < mb) Qout[gr + (int64_t)col * ldo] = acc[i][q];
    }
  }
}

// Q (n x mb, ldq) <- Q R^{-1} row by row by forward substitution with the
// upper-triangular R (mb x mb, ld mb, type TS): one thread per row, R in
// shared memory (ld 64), the substitution in FP64 whatever the storage type T
// (the result is rounded to T once).  Each row's solve is backward stable,
// (q + dq) R = q' with |dq| <= u |q| |R| elementwise, whatever the condition
// of R, unlike the product with an explicit inverse, whose error grows with
// cond(R).  The FP64 arithmetic matters for FP32 storage: a substitution in
// FP32 is backward stable in FP32 too, but its forward error u_32 cond(R) in
// a numerically rank-deficient block leaves the block's columns dependent in
// a way the second projection pass cannot undo.
template <class T, class TS>
__global__ void __launch_bounds__(128) trsm_rows_kernel(int64_t n, int mb, T* __restrict__ Q, int64_t ldq,
                                                        const TS* __restrict__ R, const int* __restrict__ active) {
  if (active && *active == 0) return;
  __shared__ double Rs[64 * 64];
  for (int t = threadIdx.x; t < mb * mb; t += blockDim.x) Rs[(t % mb) + 64 * (t / mb)] = (double)R[t];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  // in place, column sweep: x_j = v_j / r_jj, then v_l -= x_j r_jl for l > j
  double v[64];
#pragma unroll
  for (int j = 0; j < 64; ++j) v[j] = j < mb ? (double)Q[i + (int64_t)j * ldq] : 0.0;
#pragma unroll
  for (int j = 0; j < 64; ++j) {
    if (j < mb) {
      v[j] /= Rs[j + 64 * j];
#pragma unroll
      for (int l = j + 1; l < 64; ++l) v[l] -= v[j] * Rs[j + 64 * l];
    }
  }
#pragma unroll
  for (int j = 0; j < 64; ++j)
    if (j < mb) Q[i + (int64_t)j * ldq] = (T)v[j];
}

}  // namespace

template <class T, class TS>
rbgs_status trsm_rows(int64_t n, int mb, T* Q, int64_t ldq, const TS* R, const int* active, cudaStream_t st) {
  if (mb < 1 || mb > 64) return RBGS_EINVAL;
  if (n == 0) return RBGS_OK;
  trsm_rows_kernel<T, TS><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n, mb, Q, ldq, R, active);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}
template rbgs_status trsm_rows<double, double>(int64_t, int, double*, int64_t, const double*, const int*,
                                               cudaStream_t);
template rbgs_status trsm_rows<float, double>(int64_t, int, float*, int64_t, const double*, const int*, cudaStream_t);
template rbgs_status trsm_rows<float, float>(int64_t, int, float*, int64_t, const float*, const int*, cudaStream_t);

template <class T>
rbgs_status tall_update_simt(int64_t n, int64_t c, int64_t mb, const T* A1, int64_t lda1, const T* A2, int64_t lda2,
                             const T* G, int64_t ldg, T* Qout, int64_t ldo, const int* active, cudaStream_t st) {
  if (mb < 1 || mb > BN) return RBGS_EINVAL;
  if (n == 0) return RBGS_OK;
  const int64_t nblk = (n + BM - 1) / BM;
  tall_simt_kernel<T><<<(unsigned)nblk, NT, 0, st>>>(n, c, (int)mb, A1, lda1, A2, lda2, G, ldg, Qout, ldo, active);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}

template rbgs_status tall_update_simt<double>(int64_t, int64_t, int64_t, const double*, int64_t, const double*,
                                              int64_t, const double*, int64_t, double*, int64_t, const int*,
                                              cudaStream_t);
template rbgs_status tall_update_simt<float>(int64_t, int64_t, int64_t, const float*, int64_t, const float*, int64_t,
                                             const float*, int64_t, float*, int64_t, const int*, cudaStream_t);

}  // namespace rbgs
