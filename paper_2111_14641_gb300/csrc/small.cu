// Sketch-space kernels of Alg. 2 (k rows, k << n): the step-2 least-squares
// products (Richardson iterations of the supplement to Sec. 3.1), the
// implicit sketch S'_i = P_i - S_{1:i-1} R_{1:i-1,i} of Alg. 5, Cholesky QR of
// the k x m_p sketch for R_ii, the coefficient matrix of the fused projection,
// the second-pass bookkeeping and the step-6 norms.
//
// Every kernel takes an optional device flag `active`; when it points to 0
// the kernel returns at once.  This keeps the host loop free of
// synchronisations (the adaptive second pass is decided on the device).
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace rbgs {
namespace {

constexpr int SG_T = 64;   // output tile rows
constexpr int SG_N = 64;   // max output columns
constexpr int SG_K = 16;   // K chunk

template <class TA, class TACC>
__global__ void __launch_bounds__(256) small_gemm_part(int trans, int64_t M, int N, int64_t K, int64_t kper,
                                                       const TA* __restrict__ A, int64_t lda,
                                                       const TA* __restrict__ B, int64_t ldb,
                                                       TACC* __restrict__ part, const int* active) {
  if (active && *active == 0) return;
  __shared__ TACC As[SG_K][SG_T + 1];
  __shared__ TACC Bs[SG_K][SG_N + 1];
  const int tid = threadIdx.x;
  // Warp w owns output columns 8w .. 8w + 7, lane l rows l and l + 32: a warp
  // whose columns are all >= N does no arithmetic (N = m_p is often not a
  // multiple of 16, and the FP64 pipe is the bottleneck).
  const int warp = tid >> 5, lane = tid & 31;
  const int jw = 8 * warp;
  const bool busy = jw < N;
  const int64_t i0 = (int64_t)blockIdx.x * SG_T;
  const int split = blockIdx.y;
  const int64_t kb = (int64_t)split * kper;
  const int64_t ke = min(K, kb + kper);
  constexpr int PER = (SG_K * SG_T) / 256;  // elements per thread per chunk (A and B alike)
  TACC ra[PER], rb[PER];
  // software pipeline: the global loads of chunk l0 + SG_K are in flight while chunk l0 is used
  auto load = [&](int64_t l0) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = tid + 256 * q;
      int il, ll;
      if (trans) { ll = e % SG_K; il = e / SG_K; }   // A is K x M: contiguous in l
      else { il = e % SG_T; ll = e / SG_T; }         // A is M x K: contiguous in i
      const int64_t gi = i0 + il, gl = l0 + ll;
      ra[q] = (gi < M && gl < ke) ? (TACC)(trans ? A[gl + gi * lda] : A[gi + gl * lda]) : (TACC)0;
      const int lb = e % SG_K, j = e / SG_K;
      const int64_t gb = l0 + lb;
      rb[q] = (gb < ke && j < N) ? (TACC)B[gb + (int64_t)j * ldb] : (TACC)0;
    }
  };
  TACC acc[2][8];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[i][q] = 0;
  if (kb < ke) load(kb);
  for (int64_t l0 = kb; l0 < ke; l0 += SG_K) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = tid + 256 * q;
      int il, ll;
      if (trans) { ll = e % SG_K; il = e / SG_K; }
      else { il = e % SG_T; ll = e / SG_T; }
      As[ll][il] = ra[q];
      Bs[e % SG_K][e / SG_K] = rb[q];
    }
    __syncthreads();
    if (l0 + SG_K < ke) load(l0 + SG_K);
    if (busy) {
#pragma unroll
      for (int ll = 0; ll < SG_K; ++ll) {
        const TACC a0 = As[ll][lane], a1 = As[ll][lane + 32];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const TACC b = Bs[ll][jw + q];
          acc[0][q] += a0 * b;
          acc[1][q] += a1 * b;
        }
      }
    }
    __syncthreads();
  }
  if (busy) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int64_t gi = i0 + lane + 32 * i;
        const int j = jw + q;
        if (gi < M && j < N) part[((int64_t)split * N + j) * M + gi] = acc[i][q];
      }
  }
}

// The same product for FP64 data with double-FP32 ("double-float")
// arithmetic on the FP32 pipe: each operand is split once, a = a_hi + a_lo
// (df_split: 47 significant bits taken from the FP64 bits by integer
// operations, since the FP64 pipe that would convert is narrow), each
// product a_hi b_hi is formed exactly with its FMA error term, the cross
// terms a_hi b_lo + a_lo b_hi are added into that error, and the running sum
// is a double-float (s_hi, s_lo) kept by TwoSum (Knuth; Dekker 1971).  The
// relative error of the result is a few units of 2^-44, far below the FP32
// storage of the tall data, at about six times the FP64 pipe's rate on
// GB300.  The mixed-precision path uses it for its FP64 sketch space; the
// FP64 path keeps the FP64 kernel.
__global__ void __launch_bounds__(256) small_gemm_part_df(int trans, int64_t M, int N, int64_t K, int64_t kper,
                                                          const double* __restrict__ A, int64_t lda,
                                                          const double* __restrict__ B, int64_t ldb,
                                                          double* __restrict__ part, const int* active) {
  if (active && *active == 0) return;
  __shared__ float2 As[SG_K][SG_T + 1];
  __shared__ float2 Bs[SG_K][SG_N + 1];
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int jw = 8 * warp;
  const bool busy = jw < N;
  const int64_t i0 = (int64_t)blockIdx.x * SG_T;
  const int split = blockIdx.y;
  const int64_t kb = (int64_t)split * kper;
  const int64_t ke = min(K, kb + kper);
  constexpr int PER = (SG_K * SG_T) / 256;
  double ra[PER], rb[PER];
  auto load = [&](int64_t l0) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = tid + 256 * q;
      int il, ll;
      if (trans) { ll = e % SG_K; il = e / SG_K; }
      else { il = e % SG_T; ll = e / SG_T; }
      const int64_t gi = i0 + il, gl = l0 + ll;
      ra[q] = (gi < M && gl < ke) ? (trans ? A[gl + gi * lda] : A[gi + gl * lda]) : 0.0;
      const int lb = e % SG_K, j = e / SG_K;
      const int64_t gb = l0 + lb;
      rb[q] = (gb < ke && j < N) ? B[gb + (int64_t)j * ldb] : 0.0;
    }
  };
  float hi[2][8], lo[2][8];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int q = 0; q < 8; ++q) hi[i][q] = lo[i][q] = 0.f;
  if (kb < ke) load(kb);
  for (int64_t l0 = kb; l0 < ke; l0 += SG_K) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = tid + 256 * q;
      int il, ll;
      if (trans) { ll = e % SG_K; il = e / SG_K; }
      else { il = e % SG_T; ll = e / SG_T; }
      As[ll][il] = df_split(ra[q]);  // integer operations: no FP64 conversions
      Bs[e % SG_K][e / SG_K] = df_split(rb[q]);
    }
    __syncthreads();
    if (l0 + SG_K < ke) load(l0 + SG_K);
    if (busy) {
#pragma unroll
      for (int ll = 0; ll < SG_K; ++ll) {
        const float2 a0 = As[ll][lane], a1 = As[ll][lane + 32];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float2 b = Bs[ll][jw + q];
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            const float2 a = r ? a1 : a0;
            const float p = a.x * b.x;
            float e = fmaf(a.x, b.x, -p);
            e = fmaf(a.x, b.y, e);
            e = fmaf(a.y, b.x, e);
            float sacc, err;
            df_two_sum(hi[r][q], p, sacc, err);
            hi[r][q] = sacc;
            lo[r][q] += err + e;
          }
        }
      }
    }
    __syncthreads();
  }
  if (busy) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int64_t gi = i0 + lane + 32 * i;
        const int j = jw + q;
        if (gi < M && j < N) part[((int64_t)split * N + j) * M + gi] = (double)hi[i][q] + (double)lo[i][q];
      }
  }
}

template <class TACC, class TO>
__global__ void small_gemm_reduce(int64_t M, int N, int ks, const TACC* __restrict__ part, double alpha,
                                  double beta, TO* out, int64_t ldo, const int* active) {
  if (active && *active == 0) return;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * N) return;
  const int64_t i = idx % M;
  const int64_t j = idx / M;
  // eight independent loads in flight (the partial slices live in L2); the
  // slices are added in a fixed order, so the result is reproducible
  const TACC* pp = part + j * M + i;
  const int64_t stride = (int64_t)N * M;
  TACC s8[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) s8[u] = 0;
  int p = 0;
  for (; p + 8 <= ks; p += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) s8[u] += pp[(int64_t)(p + u) * stride];
  }
  for (; p < ks; ++p) s8[p & 7] += pp[(int64_t)p * stride];
  TACC s = ((s8[0] + s8[1]) + (s8[2] + s8[3])) + ((s8[4] + s8[5]) + (s8[6] + s8[7]));
  TO* o = out + i + j * ldo;
  const double v = alpha * (double)s;
  *o = (TO)(beta == 0.0 ? v : v + beta * (double)(*o));
}

// ---------------------------------------------------------------- Cholesky --
// G = R^T R (upper R, positive diagonal) of an mb x mb matrix, mb <= 64, and
// R^{-1}, in the arithmetic of T, one CTA of 256 threads.  With shift != 0 the
// factorization is of G + s I, s = shift * trace(G) (the shifted Cholesky QR
// of Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa 2020: keeps the first
// round of Cholesky QR from breaking down on ill-conditioned blocks).
// Column of linear index e in the column-by-column enumeration of an upper
// triangle (column b holds rows 0..b, so it starts at b (b + 1) / 2).
__device__ __forceinline__ int tri_col(int e) {
  int b = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
  while (b * (b + 1) / 2 > e) --b;
  while ((b + 1) * (b + 2) / 2 <= e) ++b;
  return b;
}
// Enumeration of an order-n upper triangle by diagonals d = l - i (diagonal d
// holds n - d entries, i = 0..n-1-d): first index of diagonal d, and the
// diagonal of linear index e.
__device__ __forceinline__ int diag_start(int d, int n) { return d * n - d * (d - 1) / 2; }
__device__ __forceinline__ int diag_of(int e, int n) {
  // the root of diag_start(d, n) = e, d = ((2n + 1) - sqrt((2n + 1)^2 - 8 e)) / 2,
  // then corrected to the exact diagonal
  const float b = 2.f * (float)n + 1.f;
  int d = (int)((b - sqrtf(fmaxf(b * b - 8.f * (float)e, 0.f))) * 0.5f);
  d = max(0, min(d, n - 1));
  while (d > 0 && diag_start(d, n) > e) --d;
  while (d + 1 < n && diag_start(d + 1, n) <= e) ++d;
  return d;
}

template <class T>
__global__ void __launch_bounds__(256) chol_inv_kernel(int mb, const T* __restrict__ G, T* __restrict__ R,
                                                       T* __restrict__ Rinv, double shift, int* flag,
                                                       const T* __restrict__ Rprev, const T* __restrict__ Rprev_inv,
                                                       const int* active) {
  if (active && *active == 0) return;
  extern __shared__ __align__(16) unsigned char chol_smem[];
  typedef T Row[65];
  Row* A = reinterpret_cast<Row*>(chol_smem);  // working matrix (upper part)
  Row* F = A + 64;                             // the factor R, row by row as it is finished
  Row* X = F + 64;                             // Gauss-Jordan work: unscaled rows of R^{-1}
  Row* P = X + 64;                             // Rprev
  Row* PI = P + 64;                            // Rprev_inv
  __shared__ T xscale[64];                     // row j of R^{-1} = X[j][:] * xscale[j]
  __shared__ T pivot_s[2];                     // 1 / sqrt of the current and the next pivot
  __shared__ T shift_s;
  __shared__ int bad_s;
  __shared__ uint16_t tri_ab[63 * 64 / 2];     // linear index -> a | b << 8 of a trailing triangle
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;  // 16 x 16 thread grid
  for (int e = tid; e < (mb - 1) * mb / 2; e += 256) {
    const int b = tri_col(e);
    tri_ab[e] = (uint16_t)((e - b * (b + 1) / 2) | (b << 8));
  }
  for (int l = ty; l < mb; l += 16)
    for (int i = tx; i < mb; i += 16) {
      A[i][l] = (i <= l) ? G[i + l * mb] : (T)0;
      F[i][l] = (T)0;
      X[i][l] = (i == l) ? (T)1 : (T)0;
      if (Rprev) {
        P[i][l] = Rprev[i + l * mb];
        PI[i][l] = Rprev_inv[i + l * mb];
      }
    }
  if (tid == 0) bad_s = 0;
  __syncthreads();
  if (shift != 0.0) {
    if (tid == 0) {
      double tr = 0.0;
      for (int i = 0; i < mb; ++i) tr += (double)A[i][i];
      shift_s = (T)(shift * tr);
    }
    __syncthreads();
    if (tid < mb) A[tid][tid] += shift_s;
    __syncthreads();
  }
  // Right-looking Cholesky, one barrier per step: row j of A is only read
  // during step j (the finished row of R goes to F), the trailing triangle
  // i <= l of rows > j is updated with A[i][l] -= A[j][i] A[j][l] / d.  The
  // SM's FP64 pipe is narrow and a warp instruction costs the same with idle
  // lanes, so the triangle is walked by a linear index (full warps); the
  // pivot's reciprocal square root is taken once per warp and broadcast.
  // The next pivot's reciprocal square root is taken by the thread that
  // finishes that pivot (the first entry of the trailing triangle) while the
  // other warps still update: it stays off the step's critical path.
  if (tid == 0) {
    T d = A[0][0];
    if (!(d > (T)0) || !isfinite((double)d)) {
      bad_s = 1;
      d = (T)1;
    }
    pivot_s[0] = rsqrt(d);
  }
  __syncthreads();
  for (int j = 0; j < mb; ++j) {
    const T rinv = pivot_s[j & 1];
    const T dinv = rinv * rinv;
    if (tid == 0) xscale[j] = rinv;  // 1 / R_jj, used by the inverse below
    for (int l = j + tid; l < mb; l += 256) F[j][l] = (l == j) ? (T)1 / rinv : A[j][l] * rinv;
    const int nt = mb - 1 - j;  // trailing order
    const int tot = nt * (nt + 1) / 2;
    for (int e = tid; e < tot; e += 256) {
      const int ab = tri_ab[e];  // a <= b < nt
      const int i = j + 1 + (ab & 255), l = j + 1 + (ab >> 8);
      const T v = A[i][l] - A[j][i] * dinv * A[j][l];
      A[i][l] = v;
      if (e == 0) {  // (j + 1, j + 1): the next pivot is final now
        T d = v;
        if (!(d > (T)0) || !isfinite((double)d)) {
          bad_s = 1;
          d = (T)1;
        }
        pivot_s[(j + 1) & 1] = rsqrt(d);
      }
    }
    __syncthreads();
  }
  // R^{-1} by Gauss-Jordan from the last pivot up, one barrier per step:
  // row j of the inverse is X[j][:] / R_jj (rows > j are finished), and every
  // row i < j subtracts R_ij times it (a j x (mb - j) rectangle, linear index).
  for (int j = mb - 1; j >= 0; --j) {
    const T fj = xscale[j];
    const int w = mb - j;
    const float rj = 1.f / (float)max(j, 1);
    for (int e = tid; e < j * w; e += 256) {
      // i = e mod j, l = j + e div j; e < 4096, so the float quotient is within one
      int q = (int)((float)e * rj), i = e - q * j;
      if (i < 0) {
        --q;
        i += j;
      } else if (i >= j) {
        ++q;
        i -= j;
      }
      const int l = j + q;
      X[i][l] -= F[i][j] * fj * X[j][l];
    }
    __syncthreads();
  }
  // rows of R^{-1} = X[j][:] / R_jj, scaled once
  for (int e = tid; e < mb * mb; e += 256) {
    const int i = e / mb, l = e % mb;
    if (i <= l) X[i][l] *= xscale[i];
  }
  __syncthreads();
  // Outputs by diagonals (equal dot-product lengths within a warp).
  const int ntri = mb * (mb + 1) / 2;
  if (Rprev) {
    // second round of Cholesky QR: R := R2 R1, R^{-1} := R1^{-1} R2^{-1} (upper triangular products)
    for (int e = tid; e < ntri; e += 256) {
      int d = diag_of(e, mb), i = e - diag_start(d, mb);
      const int l = i + d;
      T s1 = 0, s2 = 0;
      for (int t = i; t <= l; ++t) {
        s1 += F[i][t] * P[t][l];
        s2 += PI[i][t] * X[t][l];
      }
      R[i + l * mb] = s1;
      Rinv[i + l * mb] = s2;
    }
  } else {
    for (int e = tid; e < ntri; e += 256) {
      int d = diag_of(e, mb), i = e - diag_start(d, mb);
      const int l = i + d;
      R[i + l * mb] = F[i][l];
      Rinv[i + l * mb] = X[i][l];
    }
  }
  for (int e = tid; e < mb * mb; e += 256) {  // strictly lower parts are zero
    const int i = e % mb, l = e / mb;
    if (i > l) {
      R[i + l * mb] = (T)0;
      Rinv[i + l * mb] = (T)0;
    }
  }
  if (tid == 0 && bad_s && flag) atomicOr(flag, 1);
}

// Out = A * U (A k x mb, U upper mb x mb): one thread per output entry.
template <class TS, class TU>
__global__ void trmm_kernel(int64_t k, int mb, const TS* __restrict__ A, int64_t lda, const TU* __restrict__ U,
                            TS* __restrict__ Out, int64_t ldo, const int* active) {
  if (active && *active == 0) return;
  __shared__ TS Us[64][65];
  for (int e = threadIdx.x; e < mb * mb; e += blockDim.x) {
    const int i = e % mb, l = e / mb;
    Us[i][l] = (TS)U[i + l * mb];
  }
  __syncthreads();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= k * mb) return;
  const int64_t r = idx % k;
  const int j = (int)(idx / k);
  TS s = 0;
  for (int i = 0; i <= j; ++i) s += A[r + i * lda] * Us[i][j];
  Out[r + j * ldo] = s;
}

// C = A * B for upper-triangular mb x mb matrices (ld mb).
template <class T>
__global__ void tri_mul_kernel(int mb, const T* __restrict__ A, const T* __restrict__ B, T* C, const int* active) {
  if (active && *active == 0) return;
  __shared__ T As[64][65], Bs[64][65];
  for (int e = threadIdx.x; e < mb * mb; e += blockDim.x) {
    const int i = e % mb, j = e / mb;
    As[i][j] = A[i + j * mb];
    Bs[i][j] = B[i + j * mb];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < mb * mb; e += blockDim.x) {
    const int i = e % mb, j = e / mb;
    T s = 0;
    for (int t = i; t <= j; ++t) s += As[i][t] * Bs[t][j];
    C[i + j * mb] = (i <= j) ? s : (T)0;
  }
}

template <class TS, class TG>
__global__ void assemble_g_kernel(int64_t c, int mb, const TS* __restrict__ Rc, int64_t ldrc,
                                  const TS* __restrict__ Rii, const TS* __restrict__ Riinv, TG* G,
                                  int64_t ldg, double* R, int64_t ldr, const int* active) {
  if (active && *active == 0) return;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t rows = c + mb;
  if (idx >= rows * mb) return;
  const int64_t i = idx % rows;
  const int j = (int)(idx / rows);
  double g;
  if (i < c) {
    TS s = 0;
    for (int t = 0; t <= j; ++t) s += Rc[i + t * ldrc] * Riinv[t + j * mb];
    g = -(double)s;
    if (R) R[i + (int64_t)j * ldr] = (double)Rc[i + (int64_t)j * ldrc];
  } else {
    const int ii = (int)(i - c);
    g = (ii <= j) ? (double)Riinv[ii + j * mb] : 0.0;
    if (R) R[i + (int64_t)j * ldr] = (ii <= j) ? (double)Rii[ii + j * mb] : 0.0;
  }
  G[i + (int64_t)j * ldg] = (TG)g;
}

template <class TS>
__global__ void reorth_r_top(int64_t c, int mb, const TS* __restrict__ R2c, int64_t ldr2,
                             const TS* __restrict__ R2ii, double* Rcol, int64_t ldr, double* tmp,
                             const int* active) {
  if (active && *active == 0) return;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t rows = c + mb;
  if (idx >= rows * mb) return;
  const int64_t i = idx % rows;
  const int j = (int)(idx / rows);
  const double* Rold = Rcol + c;  // R_ii (old) at rows c..c+mb-1
  if (i < c) {
    TS s = 0;
    for (int t = 0; t <= j; ++t) s += R2c[i + t * ldr2] * (TS)Rold[t + (int64_t)j * ldr];
    Rcol[i + (int64_t)j * ldr] += (double)s;
  } else {
    const int ii = (int)(i - c);
    double s = 0.0;
    for (int t = ii; t <= j; ++t) s += (double)R2ii[ii + t * mb] * Rold[t + (int64_t)j * ldr];
    tmp[ii + j * mb] = (ii <= j) ? s : 0.0;
  }
}

__global__ void copy_diag_block(int64_t c, int mb, const double* __restrict__ tmp, double* Rcol, int64_t ldr,
                                const int* active) {
  if (active && *active == 0) return;
  for (int e = threadIdx.x; e < mb * mb; e += blockDim.x) {
    const int i = e % mb, j = e / mb;
    Rcol[c + i + (int64_t)j * ldr] = tmp[i + j * mb];
  }
}

template <class TS>
__global__ void reorth_decide_kernel(int64_t c, int mb, const TS* __restrict__ X, int64_t ldx, double tol,
                                     int mode, int* active, int* count, int* blk_flag) {
  __shared__ double red[1024];
  double s = 0.0;
  const int64_t tot = mode == 1 ? 0 : c * mb;  // mode 1 (every block) needs no norm
#pragma unroll 8
  for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
    const double v = (double)X[(e % c) + (e / c) * ldx];
    s += v * v;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int on = (mode == 1) ? 1 : (sqrt(red[0]) > tol ? 1 : 0);
    *active = on;
    if (blk_flag) *blk_flag = on;
    if (on) *count += 1;
  }
}

template <class T>
__global__ void round2_decide_kernel(int mb, const T* __restrict__ R1, const T* __restrict__ R1inv, T* R, T* Rinv,
                                     double thr, const int* active, int* need2, int* count) {
  __shared__ double red[2][256];
  __shared__ int on_s;
  if (active && *active == 0) {
    if (threadIdx.x == 0) *need2 = 0;
    return;
  }
  const int tot = mb * mb;
  double a = 0.0, b = 0.0;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const double x = (double)R1[e], y = (double)R1inv[e];
    a += x * x;
    b += y * y;
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      red[0][threadIdx.x] += red[0][threadIdx.x + h];
      red[1][threadIdx.x] += red[1][threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double kf = sqrt(red[0][0] * red[1][0]);
    const int on = !(kf <= thr);  // a NaN estimate keeps the second round
    on_s = on;
    *need2 = on;
    if (on && count) *count += 1;
  }
  __syncthreads();
  if (on_s) return;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    R[e] = R1[e];
    Rinv[e] = R1inv[e];
  }
}

// One conjugate-gradient step on the normal equations (S^T S) x_j = S^T p_j of
// step 2, for every column j at once (one CTA per column): with q = S^T S d
// given, alpha = rr / (d.q); x += alpha d; r -= alpha q; beta = rr' / rr;
// d = r + beta d.  A column whose d.q <= 0 (or rr = 0) stops for good (done[j]).
template <class TS>
__global__ void __launch_bounds__(256) cg_step_kernel(int64_t c, TS* X, int64_t ldx, TS* Rr, TS* D, const TS* Qq,
                                                      int64_t ld, double* rr, int* done) {
  const int j = blockIdx.x;
  __shared__ double red[256];
  __shared__ double sh_alpha, sh_beta;
  __shared__ int sh_go;
  if (done[j]) return;
  TS* x = X + (int64_t)j * ldx;
  TS* r = Rr + (int64_t)j * ld;
  TS* d = D + (int64_t)j * ld;
  const TS* q = Qq + (int64_t)j * ld;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < c; i += blockDim.x) s += (double)d[i] * (double)q[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double dq = red[0];
    sh_go = (dq > 0.0 && rr[j] > 0.0) ? 1 : 0;
    sh_alpha = sh_go ? rr[j] / dq : 0.0;
    if (!sh_go) done[j] = 1;
  }
  __syncthreads();
  if (!sh_go) return;
  const TS alpha = (TS)sh_alpha;
  double s2 = 0.0;
  for (int64_t i = threadIdx.x; i < c; i += blockDim.x) {
    x[i] += alpha * d[i];
    const TS ri = r[i] - alpha * q[i];
    r[i] = ri;
    s2 += (double)ri * (double)ri;
  }
  red[threadIdx.x] = s2;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sh_beta = rr[j] > 0.0 ? red[0] / rr[j] : 0.0;
    rr[j] = red[0];
  }
  __syncthreads();
  const TS beta = (TS)sh_beta;
  for (int64_t i = threadIdx.x; i < c; i += blockDim.x) d[i] = r[i] + beta * d[i];
}

// rr[j] = ||r_j||^2 and done[j] = 0, one CTA per column.
template <class TS>
__global__ void __launch_bounds__(256) cg_init_kernel(int64_t c, const TS* Rr, int64_t ld, double* rr, int* done) {
  const int j = blockIdx.x;
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < c; i += blockDim.x) {
    const double v = (double)Rr[i + (int64_t)j * ld];
    s += v * v;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    rr[j] = red[0];
    done[j] = 0;
  }
}

template <class TS>
__global__ void sub_mat_kernel(int64_t k, int64_t mb, const TS* A, int64_t lda, const TS* B, int64_t ldb, TS* C,
                               int64_t ldc, const int* active) {
  if (active && *active == 0) return;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= k * mb) return;
  const int64_t i = idx % k, j = idx / k;
  C[i + j * ldc] = A[i + j * lda] - B[i + j * ldb];
}

__global__ void fro_identity_kernel(int64_t m, const double* __restrict__ G, int64_t ldg, double* out) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int64_t e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int64_t i = e % m, j = e / m;
    const double d = (i == j ? 1.0 : 0.0) - G[i + j * ldg];
    s += d * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sqrt(red[0]);
}

__global__ void fro_diff_kernel(int64_t rows, int64_t cols, const double* __restrict__ A, int64_t lda,
                                const double* __restrict__ B, int64_t ldb, double* out_diff, double* out_a) {
  __shared__ double r1[1024], r2[1024];
  double s1 = 0.0, s2 = 0.0;
  for (int64_t e = threadIdx.x; e < rows * cols; e += blockDim.x) {
    const int64_t i = e % rows, j = e / rows;
    const double a = A[i + j * lda];
    const double d = a - B[i + j * ldb];
    s1 += d * d;
    s2 += a * a;
  }
  r1[threadIdx.x] = s1;
  r2[threadIdx.x] = s2;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      r1[threadIdx.x] += r1[threadIdx.x + h];
      r2[threadIdx.x] += r2[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *out_diff = sqrt(r1[0]);
    *out_a = sqrt(r2[0]);
  }
}


// ------------------------------------------------- Householder least squares --
// One panel of the Householder QR of the sketch S (the textbook least-squares
// solver of step 2, Sec. 3.1), one CTA.  B (k x w, ld ldb) holds Q_c^T S_i, the
// block's sketch after the c earlier reflectors; its rows c..k-1 (L = k - c)
// are factorised in place (the LAPACK reflector convention:
// H = I - tau v v^T, v(0) = 1, beta = -sign(alpha) ||x||).  Outputs:
//   V  (k x w, ld ldv): the reflectors written out, zero above row c + t and 1 at it;
//   T  (w x w, ld ldm): the panel's compact-WY factor, H_0 ... H_{w-1} = I - V T V^T
//      (T(t, t) = tau_t, T(0:t, t) = -tau_t T(0:t, 0:t) V(:, 0:t)^T v_t);
//   Ri (w x w, ld ldm): the inverse of the panel's R (upper, zero below).
// A zero or non-finite diagonal of R sets *flag |= 1.
// Dynamic shared memory: two 64 x 65 double arrays.
template <class TS>
__global__ void __launch_bounds__(512) hh_panel_kernel(int64_t k, int64_t c, int w, TS* B, int64_t ldb, TS* V,
                                                       int64_t ldv, TS* T, TS* Ri, int64_t ldm, int* flag) {
  extern __shared__ double hh_sm[];
  double(*Rs)[65] = reinterpret_cast<double(*)[65]>(hh_sm);            // R, then R^{-1}
  double(*G)[65] = reinterpret_cast<double(*)[65]>(hh_sm + 64 * 65);   // V^T V, then T
  __shared__ double red[16];
  __shared__ double wdot[64];
  __shared__ double tau_s[64];
  __shared__ double colv[64];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int64_t L = k - c;
  TS* A = B + c;
  for (int t = 0; t < w; ++t) {
    TS* x = A + (int64_t)t * ldb;
    double part = 0.0;
    for (int64_t r = t + 1 + tid; r < L; r += blockDim.x) {
      const double v = (double)x[r];
      part += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) red[warp] = part;
    __syncthreads();
    double sigma = 0.0;
    for (int q = 0; q < nw; ++q) sigma += red[q];
    const double alpha = (double)x[t];
    double beta = alpha, tau = 0.0, scale = 0.0;
    if (sigma > 0.0) {
      const double nrm = sqrt(alpha * alpha + sigma);
      beta = alpha >= 0.0 ? -nrm : nrm;
      tau = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    for (int64_t r = t + 1 + tid; r < L; r += blockDim.x) x[r] = (TS)((double)x[r] * scale);
    if (tid == 0) {
      tau_s[t] = tau;
      Rs[t][t] = beta;
    }
    __syncthreads();
    // w_j = v^T A(t:, j) for the later columns of the panel
    for (int j = t + 1 + warp; j < w; j += nw) {
      const TS* a = A + (int64_t)j * ldb;
      double d = 0.0;
      for (int64_t r = t + 1 + lane; r < L; r += 32) d += (double)x[r] * (double)a[r];
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      if (lane == 0) wdot[j] = d + (double)a[t];
    }
    __syncthreads();
    const int ncol = w - t - 1;
    const int64_t nrow = L - t;
    for (int64_t idx = tid; idx < nrow * ncol; idx += blockDim.x) {
      const int64_t r = t + idx % nrow;
      const int j = t + 1 + (int)(idx / nrow);
      const double v = r == t ? 1.0 : (double)x[r];
      TS* a = A + r + (int64_t)j * ldb;
      *a = (TS)((double)*a - tau * v * wdot[j]);
    }
    __syncthreads();
  }
  // R above the diagonal: row t is final once reflector t has been applied
  for (int idx = tid; idx < w * w; idx += blockDim.x) {
    const int i = idx % w, j = idx / w;
    if (i < j) Rs[i][j] = (double)A[i + (int64_t)j * ldb];
    else if (i > j) Rs[i][j] = 0.0;
  }
  // the reflectors written out
  for (int64_t idx = tid; idx < k * w; idx += blockDim.x) {
    const int64_t r = idx % k;
    const int t = (int)(idx / k);
    const int64_t rr = r - c;
    V[r + (int64_t)t * ldv] = rr < t ? (TS)0 : rr == t ? (TS)1 : A[rr + (int64_t)t * ldb];
  }
  // G(a, b) = v_a^T v_b, a < b (v_b is zero above row b and 1 at it)
  for (int idx = warp; idx < w * w; idx += nw) {
    const int a = idx % w, b = idx / w;
    if (a >= b) continue;
    double d = 0.0;
    for (int64_t r = b + 1 + lane; r < L; r += 32) d += (double)A[r + (int64_t)a * ldb] * (double)A[r + (int64_t)b * ldb];
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (lane == 0) G[a][b] = d + (double)A[b + (int64_t)a * ldb];
  }
  __syncthreads();
  if (tid == 0) {
    for (int t = 0; t < w; ++t) {
      const double d = Rs[t][t];
      if (!(d != 0.0) || !isfinite(d)) *flag |= 1;
    }
  }
  // T, column by column, in place of G (column t of G is read before it is overwritten)
  for (int t = 0; t < w; ++t) {
    if (tid < t) {
      double acc = 0.0;
      for (int q = tid; q < t; ++q) acc += G[tid][q] * G[q][t];  // G(tid, q), q < t, already holds T
      colv[tid] = -tau_s[t] * acc;
    }
    __syncthreads();
    if (tid < t) G[tid][t] = colv[tid];
    if (tid == t) G[t][t] = tau_s[t];
    __syncthreads();
  }
  // R^{-1} in place, column by column: Ri(i, j) = -(sum_{q = i+1..j} R(i, q) Ri(q, j)) / R(i, i)
  // with the columns < j already inverted; column j is computed into colv first
  for (int j = 0; j < w; ++j) {
    if (tid <= j) {
      const double rjj = 1.0 / Rs[j][j];
      double acc = 0.0;
      if (tid < j) {
        // y_i = sum_{q = i..j-1} Ri(i, q) R(q, j), then Ri(i, j) = -y_i / R(j, j)
        for (int q = tid; q < j; ++q) acc += Rs[tid][q] * Rs[q][j];
        colv[tid] = -acc * rjj;
      } else {
        colv[tid] = rjj;
      }
    }
    __syncthreads();
    if (tid <= j) Rs[tid][j] = colv[tid];
    __syncthreads();
  }
  for (int idx = tid; idx < w * w; idx += blockDim.x) {
    const int i = idx % w, j = idx / w;
    T[i + (int64_t)j * ldm] = i <= j ? (TS)G[i][j] : (TS)0;
    Ri[i + (int64_t)j * ldm] = i <= j ? (TS)Rs[i][j] : (TS)0;
  }
}

}  // namespace

thread_local int g_df_products = 0;

DfProducts::DfProducts(bool on) : prev(g_df_products) { g_df_products = on ? 1 : 0; }
DfProducts::~DfProducts() { g_df_products = prev; }

template <class TA, class TO, class TACC>
rbgs_status small_gemm(int trans, int64_t M, int64_t N, int64_t K, double alpha, const TA* A, int64_t lda,
                       const TA* B, int64_t ldb, double beta, TO* out, int64_t ldo, TACC* part, int64_t part_elems,
                       const int* active, cudaStream_t st) {
  if (N > SG_N || N < 0 || M < 0 || K < 0) return RBGS_EINVAL;
  if (M == 0 || N == 0) return RBGS_OK;
  const int64_t mt = (M + SG_T - 1) / SG_T;
  // about four 256-thread CTAs per SM (152 SMs), down to one K chunk per CTA
  int64_t ks = std::max<int64_t>(1, 4 * 152 / mt);
  ks = std::min<int64_t>(ks, std::max<int64_t>(1, (K + SG_K - 1) / SG_K));
  ks = std::min<int64_t>(ks, std::max<int64_t>(1, part_elems / (M * N)));
  if (ks * M * N > part_elems) return RBGS_EINVAL;
  int64_t kper = (K + ks - 1) / ks;
  kper = std::max<int64_t>(SG_K, (kper + SG_K - 1) / SG_K * SG_K);
  ks = std::max<int64_t>(1, (K + kper - 1) / kper);
  dim3 grid((unsigned)mt, (unsigned)ks);
  if constexpr (sizeof(TA) == 8 && sizeof(TACC) == 8) {
    if (g_df_products)
      small_gemm_part_df<<<grid, 256, 0, st>>>(trans, M, (int)N, K, kper, (const double*)A, lda, (const double*)B, ldb,
                                               (double*)part, active);
    else
      small_gemm_part<TA, TACC><<<grid, 256, 0, st>>>(trans, M, (int)N, K, kper, A, lda, B, ldb, part, active);
  } else {
    small_gemm_part<TA, TACC><<<grid, 256, 0, st>>>(trans, M, (int)N, K, kper, A, lda, B, ldb, part, active);
  }
  RBGS_LAUNCH_CHECK();
  const int64_t tot = M * N;
  small_gemm_reduce<TACC, TO><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(M, (int)N, (int)ks, part, alpha, beta,
                                                                            out, ldo, active);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}

#define INST_SG(TA, TO, TACC)                                                                                  \
  template rbgs_status small_gemm<TA, TO, TACC>(int, int64_t, int64_t, int64_t, double, const TA*, int64_t, \
                                                const TA*, int64_t, double, TO*, int64_t, TACC*, int64_t,   \
                                                const int*, cudaStream_t);
INST_SG(double, double, double)
INST_SG(float, float, float)
INST_SG(float, double, double)
#undef INST_SG

template <class T>
rbgs_status chol_inv(int mb, const T* G, T* R, T* Rinv, double shift, int* flag, const T* Rprev, const T* Rprev_inv,
                     const int* active, cudaStream_t st) {
  if (mb < 1 || mb > 64) return RBGS_EINVAL;
  const int smem = (int)(5 * 64 * 65 * sizeof(T));
  RBGS_CUDA_TRY(cudaFuncSetAttribute(chol_inv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  chol_inv_kernel<T><<<1, 256, smem, st>>>(mb, G, R, Rinv, shift, flag, Rprev, Rprev_inv, active);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}
template rbgs_status chol_inv<double>(int, const double*, double*, double*, double, int*, const double*,
                                      const double*, const int*, cudaStream_t);
template rbgs_status chol_inv<float>(int, const float*, float*, float*, double, int*, const float*, const float*,
                                     const int*, cudaStream_t);

template <class TS>
rbgs_status trmm_right_upper(int64_t k, int mb, const TS* A, int64_t lda, const TS* U, TS* Out, int64_t ldo,
                             const int* active, cudaStream_t st) {
  if (mb < 1 || mb > 64) return RBGS_EINVAL;
  if (k == 0) return RBGS_OK;
  const int64_t tot = k * mb;
  trmm_kernel<TS, TS><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(k, mb, A, lda, U, Out, ldo, active);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}
template rbgs_status trmm_right_upper<double>(int64_t, int, const double*, int64_t, const double*, double*, int64_t,
                                              const int*, cudaStream_t);
template rbgs_status trmm_right_upper<float>(int64_t, int, const float*, int64_t, const float*, float*, int64_t,
                                             const int*, cudaStream_t);

template <class T>
rbgs_status tri_mul(int mb, const T* A, const T* B, T* C, const int* active, cudaStream_t st) {
  tri_mul_kernel<T><<<1, 256, 0, st>>>(mb, A, B, C, active);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}
template rbgs_status tri_mul<double>(int, const double*, const double*, double*, const int*, cudaStream_t);
template rbgs_status tri_mul<float>(int, const float*, const float*, float*, const int*, cudaStream_t);

template <class TS, class TG>
rbgs_status assemble_g(int64_t c, int mb, const TS* Rc, int64_t ldrc, const TS* Rii, const TS* Riinv, TG* G,
                       int64_t ldg, double* R, int64_t ldr, const int* active, cudaStream_t st) {
  const int64_t tot = (c + mb) * mb;
  assemble_g_kernel<TS, TG><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(c, mb, Rc, ldrc, Rii, Riinv, G, ldg, R,
                                                                           ldr, active);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}
template rbgs_status assemble_g<double, double>(int64_t, int, const double*, int64_t, const double*, const double*,
                                                double*, int64_t, double*, int64_t, const int*, cudaStream_t);
template rbgs_status assemble_g<float, double>(int64_t, int, const float*, int64_t, const float*, const float*,
                                               double*, int64_t, double*, int64_t, const int*, cudaStream_t);
template rbgs_status assemble_g<float, float>(int64_t, int, const float*, int64_t, const float*, const float*,
                                              float*, int64_t, double*, int64_t, const int*, cudaStream_t);
template rbgs_status assemble_g<double, float>(int64_t, int, const double*, int64_t, const double*, const double*,
                                               float*, int64_t, double*, int64_t, const int*, cudaStream_t);

template <class TS>
rbgs_status reorth_update_r(int64_t c, int mb, const TS* R2c, int64_t ldr2, const TS* R2ii, double* Rcol,
                            int64_t ldr, double* tmp, const int* active, cudaStream_t st) {
  const int64_t tot = (c + mb) * mb;
  reorth_r_top<TS><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(c, mb, R2c, ldr2, R2ii, Rcol, ldr, tmp, active);
  RBGS_LAUNCH_CHECK();
  copy_diag_block<<<1, 256, 0, st>>>(c, mb, tmp, Rcol, ldr, active);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}
template rbgs_status reorth_update_r<double>(int64_t, int, const double*, int64_t, const double*, double*, int64_t,
                                             double*, const int*, cudaStream_t);
template rbgs_status reorth_update_r<float>(int64_t, int, const float*, int64_t, const float*, double*, int64_t,
                                            double*, const int*, cudaStream_t);

template <class TS>
rbgs_status reorth_decide(int64_t c, int mb, const TS* X, int64_t ldx, double tol, int mode, int* active, int* count,
                          int* blk_flag, cudaStream_t st) {
  reorth_decide_kernel<TS><<<1, 1024, 0, st>>>(c, mb, X, ldx, tol, mode, active, count, blk_flag);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}
template rbgs_status reorth_decide<double>(int64_t, int, const double*, int64_t, double, int, int*, int*, int*,
                                           cudaStream_t);
template rbgs_status reorth_decide<float>(int64_t, int, const float*, int64_t, double, int, int*, int*, int*,
                                          cudaStream_t);

template <class T>
rbgs_status round2_decide(int mb, const T* R1, const T* R1inv, T* R, T* Rinv, double thr, const int* active,
                          int* need2, int* count, cudaStream_t st) {
  if (mb < 1) return RBGS_EINVAL;
  round2_decide_kernel<T><<<1, 256, 0, st>>>(mb, R1, R1inv, R, Rinv, thr, active, need2, count);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}
template rbgs_status round2_decide<double>(int, const double*, const double*, double*, double*, double, const int*,
                                           int*, int*, cudaStream_t);
template rbgs_status round2_decide<float>(int, const float*, const float*, float*, float*, double, const int*,
                                          int*, int*, cudaStream_t);

template <class TS>
rbgs_status cg_init(int64_t c, int mb, const TS* Rr, int64_t ld, double* rr, int* done, cudaStream_t st) {
  cg_init_kernel<TS><<<mb, 256, 0, st>>>(c, Rr, ld, rr, done);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}
template <class TS>
rbgs_status cg_step(int64_t c, int mb, TS* X, int64_t ldx, TS* Rr, TS* D, const TS* Qq, int64_t ld, double* rr,
                    int* done, cudaStream_t st) {
  cg_step_kernel<TS><<<mb, 256, 0, st>>>(c, X, ldx, Rr, D, Qq, ld, rr, done);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}
template rbgs_status cg_init<double>(int64_t, int, const double*, int64_t, double*, int*, cudaStream_t);
template rbgs_status cg_init<float>(int64_t, int, const float*, int64_t, double*, int*, cudaStream_t);
template rbgs_status cg_step<double>(int64_t, int, double*, int64_t, double*, double*, const double*, int64_t,
                                     double*, int*, cudaStream_t);
template rbgs_status cg_step<float>(int64_t, int, float*, int64_t, float*, float*, const float*, int64_t, double*,
                                    int*, cudaStream_t);

template <class TS>
rbgs_status sub_mat(int64_t k, int64_t mb, const TS* A, int64_t lda, const TS* B, int64_t ldb, TS* C, int64_t ldc,
                    const int* active, cudaStream_t st) {
  const int64_t tot = k * mb;
  if (tot == 0) return RBGS_OK;
  sub_mat_kernel<TS><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(k, mb, A, lda, B, ldb, C, ldc, active);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}
template rbgs_status sub_mat<double>(int64_t, int64_t, const double*, int64_t, const double*, int64_t, double*,
                                     int64_t, const int*, cudaStream_t);
template rbgs_status sub_mat<float>(int64_t, int64_t, const float*, int64_t, const float*, int64_t, float*, int64_t,
                                    const int*, cudaStream_t);

rbgs_status fro_identity_defect(int64_t m, const double* G, int64_t ldg, double* out, cudaStream_t st) {
  fro_identity_kernel<<<1, 1024, 0, st>>>(m, G, ldg, out);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}

rbgs_status fro_norm_diff(int64_t rows, int64_t cols, const double* A, int64_t lda, const double* B, int64_t ldb,
                          double* out_diff, double* out_a, cudaStream_t st) {
  fro_diff_kernel<<<1, 1024, 0, st>>>(rows, cols, A, lda, B, ldb, out_diff, out_a);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}

template <class TS>
rbgs_status hh_panel(int64_t k, int64_t c, int w, TS* B, int64_t ldb, TS* V, int64_t ldv, TS* T, TS* Ri,
                     int64_t ldm, int* flag, cudaStream_t st) {
  if (w < 1 || w > 64 || k - c < w) return RBGS_EINVAL;
  const int smem = (int)(2 * 64 * 65 * sizeof(double));
  RBGS_CUDA_TRY(cudaFuncSetAttribute(hh_panel_kernel<TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  hh_panel_kernel<TS><<<1, 512, smem, st>>>(k, c, w, B, ldb, V, ldv, T, Ri, ldm, flag);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}
template rbgs_status hh_panel<double>(int64_t, int64_t, int, double*, int64_t, double*, int64_t, double*, double*,
                                      int64_t, int*, cudaStream_t);
template rbgs_status hh_panel<float>(int64_t, int64_t, int, float*, int64_t, float*, int64_t, float*, float*,
                                     int64_t, int*, cudaStream_t);

}  // namespace rbgs
