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
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.x * SG_T;
  const int split = blockIdx.y;
  const int64_t kb = (int64_t)split * kper;
  const int64_t ke = min(K, kb + kper);
  TACC acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[i][q] = 0;
  for (int64_t l0 = kb; l0 < ke; l0 += SG_K) {
    for (int e = tid; e < SG_K * SG_T; e += 256) {
      int il, ll;
      if (trans) { ll = e % SG_K; il = e / SG_K; }   // A is K x M: contiguous in l
      else { il = e % SG_T; ll = e / SG_T; }         // A is M x K: contiguous in i
      const int64_t gi = i0 + il, gl = l0 + ll;
      TACC v = 0;
      if (gi < M && gl < ke) v = (TACC)(trans ? A[gl + gi * lda] : A[gi + gl * lda]);
      As[ll][il] = v;
    }
    for (int e = tid; e < SG_K * SG_N; e += 256) {
      const int ll = e % SG_K, j = e / SG_K;
      const int64_t gl = l0 + ll;
      Bs[ll][j] = (gl < ke && j < N) ? (TACC)B[gl + (int64_t)j * ldb] : (TACC)0;
    }
    __syncthreads();
#pragma unroll
    for (int ll = 0; ll < SG_K; ++ll) {
      TACC a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[ll][ty + 16 * i];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = Bs[ll][tx + 16 * q];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] += a[i] * b[q];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t gi = i0 + ty + 16 * i;
      const int j = tx + 16 * q;
      if (gi < M && j < N) part[((int64_t)split * N + j) * M + gi] = acc[i][q];
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
  TACC s = 0;
  for (int p = 0; p < ks; ++p) s += part[((int64_t)p * N + j) * M + i];
  TO* o = out + i + j * ldo;
  const double v = alpha * (double)s;
  *o = (TO)(beta == 0.0 ? v : v + beta * (double)(*o));
}

// ---------------------------------------------------------------- Cholesky --
__global__ void chol_inv_kernel(int mb, const double* __restrict__ G, double* __restrict__ R,
                                double* __restrict__ Rinv, int* flag, const int* active) {
  if (active && *active == 0) return;
  __shared__ double Rs[64][65];
  const int t = threadIdx.x;  // column index l
  for (int e = t; e < mb * mb; e += blockDim.x) {
    const int i = e % mb, l = e / mb;
    Rs[i][l] = (i <= l) ? G[i + l * mb] : 0.0;
  }
  __syncthreads();
  int bad = 0;
  for (int j = 0; j < mb; ++j) {
    // pivot: d = G_jj - sum_{i<j} R_ij^2 (kept in Rs[j][j] as it is updated)
    if (t == 0) {
      double d = Rs[j][j];
      if (!(d > 0.0) || !isfinite(d)) {
        bad = 1;
        d = 1.0;
      }
      Rs[j][j] = sqrt(d);
    }
    __syncthreads();
    if (t > j && t < mb) Rs[j][t] /= Rs[j][j];
    __syncthreads();
    // trailing update: Rs[i][l] -= R_ji R_jl for j < i <= l
    for (int e = t; e < mb * mb; e += blockDim.x) {
      const int i = e % mb, l = e / mb;
      if (i > j && i <= l) Rs[i][l] -= Rs[j][i] * Rs[j][l];
    }
    __syncthreads();
  }
  if (t == 0 && bad && flag) atomicOr(flag, 1);
  for (int e = t; e < mb * mb; e += blockDim.x) {
    const int i = e % mb, l = e / mb;
    R[i + l * mb] = (i <= l) ? Rs[i][l] : 0.0;
  }
  // inverse of the upper factor: column l solves R x = e_l by back substitution
  if (t < mb) {
    const int l = t;
    double x[64];
#pragma unroll 1
    for (int i = mb - 1; i >= 0; --i) {
      double s = (i == l) ? 1.0 : 0.0;
      if (i <= l) {
        for (int q = i + 1; q <= l; ++q) s -= Rs[i][q] * x[q];
        x[i] = s / Rs[i][i];
      } else {
        x[i] = 0.0;
      }
    }
    for (int i = 0; i < mb; ++i) Rinv[i + l * mb] = x[i];
  }
}

template <class TS>
__global__ void trmm_kernel(int64_t k, int mb, TS* A, int64_t lda, const double* __restrict__ U,
                            const int* active) {
  if (active && *active == 0) return;
  __shared__ TS Us[64][64];
  for (int e = threadIdx.x; e < mb * mb; e += blockDim.x) {
    const int i = e % mb, l = e / mb;
    Us[i][l] = (TS)U[i + l * mb];
  }
  __syncthreads();
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= k) return;
  // in place, columns from the last: A[r][j] = sum_{i<=j} A[r][i] U[i][j]
  for (int j = mb - 1; j >= 0; --j) {
    TS s = 0;
    for (int i = 0; i <= j; ++i) s += A[r + i * lda] * Us[i][j];
    A[r + j * lda] = s;
  }
}

__global__ void tri_mul_kernel(int mb, const double* __restrict__ A, const double* __restrict__ B, double* C,
                               const int* active) {
  if (active && *active == 0) return;
  for (int e = threadIdx.x; e < mb * mb; e += blockDim.x) {
    const int i = e % mb, j = e / mb;
    double s = 0.0;
    for (int t = i; t <= j; ++t) s += A[i + t * mb] * B[t + j * mb];
    C[i + j * mb] = (i <= j) ? s : 0.0;
  }
}

template <class TS, class TG>
__global__ void assemble_g_kernel(int64_t c, int mb, const TS* __restrict__ Rc, int64_t ldrc,
                                  const double* __restrict__ Rii, const double* __restrict__ Riinv, TG* G,
                                  int64_t ldg, double* R, int64_t ldr, const int* active) {
  if (active && *active == 0) return;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t rows = c + mb;
  if (idx >= rows * mb) return;
  const int64_t i = idx % rows;
  const int j = (int)(idx / rows);
  double g;
  if (i < c) {
    double s = 0.0;
    for (int t = 0; t <= j; ++t) s += (double)Rc[i + t * ldrc] * Riinv[t + j * mb];
    g = -s;
    if (R) R[i + (int64_t)j * ldr] = (double)Rc[i + (int64_t)j * ldrc];
  } else {
    const int ii = (int)(i - c);
    g = (ii <= j) ? Riinv[ii + j * mb] : 0.0;
    if (R) R[i + (int64_t)j * ldr] = (ii <= j) ? Rii[ii + j * mb] : 0.0;
  }
  G[i + (int64_t)j * ldg] = (TG)g;
}

template <class TS>
__global__ void reorth_r_top(int64_t c, int mb, const TS* __restrict__ R2c, int64_t ldr2,
                             const double* __restrict__ R2ii, double* Rcol, int64_t ldr, double* tmp,
                             const int* active) {
  if (active && *active == 0) return;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t rows = c + mb;
  if (idx >= rows * mb) return;
  const int64_t i = idx % rows;
  const int j = (int)(idx / rows);
  const double* Rold = Rcol + c;  // R_ii (old) at rows c..c+mb-1
  if (i < c) {
    double s = 0.0;
    for (int t = 0; t <= j; ++t) s += (double)R2c[i + t * ldr2] * Rold[t + (int64_t)j * ldr];
    Rcol[i + (int64_t)j * ldr] += s;
  } else {
    const int ii = (int)(i - c);
    double s = 0.0;
    for (int t = ii; t <= j; ++t) s += R2ii[ii + t * mb] * Rold[t + (int64_t)j * ldr];
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
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t e = threadIdx.x; e < c * mb; e += blockDim.x) {
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

}  // namespace

template <class TA, class TO, class TACC>
rbgs_status small_gemm(int trans, int64_t M, int64_t N, int64_t K, double alpha, const TA* A, int64_t lda,
                       const TA* B, int64_t ldb, double beta, TO* out, int64_t ldo, TACC* part, int64_t part_elems,
                       const int* active, cudaStream_t st) {
  if (N > SG_N || N < 0 || M < 0 || K < 0) return RBGS_EINVAL;
  if (M == 0 || N == 0) return RBGS_OK;
  const int64_t mt = (M + SG_T - 1) / SG_T;
  int64_t ks = std::max<int64_t>(1, 2 * 152 / mt);
  ks = std::min<int64_t>(ks, std::max<int64_t>(1, (K + 63) / 64));
  ks = std::min<int64_t>(ks, std::max<int64_t>(1, part_elems / (M * N)));
  if (ks * M * N > part_elems) return RBGS_EINVAL;
  int64_t kper = (K + ks - 1) / ks;
  kper = std::max<int64_t>(SG_K, (kper + SG_K - 1) / SG_K * SG_K);
  ks = std::max<int64_t>(1, (K + kper - 1) / kper);
  dim3 grid((unsigned)mt, (unsigned)ks);
  small_gemm_part<TA, TACC><<<grid, 256, 0, st>>>(trans, M, (int)N, K, kper, A, lda, B, ldb, part, active);
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

rbgs_status chol_inv(int mb, const double* G, double* R, double* Rinv, int* flag, const int* active,
                     cudaStream_t st) {
  if (mb < 1 || mb > 64) return RBGS_EINVAL;
  chol_inv_kernel<<<1, 64, 0, st>>>(mb, G, R, Rinv, flag, active);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}

template <class TS>
rbgs_status trmm_right_upper(int64_t k, int mb, TS* A, int64_t lda, const double* U, const int* active,
                             cudaStream_t st) {
  if (mb < 1 || mb > 64) return RBGS_EINVAL;
  if (k == 0) return RBGS_OK;
  trmm_kernel<TS><<<(unsigned)((k + 127) / 128), 128, 0, st>>>(k, mb, A, lda, U, active);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}
template rbgs_status trmm_right_upper<double>(int64_t, int, double*, int64_t, const double*, const int*,
                                              cudaStream_t);
template rbgs_status trmm_right_upper<float>(int64_t, int, float*, int64_t, const double*, const int*, cudaStream_t);

rbgs_status tri_mul(int mb, const double* A, const double* B, double* C, const int* active, cudaStream_t st) {
  tri_mul_kernel<<<1, 256, 0, st>>>(mb, A, B, C, active);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}

template <class TS, class TG>
rbgs_status assemble_g(int64_t c, int mb, const TS* Rc, int64_t ldrc, const double* Rii, const double* Riinv, TG* G,
                       int64_t ldg, double* R, int64_t ldr, const int* active, cudaStream_t st) {
  const int64_t tot = (c + mb) * mb;
  assemble_g_kernel<TS, TG><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(c, mb, Rc, ldrc, Rii, Riinv, G, ldg, R,
                                                                           ldr, active);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}
template rbgs_status assemble_g<double, double>(int64_t, int, const double*, int64_t, const double*, const double*,
                                                double*, int64_t, double*, int64_t, const int*, cudaStream_t);
template rbgs_status assemble_g<float, double>(int64_t, int, const float*, int64_t, const double*, const double*,
                                               double*, int64_t, double*, int64_t, const int*, cudaStream_t);
template rbgs_status assemble_g<float, float>(int64_t, int, const float*, int64_t, const double*, const double*,
                                              float*, int64_t, double*, int64_t, const int*, cudaStream_t);

template <class TS>
rbgs_status reorth_update_r(int64_t c, int mb, const TS* R2c, int64_t ldr2, const double* R2ii, double* Rcol,
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
template rbgs_status reorth_update_r<float>(int64_t, int, const float*, int64_t, const double*, double*, int64_t,
                                            double*, const int*, cudaStream_t);

template <class TS>
rbgs_status reorth_decide(int64_t c, int mb, const TS* X, int64_t ldx, double tol, int mode, int* active, int* count,
                          int* blk_flag, cudaStream_t st) {
  reorth_decide_kernel<TS><<<1, 256, 0, st>>>(c, mb, X, ldx, tol, mode, active, count, blk_flag);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}
template rbgs_status reorth_decide<double>(int64_t, int, const double*, int64_t, double, int, int*, int*, int*,
                                           cudaStream_t);
template rbgs_status reorth_decide<float>(int64_t, int, const float*, int64_t, double, int, int*, int*, int*,
                                          cudaStream_t);

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

}  // namespace rbgs
