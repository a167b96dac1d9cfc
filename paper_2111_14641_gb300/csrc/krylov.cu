// Kernels of the randomized block Krylov methods (Sec. 5): the 5-point
// convection-diffusion operator applied to a block of columns, the residual
// block r = B - A X with its column norms, the casts between the FP64 solution
// and the Krylov basis precision, and the small FP64 projected problems of
// block GMRES (least squares with the block Hessenberg matrix, eq. GMRESsol)
// and block FOM (its square part, eq. RFOMsol).
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace rbgs {
namespace {

// (A x)_i at point i = (ix, iy) from its value c and its four neighbours
// (zero outside).  fc == null: A = -Laplace + b . grad, central differences
// (cx = 1/hx^2, cy = 1/hy^2, ax = bx / (2 hx), ay = by / (2 hy)).  fc != null:
// -div(a grad) with the face coefficients of RBGS_OP_DIFFUSION: x faces
// (nx+1) x (ny+2) then y faces (nx+2) x (ny+1); interior point (ix, iy) is
// node (ix+1, iy+1), its east face is x face (ix+1, iy+1), its west face
// (ix, iy+1), its north face y face (ix+1, iy+1), its south face (ix+1, iy).
__device__ __forceinline__ double op_point(int64_t nx, int64_t ny, double cx, double cy, double ax, double ay,
                                           const double* __restrict__ fc, int64_t ix, int64_t iy, double c, double w,
                                           double e, double s, double no) {
  if (!fc) return cx * (2.0 * c - w - e) + cy * (2.0 * c - s - no) + ax * (e - w) + ay * (no - s);
  const double* fx = fc;
  const double* fy = fc + (nx + 1) * (ny + 2);
  const double ae = fx[(ix + 1) + (nx + 1) * (iy + 1)], aw = fx[ix + (nx + 1) * (iy + 1)];
  const double an = fy[(ix + 1) + (nx + 2) * (iy + 1)], as = fy[(ix + 1) + (nx + 2) * iy];
  return cx * (ae * (c - e) + aw * (c - w)) + cy * (an * (c - no) + as * (c - s));
}

// Y = A X on nx x ny interior points of the unit square (spacing 1/(nx+1),
// 1/(ny+1)), zero Dirichlet boundary; point (x, y) is row x + nx y.  One
// thread per point and column.
template <class TI, class TO>
__global__ void stencil5_kernel(int64_t nx, int64_t ny, double cx, double cy, double ax, double ay,
                                const double* __restrict__ fc, const TI* __restrict__ X, int64_t ldx,
                                TO* __restrict__ Y, int64_t ldy) {
  const int64_t n = nx * ny;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t col = blockIdx.y;
  const TI* x = X + col * ldx;
  const int64_t ix = i % nx, iy = i / nx;
  const double c = (double)x[i];
  const double w = ix > 0 ? (double)x[i - 1] : 0.0;
  const double e = ix + 1 < nx ? (double)x[i + 1] : 0.0;
  const double s = iy > 0 ? (double)x[i - nx] : 0.0;
  const double no = iy + 1 < ny ? (double)x[i + nx] : 0.0;
  Y[i + col * ldy] = (TO)op_point(nx, ny, cx, cy, ax, ay, fc, ix, iy, c, w, e, s, no);
}

// The same operator on FP32 columns in double-FP32 arithmetic (the FP32 pipe;
// GB300's FP64 pipe bounded the FP64 form at a small fraction of the memory
// rate).  Each result is the FP32 rounding of a sum carried to about 2^-44 of
// its terms' magnitudes, as the FP64 form's is.  Constant coefficients
// (fc == null): y = k0 c + kw w + ke e + ks s + kn no with the five split
// coefficients k (the FP64 values of the FP64 form, split on the host).
// Face coefficients: y = sum over the four faces of (cx or cy) a_f (c - x_f),
// each difference exact as a TwoSum pair, each face product cx a_f a
// double-float.  Grid: x over rows of the grid, y over grid lines, z over
// columns (no integer division).
__global__ void __launch_bounds__(256) stencil5_df_kernel(int64_t nx, int64_t ny, float2 k0, float2 kw, float2 ke,
                                                          float2 ks, float2 kn, float2 cxs, float2 cys,
                                                          const double* __restrict__ fc, const float* __restrict__ X,
                                                          int64_t ldx, float* __restrict__ Y, int64_t ldy) {
  const int64_t ix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t iy = blockIdx.y;
  if (ix >= nx) return;
  const int64_t col = blockIdx.z;
  const float* x = X + col * ldx;
  const int64_t i = ix + nx * iy;
  const float c = x[i];
  const float w = ix > 0 ? x[i - 1] : 0.f;
  const float e = ix + 1 < nx ? x[i + 1] : 0.f;
  const float s = iy > 0 ? x[i - nx] : 0.f;
  const float no = iy + 1 < ny ? x[i + nx] : 0.f;
  float hi = 0.f, lo = 0.f;
  if (!fc) {
    df_fma(k0, c, hi, lo);
    df_fma(kw, w, hi, lo);
    df_fma(ke, e, hi, lo);
    df_fma(ks, s, hi, lo);
    df_fma(kn, no, hi, lo);
  } else {
    const double* fx = fc;
    const double* fy = fc + (nx + 1) * (ny + 2);
    const double af[4] = {fx[(ix + 1) + (nx + 1) * (iy + 1)], fx[ix + (nx + 1) * (iy + 1)],
                          fy[(ix + 1) + (nx + 2) * (iy + 1)], fy[(ix + 1) + (nx + 2) * iy]};
    const float xf[4] = {e, w, no, s};
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const float2 h = f < 2 ? cxs : cys;
      const float2 a = df_split(af[f]);
      // the face product h a as a double-float (p, q)
      const float p = h.x * a.x;
      float q = fmaf(h.x, a.x, -p);
      q = fmaf(h.x, a.y, q);
      q = fmaf(h.y, a.x, q);
      // the difference c - x_f exactly, (d, dl)
      float d, dl;
      df_two_sum(c, -xf[f], d, dl);
      // (p + q)(d + dl): p d exactly with its error, the cross terms into the error
      const float t = p * d;
      float te = fmaf(p, d, -t);
      te = fmaf(p, dl, te);
      te = fmaf(q, d, te);
      float sh, sl;
      df_two_sum(hi, t, sh, sl);
      hi = sh;
      lo += sl + te;
    }
  }
  Y[i + col * ldy] = hi + lo;
}

// Face coefficients of -div(a grad) (layout of RBGS_OP_DIFFUSION): harmonic
// means of the node values a ((nx+2) x (ny+2)).
__global__ void diffusion_faces_kernel(int64_t nx, int64_t ny, const double* __restrict__ a,
                                       double* __restrict__ fc) {
  const int64_t nfx = (nx + 1) * (ny + 2), nfy = (nx + 2) * (ny + 1);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nfx + nfy) return;
  double p, q;
  if (t < nfx) {
    const int64_t i = t % (nx + 1), j = t / (nx + 1);
    p = a[i + (nx + 2) * j];
    q = a[i + 1 + (nx + 2) * j];
  } else {
    const int64_t u = t - nfx;
    const int64_t i = u % (nx + 2), j = u / (nx + 2);
    p = a[i + (nx + 2) * j];
    q = a[i + (nx + 2) * (j + 1)];
  }
  fc[t] = 2.0 * p * q / (p + q);
}

// r = B - A X (FP64), and the partial sums of ||r_j||^2 per block of rows.
__global__ void residual_kernel(int64_t nx, int64_t ny, double cx, double cy, double ax, double ay,
                                const double* __restrict__ fc, const double* __restrict__ B, int64_t ldb,
                                const double* __restrict__ X, int64_t ldx, double* __restrict__ r, int64_t ldr,
                                double* __restrict__ part) {
  __shared__ double red[8];
  const int64_t n = nx * ny;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t col = blockIdx.y;
  double v = 0.0;
  if (i < n) {
    const double* x = X + col * ldx;
    const int64_t ix = i % nx, iy = i / nx;
    const double c = x[i];
    const double w = ix > 0 ? x[i - 1] : 0.0;
    const double e = ix + 1 < nx ? x[i + 1] : 0.0;
    const double s = iy > 0 ? x[i - nx] : 0.0;
    const double no = iy + 1 < ny ? x[i + nx] : 0.0;
    const double ax_i = op_point(nx, ny, cx, cy, ax, ay, fc, ix, iy, c, w, e, s, no);
    v = B[i + col * ldb] - ax_i;
    r[i + col * ldr] = v;
  }
  double sq = v * v;
#pragma unroll
  for (int o = 16; o; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[col * gridDim.x + blockIdx.x] = t;
  }
}

// Partial sums of ||A_j||^2 per block of 256 rows.
__global__ void sqnorm_part_kernel(int64_t n, const double* __restrict__ A, int64_t lda, double* __restrict__ part) {
  __shared__ double red[8];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t col = blockIdx.y;
  const double v = i < n ? A[i + col * lda] : 0.0;
  double sq = v * v;
#pragma unroll
  for (int o = 16; o; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[col * gridDim.x + blockIdx.x] = t;
  }
}

// norms[j] = sqrt(sum of part[j, :]) (one warp per column, fixed order).
__global__ void colnorm_finish_kernel(int64_t ncols, int nparts, const double* __restrict__ part,
                                      double* __restrict__ norms) {
  const int col = blockIdx.x;
  double s = 0.0;
  for (int t = threadIdx.x; t < nparts; t += 32) s += part[(int64_t)col * nparts + t];
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) norms[col] = sqrt(s);
}

template <class TI, class TO>
__global__ void cast_cols_kernel(int64_t n, int64_t ncols, const TI* __restrict__ A, int64_t lda,
                                 TO* __restrict__ B, int64_t ldb) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * ncols) return;
  const int64_t i = idx % n, j = idx / n;
  B[i + j * ldb] = (TO)A[i + j * lda];
}

template <class TD>
__global__ void add_cols_kernel(int64_t n, int64_t ncols, const TD* __restrict__ D, int64_t ldd,
                                double* __restrict__ X, int64_t ldx) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * ncols) return;
  const int64_t i = idx % n, j = idx / n;
  X[i + j * ldx] += (double)D[i + j * ldd];
}

// min || H z - F || for H (M x N, M >= N, zero below its bw-th subdiagonal)
// and nrhs right sides, by Householder reflectors of at most bw + 1 rows;
// H and F are overwritten (in global memory, L2-resident), Z = the solution
// (N x nrhs).  One CTA: the columns are sequential, the updates of one
// reflector are spread over the threads; the back substitution runs one warp
// per right side.  *flag gets 1 on a zero pivot.
__global__ void __launch_bounds__(256) banded_ls_kernel(int M, int N, int bw, double* __restrict__ H, int ldh,
                                                        double* __restrict__ F, int ldf, int nrhs,
                                                        double* __restrict__ Z, int ldz, int* flag) {
  __shared__ double v[72];
  __shared__ double beta_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int j = 0; j < N; ++j) {
    const int L = min(bw + 1, M - j);
    if (warp == 0) {
      double ss = 0.0;
      for (int t = lane; t < L; t += 32) {
        const double a = H[j + t + (int64_t)j * ldh];
        v[t] = a;
        ss += a * a;
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      __syncwarp();
      if (lane == 0) {
        const double nrm = sqrt(ss);
        const double a0 = v[0];
        if (nrm == 0.0) {
          beta_s = 0.0;  // nothing to eliminate
        } else {
          const double alpha = a0 >= 0.0 ? -nrm : nrm;
          v[0] = a0 - alpha;
          const double vtv = ss - a0 * a0 + v[0] * v[0];
          beta_s = vtv > 0.0 ? 2.0 / vtv : 0.0;
          H[j + (int64_t)j * ldh] = alpha;
        }
      }
    }
    __syncthreads();
    const double beta = beta_s;
    if (beta != 0.0) {
      // columns j+1..N-1 of H and the right sides
      const int ncol = (N - j - 1) + nrhs;
      for (int q = tid; q < ncol; q += blockDim.x) {
        double* col = q < N - j - 1 ? H + (int64_t)(j + 1 + q) * ldh : F + (int64_t)(q - (N - j - 1)) * ldf;
        double w = 0.0;
        for (int t = 0; t < L; ++t) w += v[t] * col[j + t];
        w *= beta;
        for (int t = 0; t < L; ++t) col[j + t] -= w * v[t];
      }
      for (int t = 1 + tid; t < L; t += blockDim.x) H[j + t + (int64_t)j * ldh] = 0.0;
    }
    __syncthreads();
  }
  // back substitution, one warp per right side
  for (int r = warp; r < nrhs; r += blockDim.x >> 5) {
    for (int i = N - 1; i >= 0; --i) {
      double s = 0.0;
      for (int t = i + 1 + lane; t < N; t += 32) s += H[i + (int64_t)t * ldh] * Z[t + (int64_t)r * ldz];
#pragma unroll
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) {
        const double d = H[i + (int64_t)i * ldh];
        if (d == 0.0 || !isfinite(d)) {
          atomicOr(flag, 1);
          Z[i + (int64_t)r * ldz] = 0.0;
        } else {
          Z[i + (int64_t)r * ldz] = (F[i + (int64_t)r * ldf] - s) / d;
        }
      }
      __syncwarp();
    }
  }
}

void stencil_coeffs(const rbgs_op& op, double& cx, double& cy, double& ax, double& ay) {
  const double hx = 1.0 / (double)(op.nx + 1), hy = 1.0 / (double)(op.ny + 1);
  cx = 1.0 / (hx * hx);
  cy = 1.0 / (hy * hy);
  const bool diff = op.kind == RBGS_OP_DIFFUSION;
  ax = diff ? 0.0 : op.bx / (2.0 * hx);
  ay = diff ? 0.0 : op.by / (2.0 * hy);
}

const double* op_faces(const rbgs_op& op) { return op.kind == RBGS_OP_DIFFUSION ? op.coef : nullptr; }

}  // namespace

template <class TI, class TO>
rbgs_status stencil_apply_t(const rbgs_op& op, const TI* X, int64_t ldx, int64_t ncols, TO* Y, int64_t ldy,
                            cudaStream_t st) {
  const int64_t n = op.nx * op.ny;
  if (ncols == 0 || n == 0) return RBGS_OK;
  double cx, cy, ax, ay;
  stencil_coeffs(op, cx, cy, ax, ay);
  if constexpr (sizeof(TI) == 4 && sizeof(TO) == 4) {
    if (op.ny <= 65535 && ncols <= 65535) {
      auto split = [](double v) {
        const float hi = (float)v;
        return make_float2(hi, (float)(v - (double)hi));
      };
      dim3 grid((unsigned)((op.nx + 255) / 256), (unsigned)op.ny, (unsigned)ncols);
      stencil5_df_kernel<<<grid, 256, 0, st>>>(op.nx, op.ny, split(2.0 * cx + 2.0 * cy), split(-cx - ax),
                                               split(-cx + ax), split(-cy - ay), split(-cy + ay), split(cx),
                                               split(cy), op_faces(op), (const float*)X, ldx, (float*)Y, ldy);
      RBGS_LAUNCH_CHECK();
      return RBGS_OK;
    }
  }
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)ncols);
  stencil5_kernel<TI, TO><<<grid, 256, 0, st>>>(op.nx, op.ny, cx, cy, ax, ay, op_faces(op), X, ldx, Y, ldy);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}
template rbgs_status stencil_apply_t<double, double>(const rbgs_op&, const double*, int64_t, int64_t, double*,
                                                     int64_t, cudaStream_t);
template rbgs_status stencil_apply_t<float, float>(const rbgs_op&, const float*, int64_t, int64_t, float*, int64_t,
                                                   cudaStream_t);

size_t residual_part_elems(int64_t n, int64_t ncols) { return (size_t)((n + 255) / 256) * (size_t)ncols; }

rbgs_status residual_t(const rbgs_op& op, const double* B, int64_t ldb, const double* X, int64_t ldx,
                       int64_t ncols, double* r, int64_t ldr, double* part, double* norms, cudaStream_t st) {
  const int64_t n = op.nx * op.ny;
  double cx, cy, ax, ay;
  stencil_coeffs(op, cx, cy, ax, ay);
  const unsigned nb = (unsigned)((n + 255) / 256);
  residual_kernel<<<dim3(nb, (unsigned)ncols), 256, 0, st>>>(op.nx, op.ny, cx, cy, ax, ay, op_faces(op), B, ldb, X,
                                                              ldx, r, ldr, part);
  RBGS_LAUNCH_CHECK();
  colnorm_finish_kernel<<<(unsigned)ncols, 32, 0, st>>>(ncols, (int)nb, part, norms);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}

rbgs_status colnorms_t(int64_t n, int64_t ncols, const double* A, int64_t lda, double* part, double* norms,
                       cudaStream_t st) {
  const unsigned nb = (unsigned)((n + 255) / 256);
  sqnorm_part_kernel<<<dim3(nb, (unsigned)ncols), 256, 0, st>>>(n, A, lda, part);
  RBGS_LAUNCH_CHECK();
  colnorm_finish_kernel<<<(unsigned)ncols, 32, 0, st>>>(ncols, (int)nb, part, norms);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}

template <class TI, class TO>
rbgs_status cast_cols_t(int64_t n, int64_t ncols, const TI* A, int64_t lda, TO* B, int64_t ldb, cudaStream_t st) {
  const int64_t tot = n * ncols;
  if (tot == 0) return RBGS_OK;
  cast_cols_kernel<TI, TO><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, ncols, A, lda, B, ldb);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}
template rbgs_status cast_cols_t<double, float>(int64_t, int64_t, const double*, int64_t, float*, int64_t,
                                                cudaStream_t);
template rbgs_status cast_cols_t<double, double>(int64_t, int64_t, const double*, int64_t, double*, int64_t,
                                                 cudaStream_t);
template rbgs_status cast_cols_t<float, double>(int64_t, int64_t, const float*, int64_t, double*, int64_t,
                                                cudaStream_t);

template <class TD>
rbgs_status add_cols_t(int64_t n, int64_t ncols, const TD* D, int64_t ldd, double* X, int64_t ldx, cudaStream_t st) {
  const int64_t tot = n * ncols;
  if (tot == 0) return RBGS_OK;
  add_cols_kernel<TD><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, ncols, D, ldd, X, ldx);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}
template rbgs_status add_cols_t<float>(int64_t, int64_t, const float*, int64_t, double*, int64_t, cudaStream_t);
template rbgs_status add_cols_t<double>(int64_t, int64_t, const double*, int64_t, double*, int64_t, cudaStream_t);

rbgs_status diffusion_faces(int64_t nx, int64_t ny, const double* a, double* fc, cudaStream_t st) {
  const int64_t tot = (nx + 1) * (ny + 2) + (nx + 2) * (ny + 1);
  diffusion_faces_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(nx, ny, a, fc);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}

rbgs_status banded_ls(int M, int N, int bw, double* H, int ldh, double* F, int ldf, int nrhs, double* Z, int ldz,
                      int* flag, cudaStream_t st) {
  if (N < 1 || M < N || bw < 0 || bw + 1 > 72 || nrhs < 1) return RBGS_EINVAL;
  banded_ls_kernel<<<1, 256, 0, st>>>(M, N, bw, H, ldh, F, ldf, nrhs, Z, ldz, flag);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}

}  // namespace rbgs
