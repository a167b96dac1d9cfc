// Extreme eigenpairs of the projected matrix of the randomized Rayleigh-Ritz
// method (Alg. 8, Sec. 5.4 of Balabanov & Grigori, arXiv 2111.14641).
//
// H_(1:p-1,1:p-1) is a small dense non-symmetric FP64 matrix (N = (p-1) m_p
// <= 1024).  One CTA computes, in FP64:
//   1. its Hessenberg form by Householder reflections (the reflectors are kept
//      below the subdiagonal);
//   2. all its eigenvalues by the implicit double-shift (Francis) QR iteration
//      with deflation, updating only the active window (eigenvalues only);
//   3. the m_p extreme ones (largest or smallest real part);
//   4. their eigenvectors by two steps of inverse iteration with the
//      Hessenberg matrix (complex arithmetic, partial pivoting), mapped back
//      through the reflectors;
//   5. a real basis Y of those eigenvectors, the residual estimates
//      ||H_(p,1:p-1) y|| of step 3 of Alg. 8, and the Ritz values.
// The selection and scaling follow fixed conventions: order by real part
// (ties: positive imaginary part first, each conjugate pair once); each
// eigenvector has unit 2-norm and its first largest-modulus entry real and
// positive; a real eigenvalue takes one column y, a pair a +- ib the columns
// Re y and Im y (Re y alone if one slot is left).
// The QR iteration stops after 30 N sweeps at most; the kernel then reports
// RBGS_ENOCONV through its status word.  Every loop is bounded.
#include <cfloat>

#include "common.cuh"
#include "internal.h"

namespace rbgs {
namespace {

constexpr int kEigThreads = 256;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  // Smith's algorithm
  if (fabs(b.x) >= fabs(b.y)) {
    const double r = b.y / b.x, d = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  }
  const double r = b.x / b.y, d = b.x * r + b.y;
  return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}
__device__ __forceinline__ double cabs2(double2 a) { return hypot(a.x, a.y); }

// Sum over the CTA (red: 32 doubles of shared memory); every thread gets it.
__device__ double cta_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = lane < nw ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

struct EigArgs {
  int N, mb, mp, which;
  const double* H;  // (N + mb) x N, ld ldh: rows N.. are H_(p,1:p-1)
  int64_t ldh;
  double* A;    // N x N scratch: Hessenberg form + reflectors
  double* W;    // N x N scratch: QR iteration
  double2* L;   // N x N scratch: complex LU
  double* vals;   // 2 mp: re, im per column
  double* Y;      // N x mp (ld N)
  double* resid;  // mp
  int* status;    // 0 ok, 1 no convergence
};

__global__ void __launch_bounds__(kEigThreads) ritz_eig_kernel(EigArgs a) {
  extern __shared__ __align__(16) unsigned char eig_smem[];
  const int N = a.N, tid = threadIdx.x, T = blockDim.x;
  double* v = reinterpret_cast<double*>(eig_smem);  // N
  double* tau = v + N;                               // N
  double* wr = tau + N;                              // N
  double* wi = wr + N;                               // N
  double2* z = reinterpret_cast<double2*>(wi + N);   // N
  double2* mul = z + N;                              // N
  int* swp = reinterpret_cast<int*>(mul + N);        // N
  __shared__ double red[33];
  __shared__ double hv[3], hbeta, sh_x, sh_y, sh_z, sh_anorm;
  __shared__ int sh_l, sh_u, sh_state, sh_nr;
  __shared__ int sel[64], selpair[64], sh_nsel;
  double* A = a.A;
  double* W = a.W;
  double2* L = a.L;
  const int64_t ldn = N;
  auto AT = [&](int i, int j) -> double& { return A[i + j * ldn]; };
  auto WT = [&](int i, int j) -> double& { return W[i + j * ldn]; };

  // ---- 1. Hessenberg reduction of A = H_(1:p-1,1:p-1)
  for (int64_t e = tid; e < (int64_t)N * N; e += T) A[e] = a.H[(e % N) + (e / N) * a.ldh];
  for (int i = tid; i < N; i += T) tau[i] = 0.0;
  __syncthreads();
  for (int j = 0; j + 2 < N; ++j) {
    const int len = N - j - 1;
    double part = 0.0;
    for (int i = 1 + tid; i < len; i += T) {
      const double x = AT(j + 1 + i, j);
      part += x * x;
    }
    const double rest = cta_sum(part, red);
    if (rest == 0.0) continue;  // the column is already in Hessenberg form (tau_j = 0)
    const double x0 = AT(j + 1, j);
    const double sigma = sqrt(x0 * x0 + rest);
    const double alpha = x0 >= 0.0 ? -sigma : sigma;
    const double v0 = x0 - alpha;
    const double tj = (alpha - x0) / alpha;
    for (int i = tid; i < len; i += T) v[i] = i == 0 ? 1.0 : AT(j + 1 + i, j) / v0;
    __syncthreads();
    // from the left, columns j+1 .. N-1
    for (int c = j + 1 + tid; c < N; c += T) {
      double d = 0.0;
      for (int i = 0; i < len; ++i) d += v[i] * AT(j + 1 + i, c);
      d *= tj;
      for (int i = 0; i < len; ++i) AT(j + 1 + i, c) -= d * v[i];
    }
    __syncthreads();
    // from the right, every row
    for (int r = tid; r < N; r += T) {
      double d = 0.0;
      for (int i = 0; i < len; ++i) d += AT(r, j + 1 + i) * v[i];
      d *= tj;
      for (int i = 0; i < len; ++i) AT(r, j + 1 + i) -= d * v[i];
    }
    __syncthreads();
    for (int i = tid; i < len; i += T) AT(j + 1 + i, j) = i == 0 ? alpha : v[i];
    if (tid == 0) tau[j] = tj;
    __syncthreads();
  }
  // the work copy: the upper Hessenberg part; and a norm for the tests
  double part = 0.0;
  for (int64_t e = tid; e < (int64_t)N * N; e += T) {
    const int i = (int)(e % N), j = (int)(e / N);
    const double x = i <= j + 1 ? A[e] : 0.0;
    W[e] = x;
    part += fabs(x);
  }
  const double anorm_sum = cta_sum(part, red);
  if (tid == 0) sh_anorm = anorm_sum > 0.0 ? anorm_sum : 1.0;
  __syncthreads();
  const double anorm = sh_anorm;

  // ---- 2. eigenvalues: implicit double-shift QR on the active window [l, u]
  const int maxit = 30 * N;
  int its = 0, total = 0;  // kept by thread 0
  if (tid == 0) sh_u = N - 1;
  for (;;) {
    __syncthreads();
    if (tid == 0) {
      int u = sh_u, l = 0, state = 0;
      while (u >= 0) {
        l = 0;
        for (int i = u; i >= 1; --i) {
          double tst = fabs(WT(i - 1, i - 1)) + fabs(WT(i, i));
          if (tst == 0.0) tst = anorm;
          if (fabs(WT(i, i - 1)) <= DBL_EPSILON * tst) {
            WT(i, i - 1) = 0.0;
            l = i;
            break;
          }
        }
        if (l == u) {
          wr[u] = WT(u, u);
          wi[u] = 0.0;
          u -= 1;
          its = 0;
          continue;
        }
        if (l == u - 1) {
          const double p00 = WT(u - 1, u - 1), p01 = WT(u - 1, u), p10 = WT(u, u - 1), p11 = WT(u, u);
          const double hp = 0.5 * (p00 - p11), disc = hp * hp + p01 * p10;
          if (disc >= 0.0) {
            const double zz = hp + (hp >= 0.0 ? sqrt(disc) : -sqrt(disc));
            wr[u - 1] = p11 + zz;
            wr[u] = zz != 0.0 ? p11 - p01 * p10 / zz : p11;
            wi[u - 1] = wi[u] = 0.0;
          } else {
            const double re = p11 + hp, im = sqrt(-disc);
            wr[u - 1] = wr[u] = re;
            wi[u - 1] = im;
            wi[u] = -im;
          }
          u -= 2;
          its = 0;
          continue;
        }
        break;
      }
      if (u < 0) {
        state = 1;
      } else if (total >= maxit) {
        state = 2;
      } else {
        ++its;
        ++total;
        double s, t;
        if (its % 10 == 0) {  // exceptional shift after 10 and 20 sweeps without deflation
          const double sg = fabs(WT(u, u - 1)) + fabs(WT(u - 1, u - 2));
          s = 1.5 * sg;
          t = sg * sg;
        } else {
          s = WT(u - 1, u - 1) + WT(u, u);
          t = WT(u - 1, u - 1) * WT(u, u) - WT(u - 1, u) * WT(u, u - 1);
        }
        const double h00 = WT(l, l), h01 = WT(l, l + 1), h10 = WT(l + 1, l), h11 = WT(l + 1, l + 1);
        sh_x = h00 * h00 + h01 * h10 - s * h00 + t;
        sh_y = h10 * (h00 + h11 - s);
        sh_z = h10 * WT(l + 2, l + 1);
      }
      sh_u = u;
      sh_l = l;
      sh_state = state;
    }
    __syncthreads();
    if (sh_state != 0) break;
    const int l = sh_l, u = sh_u;
    for (int k = l; k <= u - 1; ++k) {
      if (tid == 0) {
        double x, y, zz;
        const int nr = (k + 2 <= u) ? 3 : 2;
        if (k == l) {
          x = sh_x;
          y = sh_y;
          zz = nr == 3 ? sh_z : 0.0;
        } else {
          x = WT(k, k - 1);
          y = WT(k + 1, k - 1);
          zz = nr == 3 ? WT(k + 2, k - 1) : 0.0;
        }
        const double sc = fabs(x) + fabs(y) + fabs(zz);
        if (sc == 0.0) {
          hbeta = 0.0;
        } else {
          x /= sc;
          y /= sc;
          zz /= sc;
          const double sg = sqrt(x * x + y * y + zz * zz);
          const double al = x >= 0.0 ? -sg : sg;
          hv[0] = x - al;
          hv[1] = y;
          hv[2] = zz;
          hbeta = 1.0 / (sg * (sg + fabs(x)));
        }
        sh_nr = nr;
      }
      __syncthreads();
      const double beta = hbeta;
      if (beta != 0.0) {
        const int nr = sh_nr;
        const double v0 = hv[0], v1 = hv[1], v2 = nr == 3 ? hv[2] : 0.0;
        const int c0 = k - 1 > l ? k - 1 : l;
        for (int c = c0 + tid; c <= u; c += T) {
          double d = v0 * WT(k, c) + v1 * WT(k + 1, c);
          if (nr == 3) d += v2 * WT(k + 2, c);
          d *= beta;
          WT(k, c) -= d * v0;
          WT(k + 1, c) -= d * v1;
          if (nr == 3) WT(k + 2, c) -= d * v2;
        }
        __syncthreads();
        const int r1 = k + 3 < u ? k + 3 : u;
        for (int r = l + tid; r <= r1; r += T) {
          double d = WT(r, k) * v0 + WT(r, k + 1) * v1;
          if (nr == 3) d += WT(r, k + 2) * v2;
          d *= beta;
          WT(r, k) -= d * v0;
          WT(r, k + 1) -= d * v1;
          if (nr == 3) WT(r, k + 2) -= d * v2;
        }
      }
      __syncthreads();
    }
  }
  if (sh_state == 2) {
    if (tid == 0) *a.status = 1;
    return;
  }

  // ---- 3. the m_p extreme eigenvalues (each conjugate pair once)
  if (tid == 0) {
    int col = 0, ns = 0;
    for (int guard = 0; guard < N && col < a.mp; ++guard) {
      int best = -1;
      for (int i = 0; i < N; ++i) {
        if (wi[i] < 0.0 || wi[i] != wi[i]) continue;
        bool taken = false;
        for (int q = 0; q < ns; ++q) taken |= sel[q] == i;
        if (taken) continue;
        if (best < 0) {
          best = i;
          continue;
        }
        const double kb = a.which == 0 ? -wr[best] : wr[best], ki = a.which == 0 ? -wr[i] : wr[i];
        if (ki < kb || (ki == kb && wi[i] > wi[best])) best = i;
      }
      if (best < 0) break;
      sel[ns] = best;
      selpair[ns] = (wi[best] > 0.0 && col + 1 < a.mp) ? 1 : 0;
      col += 1 + selpair[ns];
      ++ns;
    }
    sh_nsel = ns;
  }
  __syncthreads();

  // ---- 4-5. eigenvectors by inverse iteration, mapped back, scaled; Y, values, residuals
  int col = 0;
  for (int q = 0; q < sh_nsel; ++q) {
    const double2 mu = make_double2(wr[sel[q]], wi[sel[q]]);
    // L = Hessenberg(A) - mu I
    for (int64_t e = tid; e < (int64_t)N * N; e += T) {
      const int i = (int)(e % N), j = (int)(e / N);
      double re = i <= j + 1 ? A[e] : 0.0, im = 0.0;
      if (i == j) {
        re -= mu.x;
        im = -mu.y;
      }
      L[e] = make_double2(re, im);
    }
    __syncthreads();
    const double tiny = DBL_EPSILON * anorm;
    for (int k = 0; k + 1 < N; ++k) {
      if (tid == 0) {
        double2 p = L[k + k * ldn], b = L[(k + 1) + k * ldn];
        const int s = cabs2(b) > cabs2(p) ? 1 : 0;
        if (s) {
          const double2 t = p;
          p = b;
          b = t;
        }
        if (cabs2(p) == 0.0) p = make_double2(tiny, 0.0);
        L[k + k * ldn] = p;
        L[(k + 1) + k * ldn] = make_double2(0.0, 0.0);
        swp[k] = s;
        mul[k] = cdiv(b, p);
      }
      __syncthreads();
      const int s = swp[k];
      const double2 m = mul[k];
      for (int c = k + 1 + tid; c < N; c += T) {
        double2 top = L[k + c * ldn], bot = L[(k + 1) + c * ldn];
        if (s) {
          const double2 t = top;
          top = bot;
          bot = t;
        }
        const double2 mt = cmul(m, top);
        L[k + c * ldn] = top;
        L[(k + 1) + c * ldn] = make_double2(bot.x - mt.x, bot.y - mt.y);
      }
      __syncthreads();
    }
    if (tid == 0 && cabs2(L[(N - 1) + (N - 1) * ldn]) == 0.0) L[(N - 1) + (N - 1) * ldn] = make_double2(tiny, 0.0);
    for (int i = tid; i < N; i += T) z[i] = make_double2(1.0 + 0.25 * (double)(i % 3), 0.0);
    __syncthreads();
    for (int sweep = 0; sweep < 2; ++sweep) {
      if (tid == 0) {  // forward elimination of the right-hand side
        for (int k = 0; k + 1 < N; ++k) {
          if (swp[k]) {
            const double2 t = z[k];
            z[k] = z[k + 1];
            z[k + 1] = t;
          }
          const double2 mt = cmul(mul[k], z[k]);
          z[k + 1] = make_double2(z[k + 1].x - mt.x, z[k + 1].y - mt.y);
        }
      }
      __syncthreads();
      for (int i = N - 1; i >= 0; --i) {  // back substitution, column by column
        if (tid == 0) z[i] = cdiv(z[i], L[i + i * ldn]);
        __syncthreads();
        const double2 zi = z[i];
        for (int r = tid; r < i; r += T) {
          const double2 t = cmul(L[r + i * ldn], zi);
          z[r] = make_double2(z[r].x - t.x, z[r].y - t.y);
        }
        __syncthreads();
      }
      double pn = 0.0;
      for (int i = tid; i < N; i += T) pn += z[i].x * z[i].x + z[i].y * z[i].y;
      const double nrm = sqrt(cta_sum(pn, red));
      const double sc = nrm > 0.0 ? 1.0 / nrm : 1.0;
      for (int i = tid; i < N; i += T) z[i] = make_double2(z[i].x * sc, z[i].y * sc);
      __syncthreads();
    }
    // back through the reflectors: y = P_0 P_1 ... P_(N-3) z
    for (int j = N - 3; j >= 0; --j) {
      const double tj = tau[j];
      if (tj == 0.0) continue;  // uniform across the CTA
      const int len = N - j - 1;
      double dr = 0.0, di = 0.0;
      for (int i = tid; i < len; i += T) {
        const double vi = i == 0 ? 1.0 : AT(j + 1 + i, j);
        dr += vi * z[j + 1 + i].x;
        di += vi * z[j + 1 + i].y;
      }
      dr = cta_sum(dr, red) * tj;
      di = cta_sum(di, red) * tj;
      for (int i = tid; i < len; i += T) {
        const double vi = i == 0 ? 1.0 : AT(j + 1 + i, j);
        z[j + 1 + i] = make_double2(z[j + 1 + i].x - dr * vi, z[j + 1 + i].y - di * vi);
      }
      __syncthreads();
    }
    // unit 2-norm, first largest-modulus entry real and positive
    double pn = 0.0;
    for (int i = tid; i < N; i += T) pn += z[i].x * z[i].x + z[i].y * z[i].y;
    const double nrm = sqrt(cta_sum(pn, red));
    if (tid == 0) {
      int im = 0;
      double best = -1.0;
      for (int i = 0; i < N; ++i) {
        const double m = z[i].x * z[i].x + z[i].y * z[i].y;
        if (m > best) {
          best = m;
          im = i;
        }
      }
      const double mag = sqrt(best);
      // multiply by conj(z_im) / (|z_im| nrm)
      const double inv = (mag > 0.0 && nrm > 0.0) ? 1.0 / (mag * nrm) : 1.0;
      hv[0] = z[im].x * inv;
      hv[1] = -z[im].y * inv;
    }
    __syncthreads();
    const double2 ph = make_double2(hv[0], hv[1]);
    for (int i = tid; i < N; i += T) z[i] = cmul(z[i], ph);
    __syncthreads();
    // residual estimate ||H_(p,1:p-1) y||
    double rs = 0.0;
    for (int r = 0; r < a.mb; ++r) {
      double pr = 0.0, pi = 0.0;
      for (int c = tid; c < N; c += T) {
        const double h = a.H[(N + r) + (int64_t)c * a.ldh];
        pr += h * z[c].x;
        pi += h * z[c].y;
      }
      pr = cta_sum(pr, red);
      pi = cta_sum(pi, red);
      rs += pr * pr + pi * pi;
    }
    rs = sqrt(rs);
    for (int i = tid; i < N; i += T) a.Y[i + (int64_t)col * N] = z[i].x;
    if (tid == 0) {
      a.vals[2 * col] = mu.x;
      a.vals[2 * col + 1] = mu.y;
      a.resid[col] = rs;
    }
    ++col;
    if (selpair[q]) {
      for (int i = tid; i < N; i += T) a.Y[i + (int64_t)col * N] = z[i].y;
      if (tid == 0) {
        a.vals[2 * col] = mu.x;
        a.vals[2 * col + 1] = -mu.y;
        a.resid[col] = rs;
      }
      ++col;
    }
    __syncthreads();
  }
  // columns beyond the selection (fewer eigenvalues than m_p): zero
  for (; col < a.mp; ++col) {
    for (int i = tid; i < N; i += T) a.Y[i + (int64_t)col * N] = 0.0;
    if (tid == 0) {
      a.vals[2 * col] = a.vals[2 * col + 1] = 0.0;
      a.resid[col] = 0.0;
    }
  }
  if (tid == 0) *a.status = 0;
}

__global__ void scale_cols_kernel(int64_t n, int64_t ncols, const double* __restrict__ s, double* X, int64_t ldx) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * ncols) return;
  const int64_t i = idx % n, j = idx / n;
  const double d = s[j];
  X[i + j * ldx] *= d > 0.0 ? 1.0 / d : 1.0;
}

}  // namespace

size_t ritz_eig_scratch_bytes(int N) { return (size_t)N * N * (8 + 8 + 16) + 1024; }

rbgs_status ritz_eig(int N, int mb, int mp, int which, const double* H, int64_t ldh, double* vals, double* Y,
                     double* resid, void* scratch, int* status, cudaStream_t st) {
  if (N < 1 || N > kRitzMaxN || mp < 1 || mp > 64 || mb < 1 || ldh < N + mb || (which != 0 && which != 1))
    return RBGS_EINVAL;
  EigArgs a;
  a.N = N;
  a.mb = mb;
  a.mp = mp;
  a.which = which;
  a.H = H;
  a.ldh = ldh;
  char* w = (char*)scratch;
  a.A = (double*)w;
  a.W = a.A + (size_t)N * N;
  a.L = (double2*)(a.W + (size_t)N * N);
  a.vals = vals;
  a.Y = Y;
  a.resid = resid;
  a.status = status;
  const size_t smem = (size_t)N * (8 * 4 + 16 * 2 + 4) + 16;
  RBGS_CUDA_TRY(cudaFuncSetAttribute(ritz_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ritz_eig_kernel<<<1, kEigThreads, smem, st>>>(a);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}

rbgs_status scale_cols(int64_t n, int64_t ncols, const double* norms, double* X, int64_t ldx, cudaStream_t st) {
  const int64_t tot = n * ncols;
  if (tot == 0) return RBGS_OK;
  scale_cols_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, ncols, norms, X, ldx);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}

}  // namespace rbgs
