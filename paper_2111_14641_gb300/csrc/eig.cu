// Extreme eigenpairs of the projected matrix of the randomized Rayleigh-Ritz
// method (Alg. 8, Sec. 5.4 of Balabanov & Grigori, arXiv 2111.14641).
//
// H_(1:p-1,1:p-1) is a small dense non-symmetric matrix (N = (p-1) m_p <=
// 1024) in block upper Hessenberg form: H[i, j] = 0 for i > j + m_p.  One CTA
//   1. reduces an FP32 copy to Hessenberg form (Householder reflections);
//   2. estimates all eigenvalues in FP32 by the implicit double-shift (Francis)
//      QR iteration with deflation, on the active window only;
//   3. picks the m_p extreme estimates (largest or smallest real part);
//   4. refines each in FP64 by Rayleigh-quotient iteration on H itself (complex
//      arithmetic; each step an LU with partial pivoting inside the m_p-wide
//      lower band, O(N^2 m_p), and one solve), which gives the eigenvector of H
//      and the eigenvalue to FP64 accuracy;
//   5. orders the refined pairs, and writes a real basis Y of the vectors, the
//      residual estimates ||H_(p,1:p-1) y|| of step 3 of Alg. 8 and the Ritz
//      values.
// On GB300 a warp-wide FP64 instruction occupies one SM's FP64 pipe for tens of
// cycles, which makes the sequential bulge chase of the QR iteration slow in
// FP64; it only has to separate the eigenvalues, so it runs in FP32.
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

constexpr int kEigThreads = 512;
constexpr int kRqiSteps = 3;  // inverse-iteration steps, each shifted by the latest Rayleigh quotient
constexpr int kExtraCols = 2;  // candidates beyond m_p columns, in case two refine to one eigenvalue
constexpr int kMaxCand = 64 + kExtraCols;

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

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the CTA (red: 33 doubles of shared memory); every thread gets it.
__device__ double cta_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = lane < nw ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// The QR iteration reads and writes only entries with i <= j + 3 (the
// Hessenberg form and the bulge), which fit in shared memory for N up to about
// 320 when packed by columns (column j holds rows 0 .. min(j + 3, N - 1) at
// off[j]); otherwise the iteration works on the dense matrix in global memory.
struct QrMat {
  float* p;
  const int* off;  // null: dense, ld N
  int64_t N;
  __device__ __forceinline__ float& operator()(int i, int j) const { return off ? p[off[j] + i] : p[i + j * N]; }
};

__host__ __device__ inline int64_t qr_band_len(int64_t N, int64_t j) { return j + 4 < N ? j + 4 : N; }

struct EigArgs {
  int N, mb, mp, which;
  const double* H;  // (N + mb) x N, ld ldh: rows N.. are H_(p,1:p-1)
  int64_t ldh;
  float* W;        // N x N scratch: FP32 Hessenberg form, then the QR iteration
  double2* L;      // N x N scratch: complex LU of H - mu I
  double2* M;      // N x mb scratch: the LU's multipliers
  double2* Z;      // N x mp scratch: refined eigenvectors
  double* vals;    // 2 mp: re, im per column
  double* Y;       // N x mp (ld N)
  double* resid;   // mp
  int* status;     // 0 ok, 1 no convergence
  int packed;      // the QR iteration runs on the band in shared memory
};

// Step 2 on the Hessenberg matrix W (entries with i <= j + 3 are read and
// written), by the CTA's threads t = 0 .. nt - 1.  Writes wr, wi (shifted back
// by sigma0); returns 1 when every eigenvalue is found, 2 after maxit sweeps.
struct QrShared {
  float v[3], beta, x, y, z;
  int l, u, state, nr;
};

__device__ int qr_eigenvalues(const QrMat Wq, int N, double sigma0, double anorm, double* wr, double* wi,
                              QrShared& q, int t, int nt) {
  auto SYNC = [] { __syncthreads(); };
  const int maxit = 30 * N;
  int its = 0, total = 0;  // kept by thread 0
  if (t == 0) q.u = N - 1;
  for (;;) {
    SYNC();
    if (t == 0) {
      int u = q.u, l = 0, state = 0;
      while (u >= 0) {
        l = 0;
        for (int i = u; i >= 1; --i) {
          float tst = fabsf(Wq(i - 1, i - 1)) + fabsf(Wq(i, i));
          if (tst == 0.f) tst = (float)anorm;
          if (fabsf(Wq(i, i - 1)) <= FLT_EPSILON * tst) {
            Wq(i, i - 1) = 0.f;
            l = i;
            break;
          }
        }
        if (l == u) {
          wr[u] = (double)Wq(u, u) + sigma0;
          wi[u] = 0.0;
          u -= 1;
          its = 0;
          continue;
        }
        if (l == u - 1) {
          const double p00 = Wq(u - 1, u - 1), p01 = Wq(u - 1, u), p10 = Wq(u, u - 1), p11 = Wq(u, u);
          const double hp = 0.5 * (p00 - p11), disc = hp * hp + p01 * p10;
          if (disc >= 0.0) {
            const double zz = hp + (hp >= 0.0 ? sqrt(disc) : -sqrt(disc));
            wr[u - 1] = p11 + zz + sigma0;
            wr[u] = (zz != 0.0 ? p11 - p01 * p10 / zz : p11) + sigma0;
            wi[u - 1] = wi[u] = 0.0;
          } else {
            const double re = p11 + hp + sigma0, im = sqrt(-disc);
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
        // first column of (W - s1 I)(W - s2 I), s1 and s2 the eigenvalues of the trailing 2 x 2
        // block, written with differences of diagonal entries (no cancellation of large squares)
        const float h00 = Wq(l, l), h01 = Wq(l, l + 1), h10 = Wq(l + 1, l), h11 = Wq(l + 1, l + 1);
        if (its % 10 == 0) {  // exceptional shift after 10 and 20 sweeps without deflation
          const float sg = fabsf(Wq(u, u - 1)) + fabsf(Wq(u - 1, u - 2));
          const float ssum = 1.5f * sg, sprod = sg * sg;
          q.x = h00 * (h00 - ssum) + sprod + h01 * h10;
          q.y = h10 * (h00 + h11 - ssum);
        } else {
          const float ta = Wq(u - 1, u - 1), tb = Wq(u - 1, u), tc = Wq(u, u - 1), td = Wq(u, u);
          q.x = (h00 - ta) * (h00 - td) - tb * tc + h01 * h10;
          q.y = h10 * ((h00 - ta) + (h11 - td));
        }
        q.z = h10 * Wq(l + 2, l + 1);
      }
      q.u = u;
      q.l = l;
      q.state = state;
    }
    SYNC();
    if (q.state != 0) break;
    const int l = q.l, u = q.u;
    for (int k = l; k <= u - 1; ++k) {
      if (t == 0) {
        float x, y, zz;
        const int nr = (k + 2 <= u) ? 3 : 2;
        if (k == l) {
          x = q.x;
          y = q.y;
          zz = nr == 3 ? q.z : 0.f;
        } else {
          x = Wq(k, k - 1);
          y = Wq(k + 1, k - 1);
          zz = nr == 3 ? Wq(k + 2, k - 1) : 0.f;
        }
        const float sc = fabsf(x) + fabsf(y) + fabsf(zz);
        if (sc == 0.f) {
          q.beta = 0.f;
        } else {
          const float is = 1.f / sc;
          x *= is;
          y *= is;
          zz *= is;
          const float sg = sqrtf(x * x + y * y + zz * zz);
          const float al = x >= 0.f ? -sg : sg;
          q.v[0] = x - al;
          q.v[1] = y;
          q.v[2] = zz;
          q.beta = 1.f / (sg * (sg + fabsf(x)));
        }
        q.nr = nr;
      }
      SYNC();
      const float beta = q.beta;
      if (beta != 0.f) {
        const int nr = q.nr;
        const float v0 = q.v[0], v1 = q.v[1], v2 = nr == 3 ? q.v[2] : 0.f;
        const int c0 = k - 1 > l ? k - 1 : l;
        for (int c = c0 + t; c <= u; c += nt) {
          float d = v0 * Wq(k, c) + v1 * Wq(k + 1, c);
          if (nr == 3) d += v2 * Wq(k + 2, c);
          d *= beta;
          Wq(k, c) -= d * v0;
          Wq(k + 1, c) -= d * v1;
          if (nr == 3) Wq(k + 2, c) -= d * v2;
        }
        SYNC();
        const int r1 = k + 3 < u ? k + 3 : u;
        for (int r = l + t; r <= r1; r += nt) {
          float d = Wq(r, k) * v0 + Wq(r, k + 1) * v1;
          if (nr == 3) d += Wq(r, k + 2) * v2;
          d *= beta;
          Wq(r, k) -= d * v0;
          Wq(r, k + 1) -= d * v1;
          if (nr == 3) Wq(r, k + 2) -= d * v2;
        }
      }
      SYNC();
    }
  }
  return q.state;
}

__global__ void __launch_bounds__(kEigThreads) ritz_eig_kernel(EigArgs a) {
  extern __shared__ __align__(16) unsigned char eig_smem[];
  const int N = a.N, mb = a.mb, tid = threadIdx.x, T = blockDim.x;
  const int lane = tid & 31, wp = tid >> 5, nw = T >> 5;
  double* wr = reinterpret_cast<double*>(eig_smem);  // N
  double* wi = wr + N;                                // N
  double2* z = reinterpret_cast<double2*>(wi + N);    // N
  float* v = reinterpret_cast<float*>(z + N);         // N
  int* piv = reinterpret_cast<int*>(v + N);           // N
  int* off = piv + N;                                 // N + 1 (packed band offsets)
  float* band = reinterpret_cast<float*>(off + N + 1);  // the packed band (when a.packed)
  __shared__ double red[33];
  __shared__ double sh_sigma;
  __shared__ double2 sh_mu, sh_ph, mulk[64];
  __shared__ int sel[kMaxCand], sh_nsel;
  __shared__ double2 mu_ref[kMaxCand];
  __shared__ double res_ref[kMaxCand];
  float* W = a.W;
  double2* L = a.L;
  const int64_t ldn = N;
  auto WT = [&](int i, int j) -> float& { return W[i + j * ldn]; };
  auto HT = [&](int i, int j) -> double { return a.H[i + (int64_t)j * a.ldh]; };

  // ---- 1. FP32 Hessenberg form of H_(1:p-1,1:p-1) - sigma I, sigma the mean of the
  // diagonal (taken in FP64, so that FP32 resolves the spread of the spectrum around it)
  double dsum = 0.0;
  for (int i = tid; i < N; i += T) dsum += HT(i, i);
  dsum = cta_sum(dsum, red);
  const double sigma0 = dsum / N;
  double part = 0.0;
  for (int64_t e = tid; e < (int64_t)N * N; e += T) {
    const int i = (int)(e % N), j = (int)(e / N);
    const double h = a.H[i + (int64_t)j * a.ldh];
    W[e] = (float)(i == j ? h - sigma0 : h);
    part += fabs(h);
  }
  const double anorm_sum = cta_sum(part, red);
  const double anorm = anorm_sum > 0.0 ? anorm_sum / N : 1.0;  // a scale of the entries' magnitude
  for (int j = 0; j + 2 < N; ++j) {
    const int len = N - j - 1;
    double pr = 0.0;
    for (int i = 1 + tid; i < len; i += T) {
      const double x = WT(j + 1 + i, j);
      pr += x * x;
    }
    const double rest = cta_sum(pr, red);
    if (rest == 0.0) continue;  // uniform: the column is already reduced
    const float x0 = WT(j + 1, j);
    const float sigma = (float)sqrt((double)x0 * x0 + rest);
    const float alpha = x0 >= 0.f ? -sigma : sigma;
    const float v0 = x0 - alpha;
    const float tj = (alpha - x0) / alpha;
    for (int i = tid; i < len; i += T) v[i] = i == 0 ? 1.f : WT(j + 1 + i, j) / v0;
    __syncthreads();
    for (int c = j + 1 + wp; c < N; c += nw) {  // from the left: a warp per column
      float d = 0.f;
      for (int i = lane; i < len; i += 32) d += v[i] * WT(j + 1 + i, c);
      d = warp_sum(d) * tj;
      for (int i = lane; i < len; i += 32) WT(j + 1 + i, c) -= d * v[i];
    }
    __syncthreads();
    for (int r = tid; r < N; r += T) {  // from the right: a thread per row
      float d = 0.f;
      for (int i = 0; i < len; ++i) d += WT(r, j + 1 + i) * v[i];
      d *= tj;
      for (int i = 0; i < len; ++i) WT(r, j + 1 + i) -= d * v[i];
    }
    __syncthreads();
    for (int i = tid; i < len; i += T) WT(j + 1 + i, j) = i == 0 ? alpha : 0.f;
    __syncthreads();
  }

  // ---- 2. FP32 eigenvalue estimates: implicit double-shift QR on the active window [l, u]
  QrMat Wq{W, nullptr, N};
  if (a.packed) {
    if (tid == 0) {
      int o = 0;
      for (int j = 0; j < N; ++j) {
        off[j] = o;
        o += (int)qr_band_len(N, j);
      }
      off[N] = o;
    }
    __syncthreads();
    for (int j = wp; j < N; j += nw)
      for (int i = lane; i < qr_band_len(N, j); i += 32) band[off[j] + i] = WT(i, j);
    __syncthreads();
    Wq = QrMat{band, off, N};
  }
  __shared__ QrShared qs;
  // (one warp alone, without CTA-wide barriers, measured twice as slow)
  const int qstate = qr_eigenvalues(Wq, N, sigma0, anorm, wr, wi, qs, tid, T);
  __syncthreads();
  if (qstate == 2) {
    if (tid == 0) *a.status = 1;
    return;
  }

  // ---- 3. the extreme estimates (each conjugate pair once), enough for mp columns and a margin
  if (tid == 0) {
    int col = 0, ns = 0;
    for (int guard = 0; guard < N && col < a.mp + kExtraCols && ns < kMaxCand; ++guard) {
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
      col += wi[best] > 0.0 ? 2 : 1;
      ++ns;
    }
    sh_nsel = ns;
  }
  __syncthreads();

  // ---- 4. FP64 Rayleigh-quotient iteration on H for each estimate
  const double tiny = DBL_EPSILON * anorm;
  for (int q = 0; q < sh_nsel; ++q) {
    if (tid == 0) sh_mu = make_double2(wr[sel[q]], wi[sel[q]]);
    for (int i = tid; i < N; i += T) z[i] = make_double2(1.0 + 0.25 * (double)(i % 3), 0.0);
    __syncthreads();
    for (int step = 0; step < kRqiSteps; ++step) {
      const double2 shift = sh_mu;
      // L = H - shift I (only the band below the diagonal is non-zero)
      for (int64_t e = tid; e < (int64_t)N * N; e += T) {  // entries below the band are never read
        const int i = (int)(e % N), j = (int)(e / N);
        if (i > j + mb) continue;
        double re = HT(i, j), im = 0.0;
        if (i == j) {
          re -= shift.x;
          im = -shift.y;
        }
        L[e] = make_double2(re, im);
      }
      __syncthreads();
      for (int k = 0; k + 1 < N; ++k) {
        const int ke = k + mb < N - 1 ? k + mb : N - 1;  // last row with a non-zero in column k
        if (wp == 0) {  // pivot: the first row of largest modulus among k .. ke (mb + 1 <= 65 rows)
          double best = -1.0;
          int p = k;
          for (int i = k + lane; i <= ke; i += 32) {
            const double m = cabs2(L[i + k * ldn]);
            if (m > best) {
              best = m;
              p = i;
            }
          }
  #pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int op = __shfl_xor_sync(0xffffffffu, p, o);
            if (ob > best || (ob == best && op < p)) {
              best = ob;
              p = op;
            }
          }
          if (lane == 0) {
            piv[k] = p;
            if (best == 0.0) L[p + k * ldn] = make_double2(tiny, 0.0);
          }
        }
        __syncthreads();
        const int p = piv[k];
        if (p != k)
          for (int c = k + tid; c < N; c += T) {
            const double2 t = L[k + c * ldn];
            L[k + c * ldn] = L[p + c * ldn];
            L[p + c * ldn] = t;
          }
        __syncthreads();
        const double2 pk = L[k + k * ldn];
        for (int i = k + 1 + tid; i <= ke; i += T) {
          const double2 m = cdiv(L[i + k * ldn], pk);
          a.M[(int64_t)k * mb + (i - k - 1)] = m;
          mulk[i - k - 1] = m;
        }
        __syncthreads();
        const int nb = ke - k;
        const int64_t cnt = (int64_t)nb * (N - k - 1);
        for (int64_t e = tid; e < cnt; e += T) {  // (row, column) pairs of the band rows, rows fastest
          const int r = (int)(e % nb), c = k + 1 + (int)(e / nb);
          const double2 t = cmul(mulk[r], L[k + c * ldn]);
          double2& dst = L[(k + 1 + r) + c * ldn];
          dst = make_double2(dst.x - t.x, dst.y - t.y);
        }
        __syncthreads();
      }
      if (tid == 0 && cabs2(L[(N - 1) + (N - 1) * ldn]) == 0.0) L[(N - 1) + (N - 1) * ldn] = make_double2(tiny, 0.0);
      __syncthreads();
      // solve (H - mu I) w = z: the row swaps and band eliminations, then U
      for (int k = 0; k + 1 < N; ++k) {
        const int ke = k + mb < N - 1 ? k + mb : N - 1;
        if (tid == 0 && piv[k] != k) {
          const double2 t = z[k];
          z[k] = z[piv[k]];
          z[piv[k]] = t;
        }
        __syncthreads();
        const double2 zk = z[k];
        for (int i = k + 1 + tid; i <= ke; i += T) {
          const double2 t = cmul(a.M[(int64_t)k * mb + (i - k - 1)], zk);
          z[i] = make_double2(z[i].x - t.x, z[i].y - t.y);
        }
        __syncthreads();
      }
      for (int i = N - 1; i >= 0; --i) {
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
      // Rayleigh quotient mu = z^H H z (z has unit norm), a warp per row of H z
      double qr = 0.0, qi = 0.0;
      for (int r = wp; r < N; r += nw) {
        double hr = 0.0, hi = 0.0;
        const int c0 = r - mb > 0 ? r - mb : 0;
        for (int c = c0 + lane; c < N; c += 32) {
          const double h = HT(r, c);
          hr += h * z[c].x;
          hi += h * z[c].y;
        }
        hr = warp_sum(hr);
        hi = warp_sum(hi);
        // conj(z_r) (hr + i hi)
        qr += z[r].x * hr + z[r].y * hi;
        qi += z[r].x * hi - z[r].y * hr;
      }
      if (lane != 0) qr = qi = 0.0;
      qr = cta_sum(qr, red);
      qi = cta_sum(qi, red);
      if (tid == 0) sh_mu = make_double2(qr, qi);
      __syncthreads();
    }
    // unit 2-norm (already), first largest-modulus entry real and positive
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
      const double inv = mag > 0.0 ? 1.0 / mag : 1.0;
      sh_ph = make_double2(z[im].x * inv, -z[im].y * inv);
    }
    __syncthreads();
    const double2 ph = sh_ph;
    double2 mu = sh_mu;
    const bool real_mu = fabs(mu.y) <= 64.0 * DBL_EPSILON * fabs(mu.x);
    // keep the member of a pair with positive imaginary part: (conj mu, conj z) is the other
    const bool flip = !real_mu && mu.y < 0.0;
    for (int i = tid; i < N; i += T) {
      double2 t = cmul(z[i], ph);
      if (real_mu) t.y = 0.0;
      if (flip) t.y = -t.y;
      a.Z[i + (int64_t)q * N] = t;
      z[i] = t;
    }
    __syncthreads();
    if (real_mu) mu.y = 0.0;
    if (flip) mu.y = -mu.y;
    // residual estimate ||H_(p,1:p-1) y||
    double rs = 0.0;
    for (int r = 0; r < mb; ++r) {
      double pr2 = 0.0, pi2 = 0.0;
      for (int c = tid; c < N; c += T) {
        const double h = HT(N + r, c);
        pr2 += h * z[c].x;
        pi2 += h * z[c].y;
      }
      pr2 = cta_sum(pr2, red);
      pi2 = cta_sum(pi2, red);
      rs += pr2 * pr2 + pi2 * pi2;
    }
    if (tid == 0) {
      mu_ref[q] = mu;
      res_ref[q] = sqrt(rs);
    }
    __syncthreads();
  }

  // ---- 5. order the refined pairs and write the columns
  if (tid == 0) {  // selection sort of the nsel refined values (sel[] is reused as the order)
    const int ns = sh_nsel;
    for (int q = 0; q < ns; ++q) sel[q] = q;
    for (int q = 0; q < ns; ++q) {
      int b = q;
      for (int r = q + 1; r < ns; ++r) {
        const double2 x = mu_ref[sel[r]], y = mu_ref[sel[b]];
        const double kx = a.which == 0 ? -x.x : x.x, ky = a.which == 0 ? -y.x : y.x;
        if (kx < ky || (kx == ky && x.y > y.y)) b = r;
      }
      const int t = sel[q];
      sel[q] = sel[b];
      sel[b] = t;
    }
  }
  __syncthreads();
  int col = 0;
  for (int q = 0; q < sh_nsel && col < a.mp; ++q) {
    const int s = sel[q];
    const double2 mu = mu_ref[s];
    bool dup = false;  // two estimates that refined to the same eigenvalue
    for (int r = 0; r < q; ++r) {
      const double2 o = mu_ref[sel[r]];
      dup |= fabs(o.x - mu.x) <= 1e-10 * (fabs(mu.x) + fabs(mu.y) + tiny) &&
             fabs(o.y - mu.y) <= 1e-10 * (fabs(mu.x) + fabs(mu.y) + tiny);
    }
    if (dup) continue;  // uniform: mu_ref and sel are shared
    // a refined vector whose imaginary part vanished belongs to a real eigenvalue
    const bool pair = mu.y > 0.0;
    for (int i = tid; i < N; i += T) a.Y[i + (int64_t)col * N] = a.Z[i + (int64_t)s * N].x;
    if (tid == 0) {
      a.vals[2 * col] = mu.x;
      a.vals[2 * col + 1] = mu.y;
      a.resid[col] = res_ref[s];
    }
    ++col;
    if (pair && col < a.mp) {
      for (int i = tid; i < N; i += T) a.Y[i + (int64_t)col * N] = a.Z[i + (int64_t)s * N].y;
      if (tid == 0) {
        a.vals[2 * col] = mu.x;
        a.vals[2 * col + 1] = -mu.y;
        a.resid[col] = res_ref[s];
      }
      ++col;
    }
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

size_t ritz_eig_scratch_bytes(int N, int mb, int mp) {
  return (size_t)N * N * (4 + 16) + (size_t)N * (size_t)(mb + mp + kExtraCols) * 16 + 4096;
}

rbgs_status ritz_eig(int N, int mb, int mp, int which, const double* H, int64_t ldh, double* vals, double* Y,
                     double* resid, void* scratch, int* status, cudaStream_t st) {
  if (N < 1 || N > kRitzMaxN || mp < 1 || mp > 64 || mb < 1 || mb > 64 || ldh < N + mb || (which != 0 && which != 1))
    return RBGS_EINVAL;
  EigArgs a;
  a.N = N;
  a.mb = mb;
  a.mp = mp;
  a.which = which;
  a.H = H;
  a.ldh = ldh;
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  char* w = (char*)scratch;
  a.L = (double2*)w;
  w += up((size_t)N * N * 16);
  a.M = (double2*)w;
  w += up((size_t)N * mb * 16);
  a.Z = (double2*)w;
  w += up((size_t)N * (mp + kExtraCols) * 16);
  a.W = (float*)w;
  a.vals = vals;
  a.Y = Y;
  a.resid = resid;
  a.status = status;
  const size_t base = (size_t)N * (8 * 2 + 16 + 4 + 4) + 4 * ((size_t)N + 1) + 16;
  size_t band = 0;
  for (int j = 0; j < N; ++j) band += (size_t)qr_band_len(N, j);
  int dev = 0, optin = 0;
  RBGS_CUDA_TRY(cudaGetDevice(&dev));
  RBGS_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t static_smem = 8192;  // the kernel's own __shared__ variables, with a margin
  a.packed = base + 4 * band + static_smem <= (size_t)optin ? 1 : 0;
  const size_t smem = a.packed ? base + 4 * band : base;
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
