/*
 * rbgs_oracle.c -- plain FP64 CPU oracle for randomized block Gram-Schmidt.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls
 * this file: only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference leg of bench.py use it.  It shares no code, header or table with
 * the CUDA library; the only thing the two have in common is the written
 * definition of the sketching matrix (Philox4x32-10 bits -> Theta entries),
 * which each side implements on its own.
 *
 * Everything is column-major double precision.  Loops are written the way
 * the paper states each step (Balabanov & Grigori, "Randomized block
 * Gram-Schmidt process for the solution of linear systems and eigenvalue
 * problems"), with no blocking or fusion beyond what a step states:
 *
 *   Sec. 2.3  sketching matrices (Rademacher, SRHT with zero padding); the
 *             Gaussian sketch is the i.i.d. N(0,1/k) matrix, and the
 *             sparse-sign sketch the block sparse JL transform (neither is in
 *             the paper).
 *   Alg. 2    RBGS: sketch W_i, sketched least squares for R_{1:i-1,i},
 *             projection Q'_i = W_i - Q_{1:i-1} R_{1:i-1,i}, sketched QR of
 *             the block (steps 4-5), optional certification (step 6).
 *   Sec. 3.1  step-2 solvers: Householder least squares; the supplement's
 *             Richardson iteration (CGS with l re-orthogonalizations) and
 *             CG on the normal equations.
 *   Alg. 4    steps 4-5 by RCholeskyQR (explicit sketch of Q'_i).
 *   Alg. 5    steps 4-5 by RCholeskyQR with postponed sketch
 *             (S'_i = P_i - S_{1:i-1} R_{1:i-1,i}).
 *   Alg. 6    steps 4-5 by l2 Householder QR followed by RCholeskyQR.
 *   Step 6    Delta = ||I - S^T S||_F, Delta~ = ||P - S R||_F / ||P||_F.
 *   Alg. 7    RBGS-Arnoldi for the 5-point convection-diffusion operator;
 *   Sec. 5.2  restarted randomized block GMRES, Sec. 5.3 block FOM.
 *
 * One extension that the paper does not contain is offered behind a flag:
 * a second projection pass per block ("reorth"), the sketched analogue of
 * re-orthogonalized BCGS (Sec. 1.2), triggered by the certification idea in
 * the remark after Alg. 5.  With reorth=0 the oracle is Alg. 2 exactly.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_THETA_GAUSS 0
#define OR_THETA_RADEMACHER 1
#define OR_THETA_SRHT 2
#define OR_THETA_IDENTITY 3
#define OR_THETA_SPARSE 4

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11).
 * Round: two 32x32->64 multiplications of counter words 0 and 2 by the
 * round multipliers, the high halves xor-ed with the other two words and the
 * key; the key is bumped by the Weyl constants between rounds.           */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox_call(uint64_t seed, uint32_t a, uint32_t b, uint32_t purpose, uint32_t d, uint32_t out[4]) {
  uint32_t ctr[4] = {a, b, purpose, d};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  or_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* Entries of Theta (k x n).  Definitions (project convention; the paper only
 * asks for a seeded generator, Sec. 2.3):
 *  Gaussian   theta_{r,j} = z / sqrt(k), z from Box-Muller on the Philox
 *             block with counter (j_lo, r>>1, 0, j_hi); even r takes the
 *             cosine branch, odd r the sine branch.
 *  Rademacher theta_{r,j} = +-1/sqrt(k), the sign is bit (r & 31) of word
 *             (r>>5)&3 of the block with counter (j_lo, r>>7, 1, j_hi); a set
 *             bit means -1.
 *  SRHT       theta_{r,j} = D_j * (-1)^{popcount(s_r & j)} / sqrt(k), D_j the
 *             sign bit (j & 31) of word (j>>5)&3 of block (j>>7, 0, 2, 0),
 *             s_0 < ... < s_{k-1} the sampled rows of the n' x n' Sylvester
 *             Hadamard matrix, n' = 2^ceil(log2 n).
 *  Sparse     sign (not in the paper): the block construction of the sparse
 *             Johnson-Lindenstrauss transform (Kane and Nelson, J. ACM 2014).
 *             With z = min(8, k), the rows split into z segments
 *             [floor(s k / z), floor((s+1) k / z)); column j has exactly one
 *             nonzero in each segment s, +-1/sqrt(z), at offset
 *             (x >> 1) mod (segment size), negative when bit 0 of x is set,
 *             x = word s&3 of the block with counter (j_lo, s>>2, 4, j_hi). */
static double gauss_pair(uint64_t seed, int64_t j, int64_t rpair, int which) {
  uint32_t x[4];
  philox_call(seed, (uint32_t)(j & 0xffffffff), (uint32_t)rpair, 0u, (uint32_t)(j >> 32), x);
  double u1 = ((double)(x[0] >> 5) * 67108864.0 + (double)(x[1] >> 6) + 0.5) * (1.0 / 9007199254740992.0);
  double u2 = ((double)(x[2] >> 5) * 67108864.0 + (double)(x[3] >> 6) + 0.5) * (1.0 / 9007199254740992.0);
  double rad = sqrt(-2.0 * log(u1));
  double ang = 2.0 * M_PI * u2;
  return which ? rad * sin(ang) : rad * cos(ang);
}

double or_theta_gauss_entry(uint64_t seed, int64_t k, int64_t r, int64_t j) {
  return gauss_pair(seed, j, r >> 1, (int)(r & 1)) / sqrt((double)k);
}

double or_theta_rademacher_entry(uint64_t seed, int64_t k, int64_t r, int64_t j) {
  uint32_t x[4];
  philox_call(seed, (uint32_t)(j & 0xffffffff), (uint32_t)(r >> 7), 1u, (uint32_t)(j >> 32), x);
  uint32_t bit = (x[(r >> 5) & 3] >> (r & 31)) & 1u;
  return (bit ? -1.0 : 1.0) / sqrt((double)k);
}

int64_t or_srht_padded(int64_t n) {
  int64_t np = 1;
  while (np < n) np <<= 1;
  return np;
}

double or_srht_sign(uint64_t seed, int64_t j) {
  uint32_t x[4];
  philox_call(seed, (uint32_t)(j >> 7), 0u, 2u, 0u, x);
  uint32_t bit = (x[(j >> 5) & 3] >> (j & 31)) & 1u;
  return bit ? -1.0 : 1.0;
}

/* The z nonzeros of column j of the sparse-sign Theta: rows[s] (segment s)
 * and signs[s] = +-1.  Returns z = min(8, k).                               */
int or_sparse_column(uint64_t seed, int64_t k, int64_t j, int64_t* rows, double* signs) {
  int z = k < 8 ? (int)k : 8;
  for (int s = 0; s < z; ++s) {
    uint32_t x[4];
    philox_call(seed, (uint32_t)(j & 0xffffffff), (uint32_t)(s >> 2), 4u, (uint32_t)(j >> 32), x);
    uint32_t w = x[s & 3];
    int64_t lo = (int64_t)s * k / z, hi = (int64_t)(s + 1) * k / z;
    rows[s] = lo + (int64_t)((w >> 1) % (uint32_t)(hi - lo));
    signs[s] = (w & 1u) ? -1.0 : 1.0;
  }
  return z;
}

static int cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x > y) - (x < y);
}

/* k distinct rows of [0, np), uniform without replacement (Floyd's
 * algorithm): for t = 0..k-1 with J = np-k+t, draw v uniform in [0, J] from
 * the block (t, 0, 3, 0) as (word1:word0) mod (J+1); keep v unless already
 * chosen, else keep J.  The set is returned sorted ascending.  Returns 0, or
 * -1 when k > np.                                                          */
int or_srht_samples(uint64_t seed, int64_t np, int64_t k, int64_t* out) {
  if (k > np || k < 0) return -1;
  /* membership by sorted insertion; plain O(k^2) keeps it obviously right */
  int64_t cnt = 0;
  for (int64_t t = 0; t < k; ++t) {
    int64_t J = np - k + t;
    uint32_t x[4];
    philox_call(seed, (uint32_t)t, 0u, 3u, 0u, x);
    uint64_t r64 = ((uint64_t)x[1] << 32) | (uint64_t)x[0];
    int64_t v = (int64_t)(r64 % (uint64_t)(J + 1));
    int found = 0;
    for (int64_t q = 0; q < cnt; ++q)
      if (out[q] == v) { found = 1; break; }
    out[cnt++] = found ? J : v;
  }
  qsort(out, (size_t)k, sizeof(int64_t), cmp_i64);
  return 0;
}

static int popcount64(uint64_t v) {
  int c = 0;
  while (v) { v &= v - 1; ++c; }
  return c;
}

double or_theta_srht_entry(uint64_t seed, int64_t k, int64_t n, const int64_t* samples, int64_t r, int64_t j) {
  (void)n;
  double h = (popcount64((uint64_t)(samples[r] & j)) & 1) ? -1.0 : 1.0;
  return or_srht_sign(seed, j) * h / sqrt((double)k);
}

/* Dense Theta (k x n, column-major, ld = k) straight from the entry
 * definitions.  For small cases and tests only.                            */
int or_theta_dense(int type, int64_t k, int64_t n, uint64_t seed, double* T) {
  int64_t* samples = NULL;
  if (type == OR_THETA_SRHT) {
    samples = (int64_t*)malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
    if (or_srht_samples(seed, or_srht_padded(n), k, samples)) { free(samples); return -1; }
  }
  for (int64_t j = 0; j < n; ++j)
    for (int64_t r = 0; r < k; ++r) {
      double v;
      if (type == OR_THETA_GAUSS) v = or_theta_gauss_entry(seed, k, r, j);
      else if (type == OR_THETA_RADEMACHER) v = or_theta_rademacher_entry(seed, k, r, j);
      else if (type == OR_THETA_SRHT) v = or_theta_srht_entry(seed, k, n, samples, r, j);
      else if (type == OR_THETA_SPARSE) v = 0.0;
      else v = (r == j) ? 1.0 : 0.0;
      T[r + j * k] = v;
    }
  if (type == OR_THETA_SPARSE)
    for (int64_t j = 0; j < n; ++j) {
      int64_t rows[8];
      double signs[8];
      int z = or_sparse_column(seed, k, j, rows, signs);
      for (int s = 0; s < z; ++s) T[rows[s] + j * k] = signs[s] / sqrt((double)z);
    }
  free(samples);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Theta * X for X n x ncols (ldx), Y k x ncols (ldy).                       */

typedef struct {
  int type;
  int64_t k, n, ncols, ldx, ldy;
  uint64_t seed;
  const double* X;
  double* Y;
  const int64_t* samples;
  int64_t lo, hi; /* range of the parallel index */
} theta_job;

/* Gaussian / Rademacher: each worker owns a range of Theta rows [lo, hi),
 * regenerates theta_{r,j} for its rows and accumulates y_r = sum_j theta_{r,j} x_j. */
static void* theta_dense_worker(void* arg) {
  theta_job* J = (theta_job*)arg;
  for (int64_t r = J->lo; r < J->hi; ++r)
    for (int64_t c = 0; c < J->ncols; ++c) J->Y[r + c * J->ldy] = 0.0;
  for (int64_t j = 0; j < J->n; ++j) {
    for (int64_t r = J->lo; r < J->hi; ++r) {
      double t = (J->type == OR_THETA_GAUSS) ? or_theta_gauss_entry(J->seed, J->k, r, j)
                                             : or_theta_rademacher_entry(J->seed, J->k, r, j);
      for (int64_t c = 0; c < J->ncols; ++c) J->Y[r + c * J->ldy] += t * J->X[j + c * J->ldx];
    }
  }
  return NULL;
}

/* Sparse sign: each worker owns a range of columns of X and scatters every
 * row x_j into the z rows of column j of Theta.                             */
static void* theta_sparse_worker(void* arg) {
  theta_job* J = (theta_job*)arg;
  int64_t rows[8];
  double signs[8];
  for (int64_t c = J->lo; c < J->hi; ++c) {
    for (int64_t r = 0; r < J->k; ++r) J->Y[r + c * J->ldy] = 0.0;
    for (int64_t j = 0; j < J->n; ++j) {
      int z = or_sparse_column(J->seed, J->k, j, rows, signs);
      double v = J->X[j + c * J->ldx] / sqrt((double)z);
      for (int s = 0; s < z; ++s) J->Y[rows[s] + c * J->ldy] += signs[s] * v;
    }
  }
  return NULL;
}

/* Sylvester-ordered Walsh-Hadamard transform y = H x, in place, length 2^q.
 * H_{2N} = [[H_N, H_N], [H_N, -H_N]] applied level by level.               */
void or_fwht(double* x, int64_t len) {
  for (int64_t h = 1; h < len; h <<= 1)
    for (int64_t i = 0; i < len; i += 2 * h)
      for (int64_t j = i; j < i + h; ++j) {
        double a = x[j], b = x[j + h];
        x[j] = a + b;
        x[j + h] = a - b;
      }
}

/* SRHT: each worker owns a range of columns of X.  Per column: zero-pad to
 * n', multiply by D, Hadamard transform, keep the sampled entries, scale.  */
static void* theta_srht_worker(void* arg) {
  theta_job* J = (theta_job*)arg;
  int64_t np = or_srht_padded(J->n);
  double* buf = (double*)malloc(sizeof(double) * (size_t)np);
  double* sgn = (double*)malloc(sizeof(double) * (size_t)np);
  for (int64_t j = 0; j < np; ++j) sgn[j] = or_srht_sign(J->seed, j);
  double scale = 1.0 / sqrt((double)J->k);
  for (int64_t c = J->lo; c < J->hi; ++c) {
    for (int64_t j = 0; j < np; ++j) buf[j] = (j < J->n) ? sgn[j] * J->X[j + c * J->ldx] : 0.0;
    or_fwht(buf, np);
    for (int64_t r = 0; r < J->k; ++r) J->Y[r + c * J->ldy] = scale * buf[J->samples[r]];
  }
  free(buf);
  free(sgn);
  return NULL;
}

static int g_threads = 1;
void or_set_threads(int t) { g_threads = t < 1 ? 1 : t; }
int or_get_threads(void) { return g_threads; }

int or_theta_apply(int type, int64_t k, int64_t n, uint64_t seed, const double* X, int64_t ldx, int64_t ncols,
                   double* Y, int64_t ldy) {
  if (type == OR_THETA_IDENTITY) {
    if (k != n) return -1;
    for (int64_t c = 0; c < ncols; ++c)
      for (int64_t r = 0; r < n; ++r) Y[r + c * ldy] = X[r + c * ldx];
    return 0;
  }
  int64_t* samples = NULL;
  if (type == OR_THETA_SRHT) {
    samples = (int64_t*)malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
    if (or_srht_samples(seed, or_srht_padded(n), k, samples)) { free(samples); return -1; }
  }
  int nt = g_threads;
  int64_t total = (type == OR_THETA_SRHT || type == OR_THETA_SPARSE) ? ncols : k;
  if (nt > total) nt = (int)(total > 0 ? total : 1);
  pthread_t th[256];
  theta_job jobs[256];
  if (nt > 256) nt = 256;
  for (int t = 0; t < nt; ++t) {
    theta_job* J = &jobs[t];
    J->type = type; J->k = k; J->n = n; J->ncols = ncols; J->ldx = ldx; J->ldy = ldy;
    J->seed = seed; J->X = X; J->Y = Y; J->samples = samples;
    if (type == OR_THETA_GAUSS) { /* keep Gaussian row pairs on one worker */
      int64_t pairs = (k + 1) / 2;
      J->lo = 2 * (pairs * t / nt);
      J->hi = 2 * (pairs * (t + 1) / nt);
      if (J->hi > k) J->hi = k;
    } else {
      J->lo = total * t / nt;
      J->hi = total * (t + 1) / nt;
    }
    void* (*fn)(void*) = (type == OR_THETA_SRHT)     ? theta_srht_worker
                         : (type == OR_THETA_SPARSE) ? theta_sparse_worker
                                                     : theta_dense_worker;
    if (nt == 1) fn(J);
    else pthread_create(&th[t], NULL, fn, J);
  }
  if (nt > 1)
    for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
  free(samples);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Dense building blocks (column-major).                                     */

/* C (m x n) = alpha * op(A) * op(B) + beta * C, plain triple loop.          */
static void gemm(int ta, int tb, int64_t m, int64_t n, int64_t kk, double alpha, const double* A, int64_t lda,
                 const double* B, int64_t ldb, double beta, double* C, int64_t ldc) {
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) {
      double s = 0.0;
      for (int64_t l = 0; l < kk; ++l) {
        double a = ta ? A[l + i * lda] : A[i + l * lda];
        double b = tb ? B[j + l * ldb] : B[l + j * ldb];
        s += a * b;
      }
      C[i + j * ldc] = alpha * s + (beta == 0.0 ? 0.0 : beta * C[i + j * ldc]);
    }
}

/* Householder QR of A (m x n, m >= n) in place (LAPACK-style compact form:
 * R in the upper triangle, v_j below the diagonal with implicit unit head,
 * tau[j]).  Returns 0.  R's diagonal sign is whatever the reflectors give;
 * callers that need a positive diagonal flip signs afterwards.              */
void or_householder_qr(int64_t m, int64_t n, double* A, int64_t lda, double* tau) {
  for (int64_t j = 0; j < n; ++j) {
    double* a = A + j + j * lda;
    double norm2 = 0.0;
    for (int64_t i = 0; i < m - j; ++i) norm2 += a[i] * a[i];
    double alpha = a[0];
    double norm = sqrt(norm2);
    if (norm == 0.0) { tau[j] = 0.0; continue; }
    double beta = (alpha >= 0.0) ? -norm : norm;
    double v0 = alpha - beta;
    for (int64_t i = 1; i < m - j; ++i) a[i] /= v0;
    tau[j] = (beta - alpha) / beta;
    a[0] = beta;
    /* apply H = I - tau v v^T to the trailing columns */
    for (int64_t c = j + 1; c < n; ++c) {
      double* x = A + j + c * lda;
      double s = x[0];
      for (int64_t i = 1; i < m - j; ++i) s += a[i] * x[i];
      s *= tau[j];
      x[0] -= s;
      for (int64_t i = 1; i < m - j; ++i) x[i] -= s * a[i];
    }
  }
}

/* Apply Q^T (from or_householder_qr of an m x n matrix) to B (m x nb).       */
static void householder_apply_qt(int64_t m, int64_t n, const double* A, int64_t lda, const double* tau, double* B,
                                 int64_t ldb, int64_t nb) {
  for (int64_t j = 0; j < n; ++j) {
    if (tau[j] == 0.0) continue;
    const double* v = A + j + j * lda;
    for (int64_t c = 0; c < nb; ++c) {
      double* x = B + j + c * ldb;
      double s = x[0];
      for (int64_t i = 1; i < m - j; ++i) s += v[i] * x[i];
      s *= tau[j];
      x[0] -= s;
      for (int64_t i = 1; i < m - j; ++i) x[i] -= s * v[i];
    }
  }
}

/* Apply Q (from or_householder_qr) to B (m x nb): B <- H_0 H_1 ... H_{n-1} B. */
static void householder_apply_q(int64_t m, int64_t n, const double* A, int64_t lda, const double* tau, double* B,
                                int64_t ldb, int64_t nb) {
  for (int64_t j = n - 1; j >= 0; --j) {
    if (tau[j] == 0.0) continue;
    const double* v = A + j + j * lda;
    for (int64_t c = 0; c < nb; ++c) {
      double* x = B + j + c * ldb;
      double s = x[0];
      for (int64_t i = 1; i < m - j; ++i) s += v[i] * x[i];
      s *= tau[j];
      x[0] -= s;
      for (int64_t i = 1; i < m - j; ++i) x[i] -= s * v[i];
    }
  }
}

/* R factor (n x n, ldr) of the thin QR of A (m x n), positive diagonal.
 * A is not modified.  Returns -1 if a diagonal entry is zero or not finite. */
int or_qr_r(int64_t m, int64_t n, const double* A, int64_t lda, double* R, int64_t ldr) {
  double* W = (double*)malloc(sizeof(double) * (size_t)(m * n > 0 ? m * n : 1));
  double* tau = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) W[i + j * m] = A[i + j * lda];
  or_householder_qr(m, n, W, m, tau);
  int bad = 0;
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t i = 0; i < n; ++i) R[i + j * ldr] = (i <= j) ? W[i + j * m] : 0.0;
  }
  for (int64_t i = 0; i < n; ++i) {
    double d = R[i + i * ldr];
    if (!(d != 0.0) || !isfinite(d)) bad = 1;
    if (d < 0.0)
      for (int64_t j = i; j < n; ++j) R[i + j * ldr] = -R[i + j * ldr];
  }
  free(W);
  free(tau);
  return bad ? -1 : 0;
}

/* Thin Householder QR with explicit Q (m x n) and positive-diagonal R.      */
int or_qr_full(int64_t m, int64_t n, const double* A, int64_t lda, double* Q, int64_t ldq, double* R, int64_t ldr) {
  double* W = (double*)malloc(sizeof(double) * (size_t)(m * n > 0 ? m * n : 1));
  double* tau = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) W[i + j * m] = A[i + j * lda];
  or_householder_qr(m, n, W, m, tau);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) R[i + j * ldr] = (i <= j) ? W[i + j * m] : 0.0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) Q[i + j * ldq] = (i == j) ? 1.0 : 0.0;
  householder_apply_q(m, n, W, m, tau, Q, ldq, n);
  int bad = 0;
  for (int64_t i = 0; i < n; ++i) {
    double d = R[i + i * ldr];
    if (!(d != 0.0) || !isfinite(d)) bad = 1;
    if (d < 0.0) {
      for (int64_t j = i; j < n; ++j) R[i + j * ldr] = -R[i + j * ldr];
      for (int64_t r = 0; r < m; ++r) Q[r + i * ldq] = -Q[r + i * ldq];
    }
  }
  free(W);
  free(tau);
  return bad ? -1 : 0;
}

/* X <- X * U^{-1} for upper-triangular U (nb x nb), X (m x nb): forward
 * substitution over the columns of X, row by row.                         */
typedef struct {
  double* X;
  int64_t ldx, nb, lo, hi;
  const double* U;
  int64_t ldu;
} trsm_job;

static void* trsm_worker(void* arg) {
  trsm_job* J = (trsm_job*)arg;
  for (int64_t r = J->lo; r < J->hi; ++r)
    for (int64_t j = 0; j < J->nb; ++j) {
      double s = J->X[r + j * J->ldx];
      for (int64_t l = 0; l < j; ++l) s -= J->X[r + l * J->ldx] * J->U[l + j * J->ldu];
      J->X[r + j * J->ldx] = s / J->U[j + j * J->ldu];
    }
  return NULL;
}

static void trsm_right_upper(int64_t m, int64_t nb, const double* U, int64_t ldu, double* X, int64_t ldx) {
  int nt = g_threads;
  if (nt > 256) nt = 256;
  if (m < 4096) nt = 1;
  pthread_t th[256];
  trsm_job jobs[256];
  for (int t = 0; t < nt; ++t) {
    jobs[t] = (trsm_job){X, ldx, nb, m * t / nt, m * (t + 1) / nt, U, ldu};
    if (nt == 1) trsm_worker(&jobs[t]);
    else pthread_create(&th[t], NULL, trsm_worker, &jobs[t]);
  }
  if (nt > 1)
    for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
}

/* Step 3 of Alg. 2: Qp = W_i - Q_{1:i-1} R_{1:i-1,i}, rows split over threads. */
typedef struct {
  const double* W;
  int64_t ldw;
  const double* Q;
  int64_t ldq;
  const double* Rc;
  int64_t ldr;
  double* Qp;
  int64_t ldqp;
  int64_t c, mp, lo, hi;
} proj_job;

static void* proj_worker(void* arg) {
  proj_job* J = (proj_job*)arg;
  for (int64_t j = 0; j < J->mp; ++j)
    for (int64_t r = J->lo; r < J->hi; ++r) {
      double s = 0.0;
      for (int64_t l = 0; l < J->c; ++l) s += J->Q[r + l * J->ldq] * J->Rc[l + j * J->ldr];
      J->Qp[r + j * J->ldqp] = J->W[r + j * J->ldw] - s;
    }
  return NULL;
}

static void project(int64_t n, int64_t c, int64_t mp, const double* W, int64_t ldw, const double* Q, int64_t ldq,
                    const double* Rc, int64_t ldr, double* Qp, int64_t ldqp) {
  int nt = g_threads;
  if (nt > 256) nt = 256;
  if (n < 4096) nt = 1;
  pthread_t th[256];
  proj_job jobs[256];
  for (int t = 0; t < nt; ++t) {
    jobs[t] = (proj_job){W, ldw, Q, ldq, Rc, ldr, Qp, ldqp, c, mp, n * t / nt, n * (t + 1) / nt};
    if (nt == 1) proj_worker(&jobs[t]);
    else pthread_create(&th[t], NULL, proj_worker, &jobs[t]);
  }
  if (nt > 1)
    for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------------ */
/* Step 2 solvers: X (c x mp) = argmin_Y ||S Y - P||_F, S k x c, P k x mp.   */

#define OR_LS_HOUSEHOLDER 0
#define OR_LS_RICHARDSON 1
#define OR_LS_CG 2

/* Householder least squares: QR of S, Y = R^{-1} (Q^T P)_{1:c}.             */
static int ls_householder(int64_t k, int64_t c, const double* S, int64_t lds, const double* P, int64_t ldp,
                          int64_t mp, double* X, int64_t ldx) {
  double* A = (double*)malloc(sizeof(double) * (size_t)(k * c));
  double* tau = (double*)malloc(sizeof(double) * (size_t)c);
  double* B = (double*)malloc(sizeof(double) * (size_t)(k * mp));
  for (int64_t j = 0; j < c; ++j)
    for (int64_t i = 0; i < k; ++i) A[i + j * k] = S[i + j * lds];
  for (int64_t j = 0; j < mp; ++j)
    for (int64_t i = 0; i < k; ++i) B[i + j * k] = P[i + j * ldp];
  or_householder_qr(k, c, A, k, tau);
  householder_apply_qt(k, c, A, k, tau, B, k, mp);
  int bad = 0;
  for (int64_t j = 0; j < mp; ++j)
    for (int64_t i = c - 1; i >= 0; --i) {
      double s = B[i + j * k];
      for (int64_t l = i + 1; l < c; ++l) s -= A[i + l * k] * X[l + j * ldx];
      double d = A[i + i * k];
      if (d == 0.0) bad = 1;
      X[i + j * ldx] = s / d;
    }
  free(A);
  free(tau);
  free(B);
  return bad ? -1 : 0;
}

/* Richardson iteration on the normal equations (the supplement's CGS with l
 * re-orthogonalizations): X <- 0; repeat l times X <- X + S^T (P - S X).   */
static void ls_richardson(int64_t k, int64_t c, const double* S, int64_t lds, const double* P, int64_t ldp, int64_t mp,
                          int l, double* X, int64_t ldx) {
  double* Res = (double*)malloc(sizeof(double) * (size_t)(k * mp));
  double* Dx = (double*)malloc(sizeof(double) * (size_t)(c * mp));
  for (int64_t j = 0; j < mp; ++j)
    for (int64_t i = 0; i < c; ++i) X[i + j * ldx] = 0.0;
  for (int it = 0; it < l; ++it) {
    /* Res = P - S X */
    gemm(0, 0, k, mp, c, 1.0, S, lds, X, ldx, 0.0, Res, k);
    for (int64_t j = 0; j < mp; ++j)
      for (int64_t i = 0; i < k; ++i) Res[i + j * k] = P[i + j * ldp] - Res[i + j * k];
    /* X += S^T Res */
    gemm(1, 0, c, mp, k, 1.0, S, lds, Res, k, 0.0, Dx, c);
    for (int64_t j = 0; j < mp; ++j)
      for (int64_t i = 0; i < c; ++i) X[i + j * ldx] += Dx[i + j * c];
  }
  free(Res);
  free(Dx);
}

/* l iterations of conjugate gradients on (S^T S) x = S^T p, per column,
 * starting from x = 0 (the supplement's "other methods").                  */
static void ls_cg(int64_t k, int64_t c, const double* S, int64_t lds, const double* P, int64_t ldp, int64_t mp, int l,
                  double* X, int64_t ldx) {
  double* r = (double*)malloc(sizeof(double) * (size_t)c);
  double* p = (double*)malloc(sizeof(double) * (size_t)c);
  double* t = (double*)malloc(sizeof(double) * (size_t)k);
  double* q = (double*)malloc(sizeof(double) * (size_t)c);
  for (int64_t col = 0; col < mp; ++col) {
    double* x = X + col * ldx;
    const double* b = P + col * ldp;
    for (int64_t i = 0; i < c; ++i) x[i] = 0.0;
    /* r = S^T b */
    for (int64_t i = 0; i < c; ++i) {
      double s = 0.0;
      for (int64_t h = 0; h < k; ++h) s += S[h + i * lds] * b[h];
      r[i] = s;
      p[i] = s;
    }
    double rr = 0.0;
    for (int64_t i = 0; i < c; ++i) rr += r[i] * r[i];
    for (int it = 0; it < l && rr > 0.0; ++it) {
      /* q = S^T (S p) */
      for (int64_t h = 0; h < k; ++h) {
        double s = 0.0;
        for (int64_t i = 0; i < c; ++i) s += S[h + i * lds] * p[i];
        t[h] = s;
      }
      double pq = 0.0;
      for (int64_t i = 0; i < c; ++i) {
        double s = 0.0;
        for (int64_t h = 0; h < k; ++h) s += S[h + i * lds] * t[h];
        q[i] = s;
        pq += p[i] * s;
      }
      if (pq <= 0.0) break;
      double alpha = rr / pq;
      for (int64_t i = 0; i < c; ++i) {
        x[i] += alpha * p[i];
        r[i] -= alpha * q[i];
      }
      double rr_new = 0.0;
      for (int64_t i = 0; i < c; ++i) rr_new += r[i] * r[i];
      double beta = rr_new / rr;
      rr = rr_new;
      for (int64_t i = 0; i < c; ++i) p[i] = r[i] + beta * p[i];
    }
  }
  free(r);
  free(p);
  free(t);
  free(q);
}

static int solve_ls(int ls, int ls_iters, int64_t k, int64_t c, const double* S, int64_t lds, const double* P,
                    int64_t ldp, int64_t mp, double* X, int64_t ldx) {
  if (c == 0) return 0;
  if (ls == OR_LS_HOUSEHOLDER) return ls_householder(k, c, S, lds, P, ldp, mp, X, ldx);
  if (ls == OR_LS_RICHARDSON) { ls_richardson(k, c, S, lds, P, ldp, mp, ls_iters, X, ldx); return 0; }
  ls_cg(k, c, S, lds, P, ldp, mp, ls_iters, X, ldx);
  return 0;
}

typedef struct or_stencil or_stencil;
static int rbgs_core(const double* W, int64_t n, int64_t m, int64_t ldw, int64_t mp, int theta, int64_t k,
                     uint64_t seed, int variant, int ls, int ls_iters, int ls_iters_first, int reorth,
                     const or_stencil* op, double* Q, int64_t ldq, double* R, int64_t ldr, double* S_out,
                     double* P_out, double* stats);

/* ------------------------------------------------------------------------ */
/* Steps 4-5 of Alg. 2 on the block Qp (n x mp, in place -> Q_i).            *
 * Outputs R_ii (mp x mp) and S_i = Theta Q_i (k x mp).                      *
 * Spp carries the implicit sketch S'_i needed by Alg. 5.                    */
static int interblock(int variant, int64_t n, int64_t mp, double* Qp, int64_t ldq, const double* Spp, int64_t lds,
                      int theta, int64_t k, uint64_t seed, double* Rii, int64_t ldr, double* Si, int64_t ldsi) {
  double* Sp = (double*)malloc(sizeof(double) * (size_t)(k * mp));
  int rc = 0;
  if (variant == 1 || variant == 3) {
    /* Column by column within the block: single-vector RGS (1: each new
       column's sketch taken explicitly, as in Alg. 4) or vRCholeskyQR (3,
       Alg. 3: the sketch taken implicitly, as in Alg. 5).  Both are RBGS with
       one-column blocks on Q'_i itself (Householder least squares). */
    double* Qc = (double*)malloc(sizeof(double) * (size_t)(n * mp));
    double* Rc = (double*)malloc(sizeof(double) * (size_t)(mp * mp));
    for (int64_t j = 0; j < mp; ++j)
      for (int64_t i = 0; i < n; ++i) Qc[i + j * n] = Qp[i + j * ldq];
    rc |= rbgs_core(Qc, n, mp, n, 1, theta, k, seed, variant == 1 ? 4 : 5, 0, 0, 0, 0, NULL, Qp, ldq, Rc, mp, NULL,
                    NULL, NULL) ? 1 : 0;
    for (int64_t j = 0; j < mp; ++j)
      for (int64_t i = 0; i < mp; ++i) Rii[i + j * ldr] = Rc[i + j * mp];
    free(Qc);
    free(Rc);
  } else if (variant == 5) {
    /* Alg. 5: S'_i is P_i - S_{1:i-1} R_{1:i-1,i}, given by the caller.    */
    for (int64_t j = 0; j < mp; ++j)
      for (int64_t i = 0; i < k; ++i) Sp[i + j * k] = Spp[i + j * lds];
    rc |= or_qr_r(k, mp, Sp, k, Rii, ldr);
    trsm_right_upper(n, mp, Rii, ldr, Qp, ldq);
  } else if (variant == 4) {
    /* Alg. 4: S'_i = Theta Q'_i, R_ii = R of qr(S'_i), Q_i = Q'_i R_ii^{-1}. */
    or_theta_apply(theta, k, n, seed, Qp, ldq, mp, Sp, k);
    rc |= or_qr_r(k, mp, Sp, k, Rii, ldr);
    trsm_right_upper(n, mp, Rii, ldr, Qp, ldq);
  } else {
    /* Alg. 6: Q'_i = Q* R' (l2 Householder), then Alg. 4 on Q*, R_ii = R'' R'. */
    double* Qs = (double*)malloc(sizeof(double) * (size_t)(n * mp));
    double* R1 = (double*)malloc(sizeof(double) * (size_t)(mp * mp));
    double* R2 = (double*)malloc(sizeof(double) * (size_t)(mp * mp));
    rc |= or_qr_full(n, mp, Qp, ldq, Qs, n, R1, mp);
    or_theta_apply(theta, k, n, seed, Qs, n, mp, Sp, k);
    rc |= or_qr_r(k, mp, Sp, k, R2, mp);
    trsm_right_upper(n, mp, R2, mp, Qs, n);
    for (int64_t j = 0; j < mp; ++j)
      for (int64_t i = 0; i < n; ++i) Qp[i + j * ldq] = Qs[i + j * n];
    gemm(0, 0, mp, mp, mp, 1.0, R2, mp, R1, mp, 0.0, Rii, ldr);
    free(Qs);
    free(R1);
    free(R2);
  }
  /* step 5: S_i = Theta Q_i */
  or_theta_apply(theta, k, n, seed, Qp, ldq, mp, Si, ldsi);
  free(Sp);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Alg. 2.  W n x m (ldw), block size mp (the last of the p = ceil(m / mp)
 * blocks takes the remaining columns).  Outputs Q (n x m, ldq),
 * R (m x m, ldr, upper triangular), and, when non-NULL, S = Theta Q and
 * P = Theta W (k x m, ld k).  stats (when non-NULL) receives
 * {Delta, Delta~, number of second passes}.  With reorth, ls_iters_first > 0
 * sets the Richardson count of the first (provisional) pass.  Returns 0, -1
 * on bad arguments, -2 on a breakdown (zero or non-finite R_ii diagonal).   */
/* ------------------------------------------------------------------------ */
/* The 5-point convection-diffusion operator A u = -Laplace(u) + b . grad(u) on
 * the unit square, nx x ny interior points with spacing hx = 1/(nx+1),
 * hy = 1/(ny+1), zero Dirichlet boundary, central differences; point (x, y)
 * is row x + nx y.  (The synthetic operator of the Krylov experiments.)     */
struct or_stencil {
  int64_t nx, ny;
  double bx, by;
};

void or_stencil5_apply(const or_stencil* op, const double* X, int64_t ldx, int64_t ncols, double* Y, int64_t ldy) {
  const int64_t nx = op->nx, ny = op->ny;
  const double hx = 1.0 / (double)(nx + 1), hy = 1.0 / (double)(ny + 1);
  const double cx = 1.0 / (hx * hx), cy = 1.0 / (hy * hy);
  const double ax = op->bx / (2.0 * hx), ay = op->by / (2.0 * hy);
  for (int64_t j = 0; j < ncols; ++j) {
    const double* x = X + j * ldx;
    double* y = Y + j * ldy;
    for (int64_t iy = 0; iy < ny; ++iy)
      for (int64_t ix = 0; ix < nx; ++ix) {
        const int64_t i = ix + nx * iy;
        const double w = ix > 0 ? x[i - 1] : 0.0, e = ix + 1 < nx ? x[i + 1] : 0.0;
        const double so = iy > 0 ? x[i - nx] : 0.0, no = iy + 1 < ny ? x[i + nx] : 0.0;
        y[i] = cx * (2.0 * x[i] - w - e) + cy * (2.0 * x[i] - so - no) + ax * (e - w) + ay * (no - so);
      }
  }
}

/* RBGS, optionally as the block Arnoldi process of Alg. 7: with op, block 1
 * is W_1 = B (the given W) and every later block is W_i = A Q_{i-1}.       */
static int rbgs_core(const double* W, int64_t n, int64_t m, int64_t ldw, int64_t mp, int theta, int64_t k,
                     uint64_t seed, int variant, int ls, int ls_iters, int ls_iters_first, int reorth,
                     const or_stencil* op, double* Q, int64_t ldq, double* R, int64_t ldr, double* S_out,
                     double* P_out, double* stats) {
  /* m need not be a multiple of mp: the last block takes the m - (p-1) mp
     remaining columns (the Arnoldi process needs equal blocks) */
  if (mp <= 0 || n < 1 || k < m || ldw < n || ldq < n || ldr < m) return -1;
  if (op && m % mp != 0) return -1;
  if (theta == OR_THETA_SRHT && k > or_srht_padded(n)) return -1;
  if (theta != OR_THETA_SRHT && k > n) return -1;
  int64_t p = (m + mp - 1) / mp;
  double* S = (double*)calloc((size_t)(k * m), sizeof(double));
  double* P = (double*)calloc((size_t)(k * m), sizeof(double));
  double* Spp = (double*)malloc(sizeof(double) * (size_t)(k * mp));
  double* Rc = (double*)malloc(sizeof(double) * (size_t)(m * mp));
  double* Rii = (double*)malloc(sizeof(double) * (size_t)(mp * mp));
  double* R2 = (double*)malloc(sizeof(double) * (size_t)(m * mp));
  double* R2ii = (double*)malloc(sizeof(double) * (size_t)(mp * mp));
  double* Tmp = (double*)malloc(sizeof(double) * (size_t)(m * mp));
  double* Qtmp = (double*)malloc(sizeof(double) * (size_t)(n * mp));
  double* Wop = op ? (double*)malloc(sizeof(double) * (size_t)(n * mp)) : NULL;
  int rc = 0;
  int passes2 = 0;
  for (int64_t j = 0; j < m; ++j)
    for (int64_t i = 0; i < m; ++i) R[i + j * ldr] = 0.0;

  for (int64_t blk = 0; blk < p; ++blk) {
    int64_t c = blk * mp; /* columns already orthogonalized */
    const int64_t w = m - c < mp ? m - c : mp; /* this block's width */
    const double* Wi = W + c * ldw;
    int64_t ldwi = ldw;
    if (op && blk > 0) { /* Alg. 7, step 2: W_i = A Q_{i-1} */
      or_stencil5_apply(op, Q + (c - mp) * ldq, ldq, w, Wop, n);
      Wi = Wop;
      ldwi = n;
    }
    double* Qi = Q + c * ldq;
    double* Pi = P + c * k;
    double* Si = S + c * k;
    /* step 1: P_i = Theta W_i */
    or_theta_apply(theta, k, n, seed, Wi, ldwi, w, Pi, k);
    /* step 2: R_{1:i-1,i} = argmin ||S_{1:i-1} Y - P_i||_F (with a second pass
       to follow, the first may use its own iteration count) */
    if (c > 0 && solve_ls(ls, (reorth && ls_iters_first > 0) ? ls_iters_first : ls_iters, k, c, S, k, Pi, k, w, Rc,
                          m))
      rc = -2;
    /* step 3: Q'_i = W_i - Q_{1:i-1} R_{1:i-1,i} */
    project(n, c, w, Wi, ldwi, Q, ldq, Rc, m, Qi, ldq);
    /* implicit sketch for Alg. 5: S'_i = P_i - S_{1:i-1} R_{1:i-1,i} */
    if (c > 0) gemm(0, 0, k, w, c, 1.0, S, k, Rc, m, 0.0, Spp, k);
    for (int64_t j = 0; j < w; ++j)
      for (int64_t i = 0; i < k; ++i) Spp[i + j * k] = Pi[i + j * k] - (c > 0 ? Spp[i + j * k] : 0.0);
    /* steps 4-5 */
    if (interblock(variant, n, w, Qi, ldq, Spp, k, theta, k, seed, Rii, mp, Si, k)) rc = -2;

    if (reorth && c > 0) {
      /* second pass (extension): treat Q_i as the block to orthogonalize. */
      ++passes2;
      if (solve_ls(ls, ls_iters, k, c, S, k, Si, k, w, R2, m)) rc = -2;
      for (int64_t j = 0; j < w; ++j)
        for (int64_t i = 0; i < n; ++i) Qtmp[i + j * n] = Qi[i + j * ldq];
      project(n, c, w, Qtmp, n, Q, ldq, R2, m, Qi, ldq);
      gemm(0, 0, k, w, c, 1.0, S, k, R2, m, 0.0, Spp, k);
      for (int64_t j = 0; j < w; ++j)
        for (int64_t i = 0; i < k; ++i) Spp[i + j * k] = Si[i + j * k] - Spp[i + j * k];
      if (interblock(variant, n, w, Qi, ldq, Spp, k, theta, k, seed, R2ii, mp, Si, k)) rc = -2;
      /* R_{1:i-1,i} += R2 R_ii ; R_ii <- R2_ii R_ii */
      gemm(0, 0, c, w, w, 1.0, R2, m, Rii, mp, 0.0, Tmp, m);
      for (int64_t j = 0; j < w; ++j)
        for (int64_t i = 0; i < c; ++i) Rc[i + j * m] += Tmp[i + j * m];
      gemm(0, 0, w, w, w, 1.0, R2ii, mp, Rii, mp, 0.0, Tmp, mp);
      for (int64_t j = 0; j < w; ++j)
        for (int64_t i = 0; i < w; ++i) Rii[i + j * mp] = Tmp[i + j * mp];
    }
    /* assemble column block i of R */
    for (int64_t j = 0; j < w; ++j) {
      for (int64_t i = 0; i < c; ++i) R[i + (c + j) * ldr] = Rc[i + j * m];
      for (int64_t i = 0; i < w; ++i) R[c + i + (c + j) * ldr] = Rii[i + j * mp];
    }
  }
  if (stats) {
    /* step 6: Delta = ||I - S^T S||_F, Delta~ = ||P - S R||_F / ||P||_F */
    double d = 0.0, num = 0.0, den = 0.0;
    for (int64_t j = 0; j < m; ++j)
      for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t h = 0; h < k; ++h) s += S[h + i * k] * S[h + j * k];
        double e = (i == j ? 1.0 : 0.0) - s;
        d += e * e;
      }
    for (int64_t j = 0; j < m; ++j)
      for (int64_t h = 0; h < k; ++h) {
        double s = 0.0;
        for (int64_t i = 0; i <= j; ++i) s += S[h + i * k] * R[i + j * ldr];
        double e = P[h + j * k] - s;
        num += e * e;
        den += P[h + j * k] * P[h + j * k];
      }
    stats[0] = sqrt(d);
    stats[1] = den > 0 ? sqrt(num / den) : 0.0;
    stats[2] = (double)passes2;
  }
  if (S_out) memcpy(S_out, S, sizeof(double) * (size_t)(k * m));
  if (P_out) memcpy(P_out, P, sizeof(double) * (size_t)(k * m));
  free(S); free(P); free(Spp); free(Rc); free(Rii); free(R2); free(R2ii); free(Tmp); free(Qtmp); free(Wop);
  return rc;
}

int or_rbgs(const double* W, int64_t n, int64_t m, int64_t ldw, int64_t mp, int theta, int64_t k, uint64_t seed,
            int variant, int ls, int ls_iters, int ls_iters_first, int reorth, double* Q, int64_t ldq, double* R,
            int64_t ldr, double* S_out, double* P_out, double* stats) {
  return rbgs_core(W, n, m, ldw, mp, theta, k, seed, variant, ls, ls_iters, ls_iters_first, reorth, NULL, Q, ldq, R,
                   ldr, S_out, P_out, stats);
}

/* Alg. 7 (RBGS-Arnoldi) for the stencil operator: Q = Q_(1:p) (n x p mp) and
 * R = R_(1:p,1:p); the block Hessenberg matrix is H = R_(1:p,2:p), so that
 * A Q_(1:p-1) = Q_(1:p) H.                                                  */
int or_rbgs_arnoldi(int64_t nx, int64_t ny, double bx, double by, const double* B, int64_t ldb, int64_t mp,
                    int64_t p, int theta, int64_t k, uint64_t seed, int variant, int ls, int ls_iters,
                    int ls_iters_first, int reorth, double* Q, int64_t ldq, double* R, int64_t ldr, double* stats) {
  or_stencil op = {nx, ny, bx, by};
  return rbgs_core(B, nx * ny, p * mp, ldb, mp, theta, k, seed, variant, ls, ls_iters, ls_iters_first, reorth, &op, Q,
                   ldq, R, ldr, NULL, NULL, stats);
}

/* Least squares min ||A z - b|| (A m x n, m >= n, full rank) for nrhs right
 * sides by Householder QR; A and B are overwritten, Z (n x nrhs) receives z. */
static int householder_ls(int64_t m, int64_t n, double* A, int64_t lda, double* B, int64_t ldb, int64_t nrhs,
                          double* Z, int64_t ldz) {
  double* tau = (double*)malloc(sizeof(double) * (size_t)n);
  or_householder_qr(m, n, A, lda, tau);
  householder_apply_qt(m, n, A, lda, tau, B, ldb, nrhs);
  free(tau);
  for (int64_t r = 0; r < nrhs; ++r)
    for (int64_t i = n - 1; i >= 0; --i) {
      double s = B[i + r * ldb];
      for (int64_t t = i + 1; t < n; ++t) s -= A[i + t * lda] * Z[t + r * ldz];
      if (A[i + i * lda] == 0.0) return -2;
      Z[i + r * ldz] = s / A[i + i * lda];
    }
  return 0;
}

/* Restarted randomized block GMRES (Sec. 5.2) or FOM (Sec. 5.3) for A X = B
 * (n x mp, FP64).  Each cycle runs Alg. 7 on the residual block r = B - A X
 * with p blocks and takes the coordinates z of the correction in Q_(1:p-1):
 *   GMRES: z = argmin || H z - R_(1:p,1) ||   (H = R_(1:p,2:p), eq. GMRESsol)
 *   FOM:   z = H_(1:p-1,1:p-1)^{-1} R_(1:p-1,1)                 (eq. RFOMsol)
 * then X += Q_(1:p-1) z.  Stops when max_j ||r_j|| / ||b_j|| <= rtol or after
 * max_cycles cycles; relres (mp) receives the final relative residuals.
 * method: 0 = GMRES, 1 = FOM.  Returns the number of cycles run, or < 0.   */
int or_block_krylov(int method, int64_t nx, int64_t ny, double bx, double by, const double* B, int64_t ldb,
                    double* X, int64_t ldx, int64_t mp, int64_t p, int theta, int64_t k, uint64_t seed, int variant,
                    int ls, int ls_iters, int ls_iters_first, int reorth, double rtol, int64_t max_cycles,
                    double* relres) {
  or_stencil op = {nx, ny, bx, by};
  const int64_t n = nx * ny, m = p * mp, nk = m - mp;
  if (p < 2 || mp < 1 || k < m) return -1;
  double* r = (double*)malloc(sizeof(double) * (size_t)(n * mp));
  double* Q = (double*)malloc(sizeof(double) * (size_t)(n * m));
  double* R = (double*)malloc(sizeof(double) * (size_t)(m * m));
  double* H = (double*)malloc(sizeof(double) * (size_t)(m * nk));
  double* rhs = (double*)malloc(sizeof(double) * (size_t)(m * mp));
  double* Z = (double*)malloc(sizeof(double) * (size_t)(nk * mp));
  double* bn = (double*)malloc(sizeof(double) * (size_t)mp);
  int64_t cyc = 0;
  int rc = 0;
  for (int64_t j = 0; j < mp; ++j) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += B[i + j * ldb] * B[i + j * ldb];
    bn[j] = sqrt(s) > 0.0 ? sqrt(s) : 1.0;
  }
  for (;;) {
    or_stencil5_apply(&op, X, ldx, mp, r, n);
    double worst = 0.0;
    for (int64_t j = 0; j < mp; ++j) {
      double s = 0.0;
      for (int64_t i = 0; i < n; ++i) {
        r[i + j * n] = B[i + j * ldb] - r[i + j * n];
        s += r[i + j * n] * r[i + j * n];
      }
      relres[j] = sqrt(s) / bn[j];
      if (relres[j] > worst) worst = relres[j];
    }
    if (worst <= rtol || cyc >= max_cycles) break;
    if (rbgs_core(r, n, m, n, mp, theta, k, seed, variant, ls, ls_iters, ls_iters_first, reorth, &op, Q, n, R, m, NULL,
                  NULL, NULL)) {
      rc = -2;
      break;
    }
    if (method == 0) {
      for (int64_t j = 0; j < nk; ++j)
        for (int64_t i = 0; i < m; ++i) H[i + j * m] = R[i + (mp + j) * m];
      for (int64_t j = 0; j < mp; ++j)
        for (int64_t i = 0; i < m; ++i) rhs[i + j * m] = R[i + j * m];
      if (householder_ls(m, nk, H, m, rhs, m, mp, Z, nk)) { rc = -2; break; }
    } else {
      for (int64_t j = 0; j < nk; ++j)
        for (int64_t i = 0; i < nk; ++i) H[i + j * nk] = R[i + (mp + j) * m];
      for (int64_t j = 0; j < mp; ++j)
        for (int64_t i = 0; i < nk; ++i) rhs[i + j * nk] = R[i + j * m];
      if (householder_ls(nk, nk, H, nk, rhs, nk, mp, Z, nk)) { rc = -2; break; }
    }
    /* X += Q_(1:p-1) z */
    gemm(0, 0, n, mp, nk, 1.0, Q, n, Z, nk, 1.0, X, ldx);
    ++cyc;
  }
  free(r); free(Q); free(R); free(H); free(rhs); free(Z); free(bn);
  return rc ? rc : (int)cyc;
}

/* Closed form of RBGS in exact arithmetic: R = R factor (positive diagonal)
 * of the thin QR of Theta W; Q = W R^{-1}.  This is the same factorization
 * as RCholeskyQR of W (remark after Alg. 5).                               */
int or_rcholqr(const double* W, int64_t n, int64_t m, int64_t ldw, int theta, int64_t k, uint64_t seed, double* Q,
               int64_t ldq, double* R, int64_t ldr) {
  double* P = (double*)malloc(sizeof(double) * (size_t)(k * m));
  if (or_theta_apply(theta, k, n, seed, W, ldw, m, P, k)) { free(P); return -1; }
  int rc = or_qr_r(k, m, P, k, R, ldr);
  for (int64_t j = 0; j < m; ++j)
    for (int64_t i = 0; i < n; ++i) Q[i + j * ldq] = W[i + j * ldw];
  trsm_right_upper(n, m, R, ldr, Q, ldq);
  free(P);
  return rc ? -2 : 0;
}

/* Exported step-2 solver, for tests of the supplement's error bounds.       */
int or_ls_solve(int ls, int ls_iters, int64_t k, int64_t c, const double* S, int64_t lds, const double* P, int64_t ldp,
                int64_t mp, double* X, int64_t ldx) {
  return solve_ls(ls, ls_iters, k, c, S, lds, P, ldp, mp, X, ldx);
}
