// Internal interfaces between the librbgs translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/rbgs.h"

namespace rbgs {

// ---------------------------------------------------------------- sketches --
// SRHT plan: sampled Hadamard rows split as i = i_hi * B + i_lo with the tile
// length B = min(n', kSrhtTile); L = sorted distinct i_lo values.
constexpr int kSrhtTile = 16384;

struct SrhtPlan {
  uint64_t seed = 0;
  int64_t n = 0, np = 0, k = 0;
  int B = 0, T = 0, L = 0;   // tile length, number of tiles, distinct low indices
  int* d_lvals = nullptr;    // [L]  distinct low indices (sorted)
  int* d_rhi = nullptr;      // [k]  i_hi of sample r
  int* d_rl = nullptr;       // [k]  position of i_lo(sample r) in lvals
  int* d_off = nullptr;      // [L+1] CSR offsets: samples whose low index is lvals[l]
  int* d_rs = nullptr;       // [k]  sample indices grouped by low index
  std::vector<int64_t> samples;
};

// Host: k distinct sorted rows of the n' x n' Hadamard matrix (Floyd's
// algorithm on the Philox stream of purpose 3).
int srht_samples_host(uint64_t seed, int64_t np, int64_t k, int64_t* out);

// Cached per (device, seed, n, k).
rbgs_status srht_plan_get(uint64_t seed, int64_t n, int64_t k, const SrhtPlan** plan);
void srht_plans_release();

// Scratch (bytes) needed by sketch_apply for `ncols` columns.
size_t sketch_scratch_bytes(rbgs_sketch kind, int64_t k, int64_t n, int64_t ncols, bool fp64);

// Y (k x ncols, ldy) = Theta X (n x ncols, ldx).  TX = float|double input,
// TY = float|double output; the arithmetic is double iff TX is double.
template <class TX, class TY>
rbgs_status sketch_apply_t(rbgs_sketch kind, int64_t k, int64_t n, uint64_t seed, const TX* X, int64_t ldx,
                           int64_t ncols, TY* Y, int64_t ldy, void* scratch, size_t scratch_bytes,
                           cudaStream_t st, const int* active = nullptr);

// Two-source form: Y1 = Theta X1 and Y2 = Theta X2 in one pass (the SRHT
// transforms all columns in the same launches).
template <class TX, class TY>
rbgs_status sketch_apply2_t(rbgs_sketch kind, int64_t k, int64_t n, uint64_t seed, const TX* X1, int64_t ldx1,
                            int64_t nc1, TY* Y1, int64_t ldy1, const TX* X2, int64_t ldx2, int64_t nc2, TY* Y2,
                            int64_t ldy2, void* scratch, size_t scratch_bytes, cudaStream_t st,
                            const int* active = nullptr);

// --------------------------------------------------------------- tall ops ---
// Qout (n x mb) = [A1 (n x c) | A2 (n x mb)] * G ((c+mb) x mb, ldg).  Qout may
// alias A2 exactly.  mb <= 64.
template <class T>
rbgs_status tall_update_simt(int64_t n, int64_t c, int64_t mb, const T* A1, int64_t lda1, const T* A2, int64_t lda2,
                             const T* G, int64_t ldg, T* Qout, int64_t ldo, const int* active, cudaStream_t st);

// tcgen05 3xTF32 version; Gsplit is the TF32 hi/lo split of G in the B-operand
// layout (tc_split_g).  Needs 16-byte aligned A1/A2 and ld % 4 == 0; *err is
// set (1, 2, 3) when a bounded device-side wait expires.
rbgs_status tall_update_tc(int64_t n, int64_t c, int64_t mb, const float* A1, int64_t lda1, const float* A2,
                           int64_t lda2, const float* Gsplit, float* Qout, int64_t ldo, const int* active, int* err,
                           cudaStream_t st);
size_t tc_gsplit_floats(int64_t K);  // floats needed for the split G of K rows
// Build the split operand of the tensor-core kernel from the FP64 G.
rbgs_status tc_split_g(int64_t K, int64_t mb, const double* G, int64_t ldg, float* Gsplit, const int* active,
                       cudaStream_t st);

// FP16 hi/lo split tensor-core version (tall_h3.cu).  The previous basis is
// pre-split in a tiled layout (per 128-row tile, h3_nch_row(m) chunks of 64
// columns, 32 KB each); the block's own columns `raw` (FP32) are split in the
// kernel.  h3_prepare builds the split G (B) and the scales from the sketch of
// the raw block (Sraw, k x mb) or from its column maxima (rawmax); qscale are
// the per-column scales of the pre-split basis (null: 2^9 for every column).
int64_t h3_nch_row(int64_t m);
size_t h3_qs_bytes(int64_t n, int64_t m);
size_t h3_b_bytes(int64_t c);
// Output-column shift that aligns the split copy of columns cs_out.. to 8-column groups.
int h3_shift(int64_t cs_out, int64_t mb, bool split_out);
template <class TS>
rbgs_status h3_prepare(int64_t c, int64_t mb, const double* G, int64_t ldg, const TS* Sraw, int64_t k,
                       const float* rawmax, const float* qscale, int jsh, unsigned char* B, float* scales,
                       const int* active, cudaStream_t st);
rbgs_status tall_update_h3(int64_t n, int64_t c, int64_t mb, const unsigned char* qs, int64_t nch_row,
                           const float* raw, int64_t ldr, const unsigned char* B, const float* scales, float* Qout,
                           int64_t ldo, unsigned char* qs_out, int64_t cs_out, int jsh, const int* active, int* err,
                           cudaStream_t st);
rbgs_status h3_colmax(int64_t n, int64_t cols, const float* A, int64_t lda, unsigned int* mx, cudaStream_t st);
rbgs_status h3_scales_from_max(int64_t cols, const unsigned int* mx, float* scale, cudaStream_t st);
rbgs_status h3_split(int64_t n, int64_t cols, const float* A, int64_t lda, const float* scale, int64_t nch_row,
                     unsigned char* qs, cudaStream_t st);

// --------------------------------------------------------- Krylov (Sec. 5) --
template <class TI, class TO>
rbgs_status stencil_apply_t(const rbgs_op& op, const TI* X, int64_t ldx, int64_t ncols, TO* Y, int64_t ldy,
                            cudaStream_t st);
size_t residual_part_elems(int64_t n, int64_t ncols);
// r = B - A X (FP64) and norms[j] = ||r_j|| (part: residual_part_elems scratch)
rbgs_status residual_t(const rbgs_op& op, const double* B, int64_t ldb, const double* X, int64_t ldx,
                       int64_t ncols, double* r, int64_t ldr, double* part, double* norms, cudaStream_t st);
rbgs_status colnorms_t(int64_t n, int64_t ncols, const double* A, int64_t lda, double* part, double* norms,
                       cudaStream_t st);
template <class TI, class TO>
rbgs_status cast_cols_t(int64_t n, int64_t ncols, const TI* A, int64_t lda, TO* B, int64_t ldb, cudaStream_t st);
template <class TD>
rbgs_status add_cols_t(int64_t n, int64_t ncols, const TD* D, int64_t ldd, double* X, int64_t ldx, cudaStream_t st);
// min ||H z - F|| with H (M x N) zero below its bw-th subdiagonal (overwrites H, F)
rbgs_status banded_ls(int M, int N, int bw, double* H, int ldh, double* F, int ldf, int nrhs, double* Z, int ldz,
                      int* flag, cudaStream_t st);

// ------------------------------------------------------------ sketch space --
// out (M x N, ldo) = alpha * op(A) * B + beta * out, op(A) = A (TRANS=0, A M x K)
// or A^T (TRANS=1, A K x M); B K x N; N <= 64.  TA/TB input, TO output type,
// accumulation in TACC.  Uses `part` scratch of ksplit * M * N TACC.
template <class TA, class TO, class TACC>
rbgs_status small_gemm(int trans, int64_t M, int64_t N, int64_t K, double alpha, const TA* A, int64_t lda,
                       const TA* B, int64_t ldb, double beta, TO* out, int64_t ldo, TACC* part, int64_t part_elems,
                       const int* active, cudaStream_t st);
// While an instance is alive on this host thread, the FP64 small products
// run in double-FP32 arithmetic on the FP32 pipe (about 2^-44 relative): the
// mixed-precision path's FP64 sketch space with opts.fine = 2.  The dense
// sketches keep their FP64 sums.  The FP64 path never sets it.
extern thread_local int g_df_products;
struct DfProducts {
  explicit DfProducts(bool on);
  ~DfProducts();
  int prev;
};

// Cholesky G (+ shift * trace(G) I) = R^T R (upper R, positive diagonal) of an
// mb x mb matrix and R^{-1}, in the arithmetic of T; sets *flag |= 1 on a
// non-positive or non-finite pivot.
// With Rprev != null (a second Cholesky QR round) R and Rinv receive the
// products R_new Rprev and Rprev_inv R_new^{-1}.
template <class T>
rbgs_status chol_inv(int mb, const T* G, T* R, T* Rinv, double shift, int* flag, const T* Rprev, const T* Rprev_inv,
                     const int* active, cudaStream_t st);

// One panel of the blocked Householder QR of the sketch (step 2 by Householder
// least squares): rows c..k-1 of B (k x w, ld ldb, holding Q_c^T S_i) factorised
// in place; writes the explicit reflectors V (k x w, ld ldv), the panel's
// compact-WY factor T and the inverse of its R (w x w each, ld ldm, zero below
// the diagonal); *flag |= 1 on a zero or non-finite diagonal of R.  w <= 64.
template <class TS>
rbgs_status hh_panel(int64_t k, int64_t c, int w, TS* B, int64_t ldb, TS* V, int64_t ldv, TS* T, TS* Ri,
                     int64_t ldm, int* flag, cudaStream_t st);

// Out (k x mb, ldo) = A (k x mb, lda) * U (U upper mb x mb, ld mb).
template <class TS>
rbgs_status trmm_right_upper(int64_t k, int mb, const TS* A, int64_t lda, const TS* U, TS* Out, int64_t ldo,
                             const int* active, cudaStream_t st);

// C (mb x mb) = A * B for upper-triangular mb x mb matrices (ld mb).
template <class T>
rbgs_status tri_mul(int mb, const T* A, const T* B, T* C, const int* active, cudaStream_t st);

// Coefficient matrix of the fused projection + triangular solve and the R
// column block:  G = [-Rc * Rii^{-1} ; Rii^{-1}]  ((c+mb) x mb, ldg), written
// as TG; when `R` is non-null also R[0:c, col] = Rc, R[c:c+mb, col] = Rii.
template <class TS, class TG>
rbgs_status assemble_g(int64_t c, int mb, const TS* Rc, int64_t ldrc, const TS* Rii, const TS* Riinv,
                       TG* G, int64_t ldg, double* R, int64_t ldr, const int* active, cudaStream_t st);

// Second-pass update of the R column block:
//   R[0:c, col] += R2c * Rii_old ;  R[c:c+mb, col] = R2ii * Rii_old
// with Rii_old read from R[c:c+mb, col] (upper part).
template <class TS>
rbgs_status reorth_update_r(int64_t c, int mb, const TS* R2c, int64_t ldr2, const TS* R2ii, double* Rcol,
                            int64_t ldr, double* tmp, const int* active, cudaStream_t st);

// Adaptive second pass: flag = (||X||_F > tol) with X c x mb; counts passes.
template <class TS>
rbgs_status reorth_decide(int64_t c, int mb, const TS* X, int64_t ldx, double tol, int mode, int* active,
                          int* count, int* blk_flag, cudaStream_t st);

// Whether a Cholesky QR round may be the last one: with R1 and R1^{-1} from
// one round, need2 = (active) and ||R1||_F ||R1^{-1}||_F > thr.  When the round
// is the last one, R1 and R1inv are copied into R and Rinv (mb x mb, ld mb);
// count is incremented for every second round that will run.
template <class T>
rbgs_status round2_decide(int mb, const T* R1, const T* R1inv, T* R, T* Rinv, double thr, const int* active,
                          int* need2, int* count, cudaStream_t st);

// Alg. 8, step 2-3: the mp extreme eigenpairs of the N x N matrix H (ld ldh,
// N + mb rows: rows N.. are H_(p,1:p-1)); which 0 = largest real part, 1 =
// smallest.  vals: 2 mp doubles (re, im per column), Y: N x mp (ld N), resid:
// mp residual estimates; *status = 0 or 1 (QR iteration did not converge).
// scratch: ritz_eig_scratch_bytes(N, mb, mp).  One CTA (FP32 estimates, FP64 refinement).
constexpr int kRitzMaxN = RBGS_RITZ_MAX_N;
size_t ritz_eig_scratch_bytes(int N, int mb, int mp);
rbgs_status ritz_eig(int N, int mb, int mp, int which, const double* H, int64_t ldh, double* vals, double* Y,
                     double* resid, void* scratch, int* status, cudaStream_t st);
// X[:, j] /= norms[j] (n x ncols, double)
rbgs_status scale_cols(int64_t n, int64_t ncols, const double* norms, double* X, int64_t ldx, cudaStream_t st);

// Conjugate gradients on the normal equations of step 2, column by column:
// cg_init sets rr = ||r_j||^2 (r = S^T p); cg_step performs one step given
// q = S^T S d (all c x mb with leading dimension ld; X with ldx).
template <class TS>
rbgs_status cg_init(int64_t c, int mb, const TS* Rr, int64_t ld, double* rr, int* done, cudaStream_t st);
template <class TS>
rbgs_status cg_step(int64_t c, int mb, TS* X, int64_t ldx, TS* Rr, TS* D, const TS* Qq, int64_t ld, double* rr,
                    int* done, cudaStream_t st);

// Elementwise C = A - B (k x mb) in TS.
template <class TS>
rbgs_status sub_mat(int64_t k, int64_t mb, const TS* A, int64_t lda, const TS* B, int64_t ldb, TS* C, int64_t ldc,
                    const int* active, cudaStream_t st);

// Q <- Q R^{-1} by a row-wise forward substitution (tall_simt.cu).
template <class T, class TS>
rbgs_status trsm_rows(int64_t n, int mb, T* Q, int64_t ldq, const TS* R, const int* active, cudaStream_t st);

// Face coefficients of RBGS_OP_DIFFUSION from node values (krylov.cu).
rbgs_status diffusion_faces(int64_t nx, int64_t ny, const double* a, double* fc, cudaStream_t st);

// The tensor-core 3 x 3 convolution (unet_tc.cu): out = conv3x3(in) with
// bfloat16 NHWC input (ld_in, channel offset off_in), weights packed by
// conv_tc_pack (flip: the backward convolution's flipped, transposed weights
// of a layer with cin and cout exchanged), bias and relu optional, output
// bfloat16 (out_bf16) or FP32.
bool conv_tc_supported(int N, int cin, int cout, int64_t ld_in, int off_in, int64_t ld_out, int off_out);
size_t conv_tc_pack_bytes(int cin, int cout);
rbgs_status conv_tc_pack(int cin, int cout, const float* w, int flip, void* packed, cudaStream_t st);
rbgs_status conv_tc(int N, int batch, int cin, int cout, const void* in, int64_t ld_in, int off_in, const void* packed,
                    const float* bias, int relu, void* out, int out_bf16, int64_t ld_out, int off_out, int* err,
                    cudaStream_t st);

// The U-Net preconditioner (unet.cu): Z (n x ncols, ldz) = M(Q) column by
// column, M(q) = s (h^2 / 8) U-Net(q / s), s = ||q|| / sqrt(n), h = 1 / (N + 1).
template <class T>
rbgs_status unet_precondition(const rbgs_unet& net, const float* params, int N, int ncols, const T* Q, int64_t ldq,
                              T* Z, int64_t ldz, cudaStream_t st);
bool unet_valid(const rbgs_unet* net, int64_t N);
// Frees the U-Net buffers of device dev (rbgs_release_workspace).
void unet_release(int dev);

// Forgets the no-allocation entry point's looked-up scratch address on device
// dev (noalloc.cu); the next call there looks it up again.
void noalloc_forget_device(int dev);

// Frobenius norms for step 6.
rbgs_status fro_identity_defect(int64_t m, const double* G, int64_t ldg, double* out, cudaStream_t st);
rbgs_status fro_norm_diff(int64_t rows, int64_t cols, const double* A, int64_t lda, const double* B, int64_t ldb,
                          double* out_diff, double* out_a, cudaStream_t st);

}  // namespace rbgs
