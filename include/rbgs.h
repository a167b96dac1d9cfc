/*
 * rbgs.h -- C ABI of librbgs: randomized block Gram-Schmidt (RBGS) on one
 * NVIDIA GB300 (sm_103a).
 *
 * Method: Balabanov & Grigori, "Randomized block Gram-Schmidt process for the
 * solution of linear systems and eigenvalue problems", arXiv 2111.14641.
 *
 * Conventions shared by every entry point
 *  - Matrices are column-major with an explicit leading dimension (ld >= rows).
 *  - Pointers named W, Q, X, Y, R, ... are DEVICE pointers on the current CUDA
 *    device unless the comment says "host".  The caller owns them; the library
 *    never frees or keeps them beyond the call.
 *  - Element type: double when prec == RBGS_P_FP64, otherwise float (W, Q, X).
 *    R and the sketches Y returned to the caller are always double.
 *  - Work is enqueued on opts->stream (a cudaStream_t; NULL = legacy default).
 *    With opts->sync != 0 (the default) the call waits for its work and reports
 *    device-side failures (breakdown) in its return code.
 *  - Errors are reported only through the return code; nothing aborts, traps
 *    or prints.  Internal workspace is allocated by the library (cudaMalloc),
 *    cached per device and released by rbgs_release_workspace().
 *  - Entry points are not re-entrant for concurrent calls on different host
 *    threads (they share the cached workspace).
 */
#ifndef RBGS_H
#define RBGS_H

#include <stdint.h>

#if defined(__GNUC__)
#define RBGS_API __attribute__((visibility("default")))
#else
#define RBGS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RBGS_OK = 0,
  RBGS_EINVAL = 1,         /* an argument is out of range (sizes, ld, null pointer)          */
  RBGS_ENOMEM = 2,         /* device workspace allocation failed                            */
  RBGS_ECUDA = 3,          /* a CUDA runtime call or a kernel launch failed                  */
  RBGS_EBREAKDOWN = 4,     /* R_ii got a non-positive or non-finite pivot (rank breakdown)   */
  RBGS_ENOTCERTIFIED = 5,  /* Delta or Delta~ > 0.1, Thm. 4.1 cannot certify (on request)    */
  RBGS_ETIMEOUT = 6,       /* a bounded device-side wait expired                            */
  RBGS_ENOCONV = 7,        /* an iterative solver stopped before its tolerance               */
  RBGS_ENODEV = 8,         /* no usable sm_103 device                                        */
  RBGS_ETOOLARGE = 9       /* c + mb > RBGS_NOALLOC_MAX_K in rbgs_tall_update_noalloc        */
} rbgs_status;

/* Sketching matrices Theta (k x n).  Sec. 2.3 uses Rademacher and SRHT; the
 * Gaussian N(0, 1/k) matrix is the classical oblivious embedding, and the
 * sparse sign matrix is the block construction of the sparse JL transform
 * (Kane and Nelson 2014): z = min(8, k) row segments, one nonzero
 * +-1/sqrt(z) per segment and column (neither is in the paper).  Theta is
 * never stored: its entries are regenerated from a Philox4x32-10 counter
 * generator keyed by (seed_lo, seed_hi), counter word 2 naming the stream
 * (0 Gaussian, 1 Rademacher, 2 SRHT signs, 3 SRHT row sampling, 4 sparse
 * sign); the CPU oracle implements the same definitions independently.
 * Every kind needs k <= n, SRHT k <= 2^ceil(log2 n).                       */
typedef enum { RBGS_SK_GAUSS = 0, RBGS_SK_RADEMACHER = 1, RBGS_SK_SRHT = 2, RBGS_SK_SPARSE = 3 } rbgs_sketch;

/* Arithmetic of the tall (n-row) operations: the projection of step 3 fused
 * with R_ii^{-1}, and the sketches.
 *  FP64    double storage, double arithmetic everywhere.
 *  FP32    float storage of W and Q; SIMT FP32 tall product; sketches
 *          computed in FP32.  The sketch-space steps (least squares, block
 *          Cholesky QR, R) run in FP64 with opts->fine = 1, else in FP32.
 *  TF32X3  as FP32, but the tall product runs on the tcgen05 tensor cores
 *          with split operands (a = a_hi + a_lo in TF32, three products),
 *          accurate to about 2^-22 relative per product.
 *  F16X3   as TF32X3, with FP16 hi/lo splits under power-of-two column
 *          scales (three kind::f16 products, also about 2^-22).  rbgs_qr
 *          keeps the split of the finished Q columns in its workspace, so the
 *          previous basis streams into the tensor cores without conversion.
 *          The workspace grows by 4 bytes per element of Q.                 */
typedef enum { RBGS_P_FP64 = 0, RBGS_P_FP32 = 1, RBGS_P_TF32X3 = 2, RBGS_P_F16X3 = 3 } rbgs_prec;

typedef struct {
  int32_t prec;        /* rbgs_prec                                                      */
  int32_t ls_iters;    /* step 2: Richardson iterations X <- X + S^T (P - S X) (>= 1)   */
  int32_t reorth;      /* 0: Alg. 2 as written (one projection per block);
                          1: second projection pass on every block i > 1;
                          2: second pass only where ||S_{1:i-1}^T S_i||_F > reorth_tol */
  int32_t certify;     /* 1: compute Delta and Delta~ (step 6) into stats             */
  double reorth_tol;   /* threshold for reorth == 2                                      */
  void* stream;        /* cudaStream_t                                                   */
  int32_t sync;        /* 1: wait and report device-side status; 0: enqueue only        */
  int32_t timing;      /* 1: time the tall-update launches with CUDA events (needs sync) */
  int32_t fine;        /* FP32 / TF32X3 / F16X3: 1 = the sketch-space steps (P and S stored,
                          step-2 least squares, block Cholesky QR, R) in FP64 (the
                          paper's u_fine); 2 = the same, with the sketch-space products
                          in double-FP32 arithmetic on the FP32 pipe (about 2^-44
                          relative; GB300's FP64 pipe is narrow); the dense sketches
                          still sum in FP64; 0 = in FP32                              */
  int32_t interblock;  /* steps 4-5: 0 or 5 = Alg. 5 (the sketch of Q'_i taken implicitly as
                          P_i - S R, one tall pass per block); 4 = Alg. 4 (RCholeskyQR on
                          the explicit sketch Theta Q'_i: the projection, a sketch, and an
                          in-place scaling by R_ii^{-1}, two tall passes per block);
                          1 = single-vector RGS and 3 = vRCholeskyQR (Alg. 3): after the
                          projection, the block's columns one at a time (RBGS with
                          one-column blocks on Q'_i, explicit or implicit sketches; needs
                          reorth 0 or 1; not for the Sec. 5 solvers); 6 = Alg. 6: an l2
                          QR Q'_i = Q* R' (Cholesky QR twice, FP64 Gram matrices over
                          the n rows, four tall passes), then Alg. 4 on Q*, R_ii =
                          R'' R' (breaks down where kappa_2(Q'_i) nears 1e8; not for
                          the Sec. 5 solvers)                                            */
  int32_t ls;          /* step 2 solver: 0 = Richardson (X <- X + S^T (P - S X), ls_iters
                          steps from 0); 1 = conjugate gradients on the normal equations
                          (S^T S) X = S^T P, ls_iters steps from 0, column by column
                          (Sec. 3.1 and its supplement); 2 = Householder least squares:
                          a blocked Householder QR of S kept in compact WY form, one
                          panel appended per block, X = R_S^{-1} (Q_S^T P)_{1:c}
                          (ls_iters unused; not for the Sec. 5 solvers)                 */
  int32_t trsm;        /* with interblock 4: 1 = Q_i = Q'_i R_ii^{-1} by a row-wise triangular
                          solve (forward substitution, backward stable whatever cond(R_ii))
                          instead of the product with the explicit inverse (the remark
                          after Alg. 4), whose error grows with cond(R_ii): needed when a
                          block is numerically rank deficient in the storage precision
                          (near-duplicate columns); with FP32 storage the first
                          Cholesky round of an FP64 sketch space then takes the shift
                          of shifted Cholesky QR, so that such a block's sketch cannot
                          break it down;
                          0 = the explicit inverse (default).
                          RBGS_EINVAL with another interblock                            */
} rbgs_opts;

typedef struct {
  double delta;        /* ||I - S^T S||_F, S = Theta Q (step 6 of Alg. 2)              */
  double delta_tilde;  /* ||P - S R||_F / ||P||_F, P = Theta W                          */
  int32_t passes2;     /* blocks that took the second projection pass                   */
  int32_t certified;   /* delta <= 0.1 && delta_tilde <= 0.1 (Thm. 4.1 hypothesis)      */
  double tall_ms;      /* with opts->timing: summed duration of the tall-update launches */
  double tall_bytes;   /* algorithmic bytes those launches move (A read + Q_i written)  */
  int32_t tall_launches; /* tall-update launches that did work                          */
  int32_t chol_rounds2;  /* block Cholesky QR factorizations that took a second round
                            (always, in the FP32 sketch space; in FP64 only where
                            ||R1||_F ||R1^{-1}||_F > 4 m_p after the first round)       */
  double host_up_ms;      /* rbgs_qr_host with opts->timing: from the start of the call's
                             device work to the last column block of W on the device   */
  double host_compute_ms; /* ... to the last column block of Q final on the device      */
  double host_total_ms;   /* ... to Q and R back on the host (0 without opts->timing)   */
} rbgs_stats;

/* Fill *opts with the defaults: FP64, 2 Richardson iterations, reorth 0,
 * certify 0, reorth_tol 1e-8, default stream, sync 1.                     */
RBGS_API void rbgs_opts_default(rbgs_opts* opts);

/* RBGS QR factorization, Alg. 2 with steps 4-5 by Alg. 5 (RCholeskyQR with the
 * sketch of Q'_i obtained as P_i - S_{1:i-1} R_{1:i-1,i}, one reduction per
 * block) and step 2 by Richardson iterations (supplement to Sec. 3.1).
 *
 *  W    device, n x m, ld ldw >= n, float or double per opts->prec (read only)
 *  n    rows, 1 <= n < 2^31
 *  m    columns, m = mb * p
 *  mb   block size m_p, 1 <= mb <= 64; when mb does not divide m the last of
 *       the p = ceil(m / mb) blocks holds the m - (p - 1) mb remaining columns
 *  sketch, k, seed   Theta (k x n); m <= k; k <= n (Gaussian, Rademacher) or
 *       k <= n' = 2^ceil(log2 n) (SRHT)
 *  Q    device, n x m, ld ldq >= n, same type as W; receives the
 *       sketch-orthonormal factor ((Theta Q)^T (Theta Q) = I up to rounding)
 *  R    device, m x m double, ld ldr >= m; receives the upper-triangular
 *       factor with positive diagonal (strictly lower part set to zero)
 *  opts may be NULL (defaults); stats may be NULL (host pointer).
 * W and Q must not overlap.  Returns RBGS_OK, RBGS_EINVAL, RBGS_ENOMEM,
 * RBGS_ECUDA or RBGS_EBREAKDOWN (the last only with opts->sync).          */
RBGS_API rbgs_status rbgs_qr(const void* W, int64_t n, int64_t m, int64_t ldw, int64_t mb, rbgs_sketch sketch, int64_t k,
                    uint64_t seed, void* Q, int64_t ldq, double* R, int64_t ldr, const rbgs_opts* opts,
                    rbgs_stats* stats);

/* Many independent factorizations in one call (the same sketch kind and
 * options for all).  Each problem gives W, Q, R and its sizes as for rbgs_qr,
 * and receives status (RBGS_OK, RBGS_EBREAKDOWN or RBGS_ETIMEOUT) and
 * passes2.  The problems run on min(nstreams, count, 32) internal streams,
 * each with its own workspace and side stream, problem i on stream i mod
 * nstreams, with no host synchronisation before the end of the batch; the
 * batch starts after the work already on opts->stream and that stream waits
 * for it.  Every problem is checked as in rbgs_qr before any work starts
 * (RBGS_EINVAL).  opts->sync, timing and certify are ignored.  Returns the
 * first problem's error, else RBGS_OK.  Synchronous.  The paper has no
 * batched form; this serves many small factorizations at once.          */
typedef struct {
  const void* W;  /* n x m, ldw (device, prec type) */
  int64_t n, m, ldw, mb, k;
  uint64_t seed;
  void* Q;        /* n x m, ldq (device, prec type) */
  int64_t ldq;
  double* R;      /* m x m, ldr (device) */
  int64_t ldr;
  int32_t status; /* out */
  int32_t passes2; /* out */
} rbgs_problem;
RBGS_API rbgs_status rbgs_qr_batched(rbgs_problem* probs, int64_t count, rbgs_sketch sketch, const rbgs_opts* opts,
                                     int32_t nstreams);

/* rbgs_qr on HOST buffers: W (n x m, ldw), Q (n x m, ldq) and R (m x m, ldr)
 * are host arrays of the prec type (R double).  The library keeps device
 * copies (grown on demand, freed by rbgs_release_workspace).  Column block i
 * of W goes to the device on a copy stream ahead of the factorization, block
 * i of the factorization waits only for its own block, and each column block
 * of Q is copied back as soon as it is final, while later blocks compute; R
 * follows at the end.  With page-locked (pinned) host memory the copies
 * overlap the computation; pageable memory gives the same result without the
 * overlap.  Options and errors as rbgs_qr (no certification; stats receives
 * passes2 and chol_rounds2, and with opts->timing the copy and compute
 * timeline host_up_ms, host_compute_ms and host_total_ms instead of the
 * tall-launch timing).  Synchronous.                                        */
RBGS_API rbgs_status rbgs_qr_host(const void* W, int64_t n, int64_t m, int64_t ldw, int64_t mb, rbgs_sketch sketch,
                                  int64_t k, uint64_t seed, void* Q, int64_t ldq, double* R, int64_t ldr,
                                  const rbgs_opts* opts, rbgs_stats* stats);

/* A posteriori check of the epsilon-embedding property (Sec. 4, the
 * epsilon-embedding subsection): with a second, independent sketch Phi (the
 * same kind and size, seed seed_phi), Y = R_phi^{-1} for R_phi the R factor of
 * Phi Z, and (Theta Z) Y has orthonormal columns when Theta embeds range(Z)
 * without distortion.  Y comes from RBGS of Z with Phi (Q_phi = Z R_phi^{-1};
 * options as rbgs_qr), so (Theta Z) Y = Theta Q_phi.  *defect (host) receives
 * ||I - (Theta Q_phi)^T (Theta Q_phi)||_F, which bounds the distortion of Theta
 * on range(Z) up to that of Phi.  Z: n x m device array of the prec type.
 * Errors as rbgs_qr.  Synchronous; allocates its buffers per call.          */
RBGS_API rbgs_status rbgs_embedding_check(const void* Z, int64_t n, int64_t m, int64_t ldz, int64_t mb,
                                          rbgs_sketch sketch, int64_t k, uint64_t seed_theta, uint64_t seed_phi,
                                          const rbgs_opts* opts, double* defect);

/* Cholesky QR post-processing (the remark after Alg. 2): with R' the
 * Cholesky factor of Q^T Q, Q <- Q R'^{-1} and R <- R' R, in place, so that Q
 * becomes l2-orthonormal and W = Q R still holds.  Q: n x m device array of
 * the prec type (ldq); R: m x m device double (ldr).  Q^T Q is formed with
 * FP64 products (n m^2 FMA on the FP64 pipe), R' by a blocked Cholesky with
 * blocks of mb (<= 64) columns, and Q R'^{-1} by a forward sweep over those
 * blocks on the tall-update kernels of prec.  RBGS_EBREAKDOWN if Q^T Q is
 * not positive definite.  Synchronous (sync is ignored).                  */
RBGS_API rbgs_status rbgs_cholqr_postprocess(int32_t prec, int64_t n, int64_t m, void* Q, int64_t ldq, double* R,
                                             int64_t ldr, int64_t mb, void* stream, int32_t sync);

/* A factorization captured as a CUDA graph, for many factorizations of the
 * same shape on the same buffers (new contents of W each time): create
 * captures one rbgs_qr on W, Q, R (the pointers, sizes and options are fixed
 * in the graph) after one ordinary run that fills the library's caches; the
 * graph owns its workspace, side stream and status words.  launch replays
 * it on stream (asynchronous; with sync, waits and returns the status as
 * rbgs_qr would).  The sketch plans it uses stay cached until
 * rbgs_release_workspace, which must not be called while a graph exists.
 * Not for opts->interblock 1 or 3 (RBGS_EINVAL).  The paper has no
 * counterpart: this removes the per-launch host cost of the ~30 launches per
 * block when the blocks are small.                                          */
typedef struct rbgs_graph rbgs_graph;
RBGS_API rbgs_status rbgs_qr_graph_create(const void* W, int64_t n, int64_t m, int64_t ldw, int64_t mb,
                                          rbgs_sketch sketch, int64_t k, uint64_t seed, void* Q, int64_t ldq,
                                          double* R, int64_t ldr, const rbgs_opts* opts, rbgs_graph** out);
RBGS_API rbgs_status rbgs_qr_graph_launch(rbgs_graph* g, void* stream, int32_t sync);

/* A batch of independent factorizations (as rbgs_qr_batched) captured as one
 * CUDA graph: every problem on one of min(nstreams, count, 32) slot streams
 * with its own workspace and side stream, forked from and joined back to the
 * launching stream, so that rbgs_qr_graph_launch replays the whole batch
 * with a single graph launch (the pointers, sizes and options fixed; new
 * contents of each W each time).  The graph owns the slot streams,
 * workspaces and status words; probs (caller-owned) must stay valid while the
 * graph exists: a launch with sync writes each problem's status and passes2
 * there and returns the first problem's error.  Not for opts->interblock 1
 * or 3.  The paper has no batched form: this removes the host cost of
 * launching every kernel of every problem when the problems are small.     */
RBGS_API rbgs_status rbgs_qr_batched_graph_create(rbgs_problem* probs, int64_t count, rbgs_sketch sketch,
                                                  const rbgs_opts* opts, int32_t nstreams, rbgs_graph** out);
RBGS_API rbgs_status rbgs_qr_graph_destroy(rbgs_graph* g);

/* Y = Theta X (Sec. 2.3), the sketch of steps 1 and 5 of Alg. 2.
 *  X device n x ncols (ldx), double if prec == RBGS_P_FP64 else float.
 *  Y device k x ncols (ldy), double.  The Gaussian, Rademacher and sparse
 *  sketches sum in double for every prec; the SRHT sums in double for FP64
 *  and in float otherwise.  stream: cudaStream_t.  Synchronous only if
 *  sync != 0.                                                              */
RBGS_API rbgs_status rbgs_sketch_apply(rbgs_sketch sketch, int64_t k, int64_t n, uint64_t seed, int32_t prec, const void* X,
                              int64_t ldx, int64_t ncols, double* Y, int64_t ldy, void* stream, int32_t sync);

/* Tall update of step 3 fused with the triangular solve of Alg. 5:
 *   Qout = [Qprev | X] * G,   Qprev n x c (ldq), X n x mb (ldx),
 *   G (c + mb) x mb double (ldg), Qout n x mb (ldo), mb <= 64.
 * With G = [-R_{1:i-1,i}; I] R_ii^{-1} this is Q_i = (W_i - Q_{1:i-1}R_{1:i-1,i}) R_ii^{-1}.
 * Qout may alias X exactly (same pointer and ld); it must not overlap Qprev.
 * Types per prec as for rbgs_qr (G is rounded/split inside).             */
RBGS_API rbgs_status rbgs_tall_update(int32_t prec, int64_t n, int64_t c, int64_t mb, const void* Qprev, int64_t ldq,
                             const void* X, int64_t ldx, const double* G, int64_t ldg, void* Qout, int64_t ldo,
                             void* stream, int32_t sync);

/* rbgs_tall_update without any device allocation.  The paper has no
 * counterpart: this serves callers that cannot let a library call cudaMalloc
 * or cudaFree -- those whose device memory is all handed out by their own
 * allocator (a framework pool reserving most of HBM), and those on a latency
 * path where an allocation or free may synchronise the device.  Arguments,
 * results and precisions are those of rbgs_tall_update, except that F16X3 is
 * not offered (RBGS_EINVAL).
 * Limit: c + mb <= RBGS_NOALLOC_MAX_K, else RBGS_ETOOLARGE (checked before any
 * CUDA call).  The scratch (the FP32 copy or TF32 split of G and an error flag,
 * about 4.03 MiB) is a fixed __device__ array inside the library, present on
 * every device that loads it until the process exits.  The first call on a
 * device looks up that array's device address (with the device current);
 * make that first call before any stream capture on the device.  The address
 * is kept until rbgs_release_workspace() on that device, which a caller must
 * call after cudaDeviceReset before the next call.  All calls share the
 * array: calls whose GPU work overlaps (unordered streams, or host threads
 * calling at once) race on it and give wrong results.
 * Status: with sync != 0 a bounded device wait that expired in the TF32X3
 * kernel returns RBGS_ETIMEOUT; with sync == 0 the call returns after
 * enqueueing and that timeout is not reported (the next call clears its
 * flag), so callers that need it pass sync = 1.                           */
#define RBGS_NOALLOC_MAX_K 8192
RBGS_API rbgs_status rbgs_tall_update_noalloc(int32_t prec, int64_t n, int64_t c, int64_t mb, const void* Qprev,
                                     int64_t ldq, const void* X, int64_t ldx, const double* G, int64_t ldg,
                                     void* Qout, int64_t ldo, void* stream, int32_t sync);

/* ------------------------------------------------------------------------
 * Randomized block Krylov methods (Sec. 5).
 *
 * Operators on nx x ny interior points of the unit square (spacing
 * hx = 1/(nx+1), hy = 1/(ny+1)), zero Dirichlet boundary; point (x, y) is row
 * x + nx y, so n = nx ny.
 *  RBGS_OP_STENCIL5   the 5-point convection-diffusion operator
 *                     A u = -(u_xx + u_yy) + bx u_x + by u_y, central differences.
 *  RBGS_OP_DIFFUSION  -div(a grad u) by the cell-centred five-point scheme:
 *                     (A u)_P = sum over the four faces f of P of
 *                     a_f (u_P - u_neighbour) / h^2 (h = hx across x faces,
 *                     hy across y faces), with face coefficients coef
 *                     (device, double): first the x faces, (nx+1) x (ny+2)
 *                     values, face (i, j) between nodes (i, j) and (i+1, j) at
 *                     i + (nx+1) j; then the y faces, (nx+2) x (ny+1) values,
 *                     face (i, j) between (i, j) and (i, j+1) at i + (nx+2) j
 *                     (nodes 0-based over the (nx+2) x (ny+2) grid with the
 *                     boundary; interior node (i, j) is point (i-1, j-1)).
 *                     rbgs_diffusion_faces fills coef with the harmonic means
 *                     of node values of a.  bx, by are unused.  Not in the
 *                     paper: the problem class of the learned preconditioner. */
typedef enum { RBGS_OP_STENCIL5 = 0, RBGS_OP_DIFFUSION = 1 } rbgs_op_kind;
typedef struct {
  int32_t kind;      /* rbgs_op_kind                                                   */
  int32_t reserved;
  int64_t nx, ny;    /* interior points                                                */
  double bx, by;     /* convection velocity (RBGS_OP_STENCIL5)                        */
  const double* coef; /* face coefficients (RBGS_OP_DIFFUSION; device, caller-owned)  */
} rbgs_op;

/* coef (layout of RBGS_OP_DIFFUSION) = harmonic means 2 a_P a_Q / (a_P + a_Q)
 * of the node values a (device, (nx+2) x (ny+2), node (i, j) at
 * i + (nx+2) j, all > 0) of the two nodes of each face.  RBGS_EINVAL on a
 * null pointer or nx, ny < 1.                                               */
RBGS_API rbgs_status rbgs_diffusion_faces(int64_t nx, int64_t ny, const double* a, double* coef, void* stream,
                                          int32_t sync);

/* Y = A X for ncols columns (device, column-major).  X and Y are double if
 * prec == RBGS_P_FP64, else float.  X and Y must not overlap.               */
RBGS_API rbgs_status rbgs_op_apply(const rbgs_op* op, int32_t prec, const void* X, int64_t ldx, int64_t ncols, void* Y,
                          int64_t ldy, void* stream, int32_t sync);

/* RBGS-Arnoldi, Alg. 7: W_1 = B, then W_i = A Q_{i-1} for i = 2..p, each
 * block orthogonalized by one step of RBGS (Alg. 2 with Alg. 5, options as in
 * rbgs_qr).  B (n x mb, ldb) and Q (n x p mb, ldq) are device arrays of the
 * prec type; R (p mb x p mb, ldr) is device double.  The block Hessenberg
 * matrix is H = R(:, mb:), so that A Q(:, 0:(p-1) mb) = Q H.  Errors as rbgs_qr. */
RBGS_API rbgs_status rbgs_block_arnoldi(const rbgs_op* op, const void* B, int64_t ldb, int64_t mb, int64_t p,
                               rbgs_sketch sketch, int64_t k, uint64_t seed, void* Q, int64_t ldq, double* R,
                               int64_t ldr, const rbgs_opts* opts, rbgs_stats* stats);

/* Restarted randomized block GMRES (Sec. 5.2) for A X = B, B and X n x mb
 * device double (X holds the initial guess and receives the solution).  Each
 * cycle runs Alg. 7 with p blocks on the residual block r = B - A X (basis
 * in opts->prec; r, X and the projected problem in FP64) and sets
 *   X += Q(:, 0:(p-1) mb) z,   z = argmin || H z - R(:, 0:mb) ||
 * (eq. GMRESsol; H = R(:, mb:) block upper Hessenberg, solved by Householder
 * reflectors in FP64).  Stops when max_j ||r_j|| / ||b_j|| <= rtol or after
 * max_cycles cycles.  *cycles (host) receives the cycles run, relres (host,
 * mb values) the final relative residuals.  Returns RBGS_ENOCONV if rtol
 * was not reached; other errors as rbgs_qr.  Synchronous.                  */
RBGS_API rbgs_status rbgs_block_gmres(const rbgs_op* op, const double* B, int64_t ldb, double* X, int64_t ldx, int64_t mb,
                             int64_t p, double rtol, int64_t max_cycles, rbgs_sketch sketch, int64_t k,
                             uint64_t seed, const rbgs_opts* opts, int64_t* cycles, double* relres);

/* Restarted randomized block FOM (Sec. 5.3): as rbgs_block_gmres with
 *   z = H(0:(p-1) mb, :)^{-1} R(0:(p-1) mb, 0:mb)   (eq. RFOMsol),
 * whose residual satisfies the sketched Galerkin condition.                  */
RBGS_API rbgs_status rbgs_block_fom(const rbgs_op* op, const double* B, int64_t ldb, double* X, int64_t ldx, int64_t mb,
                           int64_t p, double rtol, int64_t max_cycles, rbgs_sketch sketch, int64_t k, uint64_t seed,
                           const rbgs_opts* opts, int64_t* cycles, double* relres);

/* Randomized Rayleigh-Ritz with restarting, Alg. 8 (Sec. 5.4), for extreme
 * eigenpairs of the operator.  Each of the n_iter iterations runs Alg. 7 with
 * p blocks from B (basis in opts->prec; B0 is the first B), sets
 * H = R(:, mb:), and takes the mb extreme eigenpairs (mu, y) of the
 * (p-1) mb x (p-1) mb matrix H_(1:p-1,1:p-1) (which: 0 = largest real part,
 * 1 = smallest); the next B is Q(:, 0:(p-1) mb) Y.  The paper leaves the
 * choice and the scaling of y open; here each y has unit 2-norm with its first
 * largest-modulus entry real and positive, a real eigenvalue gives one column
 * y of Y, a conjugate pair a +- ib the two columns Re y, Im y (Re y alone if
 * one column is left), ordered by real part (ties: positive imaginary part
 * first).  On return X (n x mb, ldx, device double) holds the last B with
 * unit columns (step 5); ritz_re, ritz_im and resid_est (host, mb values)
 * hold the Ritz value of each column and the estimate ||H_(p,1:p-1) y|| of
 * its residual (step 3).  (p-1) mb <= RBGS_RITZ_MAX_N.  The small
 * eigenproblem runs on one CTA (FP32 Hessenberg reduction and Francis
 * double-shift QR for estimates, then Rayleigh-quotient steps in FP64 on H);
 * RBGS_ENOCONV if its QR iteration does not converge within 30 (p-1) mb
 * sweeps.  A breakdown of Alg. 7 after the first iteration (the restart block
 * spans a numerically invariant subspace, so its Ritz pairs are converged)
 * ends the iterations and returns the previous iteration's pairs; in the
 * first iteration it is RBGS_EBREAKDOWN.  Other errors as rbgs_block_gmres.
 * Synchronous.                                                               */
#define RBGS_RITZ_MAX_N 1024
RBGS_API rbgs_status rbgs_rayleigh_ritz(const rbgs_op* op, const double* B0, int64_t ldb, int64_t mb, int64_t p,
                                        int64_t n_iter, int32_t which, rbgs_sketch sketch, int64_t k, uint64_t seed,
                                        const rbgs_opts* opts, double* X, int64_t ldx, double* ritz_re,
                                        double* ritz_im, double* resid_est);

/* ------------------------------------------------------------------------
 * The learned right preconditioner (not in the paper, which preconditions
 * its block GMRES with ILU(0)): a U-Net M on the residual columns of a
 * diffusion problem on an N x N grid (n = N^2), used inside randomized block
 * flexible GMRES (the flexible variant of Saad 1993 on the paper's Alg. 7 and
 * Sec. 5.2), trained by the entry points below.
 *
 * Network with L = levels (2..6) levels of width[l] channels (multiples of 8,
 * 8..64); level l works at N / 2^l (N divisible by 2^(L-1)):
 *   encoder l = 0..L-1:  a_l = relu(conv(x_l)),  s_l = relu(conv(a_l)),
 *                        x_0 = the input image, x_{l+1} = avgpool2(s_l)
 *   decoder l = L-2..0:  d_l = relu(conv([upsample2(d_{l+1}); s_l])),  d_{L-1} = s_{L-1}
 *   output:              y = conv(d_0)  (width[0] -> 1 channel, linear)
 * 3 x 3 convolutions with zero padding (cross-correlation), 2 x 2 average
 * pooling, nearest-neighbour upsampling.  Activations are stored in
 * bfloat16; every convolution multiplies bfloat16 operands (its input and
 * weights) with FP32 accumulation; y, gradients and parameters are FP32.
 * Parameters: one FP32 device vector of rbgs_unet_num_params() values, layer
 * after layer in evaluation order (enc0a, enc0b, enc1a, enc1b, ...,
 * dec{L-2}, ..., dec0, out), each as w[tap][ci][co] then b[co], tap = 3 ox +
 * oy with ox, oy in {0, 1, 2} the offset + 1 along the image's fast (x) and
 * slow (y) index.  Images: image b of a batch is column b of an n x batch
 * column-major FP32 array with leading dimension n (pixel (x, y) at x + N y).
 * The library keeps the activations of the last forward call with save != 0
 * (for rbgs_unet_backward) and its other buffers in cached device workspace
 * (freed by rbgs_release_workspace).                                        */
typedef struct {
  int32_t levels;
  int32_t width[6];
  int32_t flags;     /* bit 0: every convolution on the SIMT kernels (by default the
                        levels whose rows are multiples of 128 pixels and whose channel
                        counts are multiples of 16 use the tcgen05 tensor cores)      */
} rbgs_unet;

/* Number of parameters of the network, or -1 if its shape is invalid.      */
RBGS_API int64_t rbgs_unet_num_params(const rbgs_unet* net);

/* y = U-Net(x) for batch images of N x N (x, y device FP32, n x batch with
 * leading dimension n).  save != 0 keeps the activations for the next
 * rbgs_unet_backward call.  RBGS_EINVAL on an invalid shape or pointer;
 * with sync, RBGS_ETIMEOUT if a bounded wait of a tensor-core kernel expired. */
RBGS_API rbgs_status rbgs_unet_forward(const rbgs_unet* net, const float* params, int64_t N, int64_t batch,
                                       const float* x, float* y, int32_t save, void* stream, int32_t sync);

/* grads (device FP32, the parameter layout, overwritten) = d sum(gy * y) /
 * d params for the last forward call made with save != 0 on this device,
 * which must have had the same network, N, batch and x (x is read again).
 * RBGS_EINVAL if no such forward was saved.                                */
RBGS_API rbgs_status rbgs_unet_backward(const rbgs_unet* net, const float* params, int64_t N, int64_t batch,
                                        const float* x, const float* gy, float* grads, void* stream, int32_t sync);

/* The training loss of a batch of (x, y) with x the scaled residual image and
 * y = U-Net(x): L = 1/2 mean over images and pixels of (B_f y - x)^2 with
 * B_f = A_f h^2 / 8, A_f the RBGS_OP_DIFFUSION operator of image b's field
 * f = field[b] (face coefficients at coef + f coef_stride, device double;
 * nx = ny = N, h = 1/(N+1)), so that U-Net(x) learns B_f^{-1} x measured in
 * the residual norm.  *loss (device double) receives L and gy (device FP32,
 * n x batch, ld n) its gradient dL/dy = B_f (B_f y - x) / (n batch) (B_f is
 * symmetric).  field: device int32, batch values.                          */
RBGS_API rbgs_status rbgs_unet_residual_loss(int64_t N, int64_t batch, const double* coef, int64_t coef_stride,
                                             const int32_t* field, const float* x, const float* y, float* gy,
                                             double* loss, void* stream, int32_t sync);

/* One Adam update (Kingma and Ba 2015) of count FP32 parameters in place:
 * m and v (device FP32, zero before the first step) are the moment
 * estimates, t >= 1 the step number for the bias correction.               */
RBGS_API rbgs_status rbgs_adam_step(int64_t count, float* params, const float* grads, float* m, float* v, int64_t t,
                                    double lr, double beta1, double beta2, double eps, void* stream, int32_t sync);

/* The network's input scaling: X (device FP32, n x ncols, ldx) = the columns
 * of Q (prec type, ldq) scaled to unit root mean square, x = q / s with
 * s = ||q|| / sqrt(n) (zero columns stay zero): the images the preconditioner
 * feeds the network, for making training inputs from Krylov basis vectors. */
RBGS_API rbgs_status rbgs_unet_scale_inputs(int64_t n, int64_t ncols, int32_t prec, const void* Q, int64_t ldq,
                                            float* X, int64_t ldx, void* stream, int32_t sync);

/* The preconditioner applied to ncols (<= 64) columns: Z = M(Q) with, per
 * column, s = ||q|| / sqrt(n) and z = s (h^2 / 8) U-Net(q / s) (zero where
 * q = 0), h = 1/(N+1); positively homogeneous, M(alpha q) = alpha M(q).
 * Q, Z: device arrays of the prec type (double for RBGS_P_FP64, float
 * otherwise), n x ncols with leading dimensions ldq, ldz >= n.            */
RBGS_API rbgs_status rbgs_unet_precondition(const rbgs_unet* net, const float* params, int64_t N, int32_t prec,
                                            const void* Q, int64_t ldq, int64_t ncols, void* Z, int64_t ldz,
                                            void* stream, int32_t sync);

/* Restarted randomized block flexible GMRES for A X = B with the U-Net as a
 * right preconditioner that may differ from cycle to cycle (Saad 1993 on the
 * paper's Alg. 7 and Sec. 5.2): each cycle runs the RBGS Arnoldi process on
 * r = B - A X with W_1 = r and W_{j+1} = A Z_j, Z_j = M(Q_j), so that
 * A Z_{1:p-1} = Q H with H = R(:, mb:); z = argmin || H z - R(:, 0:mb) ||
 * (the sketched residual), X += Z z.  Plain block GMRES is the fallback and
 * the true residual decides: a cycle run with M is kept only when it brings
 * max_j ||r_j|| / ||b_j|| to at most accept (0 < accept <= 1) times its value
 * before the cycle; otherwise the cycle is repeated from the same X with
 * M = I (net == NULL runs plain block GMRES throughout).  op must be
 * RBGS_OP_DIFFUSION (or RBGS_OP_STENCIL5) with nx = ny = N.  *fallbacks
 * (host, may be NULL) receives the number of cycles that fell back.  Other
 * arguments, stopping and errors as rbgs_block_gmres; the workspace holds Z
 * (n x (p-1) mb in the basis type) besides the basis.  Synchronous.       */
RBGS_API rbgs_status rbgs_block_fgmres(const rbgs_op* op, const rbgs_unet* net, const float* params,
                                       const double* B, int64_t ldb, double* X, int64_t ldx, int64_t mb, int64_t p,
                                       double rtol, int64_t max_cycles, double accept, rbgs_sketch sketch, int64_t k,
                                       uint64_t seed, const rbgs_opts* opts, int64_t* cycles, double* relres,
                                       int64_t* fallbacks);

/* Philox4x32-10 blocks on the device: out[4i..4i+3] = philox(ctr[4i..4i+3],
 * key = (seed_lo, seed_hi)) for i < count (device pointers).              */
RBGS_API rbgs_status rbgs_philox(uint64_t seed, const uint32_t* ctr, uint32_t* out, int64_t count, void* stream, int32_t sync);

/* The nonzeros of columns j0 .. j0 + count - 1 of the sparse-sign Theta, on
 * the host (the generator the sketch kernels evaluate, exposed so that the
 * definition can be checked without a device): rows[t z + s] is the row of
 * the nonzero of column j0 + t in segment s, neg[...] = 1 where it is
 * -1/sqrt(z), z = min(8, k).  rows and neg are caller-owned host arrays of
 * count * z entries.  RBGS_EINVAL on a null pointer, k < 1, j0 < 0 or
 * count < 0.                                                                */
RBGS_API rbgs_status rbgs_sparse_sign_columns(uint64_t seed, int64_t k, int64_t j0, int64_t count, int64_t* rows,
                                              int32_t* neg);

/* Entries of the Gaussian Theta on the host (the generator the dense sketch
 * kernels evaluate, exposed so that it can be checked without a device):
 * out[t] = Theta(r[t], j[t]) for t < count, N(0, 1/k) by the Box-Muller pair
 * of column j[t] and row pair r[t] / 2 (cosine for even rows, sine for odd
 * ones), scaled as the kernels scale it.  r, j and out are caller-owned host
 * arrays of count entries.  RBGS_EINVAL on a null pointer (count > 0),
 * k < 1, count < 0, r[t] outside [0, k) or j[t] < 0.  Not in the paper,
 * which uses Rademacher and SRHT sketches (Sec. 2.3).                      */
RBGS_API rbgs_status rbgs_gaussian_entries(uint64_t seed, int64_t k, const int64_t* r, const int64_t* j, int64_t count,
                                           double* out);

/* Number of kernels this library has launched in the process so far (all
 * devices, all entry points); a counter for profiling and accounting.     */
RBGS_API int64_t rbgs_launch_count(void);

/* Release the cached device workspace of the current device, the cached
 * SRHT plans and the looked-up address of the no-allocation entry point's
 * scratch array (call it after cudaDeviceReset before any further call). */
RBGS_API rbgs_status rbgs_release_workspace(void);

/* Library version string (static storage).                               */
RBGS_API const char* rbgs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RBGS_H */
