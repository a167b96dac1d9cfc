// Host orchestrator of Alg. 2 and the C-ABI entry points of librbgs.
//
// Per block i (c = (i-1) m_p columns done), all on one stream, no host sync:
//   step 2   R_{1:i-1,i} by Richardson iterations on S_{1:i-1}, P_i (sketch space)
//   Alg. 5   S'_i = P_i - S_{1:i-1} R_{1:i-1,i};  R_ii = R factor of S'_i
//            (Cholesky QR twice, FP64 factorizations)
//   step 3+  Q_i = [Q_{1:i-1} | W_i] G_i  with  G_i = [-R_{1:i-1,i}; I] R_ii^{-1}
//            (one tall pass: projection and triangular solve fused)
//   step 5/1 S_i = Theta Q_i and P_{i+1} = Theta W_{i+1}
//   option   a second projection pass of Q_i against Q_{1:i-1} (reorth)
//   step 6   Delta, Delta~ on request.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace rbgs {

std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {

// ------------------------------------------------------------ workspace ---
struct DevWs {
  int dev = -1;
  void* ptr = nullptr;
  size_t bytes = 0;
};
std::mutex g_ws_mu;
std::vector<DevWs> g_ws;

rbgs_status workspace(size_t bytes, void** out) {
  int dev = 0;
  RBGS_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_ws_mu);
  for (auto& w : g_ws) {
    if (w.dev != dev) continue;
    if (w.bytes >= bytes) {
      *out = w.ptr;
      return RBGS_OK;
    }
    cudaDeviceSynchronize();
    cudaFree(w.ptr);
    w.ptr = nullptr;
    w.bytes = 0;
    if (cudaMalloc(&w.ptr, bytes) != cudaSuccess) {
      cudaGetLastError();
      return RBGS_ENOMEM;
    }
    w.bytes = bytes;
    *out = w.ptr;
    return RBGS_OK;
  }
  DevWs w;
  w.dev = dev;
  if (cudaMalloc(&w.ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    return RBGS_ENOMEM;
  }
  w.bytes = bytes;
  g_ws.push_back(w);
  *out = w.ptr;
  return RBGS_OK;
}

struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base((char*)b) {}
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = (T*)(base + off);
    off += count * sizeof(T);
    return p;
  }
};

template <class T>
__global__ void convert_kernel(int64_t rows, int64_t cols, const T* __restrict__ A, int64_t lda,
                               double* __restrict__ B, int64_t ldb) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * cols) return;
  const int64_t i = idx % rows, j = idx / rows;
  B[i + j * ldb] = (double)A[i + j * lda];
}

__global__ void cast_d2f_kernel(int64_t rows, int64_t cols, const double* __restrict__ A, int64_t lda,
                                float* __restrict__ B, int64_t ldb) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * cols) return;
  const int64_t i = idx % rows, j = idx / rows;
  B[i + j * ldb] = (float)A[i + j * lda];
}

__global__ void philox_kernel(uint2 key, const uint32_t* __restrict__ ctr, uint32_t* __restrict__ out,
                              int64_t count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
  const uint4 r = philox10(c, key);
  out[4 * i] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

constexpr int64_t kPartElems = 1 << 22;  // partial-sum scratch of the sketch-space GEMMs (doubles)

bool ranges_overlap(const void* a, size_t abytes, const void* b, size_t bbytes) {
  const char* pa = (const char*)a;
  const char* pb = (const char*)b;
  return pa < pb + bbytes && pb < pa + abytes;
}

// Cholesky QR twice of Sp (k x mb):  R = R2 R1, Rinv = R1^{-1} R2^{-1}, all in
// the sketch-space arithmetic TS.  The first round of the FP32 path factors the
// Gram matrix with a small diagonal shift so that it cannot break down on a
// nearly rank-deficient block; the second round removes the shift's effect.
// In FP64 the first round is unshifted and leaves an orthogonality defect of
// order eps64 kappa(Sp)^2, so the second round runs only where
// kappa_F(R1) = ||R1||_F ||R1^{-1}||_F exceeds 4 mb (decided on the device,
// flag need2; n2count counts the second rounds).
// Sp2 is a k x mb scratch for Sp R1^{-1}.
// shift64 > 0 shifts the first FP64 round too (relative to trace(G)); see
// alg4_pass.
template <class TS>
rbgs_status cholqr2(int64_t k, int mb, const TS* Sp, TS* Sp2, TS** sm, TS* part, int* flag, const int* active,
                    cudaStream_t st, TS* R, TS* Rinv, int* need2, int* n2count, double shift64 = 0.0) {
  TS *gram = sm[0], *R1 = sm[1], *R1inv = sm[2];
  const bool fp64 = sizeof(TS) == 8;
  const double shift = fp64 ? shift64 : 1e-6;
  rbgs_status s;
  s = small_gemm<TS, TS, TS>(1, mb, mb, k, 1.0, Sp, k, Sp, k, 0.0, gram, mb, part, kPartElems, active, st);
  if (s) return s;
  if ((s = chol_inv<TS>(mb, gram, R1, R1inv, shift, flag, nullptr, nullptr, active, st))) return s;
  // (the FP32 round is shifted and always followed by a second one: thr < 0)
  if ((s = round2_decide<TS>(mb, R1, R1inv, R, Rinv, fp64 ? 4.0 * mb : -1.0, active, need2, n2count, st))) return s;
  const int* act2 = need2;
  if ((s = trmm_right_upper<TS>(k, mb, Sp, k, R1inv, Sp2, k, act2, st))) return s;
  s = small_gemm<TS, TS, TS>(1, mb, mb, k, 1.0, Sp2, k, Sp2, k, 0.0, gram, mb, part, kPartElems, act2, st);
  if (s) return s;
  // second round; the kernel also forms R = R2 R1 and R^{-1} = R1^{-1} R2^{-1}
  if ((s = chol_inv<TS>(mb, gram, R, Rinv, 0.0, flag, R1, R1inv, act2, st))) return s;
  return RBGS_OK;
}

// One round of Cholesky QR with the shift (the provisional first pass of a
// two-pass block only needs an invertible R_ii).
template <class TS>
rbgs_status cholqr1(int64_t k, int mb, const TS* Sp, TS** sm, TS* part, int* flag, const int* active,
                    cudaStream_t st, TS* R, TS* Rinv, double shift64 = 0.0) {
  TS* gram = sm[0];
  const double shift = sizeof(TS) == 4 ? 1e-6 : shift64;
  rbgs_status s =
      small_gemm<TS, TS, TS>(1, mb, mb, k, 1.0, Sp, k, Sp, k, 0.0, gram, mb, part, kPartElems, active, st);
  if (s) return s;
  return chol_inv<TS>(mb, gram, R, Rinv, shift, flag, nullptr, nullptr, active, st);
}

// Step 2 by l Richardson iterations from X = 0:  X <- X + S^T (P - S X).
// X is c x mb (ldx); Res is k x mb scratch.
template <class TS>
rbgs_status richardson(int64_t k, int64_t c, int mb, const TS* S, const TS* Pi, TS* X, int64_t ldx, TS* Res, int l,
                       TS* partf, const int* active, cudaStream_t st) {
  rbgs_status s;
  s = small_gemm<TS, TS, TS>(1, c, mb, k, 1.0, S, k, Pi, k, 0.0, X, ldx, partf, kPartElems, active, st);
  if (s) return s;
  for (int it = 1; it < l; ++it) {
    RBGS_CUDA_TRY(cudaMemcpyAsync(Res, Pi, sizeof(TS) * k * mb, cudaMemcpyDeviceToDevice, st));
    s = small_gemm<TS, TS, TS>(0, k, mb, c, -1.0, S, k, X, ldx, 1.0, Res, k, partf, kPartElems, active, st);
    if (s) return s;
    s = small_gemm<TS, TS, TS>(1, c, mb, k, 1.0, S, k, Res, k, 1.0, X, ldx, partf, kPartElems, active, st);
    if (s) return s;
  }
  return RBGS_OK;
}

// A non-blocking stream per device for work that can run beside the caller's
// stream (ordered with events).
rbgs_status side_stream(cudaStream_t* out) {
  static std::mutex mu;
  static cudaStream_t streams[64] = {};
  int dev = 0;
  RBGS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return RBGS_ENODEV;
  std::lock_guard<std::mutex> lk(mu);
  if (!streams[dev]) RBGS_CUDA_TRY(cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking));
  *out = streams[dev];
  return RBGS_OK;
}

// Device buffers owned by one solver call.
struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

// The w x w identity (ld w).
// b = a for an mb x mb matrix (ld mb), converting the element type
template <class TI, class TO>
__global__ void copy_sq_kernel(int mb, const TI* a, TO* b, const int* active) {
  if (active && *active == 0) return;
  for (int t = threadIdx.x; t < mb * mb; t += blockDim.x) b[t] = (TO)a[t];
}

template <class TS>
__global__ void eye_kernel(int w, TS* I) {
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) I[e] = (e % w == e / w) ? (TS)1 : (TS)0;
}

// The status words of an inner factorization folded into the outer ones.
__global__ void merge_flags_kernel(const int* inner, int* brk, int* tmo) {
  if (threadIdx.x == 0) {
    if (inner[0]) *brk = 1;
    if (inner[3]) *tmo = 1;
  }
}

// Device copies of W, Q and R for the host-buffer entry point, kept per device
// and grown on demand (freed by rbgs_release_workspace), and its two copy streams.
struct HostPathBuf {
  int dev = -1;
  void* ptr = nullptr;
  size_t bytes = 0;
};
std::mutex g_hp_mu;
std::vector<HostPathBuf> g_hp;

rbgs_status host_path_buffer(size_t bytes, void** out) {
  int dev = 0;
  RBGS_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_hp_mu);
  for (auto& b : g_hp) {
    if (b.dev != dev) continue;
    if (b.bytes >= bytes) {
      *out = b.ptr;
      return RBGS_OK;
    }
    cudaDeviceSynchronize();
    cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
    if (cudaMalloc(&b.ptr, bytes) != cudaSuccess) {
      cudaGetLastError();
      return RBGS_ENOMEM;
    }
    b.bytes = bytes;
    *out = b.ptr;
    return RBGS_OK;
  }
  HostPathBuf b;
  b.dev = dev;
  if (cudaMalloc(&b.ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    return RBGS_ENOMEM;
  }
  b.bytes = bytes;
  g_hp.push_back(b);
  *out = b.ptr;
  return RBGS_OK;
}

void host_path_release() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> lock(g_hp_mu);
  for (auto& b : g_hp)
    if (b.dev == dev && b.ptr) {
      cudaDeviceSynchronize();
      cudaFree(b.ptr);
      b.ptr = nullptr;
      b.bytes = 0;
    }
}

// copy streams of the host-buffer entry point: [0] host to device, [1] device to host
rbgs_status copy_streams(cudaStream_t* h2d, cudaStream_t* d2h) {
  static std::mutex mu;
  static cudaStream_t streams[64][2] = {};
  int dev = 0;
  RBGS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return RBGS_ENODEV;
  std::lock_guard<std::mutex> lk(mu);
  for (int i = 0; i < 2; ++i)
    if (!streams[dev][i]) RBGS_CUDA_TRY(cudaStreamCreateWithFlags(&streams[dev][i], cudaStreamNonBlocking));
  *h2d = streams[dev][0];
  *d2h = streams[dev][1];
  return RBGS_OK;
}

// Resources of one factorization when several run side by side (rbgs_qr_batched):
// its own workspace and side stream instead of the per-device ones, and a device
// slot that receives its status words.  need_out alone asks for the workspace size.
struct QrCtx {
  void* ws = nullptr;
  size_t ws_bytes = 0;
  cudaStream_t side = nullptr;
  int* status_out = nullptr;  // 8 ints: breakdown, -, passes2, timeout, -, Cholesky second rounds
  size_t* need_out = nullptr;
  // host-buffer calls: block i of W may be read once w_ready[i] has fired, and
  // q_done[i] is recorded once column block i of Q and of R is final
  const cudaEvent_t* w_ready = nullptr;
  const cudaEvent_t* q_done = nullptr;
  // flexible Arnoldi (with op): block i > 1 is W_i = A Z_{i-1} with Z_{i-1} =
  // flex(Q_{i-1}) written to zbuf + (i-2) mb ldz (elements of the basis type)
  rbgs_status (*flex)(void* fctx, const void* Qprev, int64_t ldq, int mb, void* Z, int64_t ldz,
                      cudaStream_t st) = nullptr;
  void* flex_ctx = nullptr;
  void* zbuf = nullptr;
  int64_t ldz = 0;
};

// T: storage of W and Q; TS: storage/arithmetic of the sketch space.
template <class T, class TS>
rbgs_status qr_impl(const T* W, int64_t n, int64_t m, int64_t ldw, int mb, rbgs_sketch sketch, int64_t k,
                    uint64_t seed, T* Q, int64_t ldq, double* R, int64_t ldr, const rbgs_opts& o, rbgs_stats* stats,
                    int mode, const rbgs_op* op = nullptr, const QrCtx* ctx = nullptr) {
  // With op (Alg. 7, RBGS-Arnoldi): W holds only the first block B; every
  // later block is W_i = A Q_{i-1}, formed in the columns of Q_i.
  // mode 0: SIMT tall product; 1: TF32X3 tensor cores; 2: F16X3 tensor cores with the pre-split basis
  const bool tensor = mode != 0;
  cudaStream_t st = (cudaStream_t)o.stream;
  // fine == 2: the FP64 sketch space of FP32 storage takes its products in
  // double-FP32 arithmetic (small_gemm's df kernel) instead of on the FP64 pipe
  DfProducts df_guard(sizeof(T) == 4 && sizeof(TS) == 8 && o.fine == 2);
  // m need not be a multiple of mb: the last of the p blocks takes the
  // m - (p - 1) mb remaining columns.  Inside the block loop mb is the width of
  // the current block (every helper below reads it); mbf is the full width.
  const int mbf = mb;
  const int64_t p = (m + mb - 1) / mb;
  const int l = o.ls_iters < 1 ? 1 : o.ls_iters;
  const bool fp64 = sizeof(T) == 8;
  const size_t sk_bytes = sketch_scratch_bytes(sketch, k, n, 2 * mb, fp64) + 256;
  const bool cert = o.certify != 0 && stats != nullptr;

  // ---- carve the workspace
  size_t need = 0;
  for (int pass = 0; pass < 2; ++pass) {
    void* base = nullptr;
    if (pass == 1) {
      if (ctx && ctx->need_out) {
        *ctx->need_out = need;
        return RBGS_OK;
      }
      if (ctx && ctx->ws) {
        if (need > ctx->ws_bytes) return RBGS_ENOMEM;
        base = ctx->ws;
      } else {
        rbgs_status s = workspace(need, &base);
        if (s) return s;
      }
    }
    Carver cv(pass == 0 ? nullptr : base);
    TS* S = cv.take<TS>((size_t)k * m);
    TS* P = cv.take<TS>((size_t)k * m);
    TS* X = cv.take<TS>((size_t)m * mb);
    TS* X2 = cv.take<TS>((size_t)m * mb);
    TS* Res = cv.take<TS>((size_t)k * mb);
    TS* Sp = cv.take<TS>((size_t)k * mb);
    TS* sm[12];
    for (auto& q : sm) q = cv.take<TS>(64 * 64);
    double* tmp = cv.take<double>(64 * 64);
    T* Gmat = cv.take<T>((size_t)m * mb);
    double* Gd = tensor ? cv.take<double>((size_t)m * mb) : nullptr;
    float* Gsplit = mode == 1 ? cv.take<float>(tc_gsplit_floats(m)) : nullptr;
    unsigned char* Qs = mode == 2 ? cv.take<unsigned char>(h3_qs_bytes(n, m)) : nullptr;
    unsigned char* Bh = mode == 2 ? cv.take<unsigned char>(h3_b_bytes(m)) : nullptr;
    float* hsc = mode == 2 ? cv.take<float>(320) : nullptr;
    double* part = cv.take<double>(kPartElems);
    TS* partf = cv.take<TS>(kPartElems);
    // look-ahead of step 2 on the side stream (second X buffer, the partial
    // residuals of the next block, the side stream's partial-sum scratch)
    const bool cg = o.ls == 1;  // step 2 by conjugate gradients
    const bool hh = o.ls == 2;  // step 2 by Householder least squares
    const bool look = p > 1 && op == nullptr && !cg && !hh && (o.reorth != 0 || l == 1);
    TS* cgR = cg ? cv.take<TS>((size_t)m * mb) : nullptr;
    TS* cgD = cg ? cv.take<TS>((size_t)m * mb) : nullptr;
    TS* cgQ = cg ? cv.take<TS>((size_t)m * mb) : nullptr;
    TS* cgT = cg ? cv.take<TS>((size_t)k * mb) : nullptr;
    double* cgrr = cg ? cv.take<double>(64) : nullptr;
    int* cgdone = cg ? cv.take<int>(64) : nullptr;
    TS* Xalt = look ? cv.take<TS>((size_t)m * mb) : nullptr;
    TS* Spo[2] = {look ? cv.take<TS>((size_t)k * mb) : nullptr, look ? cv.take<TS>((size_t)k * mb) : nullptr};
    TS* partf2 = look ? cv.take<TS>(kPartElems) : nullptr;
    double* l2s = o.interblock == 6 ? cv.take<double>((size_t)8 * 64 * 64) : nullptr;  // Alg. 6 scratch
    // Householder least squares: S_{1:c} = Q_S [R_S; 0], Q_S = I - V T V^T (compact WY),
    // kept with R_S^{-1}; scratch for Q_c^T S_i, Q_c^T P and two c x mb products
    TS* hhV = hh ? cv.take<TS>((size_t)k * m) : nullptr;
    TS* hhT = hh ? cv.take<TS>((size_t)m * m) : nullptr;
    TS* hhRi = hh ? cv.take<TS>((size_t)m * m) : nullptr;
    TS* hhB = hh ? cv.take<TS>((size_t)k * mb) : nullptr;
    TS* hhY = hh ? cv.take<TS>((size_t)k * mb) : nullptr;
    TS* hhW = hh ? cv.take<TS>((size_t)m * mb) : nullptr;
    TS* hhW2 = hh ? cv.take<TS>((size_t)m * mb) : nullptr;
    void* skscr = cv.take<char>(sk_bytes);
    void* skscr2 = cv.take<char>(sk_bytes);  // the side stream's sketches of the next blocks of W
    int* flags = cv.take<int>(64);
    int* blk_on = cv.take<int>((size_t)p);
    double* cert_buf = cert ? cv.take<double>((size_t)k * m * 3 + (size_t)m * 64 + 8) : nullptr;
    if (pass == 0) {
      need = cv.off + 256;
      continue;
    }
    TS *Rii = sm[5], *Riinv = sm[6], *R2ii = sm[7], *R2iinv = sm[8], *Ieye = sm[9];
    const bool alg4 = o.interblock == 4;
    // single-vector RGS (1) and vRCholeskyQR (3, Alg. 3): after the projection, the
    // block's own columns are orthonormalised one at a time, by RBGS with one-column
    // blocks on Q'_i (explicit sketches for RGS, implicit for Alg. 3), in place
    const bool percol = o.interblock == 1 || o.interblock == 3;
    // Alg. 6: an l2 QR of Q'_i (Cholesky QR twice with FP64 Gram matrices), then Alg. 4
    const bool alg6 = o.interblock == 6;
    int* brk = flags;          // breakdown
    int* active = flags + 1;   // second pass on/off for this block
    int* npass2 = flags + 2;   // number of second passes
    int* tmo = flags + 3;      // bounded device wait expired
    int* need2 = flags + 4;    // second Cholesky QR round on/off (FP64 sketch space)
    int* n2count = flags + 5;  // second Cholesky QR rounds taken
    struct TallEv {
      cudaEvent_t a, b;
      double bytes;
      int64_t blk;
      bool pass2;
    };
    std::vector<TallEv> evs;
    const bool timing = o.timing && (o.sync || stats);
    auto ev_guard = [&]() {
      for (auto& e : evs) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
      }
    };
    struct Guard {
      std::function<void()> f;
      ~Guard() { f(); }
    } guard{ev_guard};
    RBGS_CUDA_TRY(cudaMemsetAsync(flags, 0, 64 * sizeof(int), st));
    RBGS_CUDA_TRY(cudaMemsetAsync(blk_on, 0, sizeof(int) * p, st));
    RBGS_CUDA_TRY(cudaMemset2DAsync(R, ldr * sizeof(double), 0, m * sizeof(double), m, st));

    rbgs_status s;
    // The tall update in two parts: the small preparation of its G operand
    // (splits and scales) and the tall kernel itself, which alone is timed.
    // c: basis columns read; cout: the column of Q the result occupies (where
    // the pre-split copy goes).
    auto tall_prep = [&](int64_t c, int64_t cout, const int* act, const TS* sraw, bool split_out) -> rbgs_status {
      if (mode == 2)
        return h3_prepare<TS>(c, mb, Gd, c + mb, sraw, k, nullptr, nullptr, h3_shift(cout, mb, split_out), Bh, hsc,
                              act, st);
      if (mode == 1) return tc_split_g(c + mb, mb, Gd, c + mb, Gsplit, act, st);
      return RBGS_OK;
    };
    auto tall_run = [&](int64_t c, int64_t cout, const T* X2src, int64_t ldx2, T* out, const int* act,
                        bool split_out) -> rbgs_status {
      if (mode == 2)
        return tall_update_h3(n, c, mb, Qs, h3_nch_row(m), (const float*)X2src, ldx2, Bh, hsc, (float*)out, ldq,
                              split_out ? Qs : nullptr, cout, h3_shift(cout, mb, split_out), act, tmo, st);
      if (mode == 1)
        return tall_update_tc(n, c, mb, (const float*)Q, ldq, (const float*)X2src, ldx2, Gsplit, (float*)out, ldq,
                              act, tmo, st);
      return tall_update_simt<T>(n, c, mb, Q, ldq, X2src, ldx2, Gmat, c + mb, out, ldq, act, st);
    };
    auto tall = [&](int64_t c, int64_t cout, const T* X2src, int64_t ldx2, T* out, const int* act, const TS* sraw,
                    bool split_out) -> rbgs_status {
      rbgs_status r0 = tall_prep(c, cout, act, sraw, split_out);
      if (r0) return r0;
      if (!timing) return tall_run(c, cout, X2src, ldx2, out, act, split_out);
      TallEv e;
      e.bytes = (double)sizeof(T) * (double)n * (double)(c + 2 * mb);
      e.blk = cout / mb;
      e.pass2 = act != nullptr;
      RBGS_CUDA_TRY(cudaEventCreate(&e.a));
      if (cudaEventCreate(&e.b) != cudaSuccess) {
        cudaEventDestroy(e.a);
        return RBGS_ECUDA;
      }
      evs.push_back(e);
      RBGS_CUDA_TRY(cudaEventRecord(e.a, st));
      rbgs_status r = tall_run(c, cout, X2src, ldx2, out, act, split_out);
      RBGS_CUDA_TRY(cudaEventRecord(e.b, st));
      return r;
    };
    auto make_g = [&](int64_t c, const TS* Rc, const TS* Rd, const TS* Rdinv, double* Rcol,
                      const int* act) -> rbgs_status {
      if (tensor) return assemble_g<TS, double>(c, mb, Rc, m, Rd, Rdinv, Gd, c + mb, Rcol, ldr, act, st);
      return assemble_g<TS, T>(c, mb, Rc, m, Rd, Rdinv, Gmat, c + mb, Rcol, ldr, act, st);
    };
    // the identity (ld w), for the projection G = [-X; I] of Alg. 4
    auto set_eye = [&](int w) -> rbgs_status {
      eye_kernel<TS><<<1, 256, 0, st>>>(w, Ieye);
      RBGS_LAUNCH_CHECK();
      return RBGS_OK;
    };
    if ((alg4 || percol || alg6) && (s = set_eye(mb))) return s;
    // Y (k x mb, ld k) <- Q_c^T Y in its first `rows` rows, Q_c = I - V T V^T over
    // the first c reflectors
    auto hh_apply_qt = [&](int64_t c, TS* Y, int64_t rows) -> rbgs_status {
      rbgs_status r;
      if ((r = small_gemm<TS, TS, TS>(1, c, mb, k, 1.0, hhV, k, Y, k, 0.0, hhW, m, partf, kPartElems, nullptr, st)))
        return r;
      if ((r = small_gemm<TS, TS, TS>(1, c, mb, c, 1.0, hhT, m, hhW, m, 0.0, hhW2, m, partf, kPartElems, nullptr,
                                      st)))
        return r;
      return small_gemm<TS, TS, TS>(0, rows, mb, c, -1.0, hhV, k, hhW2, m, 1.0, Y, k, partf, kPartElems, nullptr, st);
    };
    // Householder least squares: X = R_S^{-1} (Q_S^T P)_{1:c}
    auto hh_solve = [&](int64_t c, const TS* Pb, TS* Xo) -> rbgs_status {
      rbgs_status r;
      RBGS_CUDA_TRY(cudaMemcpyAsync(hhY, Pb, sizeof(TS) * k * mb, cudaMemcpyDeviceToDevice, st));
      if ((r = hh_apply_qt(c, hhY, c))) return r;
      return small_gemm<TS, TS, TS>(0, c, mb, c, 1.0, hhRi, m, hhY, k, 0.0, Xo, m, partf, kPartElems, nullptr, st);
    };
    // append the final sketch S_i (columns c..c+mb-1) to the factorization:
    // Q_c^T S_i, the panel's reflectors, then the off-diagonal blocks
    // T_12 = -T_11 (V_1^T V_2) T_22 and (R_S^{-1})_12 = -R_11^{-1} R_12 R_22^{-1}
    auto hh_extend = [&](int64_t c) -> rbgs_status {
      rbgs_status r;
      RBGS_CUDA_TRY(cudaMemcpyAsync(hhB, S + c * k, sizeof(TS) * k * mb, cudaMemcpyDeviceToDevice, st));
      if (c > 0 && (r = hh_apply_qt(c, hhB, k))) return r;
      if ((r = hh_panel<TS>(k, c, mb, hhB, k, hhV + c * k, k, hhT + c + c * m, hhRi + c + c * m, m, brk, st)))
        return r;
      if (c == 0) return RBGS_OK;
      if ((r = small_gemm<TS, TS, TS>(1, c, mb, k, 1.0, hhV, k, hhV + c * k, k, 0.0, hhW, m, partf, kPartElems,
                                      nullptr, st)))
        return r;
      if ((r = small_gemm<TS, TS, TS>(0, c, mb, c, 1.0, hhT, m, hhW, m, 0.0, hhW2, m, partf, kPartElems, nullptr,
                                      st)))
        return r;
      if ((r = small_gemm<TS, TS, TS>(0, c, mb, mb, -1.0, hhW2, m, hhT + c + c * m, m, 0.0, hhT + c * m, m, partf,
                                      kPartElems, nullptr, st)))
        return r;
      if ((r = small_gemm<TS, TS, TS>(0, c, mb, c, 1.0, hhRi, m, hhB, k, 0.0, hhW, m, partf, kPartElems, nullptr,
                                      st)))
        return r;
      return small_gemm<TS, TS, TS>(0, c, mb, mb, -1.0, hhW, m, hhRi + c + c * m, m, 0.0, hhRi + c * m, m, partf,
                                    kPartElems, nullptr, st);
    };
    if (hh) {
      RBGS_CUDA_TRY(cudaMemsetAsync(hhT, 0, sizeof(TS) * m * m, st));
      RBGS_CUDA_TRY(cudaMemsetAsync(hhRi, 0, sizeof(TS) * m * m, st));
    }
    // step 2: X (c x mb, ld m) from P (k x mb) by Richardson or by conjugate gradients
    // (`its` steps), or by Householder least squares
    auto step2 = [&](int64_t c, const TS* Pb, TS* Xo, int its) -> rbgs_status {
      if (hh) return hh_solve(c, Pb, Xo);
      if (!cg) return richardson<TS>(k, c, mb, S, Pb, Xo, m, Res, its, partf, nullptr, st);
      rbgs_status r;
      RBGS_CUDA_TRY(cudaMemset2DAsync(Xo, sizeof(TS) * m, 0, sizeof(TS) * c, mb, st));
      if ((r = small_gemm<TS, TS, TS>(1, c, mb, k, 1.0, S, k, Pb, k, 0.0, cgR, m, partf, kPartElems, nullptr, st)))
        return r;
      RBGS_CUDA_TRY(cudaMemcpy2DAsync(cgD, sizeof(TS) * m, cgR, sizeof(TS) * m, sizeof(TS) * c, mb,
                                      cudaMemcpyDeviceToDevice, st));
      if ((r = cg_init<TS>(c, mb, cgR, m, cgrr, cgdone, st))) return r;
      for (int it = 0; it < its; ++it) {
        if ((r = small_gemm<TS, TS, TS>(0, k, mb, c, 1.0, S, k, cgD, m, 0.0, cgT, k, partf, kPartElems, nullptr, st)))
          return r;
        if ((r = small_gemm<TS, TS, TS>(1, c, mb, k, 1.0, S, k, cgT, k, 0.0, cgQ, m, partf, kPartElems, nullptr, st)))
          return r;
        if ((r = cg_step<TS>(c, mb, Xo, m, cgR, cgD, cgQ, m, cgrr, cgdone, st))) return r;
      }
      return RBGS_OK;
    };
    // the inner factorization's own workspace, side stream, status words and R
    DevBuf inner_buf;
    size_t inner_need = 0;
    cudaStream_t inner_side = nullptr;
    struct SideFree {
      cudaStream_t* s;
      ~SideFree() {
        if (*s) cudaStreamDestroy(*s);
      }
    } inner_side_free{&inner_side};
    int* inner_flags = nullptr;
    double* Rinner = nullptr;
    if (percol) {
      rbgs_opts oq = o;
      oq.reorth = 0;
      oq.interblock = o.interblock == 1 ? 4 : 5;
      QrCtx cq;
      cq.need_out = &inner_need;
      if ((s = qr_impl<T, TS>(W, n, mbf, ldq, 1, sketch, k, seed, Q, ldq, R, mbf, oq, nullptr, mode, nullptr, &cq)))
        return s;
      const size_t extra = 256 + 8 * (size_t)mbf * mbf + 256;
      if (cudaMalloc(&inner_buf.p, inner_need + extra) != cudaSuccess) {
        cudaGetLastError();
        return RBGS_ENOMEM;
      }
      inner_flags = (int*)((char*)inner_buf.p + inner_need);
      Rinner = (double*)((char*)inner_buf.p + inner_need + 256);
      RBGS_CUDA_TRY(cudaStreamCreateWithFlags(&inner_side, cudaStreamNonBlocking));
    }
    auto percol_pass = [&](int64_t c, const TS* Xc, const T* src, int64_t ldsrc, T* Qo, const TS* sraw, TS* Rd,
                           TS* Sout, bool split_final) -> rbgs_status {
      rbgs_status r;
      if ((r = make_g(c, Xc, Ieye, Ieye, nullptr, nullptr))) return r;
      if ((r = tall(c, c, src, ldsrc, Qo, nullptr, sraw, false))) return r;
      rbgs_opts oq = o;
      oq.reorth = 0;
      oq.interblock = o.interblock == 1 ? 4 : 5;
      oq.sync = 0;
      oq.timing = 0;
      oq.certify = 0;
      oq.stream = st;
      QrCtx cq;
      cq.ws = inner_buf.p;
      cq.ws_bytes = inner_need;
      cq.side = inner_side;
      cq.status_out = inner_flags;
      if ((r = qr_impl<T, TS>(Qo, n, mb, ldq, 1, sketch, k, seed, Qo, ldq, Rinner, mb, oq, nullptr, mode, nullptr,
                              &cq)))
        return r;
      merge_flags_kernel<<<1, 32, 0, st>>>(inner_flags, brk, tmo);
      RBGS_LAUNCH_CHECK();
      if (sizeof(TS) == 8) {
        RBGS_CUDA_TRY(cudaMemcpyAsync(Rd, Rinner, 8 * (size_t)mb * mb, cudaMemcpyDeviceToDevice, st));
      } else if ((r = cast_cols_t<double, float>(mb, mb, Rinner, mb, (float*)Rd, mb, st))) {
        return r;
      }
      if ((r = sketch_apply_t<T, TS>(sketch, k, n, seed, Qo, ldq, mb, Sout, k, skscr, sk_bytes, st))) return r;
      if (mode == 2 && split_final) {  // the pre-split copy of Q_i for the later blocks: an identity pass
        if ((r = make_g(0, nullptr, Ieye, Ieye, nullptr, nullptr))) return r;
        if ((r = tall(0, c, Qo, ldq, Qo, nullptr, Sout, true))) return r;
      }
      return RBGS_OK;
    };
    // Steps 4-5 by Alg. 4 (RCholeskyQR on the explicit sketch) for the block
    // src - Q_{1:c} Xc written to Qo (column c of Q): the projection with
    // G = [-Xc; I], its sketch S'_i = Theta Q'_i, Cholesky QR of S'_i (one or two
    // rounds) giving Rd and Rd^{-1}, the in-place scaling Q_i = Q'_i Rd^{-1}, and
    // step 5, Sout = Theta Q_i.
    auto alg4_pass = [&](int64_t c, const TS* Xc, const T* src, int64_t ldsrc, T* Qo, const TS* sraw, bool one_round,
                         TS* Rd, TS* Rdinv, TS* Sout, bool split_final, const int* act) -> rbgs_status {
      rbgs_status r;
      if ((r = make_g(c, Xc, Ieye, Ieye, nullptr, act))) return r;
      if ((r = tall(c, c, src, ldsrc, Qo, act, sraw, false))) return r;
      if ((r = sketch_apply_t<T, TS>(sketch, k, n, seed, Qo, ldq, mb, Sp, k, skscr, sk_bytes, st, act))) return r;
      // With the row-wise solve on FP32 storage the blocks are expected to be
      // numerically rank deficient: the FP64 sketch of Q'_i may then be too
      // ill-conditioned for an FP64 Cholesky factor (a non-positive pivot).
      // Its first round takes the shift of shifted Cholesky QR (Fukaya, Kannan,
      // Nakatsukasa, Yamamoto and Yanagisawa 2020),
      // 11 (k m_p + m_p (m_p + 1)) u_64 ||S'_i||_F^2; the second round (or the
      // second pass) removes its effect.  FP64 storage keeps the unshifted
      // factor, so that its results stay those of the plain method.
      const double sh64 = (o.trsm && sizeof(T) == 4) ? 11.0 * ((double)k * mb + (double)mb * (mb + 1)) * 0x1p-53
                                                      : 0.0;
      if (one_round) r = cholqr1<TS>(k, mb, Sp, sm, partf, brk, act, st, Rd, Rdinv, sh64);
      else r = cholqr2<TS>(k, mb, Sp, Res, sm, partf, brk, act, st, Rd, Rdinv, need2, n2count, sh64);
      if (r) return r;
      if (o.trsm) {  // Q_i = Q'_i R_ii^{-1} by forward substitution, row by row
        if ((r = trsm_rows<T, TS>(n, mb, Qo, ldq, Rd, act, st))) return r;
        if ((r = sketch_apply_t<T, TS>(sketch, k, n, seed, Qo, ldq, mb, Sout, k, skscr, sk_bytes, st, act))) return r;
        if (mode == 2 && split_final) {  // the pre-split copy of Q_i: an identity pass
          if ((r = make_g(0, nullptr, Ieye, Ieye, nullptr, act))) return r;
          if ((r = tall(0, c, Qo, ldq, Qo, act, Sout, true))) return r;
        }
        return RBGS_OK;
      }
      if ((r = make_g(0, nullptr, Rd, Rdinv, nullptr, act))) return r;
      if ((r = tall(0, c, Qo, ldq, Qo, act, Sp, split_final))) return r;
      return sketch_apply_t<T, TS>(sketch, k, n, seed, Qo, ldq, mb, Sout, k, skscr, sk_bytes, st, act);
    };

    // Steps 4-5 by Alg. 6 for the block src - Q_{1:c} Xc written to Qo: the
    // projection; an l2 QR Q'_i = Q* R' by Cholesky QR twice (FP64 Gram matrices
    // over the n rows, in-place scaling on the tall kernels); Alg. 4 on Q*
    // (sketch, Cholesky QR, scaling) giving R''; R_ii = R'' R' (into Rd, in TS);
    // step 5, Sout = Theta Q_i.
    auto alg6_pass = [&](int64_t c, const TS* Xc, const T* src, int64_t ldsrc, T* Qo, const TS* sraw, TS* Rd,
                         TS* Sout, bool split_final, const int* act) -> rbgs_status {
      rbgs_status r;
      double *gram = l2s, *r1 = l2s + 4096, *r1i = l2s + 2 * 4096, *racc = l2s + 3 * 4096, *rtmp = l2s + 4 * 4096,
             *rpp = l2s + 5 * 4096;
      if ((r = make_g(c, Xc, Ieye, Ieye, nullptr, act))) return r;
      if ((r = tall(c, c, src, ldsrc, Qo, act, sraw, false))) return r;
      for (int round = 0; round < 2; ++round) {
        if (fp64)
          r = small_gemm<double, double, double>(1, mb, mb, n, 1.0, (const double*)Qo, ldq, (const double*)Qo, ldq,
                                                 0.0, gram, mb, part, kPartElems, act, st);
        else
          r = small_gemm<float, double, double>(1, mb, mb, n, 1.0, (const float*)Qo, ldq, (const float*)Qo, ldq,
                                                0.0, gram, mb, part, kPartElems, act, st);
        if (r) return r;
        // the first Cholesky round leaves R1 in racc; the second forms R' = R2 R1 in rtmp
        if ((r = chol_inv<double>(mb, gram, round == 0 ? racc : r1, r1i, 0.0, brk, nullptr, nullptr, act, st)))
          return r;
        if (round == 1 && (r = tri_mul<double>(mb, r1, racc, rtmp, act, st))) return r;
        // Qo <- Qo R_round^{-1} (the F16X3 path takes its column scales from the sketch of Qo)
        if (tensor) r = assemble_g<double, double>(0, mb, nullptr, 0, r1i, r1i, Gd, mb, nullptr, 0, act, st);
        else r = assemble_g<double, T>(0, mb, nullptr, 0, r1i, r1i, Gmat, mb, nullptr, 0, act, st);
        if (r) return r;
        if ((r = sketch_apply_t<T, TS>(sketch, k, n, seed, Qo, ldq, mb, Sp, k, skscr, sk_bytes, st, act))) return r;
        if ((r = tall(0, c, Qo, ldq, Qo, act, Sp, false))) return r;
      }
      // Alg. 4 on Q*
      if ((r = sketch_apply_t<T, TS>(sketch, k, n, seed, Qo, ldq, mb, Sp, k, skscr, sk_bytes, st, act))) return r;
      if ((r = cholqr2<TS>(k, mb, Sp, Res, sm, partf, brk, act, st, sm[10], sm[11], need2, n2count))) return r;
      if ((r = make_g(0, nullptr, sm[10], sm[11], nullptr, act))) return r;
      if ((r = tall(0, c, Qo, ldq, Qo, act, Sp, split_final))) return r;
      // R_ii = R'' R' in FP64, stored in TS
      copy_sq_kernel<TS, double><<<1, 256, 0, st>>>(mb, sm[10], rpp, act);
      RBGS_LAUNCH_CHECK();
      if ((r = tri_mul<double>(mb, rpp, rtmp, racc, act, st))) return r;
      copy_sq_kernel<double, TS><<<1, 256, 0, st>>>(mb, racc, Rd, act);
      RBGS_LAUNCH_CHECK();
      return sketch_apply_t<T, TS>(sketch, k, n, seed, Qo, ldq, mb, Sout, k, skscr, sk_bytes, st, act);
    };

    // Step 1 of block i + 1 (the sketch of W_{i+1}) depends on nothing in block
    // i, so it runs on a side stream while block i's sketch-space steps run
    // here (those keep few SMs busy); an event hands P_{i+1} over.
    cudaStream_t st2 = nullptr;
    std::vector<cudaEvent_t> evw;
    struct EvGuard {
      std::vector<cudaEvent_t>* v;
      ~EvGuard() {
        for (auto e : *v) cudaEventDestroy(e);
      }
    } evguard{&evw};
    const bool ahead = p > 1 && op == nullptr;  // the next block of W is known in advance
    if (ahead) {
      if (ctx && ctx->side) st2 = ctx->side;
      else if ((s = side_stream(&st2))) return s;
      evw.resize((size_t)p + 2, nullptr);  // [p]: start, [p + 1]: end of the previous block
      for (auto& e : evw) RBGS_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    // step 1 of the first block
    if (ctx && ctx->w_ready) RBGS_CUDA_TRY(cudaStreamWaitEvent(st, ctx->w_ready[0], 0));
    if ((s = sketch_apply_t<T, TS>(sketch, k, n, seed, W, ldw, (int64_t)std::min<int64_t>(mbf, m), P, k, skscr,
                                   sk_bytes, st)))
      return s;
    if (ahead) {  // the side stream starts after everything enqueued here so far
      RBGS_CUDA_TRY(cudaEventRecord(evw[p], st));
      RBGS_CUDA_TRY(cudaStreamWaitEvent(st2, evw[p], 0));
    }
    for (int64_t blk = 0; blk < p; ++blk) {
      const int64_t c = blk * mbf;
      mb = (int)std::min<int64_t>(mbf, m - c);  // this block's width
      if ((alg4 || percol || alg6) && mb != mbf && (s = set_eye(mb))) return s;  // the narrower last block
      if (ctx && ctx->w_ready && op == nullptr) RBGS_CUDA_TRY(cudaStreamWaitEvent(st, ctx->w_ready[blk], 0));
      const int64_t wnext = blk + 1 < p ? std::min<int64_t>(mbf, m - c - mbf) : 0;
      const T* Wi = W + c * ldw;
      int64_t ldwi = ldw;
      T* Qi = Q + c * ldq;
      TS* Pi = P + c * k;
      TS* Si = S + c * k;
      double* Rcol = R + c * ldr;
      if (op && blk > 0) {  // Alg. 7, step 2: W_i = A Q_{i-1}, then its sketch (step 1 of the block)
        if (ctx && ctx->flex) {  // flexible: W_i = A M(Q_{i-1})
          T* Zs = (T*)ctx->zbuf + (blk - 1) * mbf * ctx->ldz;
          if ((s = ctx->flex(ctx->flex_ctx, Qi - mbf * ldq, ldq, mb, Zs, ctx->ldz, st))) return s;
          if ((s = stencil_apply_t<T, T>(*op, Zs, ctx->ldz, mb, Qi, ldq, st))) return s;
        } else if ((s = stencil_apply_t<T, T>(*op, Qi - mbf * ldq, ldq, mb, Qi, ldq, st))) {
          return s;
        }
        Wi = Qi;
        ldwi = ldq;
        if ((s = sketch_apply_t<T, TS>(sketch, k, n, seed, Wi, ldwi, mb, Pi, k, skscr, sk_bytes, st))) return s;
      }
      if (ahead && blk + 1 < p) {
        if (ctx && ctx->w_ready) RBGS_CUDA_TRY(cudaStreamWaitEvent(st2, ctx->w_ready[blk + 1], 0));
        s = sketch_apply_t<T, TS>(sketch, k, n, seed, Wi + mbf * ldw, ldw, wnext, Pi + mbf * k, k, skscr2, sk_bytes,
                                  st2);
        if (s) return s;
        if (look) {
          // Step 2 of block i + 1 (one Richardson step, X = S^T P_{i+1}) over
          // the columns of S that are final once block i - 1 is done:
          // X_old = S_{1:i-1}^T P_{i+1} and Sp_old = P_{i+1} - S_{1:i-1} X_old.
          // Block i + 1 adds the block row of S_i itself.
          const TS* Pn = Pi + mbf * k;
          TS* Xn = ((blk + 1) & 1) ? Xalt : X;
          TS* So = Spo[(blk + 1) & 1];
          if (c > 0) {  // everything enqueued here so far is block i - 1 and before
            RBGS_CUDA_TRY(cudaEventRecord(evw[p + 1], st));
            RBGS_CUDA_TRY(cudaStreamWaitEvent(st2, evw[p + 1], 0));
            s = small_gemm<TS, TS, TS>(1, c, wnext, k, 1.0, S, k, Pn, k, 0.0, Xn, m, partf2, kPartElems, nullptr,
                                       st2);
            if (s) return s;
          }
          RBGS_CUDA_TRY(cudaMemcpyAsync(So, Pn, sizeof(TS) * k * wnext, cudaMemcpyDeviceToDevice, st2));
          if (c > 0) {
            s = small_gemm<TS, TS, TS>(0, k, wnext, c, -1.0, S, k, Xn, m, 1.0, So, k, partf2, kPartElems, nullptr,
                                       st2);
            if (s) return s;
          }
        }
        RBGS_CUDA_TRY(cudaEventRecord(evw[blk + 1], st2));
      }
      if (ahead && blk > 0) RBGS_CUDA_TRY(cudaStreamWaitEvent(st, evw[blk], 0));
      // step 2 and the implicit sketch of Alg. 5
      // With a second pass to follow, the first pass is provisional: one
      // Richardson step and one (shifted) Cholesky QR round; the second pass
      // (l steps, two rounds) settles the block.
      const bool provisional = o.reorth != 0 && c > 0;
      TS* Xc = X;   // R_{1:i-1,i}
      TS* Spc = Sp; // S'_i = P_i - S_{1:i-1} R_{1:i-1,i}
      if (c > 0 && look) {  // finish the look-ahead with the block row of S_{i-1}
        const int64_t c0 = c - mbf;  // the previous block is a full one
        Xc = (blk & 1) ? Xalt : X;
        Spc = Spo[blk & 1];
        s = small_gemm<TS, TS, TS>(1, mbf, mb, k, 1.0, S + c0 * k, k, Pi, k, 0.0, Xc + c0, m, partf, kPartElems,
                                   nullptr, st);
        if (s) return s;
        s = small_gemm<TS, TS, TS>(0, k, mb, mbf, -1.0, S + c0 * k, k, Xc + c0, m, 1.0, Spc, k, partf, kPartElems,
                                   nullptr, st);
        if (s) return s;
      } else if (c > 0) {
        if ((s = step2(c, Pi, X, provisional ? 1 : l))) return s;
        RBGS_CUDA_TRY(cudaMemcpyAsync(Sp, Pi, sizeof(TS) * k * mb, cudaMemcpyDeviceToDevice, st));
        s = small_gemm<TS, TS, TS>(0, k, mb, c, -1.0, S, k, X, m, 1.0, Sp, k, partf, kPartElems, nullptr, st);
        if (s) return s;
      } else {
        RBGS_CUDA_TRY(cudaMemcpyAsync(Sp, Pi, sizeof(TS) * k * mb, cudaMemcpyDeviceToDevice, st));
      }
      // (the split copy of a provisional result is not kept: the second pass rereads it as FP32)
      const bool split1 = !(o.reorth == 1 && c > 0);
      if (alg4) {
        if ((s = alg4_pass(c, Xc, Wi, ldwi, Qi, Pi, provisional, Rii, Riinv, Si, split1, nullptr))) return s;
        if ((s = make_g(c, Xc, Rii, Riinv, Rcol, nullptr))) return s;  // the R column (G is not used again)
      } else if (percol) {
        if ((s = percol_pass(c, Xc, Wi, ldwi, Qi, Pi, Rii, Si, split1))) return s;
        if ((s = make_g(c, Xc, Rii, Rii, Rcol, nullptr))) return s;  // the R column only
      } else if (alg6) {
        if ((s = alg6_pass(c, Xc, Wi, ldwi, Qi, Pi, Rii, Si, split1, nullptr))) return s;
        if ((s = make_g(c, Xc, Rii, Rii, Rcol, nullptr))) return s;  // the R column only
      } else {
        if (provisional) s = cholqr1<TS>(k, mb, Spc, sm, partf, brk, nullptr, st, Rii, Riinv);
        else s = cholqr2<TS>(k, mb, Spc, Res, sm, partf, brk, nullptr, st, Rii, Riinv, need2, n2count);
        if (s) return s;
        if ((s = make_g(c, Xc, Rii, Riinv, Rcol, nullptr))) return s;
        // step 3 fused with the triangular solve
        if ((s = tall(c, c, Wi, ldwi, Qi, nullptr, Pi, split1))) return s;
        // step 5 (the sketch of W_{i+1}, step 1 of the next block, runs on the side stream)
        if ((s = sketch_apply_t<T, TS>(sketch, k, n, seed, Qi, ldq, mb, Si, k, skscr, sk_bytes, st))) return s;
      }
      // optional second projection pass
      if (o.reorth && c > 0) {
        if (cg || hh) {
          if ((s = step2(c, Si, X2, l))) return s;
        } else {
          s = small_gemm<TS, TS, TS>(1, c, mb, k, 1.0, S, k, Si, k, 0.0, X2, m, partf, kPartElems, nullptr, st);
          if (s) return s;
        }
        if ((s = reorth_decide<TS>(c, mb, X2, m, o.reorth_tol, o.reorth, active, npass2, blk_on + blk, st))) return s;
        for (int it = 1; it < l && !cg && !hh; ++it) {
          RBGS_CUDA_TRY(cudaMemcpyAsync(Res, Si, sizeof(TS) * k * mb, cudaMemcpyDeviceToDevice, st));
          s = small_gemm<TS, TS, TS>(0, k, mb, c, -1.0, S, k, X2, m, 1.0, Res, k, partf, kPartElems, active, st);
          if (s) return s;
          s = small_gemm<TS, TS, TS>(1, c, mb, k, 1.0, S, k, Res, k, 1.0, X2, m, partf, kPartElems, active, st);
          if (s) return s;
        }
        if (alg4) {
          if ((s = alg4_pass(c, X2, Qi, ldq, Qi, Si, false, R2ii, R2iinv, Si, true, active))) return s;
        } else if (percol) {  // (the second pass always runs: reorth 2 is refused with these variants)
          if ((s = percol_pass(c, X2, Qi, ldq, Qi, Si, R2ii, Si, true))) return s;
        } else if (alg6) {
          if ((s = alg6_pass(c, X2, Qi, ldq, Qi, Si, R2ii, Si, true, active))) return s;
        } else {
          RBGS_CUDA_TRY(cudaMemcpyAsync(Sp, Si, sizeof(TS) * k * mb, cudaMemcpyDeviceToDevice, st));
          s = small_gemm<TS, TS, TS>(0, k, mb, c, -1.0, S, k, X2, m, 1.0, Sp, k, partf, kPartElems, active, st);
          if (s) return s;
          if ((s = cholqr2<TS>(k, mb, Sp, Res, sm, partf, brk, active, st, R2ii, R2iinv, need2, n2count))) return s;
          if ((s = make_g(c, X2, R2ii, R2iinv, nullptr, active))) return s;
          if ((s = tall(c, c, Qi, ldq, Qi, active, Si, true))) return s;
          if ((s = sketch_apply_t<T, TS>(sketch, k, n, seed, Qi, ldq, mb, Si, k, skscr, sk_bytes, st, active)))
            return s;
        }
        if ((s = reorth_update_r<TS>(c, mb, X2, m, R2ii, Rcol, ldr, tmp, active, st))) return s;
      }
      // S_i is final: append it to the Householder factorization of S
      if (hh && blk + 1 < p && (s = hh_extend(c))) return s;
      if (ctx && ctx->q_done) RBGS_CUDA_TRY(cudaEventRecord(ctx->q_done[blk], st));
    }
    mb = mbf;
    RBGS_LAUNCH_CHECK();

    // step 6 (optional): Delta = ||I - S^T S||_F, Delta~ = ||P - S R||_F / ||P||_F
    double* dres = (double*)(flags + 16);
    if (cert) {
      double* Sd = cert_buf;
      double* Pd = Sd + (size_t)k * m;
      double* SR = Pd + (size_t)k * m;
      double* Gt = SR + (size_t)k * m;
      const int64_t tot = k * m;
      convert_kernel<TS><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(k, m, S, k, Sd, k);
      convert_kernel<TS><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(k, m, P, k, Pd, k);
      RBGS_LAUNCH_CHECK();
      // Gram S^T S in column tiles of 64; accumulate ||I - G||_F^2 tile by tile on the host side
      double acc_d = 0.0;
      for (int64_t j0 = 0; j0 < m; j0 += 64) {
        const int64_t nc = std::min<int64_t>(64, m - j0);
        s = small_gemm<double, double, double>(1, m, nc, k, 1.0, Sd, k, Sd + j0 * k, k, 0.0, Gt, m, part, kPartElems,
                                               nullptr, st);
        if (s) return s;
        // ||I - G||_F^2 over this column tile, summed on the host
        std::vector<double> hG((size_t)m * nc);
        RBGS_CUDA_TRY(cudaMemcpyAsync(hG.data(), Gt, sizeof(double) * m * nc, cudaMemcpyDeviceToHost, st));
        RBGS_CUDA_TRY(cudaStreamSynchronize(st));
        for (int64_t jj = 0; jj < nc; ++jj)
          for (int64_t i = 0; i < m; ++i) {
            const double d = (i == j0 + jj ? 1.0 : 0.0) - hG[i + jj * m];
            acc_d += d * d;
          }
      }
      for (int64_t j0 = 0; j0 < m; j0 += 64) {
        const int64_t nc = std::min<int64_t>(64, m - j0);
        s = small_gemm<double, double, double>(0, k, nc, m, 1.0, Sd, k, R + j0 * ldr, ldr, 0.0, SR + j0 * k, k,
                                               part, kPartElems, nullptr, st);
        if (s) return s;
      }
      if ((s = fro_norm_diff(k, m, Pd, k, SR, k, dres, dres + 1, st))) return s;
      double hv[2];
      RBGS_CUDA_TRY(cudaMemcpyAsync(hv, dres, sizeof(hv), cudaMemcpyDeviceToHost, st));
      RBGS_CUDA_TRY(cudaStreamSynchronize(st));
      stats->delta = std::sqrt(acc_d);
      stats->delta_tilde = hv[1] > 0 ? hv[0] / hv[1] : 0.0;
      stats->certified = (stats->delta <= 0.1 && stats->delta_tilde <= 0.1) ? 1 : 0;
    }
    if (ctx && ctx->status_out)
      RBGS_CUDA_TRY(cudaMemcpyAsync(ctx->status_out, flags, 8 * sizeof(int), cudaMemcpyDeviceToDevice, st));
    if (o.sync || stats) {
      int hf[6] = {0, 0, 0, 0, 0, 0};
      RBGS_CUDA_TRY(cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st));
      RBGS_CUDA_TRY(cudaStreamSynchronize(st));
      if (stats) {
        stats->passes2 = hf[2];
        stats->chol_rounds2 = hf[5];
        stats->tall_ms = 0.0;
        stats->tall_bytes = 0.0;
        stats->tall_launches = 0;
        if (timing) {
          std::vector<int> on((size_t)p, 0);
          if (o.reorth) RBGS_CUDA_TRY(cudaMemcpy(on.data(), blk_on, sizeof(int) * p, cudaMemcpyDeviceToHost));
          for (auto& e : evs) {
            if (e.pass2 && !on[(size_t)e.blk]) continue;
            float ms = 0.f;
            RBGS_CUDA_TRY(cudaEventElapsedTime(&ms, e.a, e.b));
            stats->tall_ms += ms;
            stats->tall_bytes += e.bytes;
            stats->tall_launches += 1;
          }
        }
        if (!cert) {
          stats->delta = -1.0;
          stats->delta_tilde = -1.0;
          stats->certified = 0;
        }
      }
      if (hf[3]) return RBGS_ETIMEOUT;
      if (hf[0]) return RBGS_EBREAKDOWN;
    }
  }
  return RBGS_OK;
}

}  // namespace
}  // namespace rbgs

using namespace rbgs;

extern "C" {

void rbgs_opts_default(rbgs_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->prec = RBGS_P_FP64;
  o->ls_iters = 2;
  o->reorth = 0;
  o->certify = 0;
  o->reorth_tol = 1e-8;
  o->stream = nullptr;
  o->sync = 1;
  o->timing = 0;
}

int64_t rbgs_launch_count(void) { return rbgs::g_launches.load(); }

const char* rbgs_version(void) { return "librbgs 0.1 (sm_103a)"; }

}  // extern "C"

namespace {

// The argument checks of rbgs_qr (also applied to every problem of a batch).
rbgs_status check_qr(const void* W, int64_t n, int64_t m, int64_t ldw, int64_t mb, rbgs_sketch sketch, int64_t k,
                     const void* Q, int64_t ldq, const double* R, int64_t ldr, const rbgs_opts& o) {
  if (!W || !Q || !R) return RBGS_EINVAL;
  if (n < 1 || n >= ((int64_t)1 << 31) || m < 1 || mb < 1 || mb > 64) return RBGS_EINVAL;
  if (ldw < n || ldq < n || ldr < m || k < m) return RBGS_EINVAL;
  if (o.prec < RBGS_P_FP64 || o.prec > RBGS_P_F16X3 || o.reorth < 0 || o.reorth > 2) return RBGS_EINVAL;
  if (o.interblock != 0 && o.interblock != 1 && o.interblock != 3 && o.interblock != 4 && o.interblock != 5 &&
      o.interblock != 6)
    return RBGS_EINVAL;
  if ((o.interblock == 1 || o.interblock == 3) && o.reorth == 2) return RBGS_EINVAL;
  if (o.trsm != 0 && (o.trsm != 1 || o.interblock != 4)) return RBGS_EINVAL;
  if (o.ls != 0 && o.ls != 1 && o.ls != 2) return RBGS_EINVAL;
  if (sketch == RBGS_SK_SRHT) {
    int64_t np = 1;
    while (np < n) np <<= 1;
    if (k > np) return RBGS_EINVAL;
  } else if (sketch == RBGS_SK_GAUSS || sketch == RBGS_SK_RADEMACHER || sketch == RBGS_SK_SPARSE) {
    if (k > n) return RBGS_EINVAL;
  } else {
    return RBGS_EINVAL;
  }
  const size_t es = o.prec == RBGS_P_FP64 ? 8 : 4;
  if (ranges_overlap(W, es * (size_t)(ldw * (m - 1) + n), Q, es * (size_t)(ldq * (m - 1) + n))) return RBGS_EINVAL;
  if (ranges_overlap(R, 8 * (size_t)(ldr * (m - 1) + m), Q, es * (size_t)(ldq * (m - 1) + n))) return RBGS_EINVAL;
  if (o.prec == RBGS_P_FP64) return RBGS_OK;
  if (o.fine < 0 || o.fine > 2) return RBGS_EINVAL;
  // tensor-core paths: TMA needs 16-byte aligned bases and leading dimensions
  if ((o.prec == RBGS_P_TF32X3 || o.prec == RBGS_P_F16X3) &&
      (((uintptr_t)W & 15) || ((uintptr_t)Q & 15) || (ldw % 4) || (ldq % 4)))
    return RBGS_EINVAL;
  return RBGS_OK;
}

// rbgs_qr after its checks: the instance for the precisions.
rbgs_status qr_dispatch(const void* W, int64_t n, int64_t m, int64_t ldw, int64_t mb, rbgs_sketch sketch, int64_t k,
                        uint64_t seed, void* Q, int64_t ldq, double* R, int64_t ldr, const rbgs_opts& o,
                        rbgs_stats* stats, const QrCtx* ctx) {
  if (o.prec == RBGS_P_FP64)
    return qr_impl<double, double>((const double*)W, n, m, ldw, (int)mb, sketch, k, seed, (double*)Q, ldq, R, ldr, o,
                                   stats, 0, nullptr, ctx);
  const int mode = o.prec == RBGS_P_TF32X3 ? 1 : (o.prec == RBGS_P_F16X3 ? 2 : 0);
  if (o.fine)
    return qr_impl<float, double>((const float*)W, n, m, ldw, (int)mb, sketch, k, seed, (float*)Q, ldq, R, ldr, o,
                                  stats, mode, nullptr, ctx);
  return qr_impl<float, float>((const float*)W, n, m, ldw, (int)mb, sketch, k, seed, (float*)Q, ldq, R, ldr, o, stats,
                               mode, nullptr, ctx);
}

// The a posteriori check of the epsilon-embedding property (Sec. 4): RBGS of Z
// with the sketch Phi gives Q_phi = Z R_phi^{-1}; Theta Q_phi = (Theta Z) R_phi^{-1}
// should have orthonormal columns.  Returns ||I - (Theta Q_phi)^T Theta Q_phi||_F.
template <class T>
rbgs_status embedding_check_t(const T* Z, int64_t n, int64_t m, int64_t ldz, int64_t mb, rbgs_sketch sketch,
                              int64_t k, uint64_t seed_theta, uint64_t seed_phi, const rbgs_opts& o, double* defect) {
  cudaStream_t st = (cudaStream_t)o.stream;
  const bool fp64 = sizeof(T) == 8;
  const int64_t ldq = (n + 3) / 4 * 4;
  const int64_t chunk = 64;
  const size_t sk = sketch_scratch_bytes(sketch, k, n, chunk, fp64) + 256;
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t bq = up(sizeof(T) * (size_t)ldq * m), br = up(8 * (size_t)m * m), bs = up(8 * (size_t)k * m),
               bg = up(8 * (size_t)m * chunk), bp = up(8 * (size_t)kPartElems);
  DevBuf buf;
  if (cudaMalloc(&buf.p, bq + br + bs + bg + bp + sk) != cudaSuccess) {
    cudaGetLastError();
    return RBGS_ENOMEM;
  }
  char* w = (char*)buf.p;
  T* Qp = (T*)w;
  double* Rp = (double*)(w + bq);
  double* S = (double*)(w + bq + br);
  double* Gt = (double*)(w + bq + br + bs);
  double* part = (double*)(w + bq + br + bs + bg);
  void* scr = w + bq + br + bs + bg + bp;
  rbgs_status s = qr_dispatch(Z, n, m, ldz, mb, sketch, k, seed_phi, Qp, ldq, Rp, m, o, nullptr, nullptr);
  if (s) return s;
  for (int64_t j0 = 0; j0 < m; j0 += chunk) {
    const int64_t nc = std::min<int64_t>(chunk, m - j0);
    if ((s = sketch_apply_t<T, double>(sketch, k, n, seed_theta, Qp + j0 * ldq, ldq, nc, S + j0 * k, k, scr, sk, st)))
      return s;
  }
  double acc = 0.0;
  std::vector<double> hG((size_t)m * chunk);
  for (int64_t j0 = 0; j0 < m; j0 += chunk) {
    const int64_t nc = std::min<int64_t>(chunk, m - j0);
    s = small_gemm<double, double, double>(1, m, nc, k, 1.0, S, k, S + j0 * k, k, 0.0, Gt, m, part, kPartElems,
                                           nullptr, st);
    if (s) return s;
    RBGS_CUDA_TRY(cudaMemcpyAsync(hG.data(), Gt, sizeof(double) * m * nc, cudaMemcpyDeviceToHost, st));
    RBGS_CUDA_TRY(cudaStreamSynchronize(st));
    for (int64_t jj = 0; jj < nc; ++jj)
      for (int64_t i = 0; i < m; ++i) {
        const double d = (i == j0 + jj ? 1.0 : 0.0) - hG[(size_t)(i + jj * m)];
        acc += d * d;
      }
  }
  *defect = std::sqrt(acc);
  return RBGS_OK;
}

}  // namespace

extern "C" {

rbgs_status rbgs_embedding_check(const void* Z, int64_t n, int64_t m, int64_t ldz, int64_t mb, rbgs_sketch sketch,
                                 int64_t k, uint64_t seed_theta, uint64_t seed_phi, const rbgs_opts* opts,
                                 double* defect) {
  rbgs_opts o;
  if (opts) o = *opts;
  else rbgs_opts_default(&o);
  if (!defect) return RBGS_EINVAL;
  o.sync = 1;
  o.timing = 0;
  o.certify = 0;
  const int64_t ldq = (n + 3) / 4 * 4;
  const size_t es = o.prec == RBGS_P_FP64 ? 8 : 4;
  // the library's own Q and R lie elsewhere: check Z's arguments against a disjoint stand-in
  const uintptr_t qfake = (uintptr_t)Z + es * (size_t)(ldz * std::max<int64_t>(m, 1)) + 4096;
  rbgs_status s = check_qr(Z, n, m, ldz, mb, sketch, k, (const void*)(qfake & ~(uintptr_t)255), ldq,
                           (const double*)((qfake & ~(uintptr_t)255) + es * (size_t)(ldq * std::max<int64_t>(m, 1)) +
                                           4096),
                           m, o);
  if (s) return s;
  if (o.prec == RBGS_P_FP64)
    return embedding_check_t<double>((const double*)Z, n, m, ldz, mb, sketch, k, seed_theta, seed_phi, o, defect);
  return embedding_check_t<float>((const float*)Z, n, m, ldz, mb, sketch, k, seed_theta, seed_phi, o, defect);
}

rbgs_status rbgs_qr(const void* W, int64_t n, int64_t m, int64_t ldw, int64_t mb, rbgs_sketch sketch, int64_t k,
                    uint64_t seed, void* Q, int64_t ldq, double* R, int64_t ldr, const rbgs_opts* opts,
                    rbgs_stats* stats) {
  rbgs_opts o;
  if (opts) o = *opts;
  else rbgs_opts_default(&o);
  rbgs_status s = check_qr(W, n, m, ldw, mb, sketch, k, Q, ldq, R, ldr, o);
  if (s) return s;
  return qr_dispatch(W, n, m, ldw, mb, sketch, k, seed, Q, ldq, R, ldr, o, stats, nullptr);
}

rbgs_status rbgs_qr_batched(rbgs_problem* probs, int64_t count, rbgs_sketch sketch, const rbgs_opts* opts,
                            int32_t nstreams) {
  if (!probs || count < 0 || nstreams < 1) return RBGS_EINVAL;
  rbgs_opts o;
  if (opts) o = *opts;
  else rbgs_opts_default(&o);
  for (int64_t i = 0; i < count; ++i) {
    const rbgs_problem& q = probs[i];
    rbgs_status s = check_qr(q.W, q.n, q.m, q.ldw, q.mb, sketch, q.k, q.Q, q.ldq, q.R, q.ldr, o);
    if (s) return s;
  }
  if (count == 0) return RBGS_OK;
  o.sync = 0;
  o.timing = 0;
  o.certify = 0;
  const int ns = (int)std::min<int64_t>(std::min<int64_t>(nstreams, count), 32);
  // each stream's workspace holds the largest of its problems
  std::vector<size_t> need((size_t)ns, 0);
  for (int64_t i = 0; i < count; ++i) {
    const rbgs_problem& q = probs[i];
    size_t nd = 0;
    QrCtx c;
    c.need_out = &nd;
    rbgs_status s = qr_dispatch(q.W, q.n, q.m, q.ldw, q.mb, sketch, q.k, q.seed, q.Q, q.ldq, q.R, q.ldr, o, nullptr,
                                &c);
    if (s) return s;
    need[(size_t)(i % ns)] = std::max(need[(size_t)(i % ns)], nd);
  }
  struct Slot {
    cudaStream_t st = nullptr, side = nullptr;
    cudaEvent_t done = nullptr;
    void* ws = nullptr;
  };
  std::vector<Slot> slots((size_t)ns);
  int* dstat = nullptr;
  cudaEvent_t start = nullptr;
  struct Cleanup {
    std::vector<Slot>* sl;
    int** dstat;
    cudaEvent_t* start;
    ~Cleanup() {
      for (auto& x : *sl) {
        if (x.st) cudaStreamSynchronize(x.st);
        if (x.side) cudaStreamSynchronize(x.side);
        if (x.ws) cudaFree(x.ws);
        if (x.done) cudaEventDestroy(x.done);
        if (x.st) cudaStreamDestroy(x.st);
        if (x.side) cudaStreamDestroy(x.side);
      }
      if (*dstat) cudaFree(*dstat);
      if (*start) cudaEventDestroy(*start);
    }
  } cleanup{&slots, &dstat, &start};
  for (auto& x : slots) {
    RBGS_CUDA_TRY(cudaStreamCreateWithFlags(&x.st, cudaStreamNonBlocking));
    RBGS_CUDA_TRY(cudaStreamCreateWithFlags(&x.side, cudaStreamNonBlocking));
    RBGS_CUDA_TRY(cudaEventCreateWithFlags(&x.done, cudaEventDisableTiming));
  }
  for (int j = 0; j < ns; ++j) {
    if (cudaMalloc(&slots[(size_t)j].ws, need[(size_t)j]) != cudaSuccess) {
      cudaGetLastError();
      return RBGS_ENOMEM;
    }
  }
  if (cudaMalloc(&dstat, sizeof(int) * 8 * (size_t)count) != cudaSuccess) {
    cudaGetLastError();
    return RBGS_ENOMEM;
  }
  // the batch starts after the work already on the caller's stream, and that
  // stream waits for the whole batch
  cudaStream_t caller = (cudaStream_t)o.stream;
  RBGS_CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  RBGS_CUDA_TRY(cudaEventRecord(start, caller));
  for (auto& x : slots) RBGS_CUDA_TRY(cudaStreamWaitEvent(x.st, start, 0));
  for (int64_t i = 0; i < count; ++i) {
    const rbgs_problem& q = probs[i];
    Slot& x = slots[(size_t)(i % ns)];
    QrCtx c;
    c.ws = x.ws;
    c.ws_bytes = need[(size_t)(i % ns)];
    c.side = x.side;
    c.status_out = dstat + 8 * i;
    rbgs_opts oi = o;
    oi.stream = x.st;
    rbgs_status s = qr_dispatch(q.W, q.n, q.m, q.ldw, q.mb, sketch, q.k, q.seed, q.Q, q.ldq, q.R, q.ldr, oi, nullptr,
                                &c);
    if (s) return s;
  }
  for (auto& x : slots) {
    RBGS_CUDA_TRY(cudaEventRecord(x.done, x.st));
    RBGS_CUDA_TRY(cudaStreamWaitEvent(caller, x.done, 0));
  }
  std::vector<int> hs((size_t)count * 8);
  RBGS_CUDA_TRY(cudaMemcpyAsync(hs.data(), dstat, sizeof(int) * hs.size(), cudaMemcpyDeviceToHost, caller));
  RBGS_CUDA_TRY(cudaStreamSynchronize(caller));
  rbgs_status first = RBGS_OK;
  for (int64_t i = 0; i < count; ++i) {
    const int* f = hs.data() + 8 * i;
    const rbgs_status si = f[3] ? RBGS_ETIMEOUT : (f[0] ? RBGS_EBREAKDOWN : RBGS_OK);
    probs[i].status = si;
    probs[i].passes2 = f[2];
    if (si && !first) first = si;
  }
  return first;
}

rbgs_status rbgs_qr_host(const void* W, int64_t n, int64_t m, int64_t ldw, int64_t mb, rbgs_sketch sketch,
                         int64_t k, uint64_t seed, void* Q, int64_t ldq, double* R, int64_t ldr, const rbgs_opts* opts,
                         rbgs_stats* stats) {
  rbgs_opts o;
  if (opts) o = *opts;
  else rbgs_opts_default(&o);
  if (!W || !Q || !R) return RBGS_EINVAL;
  const size_t es = o.prec == RBGS_P_FP64 ? 8 : 4;
  if (n >= 1 && m >= 1 && ldw >= n && ldq >= n &&
      ranges_overlap(W, es * (size_t)(ldw * (m - 1) + n), Q, es * (size_t)(ldq * (m - 1) + n)))
    return RBGS_EINVAL;
  // the device copies: W and Q with a leading dimension that is a multiple of 4, R packed
  const int64_t ldd = (n + 3) / 4 * 4;
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t bw = up(es * (size_t)ldd * (size_t)std::max<int64_t>(m, 1));
  const size_t br = up(8 * (size_t)std::max<int64_t>(m, 1) * (size_t)std::max<int64_t>(m, 1));
  rbgs_opts oi = o;
  oi.sync = 0;
  oi.timing = 0;
  oi.certify = 0;
  // the same checks as rbgs_qr, on the device copies' layout
  {
    rbgs_status s0 = check_qr((const void*)(uintptr_t)256, n, m, ldd, mb, sketch, k,
                              (const void*)(uintptr_t)(256 + bw), ldd, (const double*)(uintptr_t)(256 + 2 * bw), m, oi);
    if (s0) return s0;
    if (ldw < n || ldq < n || ldr < m) return RBGS_EINVAL;
  }
  void* buf = nullptr;
  rbgs_status s = host_path_buffer(2 * bw + br + 256, &buf);
  if (s) return s;
  char* Wd = (char*)buf;
  char* Qd = Wd + bw;
  double* Rd = (double*)(Qd + bw);
  int* dstat = nullptr;
  cudaStream_t h2d = nullptr, d2h = nullptr;
  if ((s = copy_streams(&h2d, &d2h))) return s;
  const int64_t p = (m + mb - 1) / mb;
  std::vector<cudaEvent_t> ev((size_t)(2 * p + 2), nullptr);
  struct EvFree {
    std::vector<cudaEvent_t>* v;
    int** d;
    ~EvFree() {
      for (auto e : *v)
        if (e) cudaEventDestroy(e);
      if (*d) cudaFree(*d);
    }
  } evfree{&ev, &dstat};
  // with opts.timing the events keep times: the copy and compute timeline of the call
  for (auto& e : ev) RBGS_CUDA_TRY(cudaEventCreateWithFlags(&e, o.timing ? cudaEventDefault : cudaEventDisableTiming));
  cudaEvent_t* w_ready = ev.data();
  cudaEvent_t* q_done = ev.data() + p;
  cudaEvent_t start = ev[(size_t)(2 * p)], copied = ev[(size_t)(2 * p + 1)];
  if (cudaMalloc(&dstat, 8 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return RBGS_ENOMEM;
  }
  cudaStream_t caller = (cudaStream_t)o.stream;
  RBGS_CUDA_TRY(cudaEventRecord(start, caller));
  RBGS_CUDA_TRY(cudaStreamWaitEvent(h2d, start, 0));
  // W goes up block by block ahead of the factorization
  for (int64_t b = 0; b < p; ++b) {
    const int64_t c = b * mb, w = std::min<int64_t>(mb, m - c);
    RBGS_CUDA_TRY(cudaMemcpy2DAsync(Wd + es * (size_t)(c * ldd), es * (size_t)ldd, (const char*)W + es * (size_t)(c * ldw),
                                    es * (size_t)ldw, es * (size_t)n, (size_t)w, cudaMemcpyHostToDevice, h2d));
    RBGS_CUDA_TRY(cudaEventRecord(w_ready[b], h2d));
  }
  QrCtx ctx;
  ctx.status_out = dstat;
  ctx.w_ready = w_ready;
  ctx.q_done = q_done;
  s = qr_dispatch(Wd, n, m, ldd, mb, sketch, k, seed, Qd, ldd, Rd, m, oi, nullptr, &ctx);
  if (s) {
    cudaStreamSynchronize(h2d);
    cudaStreamSynchronize(caller);
    return s;
  }
  // each finished block of Q comes down while the next ones are computed; R at the end
  for (int64_t b = 0; b < p; ++b) {
    const int64_t c = b * mb, w = std::min<int64_t>(mb, m - c);
    RBGS_CUDA_TRY(cudaStreamWaitEvent(d2h, q_done[b], 0));
    RBGS_CUDA_TRY(cudaMemcpy2DAsync((char*)Q + es * (size_t)(c * ldq), es * (size_t)ldq, Qd + es * (size_t)(c * ldd),
                                    es * (size_t)ldd, es * (size_t)n, (size_t)w, cudaMemcpyDeviceToHost, d2h));
  }
  RBGS_CUDA_TRY(cudaMemcpy2DAsync(R, 8 * (size_t)ldr, Rd, 8 * (size_t)m, 8 * (size_t)m, (size_t)m,
                                  cudaMemcpyDeviceToHost, d2h));
  int hs[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  RBGS_CUDA_TRY(cudaMemcpyAsync(hs, dstat, sizeof(hs), cudaMemcpyDeviceToHost, d2h));
  RBGS_CUDA_TRY(cudaEventRecord(copied, d2h));
  RBGS_CUDA_TRY(cudaStreamWaitEvent(caller, copied, 0));
  RBGS_CUDA_TRY(cudaStreamSynchronize(caller));
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->delta = -1.0;
    stats->delta_tilde = -1.0;
    stats->passes2 = hs[2];
    stats->chol_rounds2 = hs[5];
    if (o.timing) {
      float up = 0.f, comp = 0.f, tot = 0.f;
      RBGS_CUDA_TRY(cudaEventElapsedTime(&up, start, w_ready[p - 1]));
      RBGS_CUDA_TRY(cudaEventElapsedTime(&comp, start, q_done[p - 1]));
      RBGS_CUDA_TRY(cudaEventElapsedTime(&tot, start, copied));
      stats->host_up_ms = up;
      stats->host_compute_ms = comp;
      stats->host_total_ms = tot;
    }
  }
  if (hs[3]) return RBGS_ETIMEOUT;
  if (hs[0]) return RBGS_EBREAKDOWN;
  return RBGS_OK;
}

// Cholesky QR post-processing (the remark after Alg. 2): R' = chol(Q^T Q),
// Q <- Q R'^{-1}, R <- R' R, so that Q becomes l2-orthonormal.  The Gram matrix
// is formed with FP64 products, R' by a blocked Cholesky (blocks of mb), and
// Q R'^{-1} by a forward sweep over column blocks on the tall kernels:
// block j becomes [Q_new(:, 0:c) | Q_j] [-R'(0:c, j) R'_jj^{-1}; R'_jj^{-1}].
rbgs_status rbgs_cholqr_postprocess(int32_t prec, int64_t n, int64_t m, void* Q, int64_t ldq, double* R, int64_t ldr,
                                    int64_t mb, void* stream, int32_t sync) {
  if (!Q || !R || n < 1 || m < 1 || ldq < n || ldr < m || mb < 1 || mb > 64) return RBGS_EINVAL;
  if (prec < RBGS_P_FP64 || prec > RBGS_P_F16X3) return RBGS_EINVAL;
  if ((prec == RBGS_P_TF32X3 || prec == RBGS_P_F16X3) && (((uintptr_t)Q & 15) || (ldq % 4))) return RBGS_EINVAL;
  const size_t es = prec == RBGS_P_FP64 ? 8 : 4;
  if (ranges_overlap(R, 8 * (size_t)(ldr * (m - 1) + m), Q, es * (size_t)(ldq * (m - 1) + n))) return RBGS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t nb = (m + mb - 1) / mb;
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t bmm = up(8 * (size_t)m * m), bt = up(8 * (size_t)mb * m), bd = up(8 * (size_t)mb * mb * nb),
               bg = up(8 * (size_t)m * mb), bpart = up(8 * (size_t)kPartElems);
  DevBuf buf;
  if (cudaMalloc(&buf.p, 3 * bmm + bt + 2 * bd + bg + bpart + 1024) != cudaSuccess) {
    cudaGetLastError();
    return RBGS_ENOMEM;
  }
  char* w = (char*)buf.p;
  double* G = (double*)w;                     // Q^T Q, m x m
  double* Rp = (double*)(w + bmm);            // R', m x m (upper)
  double* Tmp = (double*)(w + 2 * bmm);       // R' R
  double* Tb = (double*)(w + 3 * bmm);        // one block row of the Schur complement, mb x m (ld mb)
  double* Dd = (double*)(w + 3 * bmm + bt);   // diagonal blocks R'_jj, mb x mb each
  double* Di = (double*)(w + 3 * bmm + bt + bd);  // their inverses
  double* Gb = (double*)(w + 3 * bmm + bt + 2 * bd);  // coefficients of one forward-sweep block
  double* part = (double*)(w + 3 * bmm + bt + 2 * bd + bg);
  int* flag = (int*)(w + 3 * bmm + bt + 2 * bd + bg + bpart);
  RBGS_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), st));
  RBGS_CUDA_TRY(cudaMemsetAsync(Rp, 0, 8 * (size_t)m * m, st));
  rbgs_status s;
  // G = Q^T Q in FP64
  for (int64_t j0 = 0; j0 < m; j0 += 64) {
    const int64_t nc = std::min<int64_t>(64, m - j0);
    if (prec == RBGS_P_FP64)
      s = small_gemm<double, double, double>(1, m, nc, n, 1.0, (const double*)Q, ldq, (const double*)Q + j0 * ldq, ldq,
                                             0.0, G + j0 * m, m, part, kPartElems, nullptr, st);
    else
      s = small_gemm<float, double, double>(1, m, nc, n, 1.0, (const float*)Q, ldq, (const float*)Q + j0 * ldq, ldq,
                                            0.0, G + j0 * m, m, part, kPartElems, nullptr, st);
    if (s) return s;
  }
  // blocked Cholesky, row block by row block: T = G(c:c+w, c:m) - R'(0:c, c:c+w)^T R'(0:c, c:m);
  // R'_jj = chol(T(:, 0:w)); R'(c:c+w, c+w:m) = R'_jj^{-T} T(:, w:)
  for (int64_t jb = 0; jb < nb; ++jb) {
    const int64_t c = jb * mb, wd = std::min<int64_t>(mb, m - c), rest = m - c;
    RBGS_CUDA_TRY(cudaMemcpy2DAsync(Tb, 8 * (size_t)wd, G + c + c * m, 8 * (size_t)m, 8 * (size_t)wd, (size_t)rest,
                                    cudaMemcpyDeviceToDevice, st));
    if (c > 0) {
      for (int64_t t0 = 0; t0 < rest; t0 += 64) {
        const int64_t nt = std::min<int64_t>(64, rest - t0);
        s = small_gemm<double, double, double>(1, wd, nt, c, -1.0, Rp + c * m, m, Rp + (c + t0) * m, m, 1.0,
                                               Tb + t0 * wd, wd, part, kPartElems, nullptr, st);
        if (s) return s;
      }
    }
    double* Rjj = Dd + (size_t)jb * mb * mb;
    double* Rjjinv = Di + (size_t)jb * mb * mb;
    if ((s = chol_inv<double>((int)wd, Tb, Rjj, Rjjinv, 0.0, flag, nullptr, nullptr, nullptr, st))) return s;
    RBGS_CUDA_TRY(cudaMemcpy2DAsync(Rp + c + c * m, 8 * (size_t)m, Rjj, 8 * (size_t)wd, 8 * (size_t)wd, (size_t)wd,
                                    cudaMemcpyDeviceToDevice, st));
    for (int64_t t0 = wd; t0 < rest; t0 += 64) {
      const int64_t nt = std::min<int64_t>(64, rest - t0);
      s = small_gemm<double, double, double>(1, wd, nt, wd, 1.0, Rjjinv, wd, Tb + t0 * wd, wd, 0.0,
                                             Rp + c + (c + t0) * m, m, part, kPartElems, nullptr, st);
      if (s) return s;
    }
  }
  // Q <- Q R'^{-1}: the forward sweep, in place, block by block
  for (int64_t jb = 0; jb < nb; ++jb) {
    const int64_t c = jb * mb, wd = std::min<int64_t>(mb, m - c);
    s = assemble_g<double, double>(c, (int)wd, Rp + c * m, m, Dd + (size_t)jb * mb * mb, Di + (size_t)jb * mb * mb, Gb,
                                   c + wd, nullptr, 0, nullptr, st);
    if (s) return s;
    char* Qj = (char*)Q + es * (size_t)(c * ldq);
    s = rbgs_tall_update(prec, n, c, wd, c > 0 ? Q : nullptr, ldq, Qj, ldq, Gb, c + wd, Qj, ldq, stream, 0);
    if (s) return s;
  }
  // R <- R' R (both upper triangular)
  for (int64_t t0 = 0; t0 < m; t0 += 64) {
    const int64_t nt = std::min<int64_t>(64, m - t0);
    s = small_gemm<double, double, double>(0, m, nt, m, 1.0, Rp, m, R + t0 * ldr, ldr, 0.0, Tmp + t0 * m, m, part,
                                           kPartElems, nullptr, st);
    if (s) return s;
  }
  RBGS_CUDA_TRY(cudaMemcpy2DAsync(R, 8 * (size_t)ldr, Tmp, 8 * (size_t)m, 8 * (size_t)m, (size_t)m,
                                  cudaMemcpyDeviceToDevice, st));
  int hf = 0;
  RBGS_CUDA_TRY(cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  RBGS_CUDA_TRY(cudaStreamSynchronize(st));  // the buffers are freed on return
  (void)sync;
  return hf ? RBGS_EBREAKDOWN : RBGS_OK;
}

}  // extern "C"

// A captured factorization: the graph of one rbgs_qr on fixed W, Q, R with its
// own workspace, side stream and status words, so that later library calls
// (which may grow or free the shared workspace) do not touch its buffers.
struct rbgs_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t side = nullptr;
  void* ws = nullptr;
  int* status = nullptr;
  // a captured batch (rbgs_qr_batched_graph_create): one stream, side stream,
  // workspace and done event per slot, 8 status words per problem
  std::vector<cudaStream_t> streams, sides;
  std::vector<void*> wss;
  std::vector<cudaEvent_t> events;
  int64_t count = 0;
  rbgs_problem* probs = nullptr;  // the caller's array, for the per-problem statuses
};

extern "C" {

rbgs_status rbgs_qr_graph_destroy(rbgs_graph* g) {
  if (!g) return RBGS_OK;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->side) {
    cudaStreamSynchronize(g->side);
    cudaStreamDestroy(g->side);
  }
  if (g->ws) cudaFree(g->ws);
  if (g->status) cudaFree(g->status);
  for (auto x : g->streams)
    if (x) {
      cudaStreamSynchronize(x);
      cudaStreamDestroy(x);
    }
  for (auto x : g->sides)
    if (x) {
      cudaStreamSynchronize(x);
      cudaStreamDestroy(x);
    }
  for (auto x : g->wss)
    if (x) cudaFree(x);
  for (auto x : g->events)
    if (x) cudaEventDestroy(x);
  delete g;
  return RBGS_OK;
}

rbgs_status rbgs_qr_graph_create(const void* W, int64_t n, int64_t m, int64_t ldw, int64_t mb, rbgs_sketch sketch,
                                 int64_t k, uint64_t seed, void* Q, int64_t ldq, double* R, int64_t ldr,
                                 const rbgs_opts* opts, rbgs_graph** out) {
  if (!out) return RBGS_EINVAL;
  *out = nullptr;
  rbgs_opts o;
  if (opts) o = *opts;
  else rbgs_opts_default(&o);
  rbgs_status s = check_qr(W, n, m, ldw, mb, sketch, k, Q, ldq, R, ldr, o);
  if (s) return s;
  if (o.interblock == 1 || o.interblock == 3) return RBGS_EINVAL;  // they allocate inside the factorization
  o.sync = 0;
  o.timing = 0;
  o.certify = 0;
  rbgs_graph* g = new rbgs_graph();
  struct Undo {
    rbgs_graph** g;
    ~Undo() {
      if (*g) rbgs_qr_graph_destroy(*g);
    }
  } undo{&g};
  size_t need = 0;
  QrCtx cq;
  cq.need_out = &need;
  if ((s = qr_dispatch(W, n, m, ldw, mb, sketch, k, seed, Q, ldq, R, ldr, o, nullptr, &cq))) return s;
  if (cudaMalloc(&g->ws, need) != cudaSuccess || cudaMalloc(&g->status, 8 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return RBGS_ENOMEM;
  }
  RBGS_CUDA_TRY(cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking));
  QrCtx c;
  c.ws = g->ws;
  c.ws_bytes = need;
  c.side = g->side;
  c.status_out = g->status;
  // one run outside the capture builds what the library caches (sketch plans, the
  // kernels' attributes), so that the capture holds stream work only
  cudaStream_t cs = nullptr;
  RBGS_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  struct StreamFree {
    cudaStream_t s;
    ~StreamFree() {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  } csf{cs};
  o.stream = cs;
  if ((s = qr_dispatch(W, n, m, ldw, mb, sketch, k, seed, Q, ldq, R, ldr, o, nullptr, &c))) return s;
  RBGS_CUDA_TRY(cudaStreamSynchronize(cs));
  RBGS_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  s = qr_dispatch(W, n, m, ldw, mb, sketch, k, seed, Q, ldq, R, ldr, o, nullptr, &c);
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
  if (s) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (ce != cudaSuccess) {
    cudaGetLastError();
    return RBGS_ECUDA;
  }
  g->graph = graph;
  RBGS_CUDA_TRY(cudaGraphInstantiate(&g->exec, g->graph, 0));
  *out = g;
  g = nullptr;  // owned by the caller now
  return RBGS_OK;
}

rbgs_status rbgs_qr_batched_graph_create(rbgs_problem* probs, int64_t count, rbgs_sketch sketch, const rbgs_opts* opts,
                                         int32_t nstreams, rbgs_graph** out) {
  if (!out || !probs || count < 1 || nstreams < 1) return RBGS_EINVAL;
  *out = nullptr;
  rbgs_opts o;
  if (opts) o = *opts;
  else rbgs_opts_default(&o);
  if (o.interblock == 1 || o.interblock == 3) return RBGS_EINVAL;  // they allocate inside the factorization
  for (int64_t i = 0; i < count; ++i) {
    const rbgs_problem& q = probs[i];
    rbgs_status s = check_qr(q.W, q.n, q.m, q.ldw, q.mb, sketch, q.k, q.Q, q.ldq, q.R, q.ldr, o);
    if (s) return s;
  }
  o.sync = 0;
  o.timing = 0;
  o.certify = 0;
  const int ns = (int)std::min<int64_t>(std::min<int64_t>(nstreams, count), 32);
  rbgs_graph* g = new rbgs_graph();
  struct Undo {
    rbgs_graph** g;
    ~Undo() {
      if (*g) rbgs_qr_graph_destroy(*g);
    }
  } undo{&g};
  g->count = count;
  g->probs = probs;
  std::vector<size_t> need((size_t)ns, 0);
  rbgs_status s;
  for (int64_t i = 0; i < count; ++i) {
    const rbgs_problem& q = probs[i];
    size_t nd = 0;
    QrCtx c;
    c.need_out = &nd;
    if ((s = qr_dispatch(q.W, q.n, q.m, q.ldw, q.mb, sketch, q.k, q.seed, q.Q, q.ldq, q.R, q.ldr, o, nullptr, &c)))
      return s;
    need[(size_t)(i % ns)] = std::max(need[(size_t)(i % ns)], nd);
  }
  g->streams.assign((size_t)ns, nullptr);
  g->sides.assign((size_t)ns, nullptr);
  g->wss.assign((size_t)ns, nullptr);
  g->events.assign((size_t)ns + 1, nullptr);
  for (int j = 0; j < ns; ++j) {
    RBGS_CUDA_TRY(cudaStreamCreateWithFlags(&g->streams[(size_t)j], cudaStreamNonBlocking));
    RBGS_CUDA_TRY(cudaStreamCreateWithFlags(&g->sides[(size_t)j], cudaStreamNonBlocking));
    if (cudaMalloc(&g->wss[(size_t)j], need[(size_t)j]) != cudaSuccess) {
      cudaGetLastError();
      return RBGS_ENOMEM;
    }
  }
  for (auto& e : g->events) RBGS_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  if (cudaMalloc(&g->status, sizeof(int) * 8 * (size_t)count) != cudaSuccess) {
    cudaGetLastError();
    return RBGS_ENOMEM;
  }
  cudaStream_t cs = nullptr;
  RBGS_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  struct StreamFree {
    cudaStream_t s;
    ~StreamFree() {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  } csf{cs};
  // the batch from cs: fork to the slot streams, every problem on its slot, join
  auto enqueue = [&]() -> rbgs_status {
    RBGS_CUDA_TRY(cudaEventRecord(g->events[(size_t)ns], cs));
    for (auto x : g->streams) RBGS_CUDA_TRY(cudaStreamWaitEvent(x, g->events[(size_t)ns], 0));
    for (int64_t i = 0; i < count; ++i) {
      const rbgs_problem& q = probs[i];
      const size_t j = (size_t)(i % ns);
      QrCtx c;
      c.ws = g->wss[j];
      c.ws_bytes = need[j];
      c.side = g->sides[j];
      c.status_out = g->status + 8 * i;
      rbgs_opts oi = o;
      oi.stream = g->streams[j];
      rbgs_status r = qr_dispatch(q.W, q.n, q.m, q.ldw, q.mb, sketch, q.k, q.seed, q.Q, q.ldq, q.R, q.ldr, oi,
                                  nullptr, &c);
      if (r) return r;
    }
    for (int j = 0; j < ns; ++j) {
      RBGS_CUDA_TRY(cudaEventRecord(g->events[(size_t)j], g->streams[(size_t)j]));
      RBGS_CUDA_TRY(cudaStreamWaitEvent(cs, g->events[(size_t)j], 0));
    }
    return RBGS_OK;
  };
  // one run outside the capture fills the library's caches (sketch plans, kernel attributes)
  if ((s = enqueue())) return s;
  RBGS_CUDA_TRY(cudaStreamSynchronize(cs));
  RBGS_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  s = enqueue();
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
  if (s) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (ce != cudaSuccess) {
    cudaGetLastError();
    return RBGS_ECUDA;
  }
  g->graph = graph;
  RBGS_CUDA_TRY(cudaGraphInstantiate(&g->exec, g->graph, 0));
  *out = g;
  g = nullptr;
  return RBGS_OK;
}

rbgs_status rbgs_qr_graph_launch(rbgs_graph* g, void* stream, int32_t sync) {
  if (!g || !g->exec) return RBGS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  RBGS_CUDA_TRY(cudaGraphLaunch(g->exec, st));
  if (!sync) return RBGS_OK;
  if (g->count > 0) {  // a batch: every problem's status words
    std::vector<int> hs((size_t)g->count * 8);
    RBGS_CUDA_TRY(cudaMemcpyAsync(hs.data(), g->status, sizeof(int) * hs.size(), cudaMemcpyDeviceToHost, st));
    RBGS_CUDA_TRY(cudaStreamSynchronize(st));
    rbgs_status first = RBGS_OK;
    for (int64_t i = 0; i < g->count; ++i) {
      const int* f = hs.data() + 8 * i;
      const rbgs_status si = f[3] ? RBGS_ETIMEOUT : (f[0] ? RBGS_EBREAKDOWN : RBGS_OK);
      g->probs[i].status = si;
      g->probs[i].passes2 = f[2];
      if (si && !first) first = si;
    }
    return first;
  }
  int hs[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  RBGS_CUDA_TRY(cudaMemcpyAsync(hs, g->status, sizeof(hs), cudaMemcpyDeviceToHost, st));
  RBGS_CUDA_TRY(cudaStreamSynchronize(st));
  if (hs[3]) return RBGS_ETIMEOUT;
  if (hs[0]) return RBGS_EBREAKDOWN;
  return RBGS_OK;
}

rbgs_status rbgs_sketch_apply(rbgs_sketch sketch, int64_t k, int64_t n, uint64_t seed, int32_t prec, const void* X,
                              int64_t ldx, int64_t ncols, double* Y, int64_t ldy, void* stream, int32_t sync) {
  if (!X || !Y || n < 1 || k < 1 || ncols < 0 || ldx < n || ldy < k) return RBGS_EINVAL;
  if (prec < RBGS_P_FP64 || prec > RBGS_P_F16X3) return RBGS_EINVAL;
  if (sketch == RBGS_SK_SRHT) {
    int64_t np = 1;
    while (np < n) np <<= 1;
    if (k > np) return RBGS_EINVAL;
  } else if (sketch != RBGS_SK_GAUSS && sketch != RBGS_SK_RADEMACHER && sketch != RBGS_SK_SPARSE) {
    return RBGS_EINVAL;
  }
  const bool fp64 = prec == RBGS_P_FP64;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = sketch_scratch_bytes(sketch, k, n, ncols, fp64) + 256;
  void* scr = nullptr;
  rbgs_status s = workspace(bytes, &scr);
  if (s) return s;
  if (fp64) s = sketch_apply_t<double, double>(sketch, k, n, seed, (const double*)X, ldx, ncols, Y, ldy, scr, bytes, st);
  else s = sketch_apply_t<float, double>(sketch, k, n, seed, (const float*)X, ldx, ncols, Y, ldy, scr, bytes, st);
  if (s) return s;
  if (sync) RBGS_CUDA_TRY(cudaStreamSynchronize(st));
  return RBGS_OK;
}

rbgs_status rbgs_tall_update(int32_t prec, int64_t n, int64_t c, int64_t mb, const void* Qprev, int64_t ldq,
                             const void* X, int64_t ldx, const double* G, int64_t ldg, void* Qout, int64_t ldo,
                             void* stream, int32_t sync) {
  if (!X || !G || !Qout || (c > 0 && !Qprev)) return RBGS_EINVAL;
  if (n < 1 || c < 0 || mb < 1 || mb > 64 || ldx < n || ldo < n || (c > 0 && ldq < n) || ldg < c + mb)
    return RBGS_EINVAL;
  if (prec < RBGS_P_FP64 || prec > RBGS_P_F16X3) return RBGS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t K = c + mb;
  rbgs_status s;
  if (prec == RBGS_P_F16X3) {
    // the basis carries no sketch here: split it with scales from its column maxima
    if (((uintptr_t)X & 15) || (ldx % 4)) return RBGS_EINVAL;
    if (ranges_overlap(Qout, 4 * (size_t)(ldo * (mb - 1) + n), Qprev, c > 0 ? 4 * (size_t)(ldq * (c - 1) + n) : 0))
      return RBGS_EINVAL;
    const int64_t nch = h3_nch_row(c);
    const size_t qs_bytes = h3_qs_bytes(n, c), b_bytes = h3_b_bytes(c);
    const size_t need = 256 + qs_bytes + b_bytes + 4 * (320 + (size_t)c + (size_t)c + 64) + 1024;
    void* scr = nullptr;
    if ((s = workspace(need, &scr))) return s;
    char* w = (char*)scr;
    int* err = (int*)w;
    unsigned char* Qs = (unsigned char*)(w + 256);
    unsigned char* B = Qs + qs_bytes;
    float* sc = (float*)(B + b_bytes);
    float* qscale = sc + 320;
    unsigned int* mxq = (unsigned int*)(qscale + c);
    unsigned int* mxx = mxq + c;
    RBGS_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    if (c > 0) {
      if ((s = h3_colmax(n, c, (const float*)Qprev, ldq, mxq, st))) return s;
      if ((s = h3_scales_from_max(c, mxq, qscale, st))) return s;
      if ((s = h3_split(n, c, (const float*)Qprev, ldq, qscale, nch, Qs, st))) return s;
    }
    if ((s = h3_colmax(n, mb, (const float*)X, ldx, mxx, st))) return s;
    s = h3_prepare<float>(c, mb, G, ldg, nullptr, 0, (const float*)mxx, c > 0 ? qscale : nullptr, 0, B, sc,
                          nullptr, st);
    if (s) return s;
    s = tall_update_h3(n, c, mb, c > 0 ? Qs : nullptr, nch, (const float*)X, ldx, B, sc, (float*)Qout, ldo, nullptr,
                       0, 0, nullptr, err, st);
    if (s) return s;
    if (sync) {
      int herr = 0;
      RBGS_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
      RBGS_CUDA_TRY(cudaStreamSynchronize(st));
      if (herr) return RBGS_ETIMEOUT;
    }
    return RBGS_OK;
  }
  if (prec == RBGS_P_FP64) {
    s = tall_update_simt<double>(n, c, mb, (const double*)Qprev, ldq, (const double*)X, ldx, G, ldg, (double*)Qout,
                                 ldo, nullptr, st);
  } else if (prec == RBGS_P_FP32) {
    void* scr = nullptr;
    if ((s = workspace(sizeof(float) * K * mb + 256, &scr))) return s;
    float* Gf = (float*)scr;
    const int64_t tot = K * mb;
    cast_d2f_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(K, mb, G, ldg, Gf, K);
    RBGS_LAUNCH_CHECK();
    s = tall_update_simt<float>(n, c, mb, (const float*)Qprev, ldq, (const float*)X, ldx, Gf, K, (float*)Qout, ldo,
                                nullptr, st);
  } else {
    if (((uintptr_t)X & 15) || ((uintptr_t)Qout & 15) || (c > 0 && ((uintptr_t)Qprev & 15)) || (ldx % 4) ||
        (ldo % 4) || (c > 0 && (ldq % 4)))
      return RBGS_EINVAL;
    void* scr = nullptr;
    if ((s = workspace(sizeof(float) * tc_gsplit_floats(K) + 512, &scr))) return s;
    int* err = (int*)scr;
    float* Gs = (float*)((char*)scr + 256);
    RBGS_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    if ((s = tc_split_g(K, mb, G, ldg, Gs, nullptr, st))) return s;
    s = tall_update_tc(n, c, mb, (const float*)Qprev, ldq, (const float*)X, ldx, Gs, (float*)Qout, ldo, nullptr, err,
                       st);
    if (s) return s;
    if (sync) {
      int herr = 0;
      RBGS_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
      RBGS_CUDA_TRY(cudaStreamSynchronize(st));
      if (herr) return RBGS_ETIMEOUT;
    }
    return RBGS_OK;
  }
  if (s) return s;
  if (sync) RBGS_CUDA_TRY(cudaStreamSynchronize(st));
  return RBGS_OK;
}

rbgs_status rbgs_philox(uint64_t seed, const uint32_t* ctr, uint32_t* out, int64_t count, void* stream,
                        int32_t sync) {
  if (!ctr || !out || count < 0) return RBGS_EINVAL;
  if (count == 0) return RBGS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  philox_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(seed_key(seed), ctr, out, count);
  RBGS_LAUNCH_CHECK();
  if (sync) RBGS_CUDA_TRY(cudaStreamSynchronize(st));
  return RBGS_OK;
}

rbgs_status rbgs_sparse_sign_columns(uint64_t seed, int64_t k, int64_t j0, int64_t count, int64_t* rows,
                                     int32_t* neg) {
  if (!rows || !neg || k < 1 || j0 < 0 || count < 0) return RBGS_EINVAL;
  const uint2 key = seed_key(seed);
  for (int64_t t = 0; t < count; ++t) {
    int64_t r[8];
    bool g[8];
    const int z = sparse_column(key, j0 + t, k, r, g);
    for (int s = 0; s < z; ++s) {
      rows[t * z + s] = r[s];
      neg[t * z + s] = g[s] ? 1 : 0;
    }
  }
  return RBGS_OK;
}

rbgs_status rbgs_gaussian_entries(uint64_t seed, int64_t k, const int64_t* r, const int64_t* j, int64_t count,
                                  double* out) {
  if (k < 1 || count < 0 || (count > 0 && (!r || !j || !out))) return RBGS_EINVAL;
  for (int64_t t = 0; t < count; ++t)
    if (r[t] < 0 || r[t] >= k || j[t] < 0) return RBGS_EINVAL;
  const uint2 key = seed_key(seed);
  const double scale = 1.0 / std::sqrt((double)k);  // as the sketch kernels scale the entries
  for (int64_t t = 0; t < count; ++t) {
    double z0, z1;
    gauss_pair(key, j[t], (uint32_t)(r[t] >> 1), z0, z1);
    out[t] = ((r[t] & 1) ? z1 : z0) * scale;
  }
  return RBGS_OK;
}

rbgs_status rbgs_release_workspace(void) {
  int dev = 0;
  RBGS_CUDA_TRY(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lock(g_ws_mu);
    for (auto& w : g_ws)
      if (w.dev == dev && w.ptr) {
        cudaDeviceSynchronize();
        cudaFree(w.ptr);
        w.ptr = nullptr;
        w.bytes = 0;
      }
  }
  host_path_release();
  srht_plans_release();
  unet_release(dev);
  noalloc_forget_device(dev);
  return RBGS_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ Sec. 5 --

namespace {

rbgs_status check_op(const rbgs_op* op) {
  if (!op || (op->kind != RBGS_OP_STENCIL5 && op->kind != RBGS_OP_DIFFUSION) || op->nx < 1 || op->ny < 1)
    return RBGS_EINVAL;
  if (op->nx * op->ny >= ((int64_t)1 << 31)) return RBGS_EINVAL;
  if (op->kind == RBGS_OP_STENCIL5 && (!std::isfinite(op->bx) || !std::isfinite(op->by))) return RBGS_EINVAL;
  if (op->kind == RBGS_OP_DIFFUSION && !op->coef) return RBGS_EINVAL;
  return RBGS_OK;
}

rbgs_status check_sketch(rbgs_sketch sketch, int64_t n, int64_t k, int64_t m) {
  if (k < m) return RBGS_EINVAL;
  if (sketch == RBGS_SK_SRHT) {
    int64_t np = 1;
    while (np < n) np <<= 1;
    return k > np ? RBGS_EINVAL : RBGS_OK;
  }
  if (sketch == RBGS_SK_GAUSS || sketch == RBGS_SK_RADEMACHER || sketch == RBGS_SK_SPARSE)
    return k > n ? RBGS_EINVAL : RBGS_OK;
  return RBGS_EINVAL;
}

// Alg. 7 on (W = B, Q): dispatch by precision (the arguments are checked).
rbgs_status arnoldi_run(const rbgs_op& op, const void* B, int64_t ldb, int64_t mb, int64_t p, rbgs_sketch sketch,
                        int64_t k, uint64_t seed, void* Q, int64_t ldq, double* R, int64_t ldr, const rbgs_opts& o,
                        rbgs_stats* stats, const QrCtx* ctx = nullptr) {
  const int64_t n = op.nx * op.ny, m = p * mb;
  if (o.prec == RBGS_P_FP64)
    return qr_impl<double, double>((const double*)B, n, m, ldb, (int)mb, sketch, k, seed, (double*)Q, ldq, R, ldr, o,
                                   stats, 0, &op, ctx);
  const int mode = o.prec == RBGS_P_TF32X3 ? 1 : (o.prec == RBGS_P_F16X3 ? 2 : 0);
  if (o.fine)
    return qr_impl<float, double>((const float*)B, n, m, ldb, (int)mb, sketch, k, seed, (float*)Q, ldq, R, ldr, o,
                                  stats, mode, &op, ctx);
  return qr_impl<float, float>((const float*)B, n, m, ldb, (int)mb, sketch, k, seed, (float*)Q, ldq, R, ldr, o, stats,
                               mode, &op, ctx);
}

// The U-Net preconditioner as the flexible Arnoldi's hook.
struct FlexNet {
  const rbgs_unet* net;
  const float* params;
  int N;
  bool f64;
};
rbgs_status flex_unet(void* fctx, const void* Q, int64_t ldq, int mb, void* Z, int64_t ldz, cudaStream_t st) {
  const FlexNet* f = (const FlexNet*)fctx;
  if (f->f64)
    return unet_precondition<double>(*f->net, f->params, f->N, mb, (const double*)Q, ldq, (double*)Z, ldz, st);
  return unet_precondition<float>(*f->net, f->params, f->N, mb, (const float*)Q, ldq, (float*)Z, ldz, st);
}

// Restarted randomized block flexible GMRES with the U-Net preconditioner and
// plain block GMRES as the fallback (rbgs_block_fgmres).
rbgs_status fgmres_solve(const rbgs_op* op, const rbgs_unet* net, const float* params, const double* B, int64_t ldb,
                         double* X, int64_t ldx, int64_t mb, int64_t p, double rtol, int64_t max_cycles,
                         double accept, rbgs_sketch sketch, int64_t k, uint64_t seed, const rbgs_opts* opts,
                         int64_t* cycles, double* relres, int64_t* fallbacks) {
  rbgs_status s;
  if ((s = check_op(op))) return s;
  const int64_t n = op->nx * op->ny, m = p * mb, nk = m - mb;
  if (!B || !X || !relres || mb < 1 || mb > 64 || p < 2 || ldb < n || ldx < n || max_cycles < 0 || !(rtol >= 0.0) ||
      !(accept > 0.0 && accept <= 1.0))
    return RBGS_EINVAL;
  if (net && (!params || op->nx != op->ny || !unet_valid(net, op->nx))) return RBGS_EINVAL;
  if ((s = check_sketch(sketch, n, k, m))) return s;
  rbgs_opts o;
  if (opts) o = *opts;
  else rbgs_opts_default(&o);
  if (o.prec < RBGS_P_FP64 || o.prec > RBGS_P_F16X3 || o.reorth < 0 || o.reorth > 2 || o.fine < 0 || o.fine > 2 ||
      (o.interblock != 0 && o.interblock != 4 && o.interblock != 5) || (o.ls != 0 && o.ls != 1) ||
      (o.trsm != 0 && (o.trsm != 1 || o.interblock != 4)))
    return RBGS_EINVAL;
  o.sync = 1;
  o.timing = 0;
  cudaStream_t st = (cudaStream_t)o.stream;
  const bool f64 = o.prec == RBGS_P_FP64;
  const size_t es = f64 ? 8 : 4;
  const size_t part_elems = residual_part_elems(n, mb);
  const size_t bytes_q = es * (size_t)n * (size_t)m, bytes_z = es * (size_t)n * (size_t)nk,
               bytes_r = 8 * (size_t)n * (size_t)mb, bytes_d = es * (size_t)n * (size_t)mb;
  const size_t small = 8 * ((size_t)m * m + (size_t)m * nk + (size_t)m * mb + (size_t)nk * mb + 2 * mb + part_elems) +
                       4 * ((size_t)nk * mb) + 1024;
  DevBuf buf;
  if (cudaMalloc(&buf.p, bytes_q + bytes_z + 2 * bytes_r + bytes_d + small + 8192) != cudaSuccess) {
    cudaGetLastError();
    return RBGS_ENOMEM;
  }
  char* w = (char*)buf.p;
  auto take = [&](size_t b) {
    char* r = w;
    w += (b + 255) & ~(size_t)255;
    return (void*)r;
  };
  void* Qb = take(bytes_q);
  void* Zb = take(bytes_z);
  double* r = (double*)take(bytes_r);
  double* Xt = (double*)take(bytes_r);
  void* D = take(bytes_d);
  double* Rm = (double*)take(8 * (size_t)m * m);
  double* Hb = (double*)take(8 * (size_t)m * nk);
  double* Fb = (double*)take(8 * (size_t)m * mb);
  double* Zc = (double*)take(8 * (size_t)nk * mb);
  float* Zf = (float*)take(4 * (size_t)nk * mb);
  double* norms = (double*)take(8 * (size_t)mb);
  double* bnorm = (double*)take(8 * (size_t)mb);
  double* part = (double*)take(8 * part_elems);
  int* flag = (int*)take(256);
  RBGS_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), st));
  std::vector<double> hb((size_t)mb), hn((size_t)mb);
  if ((s = colnorms_t(n, mb, B, ldb, part, bnorm, st))) return s;
  RBGS_CUDA_TRY(cudaMemcpyAsync(hb.data(), bnorm, 8 * mb, cudaMemcpyDeviceToHost, st));
  RBGS_CUDA_TRY(cudaStreamSynchronize(st));
  for (auto& v : hb)
    if (!(v > 0.0)) v = 1.0;
  FlexNet fn{net, params, (int)op->nx, f64};
  QrCtx fctx;
  fctx.flex = flex_unet;
  fctx.flex_ctx = &fn;
  fctx.zbuf = Zb;
  fctx.ldz = n;
  // relative residuals of r (norms on the device) into rel[] and their maximum
  auto rel_of = [&](std::vector<double>& rel, double& worst) -> rbgs_status {
    RBGS_CUDA_TRY(cudaMemcpyAsync(hn.data(), norms, 8 * mb, cudaMemcpyDeviceToHost, st));
    RBGS_CUDA_TRY(cudaStreamSynchronize(st));
    worst = 0.0;
    for (int64_t j = 0; j < mb; ++j) {
      rel[(size_t)j] = hn[(size_t)j] / hb[(size_t)j];
      worst = std::max(worst, rel[(size_t)j]);
    }
    return RBGS_OK;
  };
  // one cycle from r into Xt = X + (Z or Q) z; with_net selects the flexible basis
  auto cycle = [&](bool with_net) -> rbgs_status {
    rbgs_status e;
    if (f64) e = cast_cols_t<double, double>(n, mb, r, n, (double*)Qb, n, st);
    else e = cast_cols_t<double, float>(n, mb, r, n, (float*)Qb, n, st);
    if (e) return e;
    if ((e = arnoldi_run(*op, Qb, n, mb, p, sketch, k, seed, Qb, n, Rm, m, o, nullptr, with_net ? &fctx : nullptr)))
      return e;
    RBGS_CUDA_TRY(cudaMemcpy2DAsync(Hb, 8 * m, Rm + mb * m, 8 * m, 8 * m, nk, cudaMemcpyDeviceToDevice, st));
    RBGS_CUDA_TRY(cudaMemcpy2DAsync(Fb, 8 * m, Rm, 8 * m, 8 * m, mb, cudaMemcpyDeviceToDevice, st));
    if ((e = banded_ls((int)m, (int)nk, (int)mb, Hb, (int)m, Fb, (int)m, (int)mb, Zc, (int)nk, flag, st))) return e;
    const void* Vb = with_net ? Zb : Qb;  // the correction lives in range(Z) (flexible) or range(Q)
    const int64_t c = nk - mb;
    if (f64) {
      e = tall_update_simt<double>(n, c, mb, (const double*)Vb, n, (const double*)Vb + c * n, n, Zc, nk, (double*)D, n,
                                   nullptr, st);
    } else {
      if ((e = cast_cols_t<double, float>(nk, mb, Zc, nk, Zf, nk, st))) return e;
      e = tall_update_simt<float>(n, c, mb, (const float*)Vb, n, (const float*)Vb + c * n, n, Zf, nk, (float*)D, n,
                                  nullptr, st);
    }
    if (e) return e;
    RBGS_CUDA_TRY(cudaMemcpy2DAsync(Xt, 8 * n, X, 8 * ldx, 8 * n, mb, cudaMemcpyDeviceToDevice, st));
    if (f64) e = add_cols_t<double>(n, mb, (const double*)D, n, Xt, n, st);
    else e = add_cols_t<float>(n, mb, (const float*)D, n, Xt, n, st);
    if (e) return e;
    int hflag = 0;
    RBGS_CUDA_TRY(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBGS_CUDA_TRY(cudaStreamSynchronize(st));
    return hflag ? RBGS_EBREAKDOWN : RBGS_OK;
  };
  std::vector<double> rel((size_t)mb), rel_t((size_t)mb);
  int64_t cyc = 0, fb = 0;
  double worst = 0.0;
  if ((s = residual_t(*op, B, ldb, X, ldx, mb, r, n, part, norms, st))) return s;
  if ((s = rel_of(rel, worst))) return s;
  for (;;) {
    if (!(worst > rtol) || cyc >= max_cycles) {
      for (int64_t j = 0; j < mb; ++j) relres[j] = rel[(size_t)j];
      if (cycles) *cycles = cyc;
      if (fallbacks) *fallbacks = fb;
      return worst <= rtol ? RBGS_OK : RBGS_ENOCONV;
    }
    bool plain = net == nullptr;
    double worst_t = 0.0;
    if (!plain) {
      s = cycle(true);
      if (s && s != RBGS_EBREAKDOWN) return s;
      if (!s) {
        if ((s = residual_t(*op, B, ldb, Xt, n, mb, r, n, part, norms, st))) return s;
        if ((s = rel_of(rel_t, worst_t))) return s;
      }
      if (s == RBGS_EBREAKDOWN || !(worst_t <= accept * worst)) {  // fall back from the same X (r is recomputed)
        plain = true;
        ++fb;
        RBGS_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), st));
        if ((s = residual_t(*op, B, ldb, X, ldx, mb, r, n, part, norms, st))) return s;
      }
    }
    if (plain) {
      if ((s = cycle(false))) return s;
      if ((s = residual_t(*op, B, ldb, Xt, n, mb, r, n, part, norms, st))) return s;
      if ((s = rel_of(rel_t, worst_t))) return s;
    }
    RBGS_CUDA_TRY(cudaMemcpy2DAsync(X, 8 * ldx, Xt, 8 * n, 8 * n, mb, cudaMemcpyDeviceToDevice, st));
    rel = rel_t;
    worst = worst_t;
    ++cyc;
  }
}


// Restarted randomized block GMRES (method 0) or FOM (method 1).
rbgs_status krylov_solve(int method, const rbgs_op* op, const double* B, int64_t ldb, double* X, int64_t ldx,
                         int64_t mb, int64_t p, double rtol, int64_t max_cycles, rbgs_sketch sketch, int64_t k,
                         uint64_t seed, const rbgs_opts* opts, int64_t* cycles, double* relres) {
  rbgs_status s;
  if ((s = check_op(op))) return s;
  const int64_t n = op->nx * op->ny, m = p * mb, nk = m - mb;
  if (!B || !X || !relres || mb < 1 || mb > 64 || p < 2 || ldb < n || ldx < n || max_cycles < 0 || !(rtol >= 0.0))
    return RBGS_EINVAL;
  if ((s = check_sketch(sketch, n, k, m))) return s;
  rbgs_opts o;
  if (opts) o = *opts;
  else rbgs_opts_default(&o);
  if (o.prec < RBGS_P_FP64 || o.prec > RBGS_P_F16X3 || o.reorth < 0 || o.reorth > 2 || o.fine < 0 || o.fine > 2 ||
      (o.interblock != 0 && o.interblock != 4 && o.interblock != 5) || (o.ls != 0 && o.ls != 1) ||
      (o.trsm != 0 && (o.trsm != 1 || o.interblock != 4)))
    return RBGS_EINVAL;
  o.sync = 1;  // one synchronisation per cycle (breakdown and convergence are read on the host)
  o.timing = 0;
  cudaStream_t st = (cudaStream_t)o.stream;
  const bool f64 = o.prec == RBGS_P_FP64;
  const size_t es = f64 ? 8 : 4;
  // buffers: basis Q (n x m), residual r (n x mb), correction D (n x mb, basis type), the
  // Arnoldi R (m x m), H and F copies, z, G in float, norms and partial sums, a flag
  const size_t part_elems = residual_part_elems(n, mb);
  const size_t bytes_q = es * (size_t)n * (size_t)m, bytes_r = 8 * (size_t)n * (size_t)mb,
               bytes_d = es * (size_t)n * (size_t)mb;
  const size_t small = 8 * ((size_t)m * m + (size_t)m * nk + (size_t)m * mb + (size_t)nk * mb + 2 * mb + part_elems) +
                       4 * ((size_t)nk * mb) + 1024;
  DevBuf buf;
  if (cudaMalloc(&buf.p, bytes_q + bytes_r + bytes_d + small + 4096) != cudaSuccess) {
    cudaGetLastError();
    return RBGS_ENOMEM;
  }
  char* w = (char*)buf.p;
  auto take = [&](size_t b) {
    char* r = w;
    w += (b + 255) & ~(size_t)255;
    return (void*)r;
  };
  void* Qb = take(bytes_q);
  double* r = (double*)take(bytes_r);
  void* D = take(bytes_d);
  double* Rm = (double*)take(8 * (size_t)m * m);
  double* Hb = (double*)take(8 * (size_t)m * nk);
  double* Fb = (double*)take(8 * (size_t)m * mb);
  double* Z = (double*)take(8 * (size_t)nk * mb);
  float* Zf = (float*)take(4 * (size_t)nk * mb);
  double* norms = (double*)take(8 * (size_t)mb);
  double* bnorm = (double*)take(8 * (size_t)mb);
  double* part = (double*)take(8 * part_elems);
  int* flag = (int*)take(256);
  RBGS_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), st));
  std::vector<double> hb((size_t)mb), hn((size_t)mb);
  if ((s = colnorms_t(n, mb, B, ldb, part, bnorm, st))) return s;
  RBGS_CUDA_TRY(cudaMemcpyAsync(hb.data(), bnorm, 8 * mb, cudaMemcpyDeviceToHost, st));
  RBGS_CUDA_TRY(cudaStreamSynchronize(st));
  for (auto& v : hb)
    if (!(v > 0.0)) v = 1.0;
  int64_t cyc = 0;
  for (;;) {
    if ((s = residual_t(*op, B, ldb, X, ldx, mb, r, n, part, norms, st))) return s;
    RBGS_CUDA_TRY(cudaMemcpyAsync(hn.data(), norms, 8 * mb, cudaMemcpyDeviceToHost, st));
    RBGS_CUDA_TRY(cudaStreamSynchronize(st));
    double worst = 0.0;
    for (int64_t j = 0; j < mb; ++j) {
      relres[j] = hn[(size_t)j] / hb[(size_t)j];
      worst = std::max(worst, relres[j]);
    }
    if (!(worst > rtol) || cyc >= max_cycles) {
      if (cycles) *cycles = cyc;
      return worst <= rtol ? RBGS_OK : RBGS_ENOCONV;
    }
    // Alg. 7 on the residual block (W_1 = r in the basis precision)
    if (f64) s = cast_cols_t<double, double>(n, mb, r, n, (double*)Qb, n, st);
    else s = cast_cols_t<double, float>(n, mb, r, n, (float*)Qb, n, st);
    if (s) return s;
    if ((s = arnoldi_run(*op, Qb, n, mb, p, sketch, k, seed, Qb, n, Rm, m, o, nullptr))) return s;
    // the projected problem in FP64: H = R(:, mb:), F = R(:, 0:mb) (GMRES) or their top nk rows (FOM)
    const int64_t M = method == 0 ? m : nk;
    RBGS_CUDA_TRY(cudaMemcpy2DAsync(Hb, 8 * M, Rm + mb * m, 8 * m, 8 * M, nk, cudaMemcpyDeviceToDevice, st));
    RBGS_CUDA_TRY(cudaMemcpy2DAsync(Fb, 8 * M, Rm, 8 * m, 8 * M, mb, cudaMemcpyDeviceToDevice, st));
    if ((s = banded_ls((int)M, (int)nk, (int)mb, Hb, (int)M, Fb, (int)M, (int)mb, Z, (int)nk, flag, st))) return s;
    // X += Q(:, 0:nk) z, the product on the tall kernel of the basis type
    const int64_t c = nk - mb;
    if (f64) {
      s = tall_update_simt<double>(n, c, mb, (const double*)Qb, n, (const double*)Qb + c * n, n, Z, nk,
                                   (double*)D, n, nullptr, st);
    } else {
      if ((s = cast_cols_t<double, float>(nk, mb, Z, nk, Zf, nk, st))) return s;
      s = tall_update_simt<float>(n, c, mb, (const float*)Qb, n, (const float*)Qb + c * n, n, Zf, nk, (float*)D, n,
                                  nullptr, st);
    }
    if (s) return s;
    if (f64) s = add_cols_t<double>(n, mb, (const double*)D, n, X, ldx, st);
    else s = add_cols_t<float>(n, mb, (const float*)D, n, X, ldx, st);
    if (s) return s;
    int hflag = 0;
    RBGS_CUDA_TRY(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBGS_CUDA_TRY(cudaStreamSynchronize(st));
    if (hflag) return RBGS_EBREAKDOWN;
    ++cyc;
  }
}

// Alg. 8: randomized Rayleigh-Ritz with restarting.
rbgs_status rayleigh_ritz(const rbgs_op* op, const double* B0, int64_t ldb, int64_t mb, int64_t p, int64_t n_iter,
                          int32_t which, rbgs_sketch sketch, int64_t k, uint64_t seed, const rbgs_opts* opts,
                          double* X, int64_t ldx, double* ritz_re, double* ritz_im, double* resid_est) {
  rbgs_status s;
  if ((s = check_op(op))) return s;
  const int64_t n = op->nx * op->ny, m = p * mb, N = m - mb;
  if (!B0 || !X || !ritz_re || !ritz_im || !resid_est || mb < 1 || mb > 64 || p < 2 || n_iter < 1 || ldb < n ||
      ldx < n || (which != 0 && which != 1) || N > kRitzMaxN)
    return RBGS_EINVAL;
  if ((s = check_sketch(sketch, n, k, m))) return s;
  rbgs_opts o;
  if (opts) o = *opts;
  else rbgs_opts_default(&o);
  if (o.prec < RBGS_P_FP64 || o.prec > RBGS_P_F16X3 || o.reorth < 0 || o.reorth > 2 || o.fine < 0 || o.fine > 2 ||
      (o.interblock != 0 && o.interblock != 4 && o.interblock != 5) || (o.ls != 0 && o.ls != 1) ||
      (o.trsm != 0 && (o.trsm != 1 || o.interblock != 4)))
    return RBGS_EINVAL;
  o.sync = 1;
  o.timing = 0;
  cudaStream_t st = (cudaStream_t)o.stream;
  const bool f64 = o.prec == RBGS_P_FP64;
  const size_t es = f64 ? 8 : 4;
  // buffers: basis Q (n x m), block B (n x mb, basis type), the Arnoldi R (m x m), Y (N x mb) in FP64
  // and the basis type, Ritz values and residual estimates, column norms, the eigen-solver's scratch
  const size_t part_elems = residual_part_elems(n, mb);
  const size_t bytes = es * (size_t)n * (size_t)m + es * (size_t)n * (size_t)mb + 8 * (size_t)m * m +
                       (8 + es) * (size_t)N * mb + 8 * (4 * (size_t)mb + part_elems) + ritz_eig_scratch_bytes((int)N, (int)mb, (int)mb) +
                       16 * 256;
  DevBuf buf;
  if (cudaMalloc(&buf.p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return RBGS_ENOMEM;
  }
  char* w = (char*)buf.p;
  auto take = [&](size_t b) {
    char* r = w;
    w += (b + 255) & ~(size_t)255;
    return (void*)r;
  };
  void* Qb = take(es * (size_t)n * m);
  void* Bb = take(es * (size_t)n * mb);
  double* Rm = (double*)take(8 * (size_t)m * m);
  double* Y = (double*)take(8 * (size_t)N * mb);
  void* Yt = take(es * (size_t)N * mb);
  double* vals = (double*)take(16 * (size_t)mb);
  double* res = (double*)take(8 * (size_t)mb);
  double* norms = (double*)take(8 * (size_t)mb);
  double* part = (double*)take(8 * part_elems);
  void* scr = take(ritz_eig_scratch_bytes((int)N, (int)mb, (int)mb));
  int* status = (int*)take(256);
  if (f64) s = cast_cols_t<double, double>(n, mb, B0, ldb, (double*)Bb, n, st);
  else s = cast_cols_t<double, float>(n, mb, B0, ldb, (float*)Bb, n, st);
  if (s) return s;
  const int64_t c = N - mb;
  for (int64_t it = 0; it < n_iter; ++it) {
    // step 1: Alg. 7 from B; H = R(:, mb:).  A breakdown after the first
    // iteration means the restart block B spans a numerically invariant
    // subspace (the Krylov space cannot grow): the previous iteration's Ritz
    // pairs, still in vals, res and B, are converged, and the iterations end.
    s = arnoldi_run(*op, Bb, n, mb, p, sketch, k, seed, Qb, n, Rm, m, o, nullptr);
    if (s == RBGS_EBREAKDOWN && it > 0) break;
    if (s) return s;
    // steps 2-3 on H_(1:p-1,1:p-1) and H_(p,1:p-1)
    RBGS_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
    if ((s = ritz_eig((int)N, (int)mb, (int)mb, which, Rm + mb * m, m, vals, Y, res, scr, status, st))) return s;
    int hs = 0;
    RBGS_CUDA_TRY(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBGS_CUDA_TRY(cudaStreamSynchronize(st));
    if (hs) return RBGS_ENOCONV;
    // step 4: B = Q(:, 0:N) Y on the tall kernel of the basis type
    if (f64) {
      s = tall_update_simt<double>(n, c, mb, (const double*)Qb, n, (const double*)Qb + c * n, n, Y, N, (double*)Bb, n,
                                   nullptr, st);
    } else {
      if ((s = cast_cols_t<double, float>(N, mb, Y, N, (float*)Yt, N, st))) return s;
      s = tall_update_simt<float>(n, c, mb, (const float*)Qb, n, (const float*)Qb + c * n, n, (const float*)Yt, N,
                                  (float*)Bb, n, nullptr, st);
    }
    if (s) return s;
  }
  // step 5: X = B with unit columns
  if (f64) s = cast_cols_t<double, double>(n, mb, (const double*)Bb, n, X, ldx, st);
  else s = cast_cols_t<float, double>(n, mb, (const float*)Bb, n, X, ldx, st);
  if (s) return s;
  if ((s = colnorms_t(n, mb, X, ldx, part, norms, st))) return s;
  if ((s = scale_cols(n, mb, norms, X, ldx, st))) return s;
  std::vector<double> hv(2 * (size_t)mb);
  RBGS_CUDA_TRY(cudaMemcpyAsync(hv.data(), vals, 16 * (size_t)mb, cudaMemcpyDeviceToHost, st));
  RBGS_CUDA_TRY(cudaMemcpyAsync(resid_est, res, 8 * (size_t)mb, cudaMemcpyDeviceToHost, st));
  RBGS_CUDA_TRY(cudaStreamSynchronize(st));
  for (int64_t j = 0; j < mb; ++j) {
    ritz_re[j] = hv[2 * (size_t)j];
    ritz_im[j] = hv[2 * (size_t)j + 1];
  }
  return RBGS_OK;
}

}  // namespace

rbgs_status rbgs_op_apply(const rbgs_op* op, int32_t prec, const void* X, int64_t ldx, int64_t ncols, void* Y,
                          int64_t ldy, void* stream, int32_t sync) {
  rbgs_status s;
  if ((s = check_op(op))) return s;
  const int64_t n = op->nx * op->ny;
  if (!X || !Y || ncols < 0 || ldx < n || ldy < n) return RBGS_EINVAL;
  if (prec < RBGS_P_FP64 || prec > RBGS_P_F16X3) return RBGS_EINVAL;
  const size_t es = prec == RBGS_P_FP64 ? 8 : 4;
  if (ncols > 0 && ranges_overlap(X, es * (size_t)(ldx * (ncols - 1) + n), Y, es * (size_t)(ldy * (ncols - 1) + n)))
    return RBGS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == RBGS_P_FP64) s = stencil_apply_t<double, double>(*op, (const double*)X, ldx, ncols, (double*)Y, ldy, st);
  else s = stencil_apply_t<float, float>(*op, (const float*)X, ldx, ncols, (float*)Y, ldy, st);
  if (s) return s;
  if (sync) RBGS_CUDA_TRY(cudaStreamSynchronize(st));
  return RBGS_OK;
}

rbgs_status rbgs_diffusion_faces(int64_t nx, int64_t ny, const double* a, double* coef, void* stream, int32_t sync) {
  if (!a || !coef || nx < 1 || ny < 1 || (nx + 2) * (ny + 2) >= ((int64_t)1 << 31)) return RBGS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  rbgs_status s = diffusion_faces(nx, ny, a, coef, st);
  if (s) return s;
  if (sync) RBGS_CUDA_TRY(cudaStreamSynchronize(st));
  return RBGS_OK;
}

rbgs_status rbgs_block_arnoldi(const rbgs_op* op, const void* B, int64_t ldb, int64_t mb, int64_t p,
                               rbgs_sketch sketch, int64_t k, uint64_t seed, void* Q, int64_t ldq, double* R,
                               int64_t ldr, const rbgs_opts* opts, rbgs_stats* stats) {
  rbgs_status s;
  if ((s = check_op(op))) return s;
  rbgs_opts o;
  if (opts) o = *opts;
  else rbgs_opts_default(&o);
  const int64_t n = op->nx * op->ny, m = p * mb;
  if (!B || !Q || !R || mb < 1 || mb > 64 || p < 1 || ldb < n || ldq < n || ldr < m) return RBGS_EINVAL;
  if ((s = check_sketch(sketch, n, k, m))) return s;
  if (o.prec < RBGS_P_FP64 || o.prec > RBGS_P_F16X3 || o.reorth < 0 || o.reorth > 2 || o.fine < 0 || o.fine > 2 ||
      (o.interblock != 0 && o.interblock != 4 && o.interblock != 5) || (o.ls != 0 && o.ls != 1) ||
      (o.trsm != 0 && (o.trsm != 1 || o.interblock != 4)))
    return RBGS_EINVAL;
  const size_t es = o.prec == RBGS_P_FP64 ? 8 : 4;
  if (o.prec >= RBGS_P_TF32X3 && (((uintptr_t)B & 15) || ((uintptr_t)Q & 15) || (ldb % 4) || (ldq % 4)))
    return RBGS_EINVAL;
  if (ranges_overlap(R, 8 * (size_t)(ldr * (m - 1) + m), Q, es * (size_t)(ldq * (m - 1) + n))) return RBGS_EINVAL;
  // B may be the first block of Q itself (it is read before Q_1 is written)
  if (B != Q && ranges_overlap(B, es * (size_t)(ldb * (mb - 1) + n), Q, es * (size_t)(ldq * (m - 1) + n)))
    return RBGS_EINVAL;
  return arnoldi_run(*op, B, ldb, mb, p, sketch, k, seed, Q, ldq, R, ldr, o, stats);
}

rbgs_status rbgs_block_gmres(const rbgs_op* op, const double* B, int64_t ldb, double* X, int64_t ldx, int64_t mb,
                             int64_t p, double rtol, int64_t max_cycles, rbgs_sketch sketch, int64_t k,
                             uint64_t seed, const rbgs_opts* opts, int64_t* cycles, double* relres) {
  return krylov_solve(0, op, B, ldb, X, ldx, mb, p, rtol, max_cycles, sketch, k, seed, opts, cycles, relres);
}

rbgs_status rbgs_block_fgmres(const rbgs_op* op, const rbgs_unet* net, const float* params, const double* B,
                              int64_t ldb, double* X, int64_t ldx, int64_t mb, int64_t p, double rtol,
                              int64_t max_cycles, double accept, rbgs_sketch sketch, int64_t k, uint64_t seed,
                              const rbgs_opts* opts, int64_t* cycles, double* relres, int64_t* fallbacks) {
  return fgmres_solve(op, net, params, B, ldb, X, ldx, mb, p, rtol, max_cycles, accept, sketch, k, seed, opts, cycles,
                      relres, fallbacks);
}

rbgs_status rbgs_block_fom(const rbgs_op* op, const double* B, int64_t ldb, double* X, int64_t ldx, int64_t mb,
                           int64_t p, double rtol, int64_t max_cycles, rbgs_sketch sketch, int64_t k, uint64_t seed,
                           const rbgs_opts* opts, int64_t* cycles, double* relres) {
  return krylov_solve(1, op, B, ldb, X, ldx, mb, p, rtol, max_cycles, sketch, k, seed, opts, cycles, relres);
}

rbgs_status rbgs_rayleigh_ritz(const rbgs_op* op, const double* B0, int64_t ldb, int64_t mb, int64_t p,
                               int64_t n_iter, int32_t which, rbgs_sketch sketch, int64_t k, uint64_t seed,
                               const rbgs_opts* opts, double* X, int64_t ldx, double* ritz_re, double* ritz_im,
                               double* resid_est) {
  return rayleigh_ritz(op, B0, ldb, mb, p, n_iter, which, sketch, k, seed, opts, X, ldx, ritz_re, ritz_im,
                       resid_est);
}
