// rbgs_tall_update_noalloc: the tall update of rbgs_tall_update with its
// scratch taken from a fixed array that the library itself holds on each
// device, instead of from the cudaMalloc-grown workspace.
//
// Who needs it: a caller whose device memory is all handed out by its own
// allocator (a framework pool that reserves most of HBM at start-up) cannot
// let a library call cudaMalloc behind its back, and a caller on a latency
// path cannot afford cudaMalloc/cudaFree, which may synchronise the device.
// This entry point calls neither, nor any other allocating routine.
//
// Scratch: one file-scope __device__ array of kNoallocBytes (about 4.03 MiB),
// present on every device that loads this library until the process exits.
// It holds
//   [0, 256)    int error flag of the tensor-core kernel (cleared by every call;
//               read back only with sync != 0, so with sync == 0 a timeout of
//               the bounded device waits is not reported);
//   [256, ...)  the FP32 copy of G (FP32 path) or its TF32 hi/lo split in the
//               tensor-core operand layout (TF32X3 path); every entry that a
//               kernel reads, padding included, is rewritten by each call.
// All calls on a device share the array and it keeps the last call's contents,
// so calls whose GPU work overlaps (different streams without ordering between
// them, or different host threads at once) race on it and give wrong results.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int64_t kNoallocMaxK = RBGS_NOALLOC_MAX_K;
constexpr int kNoallocFlagBytes = 256;
// The larger of the two G copies at K = kNoallocMaxK: the TF32 split needs
// (ceil(K/32) + 2) chunks of 2 x 64 x 32 floats; the FP32 copy K x 64 floats.
constexpr size_t kNoallocSplitFloats = (size_t)((kNoallocMaxK + 31) / 32 + 2) * 2 * 64 * 32;
constexpr size_t kNoallocBytes = kNoallocFlagBytes + 4 * kNoallocSplitFloats;
static_assert(kNoallocSplitFloats >= (size_t)kNoallocMaxK * 64, "FP32 copy of G must fit too");

constexpr int kNoallocMaxDevices = 64;

}  // namespace

// In host code this name is only a host-side stand-in for the symbol; kernels
// get the device address that noalloc_scratch() looks up.
static __device__ __align__(256) unsigned char rbgs_noalloc_scratch[kNoallocBytes];

namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoallocMaxDevices] = {};

// Device address of the scratch array on the current device.  Looked up once
// per device (the first call there), with that device current.
rbgs_status noalloc_scratch(void** out) {
  int dev = -1;
  RBGS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoallocMaxDevices) return RBGS_ENODEV;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, rbgs_noalloc_scratch);
    if (e != cudaSuccess || !p) return RBGS_ECUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return RBGS_OK;
}

// Gf (K x mb, ld K) = float(G).
__global__ void noalloc_g_to_f32(int64_t K, int64_t mb, const double* __restrict__ G, int64_t ldg,
                                 float* __restrict__ Gf) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= K * mb) return;
  const int64_t i = idx % K, j = idx / K;
  Gf[i + j * K] = (float)G[i + j * ldg];
}

}  // namespace

namespace rbgs {
// Forgets the looked-up address of the scratch array on device dev, so that
// the next call looks it up again.  rbgs_release_workspace calls this: after
// cudaDeviceReset the old context's address is stale.
void noalloc_forget_device(int dev) {
  if (dev < 0 || dev >= kNoallocMaxDevices) return;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  g_noalloc_ptr[dev] = nullptr;
}
}  // namespace rbgs

using namespace rbgs;

extern "C" rbgs_status rbgs_tall_update_noalloc(int32_t prec, int64_t n, int64_t c, int64_t mb, const void* Qprev,
                                                int64_t ldq, const void* X, int64_t ldx, const double* G, int64_t ldg,
                                                void* Qout, int64_t ldo, void* stream, int32_t sync) {
  if (!X || !G || !Qout || (c > 0 && !Qprev)) return RBGS_EINVAL;
  if (n < 1 || c < 0 || mb < 1 || mb > 64 || ldx < n || ldo < n || (c > 0 && ldq < n) || ldg < c + mb)
    return RBGS_EINVAL;
  if (prec < RBGS_P_FP64 || prec > RBGS_P_TF32X3) return RBGS_EINVAL;
  const int64_t K = c + mb;
  if (K > kNoallocMaxK) return RBGS_ETOOLARGE;
  if (prec == RBGS_P_TF32X3 &&
      (((uintptr_t)X & 15) || ((uintptr_t)Qout & 15) || (c > 0 && ((uintptr_t)Qprev & 15)) || (ldx % 4) ||
       (ldo % 4) || (c > 0 && (ldq % 4))))
    return RBGS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  rbgs_status s;
  if (prec == RBGS_P_FP64) {  // no scratch needed: G is used as given
    s = tall_update_simt<double>(n, c, mb, (const double*)Qprev, ldq, (const double*)X, ldx, G, ldg, (double*)Qout,
                                 ldo, nullptr, st);
    if (s) return s;
    if (sync) RBGS_CUDA_TRY(cudaStreamSynchronize(st));
    return RBGS_OK;
  }
  void* base = nullptr;
  if ((s = noalloc_scratch(&base))) return s;
  int* err = (int*)base;
  float* Gbuf = (float*)((char*)base + kNoallocFlagBytes);
  if (prec == RBGS_P_FP32) {
    const int64_t tot = K * mb;
    noalloc_g_to_f32<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(K, mb, G, ldg, Gbuf);
    RBGS_LAUNCH_CHECK();
    s = tall_update_simt<float>(n, c, mb, (const float*)Qprev, ldq, (const float*)X, ldx, Gbuf, K, (float*)Qout,
                                ldo, nullptr, st);
    if (s) return s;
    if (sync) RBGS_CUDA_TRY(cudaStreamSynchronize(st));
    return RBGS_OK;
  }
  if ((size_t)kNoallocFlagBytes + 4 * tc_gsplit_floats(K) > kNoallocBytes) return RBGS_ETOOLARGE;
  RBGS_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));  // the flag must start at zero
  if ((s = tc_split_g(K, mb, G, ldg, Gbuf, nullptr, st))) return s;
  s = tall_update_tc(n, c, mb, (const float*)Qprev, ldq, (const float*)X, ldx, Gbuf, (float*)Qout, ldo, nullptr, err,
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
