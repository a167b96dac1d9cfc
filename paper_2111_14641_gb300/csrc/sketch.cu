// Sketching kernels: Y = Theta X without materialising Theta (Sec. 2.3).
//
// SRHT, Theta = k^{-1/2} Samp H D with zero padding to n' = 2^ceil(log2 n):
// with the tile length B | n', H_{n'} = H_{n'/B} (x) H_B, so a sampled row
// i = i_hi B + i_lo of H D x is  sum_t (-1)^{popcount(i_hi & t)} [H_B (D x)_t]_{i_lo}.
// Stage 1 (one CTA per tile t and column): load B entries of the column,
// apply D, transform in shared memory with radix-32 register butterflies,
// keep the entries at the distinct sampled low indices.  Stage 2: for each
// sampled row, the signed sum over tiles.  Both stages are deterministic.
//
// Gaussian / Rademacher: a CTA owns 64 rows of Theta and a slice of the n
// rows of X, regenerates its Theta tile from Philox in shared memory and
// accumulates Theta_tile * X_tile; slice partials are summed in fixed order.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <unordered_set>
#include <vector>

#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace rbgs {

// ------------------------------------------------------------------ SRHT ---

int srht_samples_host(uint64_t seed, int64_t np, int64_t k, int64_t* out) {
  if (k < 0 || k > np) return -1;
  std::unordered_set<int64_t> chosen;
  chosen.reserve((size_t)k * 2 + 1);
  const uint2 key = seed_key(seed);
  for (int64_t t = 0; t < k; ++t) {
    const int64_t J = np - k + t;
    const uint4 x = philox10(make_uint4((uint32_t)t, 0u, kPurposeSrhtSample, 0u), key);
    const uint64_t r64 = ((uint64_t)x.y << 32) | (uint64_t)x.x;
    const int64_t v = (int64_t)(r64 % (uint64_t)(J + 1));
    const int64_t pick = chosen.count(v) ? J : v;
    chosen.insert(pick);
    out[t] = pick;
  }
  std::sort(out, out + k);
  return 0;
}

namespace {
struct PlanCache {
  std::mutex mu;
  std::vector<std::pair<int, SrhtPlan*>> plans;  // (device, plan)
};
PlanCache& plan_cache() {
  static PlanCache c;
  return c;
}
}  // namespace

rbgs_status srht_plan_get(uint64_t seed, int64_t n, int64_t k, const SrhtPlan** out) {
  int dev = 0;
  RBGS_CUDA_TRY(cudaGetDevice(&dev));
  PlanCache& pc = plan_cache();
  std::lock_guard<std::mutex> lock(pc.mu);
  for (auto& e : pc.plans)
    if (e.first == dev && e.second->seed == seed && e.second->n == n && e.second->k == k) {
      *out = e.second;
      return RBGS_OK;
    }
  SrhtPlan* p = new SrhtPlan();
  p->seed = seed;
  p->n = n;
  p->k = k;
  int64_t np = 1;
  while (np < n) np <<= 1;
  p->np = np;
  p->B = (int)std::min<int64_t>(np, kSrhtTile);
  p->T = (int)(np / p->B);
  p->samples.resize((size_t)k);
  if (srht_samples_host(seed, np, k, p->samples.data())) {
    delete p;
    return RBGS_EINVAL;
  }
  std::vector<int> lo((size_t)k), rhi((size_t)k), rl((size_t)k);
  for (int64_t r = 0; r < k; ++r) {
    lo[r] = (int)(p->samples[r] % p->B);
    rhi[r] = (int)(p->samples[r] / p->B);
  }
  std::vector<int> lv(lo);
  std::sort(lv.begin(), lv.end());
  lv.erase(std::unique(lv.begin(), lv.end()), lv.end());
  for (int64_t r = 0; r < k; ++r) rl[r] = (int)(std::lower_bound(lv.begin(), lv.end(), lo[r]) - lv.begin());
  p->L = (int)lv.size();
  std::vector<int> off((size_t)p->L + 1, 0), rs((size_t)k);
  for (int64_t r = 0; r < k; ++r) off[(size_t)rl[r] + 1] += 1;
  for (int l = 0; l < p->L; ++l) off[(size_t)l + 1] += off[(size_t)l];
  {
    std::vector<int> fill(off.begin(), off.end() - 1);
    for (int64_t r = 0; r < k; ++r) rs[(size_t)fill[(size_t)rl[r]]++] = (int)r;
  }
  auto release = [&]() {
    cudaFree(p->d_lvals);
    cudaFree(p->d_rhi);
    cudaFree(p->d_rl);
    cudaFree(p->d_off);
    cudaFree(p->d_rs);
    delete p;
  };
  cudaError_t e1 = cudaMalloc(&p->d_lvals, sizeof(int) * std::max<size_t>(1, lv.size()));
  cudaError_t e2 = cudaMalloc(&p->d_rhi, sizeof(int) * std::max<int64_t>(1, k));
  cudaError_t e3 = cudaMalloc(&p->d_rl, sizeof(int) * std::max<int64_t>(1, k));
  cudaError_t e4 = cudaMalloc(&p->d_off, sizeof(int) * off.size());
  cudaError_t e5 = cudaMalloc(&p->d_rs, sizeof(int) * std::max<int64_t>(1, k));
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess || e5 != cudaSuccess) {
    release();
    return RBGS_ENOMEM;
  }
  if (cudaMemcpy(p->d_lvals, lv.data(), sizeof(int) * lv.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p->d_rhi, rhi.data(), sizeof(int) * k, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p->d_rl, rl.data(), sizeof(int) * k, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p->d_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p->d_rs, rs.data(), sizeof(int) * k, cudaMemcpyHostToDevice) != cudaSuccess) {
    release();
    return RBGS_ECUDA;
  }
  pc.plans.push_back({dev, p});
  *out = p;
  return RBGS_OK;
}

void srht_plans_release() {
  PlanCache& pc = plan_cache();
  std::lock_guard<std::mutex> lock(pc.mu);
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<std::pair<int, SrhtPlan*>> keep;
  for (auto& e : pc.plans) {
    if (e.first == dev) {
      cudaFree(e.second->d_lvals);
      cudaFree(e.second->d_rhi);
      cudaFree(e.second->d_rl);
      cudaFree(e.second->d_off);
      cudaFree(e.second->d_rs);
      delete e.second;
    } else {
      keep.push_back(e);
    }
  }
  pc.plans.swap(keep);
}

namespace {

constexpr int kSrhtThreads = 512;

__device__ __forceinline__ int swz(int j) { return j ^ ((j >> 5) & 31); }

template <class TC, int R>
__device__ __forceinline__ void fwht_stage(TC* buf, int B, int lo) {
  constexpr int G = 1 << R;
  const int ngroups = B >> R;
  const int lomask = (1 << lo) - 1;
  for (int g = threadIdx.x; g < ngroups; g += blockDim.x) {
    const int base = ((g >> lo) << (lo + R)) | (g & lomask);
    TC v[G];
#pragma unroll
    for (int e = 0; e < G; ++e) v[e] = buf[swz(base + (e << lo))];
#pragma unroll
    for (int h = 1; h < G; h <<= 1) {
#pragma unroll
      for (int e = 0; e < G; ++e) {
        if ((e & h) == 0) {
          const TC a = v[e], b = v[e + h];
          v[e] = a + b;
          v[e + h] = a - b;
        }
      }
    }
#pragma unroll
    for (int e = 0; e < G; ++e) buf[swz(base + (e << lo))] = v[e];
  }
}

// Stage 1: grid (T, ncols).  z[(col * T + t) * L + l] = [H_B (D x)_t]_{lvals[l]}.
// Thread t holds the E = B / 512 entries j = t + 512 e: their loads are all in
// flight together, the transform over the top log2(E) index bits runs in
// registers, the remaining 9 bits in two shared-memory stages.
template <class TX, class TC, int E>
__global__ void __launch_bounds__(kSrhtThreads) srht_stage1(const TX* __restrict__ X, int64_t ldx, int64_t n, int B,
                                                            int logB, int T, uint2 key,
                                                            const int* __restrict__ lvals, int L,
                                                            TC* __restrict__ z, const int* active) {
  if (active && *active == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC* buf = reinterpret_cast<TC*>(smem_raw);
  uint32_t* sgn = reinterpret_cast<uint32_t*>(buf + B);
  const int t = blockIdx.x;
  const int col = blockIdx.y;
  const int tid = threadIdx.x;
  const int64_t row0 = (int64_t)t * B;
  const TX* xc = X + (int64_t)col * ldx;
  TC v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int j = tid + kSrhtThreads * e;
    const int64_t gr = row0 + j;
    v[e] = (j < B && gr < n) ? (TC)__ldg(xc + gr) : (TC)0;
  }
  const int nwords = (B + 31) >> 5;
  for (int w = tid; w < nwords; w += blockDim.x) {
    const int64_t e0 = row0 + 32 * (int64_t)w;
    const uint4 bits = srht_sign_bits(key, (uint32_t)(e0 >> 7));
    sgn[w] = word_of(bits, (int)((e0 >> 5) & 3));
  }
  __syncthreads();
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int j = tid + kSrhtThreads * e;
    if (j < B && ((sgn[j >> 5] >> (j & 31)) & 1u)) v[e] = -v[e];
  }
  // index bits 9 .. logB-1 live in e
#pragma unroll
  for (int h = 1; h < E; h <<= 1) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if ((e & h) == 0) {
        const TC a = v[e], b = v[e + h];
        v[e] = a + b;
        v[e + h] = a - b;
      }
    }
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int j = tid + kSrhtThreads * e;
    if (j < B) buf[swz(j)] = v[e];
  }
  const int lowbits = logB < 9 ? logB : 9;
  for (int lo = 0; lo < lowbits; lo += 5) {
    __syncthreads();
    const int r = min(5, lowbits - lo);
    switch (r) {
      case 5: fwht_stage<TC, 5>(buf, B, lo); break;
      case 4: fwht_stage<TC, 4>(buf, B, lo); break;
      case 3: fwht_stage<TC, 3>(buf, B, lo); break;
      case 2: fwht_stage<TC, 2>(buf, B, lo); break;
      default: fwht_stage<TC, 1>(buf, B, lo); break;
    }
  }
  __syncthreads();
  TC* zo = z + ((int64_t)col * T + t) * L;
  for (int l = tid; l < L; l += blockDim.x) zo[l] = buf[swz(lvals[l])];
}

template <class TX, class TC>
rbgs_status launch_stage1(dim3 grid, size_t smem, cudaStream_t st, const TX* X, int64_t ldx, int64_t n, int B,
                          int logB, int T, uint2 key, const int* lvals, int L, TC* z, const int* active) {
  const int E = B >= kSrhtThreads ? B / kSrhtThreads : 1;
  auto go = [&](auto kern) -> rbgs_status {
    RBGS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(TC) * kSrhtTile + 4 * kSrhtTile / 32)));
    kern<<<grid, kSrhtThreads, smem, st>>>(X, ldx, n, B, logB, T, key, lvals, L, z, active);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
  };
  switch (E) {
    case 1: return go(srht_stage1<TX, TC, 1>);
    case 2: return go(srht_stage1<TX, TC, 2>);
    case 4: return go(srht_stage1<TX, TC, 4>);
    case 8: return go(srht_stage1<TX, TC, 8>);
    case 16: return go(srht_stage1<TX, TC, 16>);
    case 32: return go(srht_stage1<TX, TC, 32>);
    default: return RBGS_EINVAL;
  }
}

// Stage 2: Y[r, col] = scale * sum_t (-1)^{popcount(rhi[r] & t)} z[col, t, rl[r]].
template <class TC, class TY>
__global__ void srht_stage2(const TC* __restrict__ z, int T, int L, const int* __restrict__ rhi,
                            const int* __restrict__ rl, int64_t k, int64_t ncols, TC scale, TY* __restrict__ Y,
                            int64_t ldy, const int* active) {
  if (active && *active == 0) return;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= k * ncols) return;
  const int64_t r = idx % k;
  const int64_t col = idx / k;
  const TC* zc = z + (int64_t)col * T * L + rl[r];
  const int hi = rhi[r];
  TC acc = 0;
  for (int t = 0; t < T; ++t) {
    const TC v = zc[(int64_t)t * L];
    acc += (__popc(hi & t) & 1) ? -v : v;
  }
  Y[r + col * ldy] = (TY)(acc * scale);
}

// Persistent, double-buffered form of stage 1 for float data (all columns of
// up to two sources): one CTA per SM walks the (column, tile) items; a bulk
// asynchronous copy brings the next tile into the second buffer while the
// current one is transformed in place.  The waits on the copies are bounded.
struct SrhtSrc {
  const float* x[2];
  int64_t ld[2];
  int64_t nc0;  // columns of source 0; the rest come from source 1
};

__device__ __forceinline__ uint32_t sk_smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool sk_mbar_wait(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > 4000000000ull) return false;
  }
}

// NB = 2: one CTA per SM prefetches the next tile into its second buffer
// while transforming the current one.  NB = 1: two CTAs per SM with one
// buffer each; the co-resident CTA computes while the other one loads.
template <int E, int NB>
__global__ void __launch_bounds__(kSrhtThreads, NB == 1 ? 2 : 1)
    srht_stage1_persist(SrhtSrc src, int64_t n, int B, int logB, int T, uint2 key, const int* __restrict__ lvals,
                        int L, float* __restrict__ z, int64_t ncols, const int* active, int* err) {
  static_assert(NB == 1 || NB == 2, "buffers");
  if (active && *active == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* bufs = reinterpret_cast<float*>(smem_raw);            // NB x B
  uint32_t* sgn = reinterpret_cast<uint32_t*>(bufs + NB * B);  // B / 32
  __shared__ __align__(8) uint64_t full[2];
  __shared__ int bad;
  const int tid = threadIdx.x;
  const int64_t nitems = ncols * T;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sk_smem_u32(&full[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sk_smem_u32(&full[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    bad = 0;
  }
  __syncthreads();
  // item -> (column, tile, source pointer, valid rows, bulk-copy bytes)
  auto item = [&](int64_t w, const float*& p, int64_t& row0, int& valid, uint32_t& bytes) {
    const int64_t col = w / T;
    const int t = (int)(w % T);
    const bool second = col >= src.nc0;
    const int64_t lc = second ? col - src.nc0 : col;
    row0 = (int64_t)t * B;
    // (a select, not src.x[index]: a runtime index would copy the parameter to local memory)
    p = (second ? src.x[1] : src.x[0]) + lc * (second ? src.ld[1] : src.ld[0]) + row0;
    const int64_t v = n - row0;
    valid = v <= 0 ? 0 : (int)(v < B ? v : B);
    bytes = ((((uintptr_t)p) & 15) == 0) ? (uint32_t)((valid * 4) & ~15) : 0u;
  };
  auto issue = [&](int64_t w, int b) {
    const float* p;
    int64_t row0;
    int valid;
    uint32_t bytes;
    item(w, p, row0, valid, bytes);
    const uint32_t bar = sk_smem_u32(&full[b]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    if (bytes)
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       sk_smem_u32(bufs + (size_t)b * B)),
                   "l"(p), "r"(bytes), "r"(bar)
                   : "memory");
  };
  // copies issued into / consumed from each buffer; a buffer with issued >
  // consumed has a copy in flight whose phase parity is (issued - 1) & 1
  int issued[2] = {0, 0}, consumed[2] = {0, 0};
  int64_t w = blockIdx.x;
  if (w < nitems) {
    if (tid == 0) issue(w, 0);
    issued[0] = 1;
  }
  for (int idx = 0; w < nitems; w += gridDim.x, ++idx) {
    const int b = NB == 2 ? (idx & 1) : 0;
    const int64_t wn = w + gridDim.x;
    if (NB == 2 && wn < nitems) {  // buffer b^1 was released at the end of the previous item
      if (tid == 0) issue(wn, b ^ 1);
      issued[b ^ 1] += 1;
    }
    const float* p;
    int64_t row0;
    int valid;
    uint32_t bytes;
    item(w, p, row0, valid, bytes);
    // sign words of this tile
    const int nwords = (B + 31) >> 5;
    for (int q = tid; q < nwords; q += blockDim.x) {
      const int64_t e0 = row0 + 32 * (int64_t)q;
      const uint4 bits = srht_sign_bits(key, (uint32_t)(e0 >> 7));
      sgn[q] = word_of(bits, (int)((e0 >> 5) & 3));
    }
    if (!sk_mbar_wait(sk_smem_u32(&full[b]), (uint32_t)(consumed[b] & 1))) bad = 1;
    consumed[b] += 1;
    __syncthreads();
    if (bad) {
      consumed[b] -= 1;  // that copy may still be in flight
      break;
    }
    float* buf = bufs + (size_t)b * B;
    const int done = (int)(bytes / 4);  // entries that arrived by the bulk copy
    float v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int j = tid + kSrhtThreads * e;
      float x = 0.f;
      if (j < done) x = buf[j];
      else if (j < valid) x = __ldg(p + j);
      if (j < B && ((sgn[j >> 5] >> (j & 31)) & 1u)) x = -x;
      v[e] = x;
    }
#pragma unroll
    for (int h = 1; h < E; h <<= 1) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        if ((e & h) == 0) {
          const float a = v[e], c = v[e + h];
          v[e] = a + c;
          v[e + h] = a - c;
        }
      }
    }
    __syncthreads();  // all reads of the raw layout done before the in-place permutation
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int j = tid + kSrhtThreads * e;
      if (j < B) buf[swz(j)] = v[e];
    }
    const int lowbits = logB < 9 ? logB : 9;
    for (int lo = 0; lo < lowbits; lo += 5) {
      __syncthreads();
      const int r = min(5, lowbits - lo);
      switch (r) {
        case 5: fwht_stage<float, 5>(buf, B, lo); break;
        case 4: fwht_stage<float, 4>(buf, B, lo); break;
        case 3: fwht_stage<float, 3>(buf, B, lo); break;
        case 2: fwht_stage<float, 2>(buf, B, lo); break;
        default: fwht_stage<float, 1>(buf, B, lo); break;
      }
    }
    __syncthreads();
    float* zo = z + w * L;  // (col * T + t) * L
    for (int l = tid; l < L; l += blockDim.x) zo[l] = buf[swz(lvals[l])];
    __syncthreads();  // buffer b may be refilled from the next iteration on
    if (NB == 1 && wn < nitems) {
      if (tid == 0) issue(wn, 0);
      issued[0] += 1;
    }
  }
  // leave no copy in flight into shared memory
  if (tid == 0) {
    for (int b = 0; b < 2; ++b)
      if (issued[b] > consumed[b] && !sk_mbar_wait(sk_smem_u32(&full[b]), (uint32_t)((issued[b] - 1) & 1))) bad = 1;
    if (bad && err) atomicExch(err, 1);
  }
  __syncthreads();
}

// Stage 1 for tiles of B = 16384 entries (every n' >= 2^14), with all indices
// known at compile time.  Entry j of a tile has 14 bits; thread t holds 32
// entries as 8 float4 and the transform runs in four register passes:
//   A: bits 0, 1 (inside a float4) and 11..13, read from the raw tile
//      (j = 4 t + 2048 q + c), with the signs of D applied on the way;
//   B: bits 2..4;  C: bits 5..7;  D: bits 8..10.
// Between the passes the tile sits in shared memory with float4 slot bits
// 0..2 xor-ed by bits 3..5 (entry bits 2..4 by 5..7), which keeps every pass's
// 16-byte accesses free of bank conflicts.  Butterflies over float4 halves use
// the packed FP32 add.
constexpr int kB16 = 16384;
constexpr int kB16Staged = 4096;  // up to this many sampled low indices are staged in shared memory

__device__ __forceinline__ int b16_phys(int j) { return j ^ (((j >> 5) & 7) << 2); }

__device__ __forceinline__ void b16_bfly(float& a0, float& a1, float& b0, float& b1) {
  const float2 a = make_float2(a0, a1), b = make_float2(b0, b1);
  const float2 s = __fadd2_rn(a, b);
  const float2 d = __ffma2_rn(b, make_float2(-1.f, -1.f), a);  // a - b in one packed instruction
  a0 = s.x;
  a1 = s.y;
  b0 = d.x;
  b1 = d.y;
}

// the three levels over the index q of v[q]
__device__ __forceinline__ void b16_levels_q(float4 (&v)[8]) {
#pragma unroll
  for (int h = 1; h < 8; h <<= 1) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if ((q & h) == 0) {
        b16_bfly(v[q].x, v[q].y, v[q + h].x, v[q + h].y);
        b16_bfly(v[q].z, v[q].w, v[q + h].z, v[q + h].w);
      }
    }
  }
}

// the two levels inside each float4 (entry bits 0 and 1)
__device__ __forceinline__ void b16_levels_in(float4 (&v)[8]) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    b16_bfly(v[q].x, v[q].y, v[q].z, v[q].w);  // bit 1
    const float x = v[q].x, y = v[q].y, z = v[q].z, w = v[q].w;
    v[q] = make_float4(x + y, x - y, z + w, z - w);  // bit 0
  }
}

__device__ __forceinline__ float b16_sign(float x, uint32_t bit_at_31) {
  return __int_as_float(__float_as_int(x) ^ (int)(bit_at_31 & 0x80000000u));
}

template <int NB>
__global__ void __launch_bounds__(kSrhtThreads, NB == 1 ? 2 : 1)
    srht_stage1_b16k(SrhtSrc src, int64_t n, int T, uint2 key, const int* __restrict__ lvals, int L,
                     float* __restrict__ z, int64_t ncols, const int* active, int* err) {
  static_assert(NB == 1 || NB == 2, "buffers");
  static_assert(kSrhtThreads == 512, "the passes assume 512 threads x 32 entries");
  constexpr int B = kB16;
  if (active && *active == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* bufs = reinterpret_cast<float*>(smem_raw);            // NB x B
  uint32_t* sgn = reinterpret_cast<uint32_t*>(bufs + NB * B);  // B / 32
  int* lv_s = reinterpret_cast<int*>(sgn + B / 32);            // the L sampled low indices, when staged
  __shared__ __align__(8) uint64_t full[2];
  __shared__ int bad;
  const int tid = threadIdx.x;
  const int64_t nitems = ncols * T;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sk_smem_u32(&full[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sk_smem_u32(&full[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    bad = 0;
  }
  const bool staged = L <= kB16Staged;  // uniform
  if (staged)
    for (int l = tid; l < L; l += blockDim.x) lv_s[l] = b16_phys(__ldg(lvals + l));
  __syncthreads();
  auto item = [&](int64_t w, const float*& p, int64_t& row0, int& valid, uint32_t& bytes) {
    const int64_t col = w / T;
    const int t = (int)(w % T);
    const bool second = col >= src.nc0;
    const int64_t lc = second ? col - src.nc0 : col;
    row0 = (int64_t)t * B;
    // (a select, not src.x[index]: a runtime index would copy the parameter to local memory)
    p = (second ? src.x[1] : src.x[0]) + lc * (second ? src.ld[1] : src.ld[0]) + row0;
    const int64_t v = n - row0;
    valid = v <= 0 ? 0 : (int)(v < B ? v : B);
    bytes = ((((uintptr_t)p) & 15) == 0) ? (uint32_t)((valid * 4) & ~15) : 0u;
  };
  auto issue = [&](int64_t w, int b) {
    const float* p;
    int64_t row0;
    int valid;
    uint32_t bytes;
    item(w, p, row0, valid, bytes);
    const uint32_t bar = sk_smem_u32(&full[b]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    if (bytes)
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       sk_smem_u32(bufs + (size_t)b * B)),
                   "l"(p), "r"(bytes), "r"(bar)
                   : "memory");
  };
  // copies issued into / consumed from each buffer (scalars: no local memory)
  int iss0 = 0, iss1 = 0, con0 = 0, con1 = 0;
  int64_t w = blockIdx.x;
  if (w < nitems) {
    if (tid == 0) issue(w, 0);
    iss0 = 1;
  }
  // per-thread slot bases (float4 units) of the four passes
  const int t7 = tid & 7, t37 = (tid >> 3) & 7;
  const int slotA = tid ^ t37;                        // + 512 q   (raw slot tid + 512 q)
  const int slotB = 8 * tid;                          // + (q ^ t7)
  const int slotC = 64 * (tid >> 3);                  // + 8 q + (t7 ^ q)
  const int slotD = (t7 ^ t37) + 8 * t37 + 512 * (tid >> 6);  // + 64 q
  for (int idx = 0; w < nitems; w += gridDim.x, ++idx) {
    const int b = NB == 2 ? (idx & 1) : 0;
    const int64_t wn = w + gridDim.x;
    if (NB == 2 && wn < nitems) {
      if (tid == 0) issue(wn, b ^ 1);
      if (b) ++iss0;
      else ++iss1;
    }
    const float* p;
    int64_t row0;
    int valid;
    uint32_t bytes;
    item(w, p, row0, valid, bytes);
    // the signs of D for this tile: one Philox block per 128 rows
    if (tid < B / 128) {
      const uint4 bits = srht_sign_bits(key, (uint32_t)((row0 >> 7) + tid));
      reinterpret_cast<uint4*>(sgn)[tid] = bits;
    }
    if (!sk_mbar_wait(sk_smem_u32(&full[b]), (uint32_t)((b ? con1 : con0) & 1))) bad = 1;
    if (b) ++con1;
    else ++con0;
    __syncthreads();
    if (bad) {
      if (b) --con1;
      else --con0;
      break;
    }
    float* buf = bufs + (size_t)b * B;
    float4* buf4 = reinterpret_cast<float4*>(buf);
    const int done = (int)(bytes / 4);
    float4 v[8];
    // pass A
    if (done == B) {
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = buf4[tid + 512 * q];
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int j = 4 * tid + 2048 * q;
        if (j + 4 <= done) {
          v[q] = buf4[tid + 512 * q];
        } else {
          float e[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) e[c] = (j + c < valid) ? __ldg(p + j + c) : 0.f;
          v[q] = make_float4(e[0], e[1], e[2], e[3]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      // entries 4 tid + 2048 q + c: bits 4 (tid & 7) + c of sign word (tid >> 3) + 64 q
      const uint32_t sw = sgn[(tid >> 3) + 64 * q] >> (4 * t7);
      v[q].x = b16_sign(v[q].x, sw << 31);
      v[q].y = b16_sign(v[q].y, sw << 30);
      v[q].z = b16_sign(v[q].z, sw << 29);
      v[q].w = b16_sign(v[q].w, sw << 28);
    }
    b16_levels_in(v);
    b16_levels_q(v);
    __syncwarp();  // the slots written below were read by lanes of this warp only
#pragma unroll
    for (int q = 0; q < 8; ++q) buf4[slotA + 512 * q] = v[q];
    __syncthreads();
    // pass B: slots 8 tid + (q ^ t7)
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = buf4[slotB + (q ^ t7)];
    b16_levels_q(v);
#pragma unroll
    for (int q = 0; q < 8; ++q) buf4[slotB + (q ^ t7)] = v[q];
    __syncthreads();
    // pass C
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = buf4[slotC + 8 * q + (t7 ^ q)];
    b16_levels_q(v);
#pragma unroll
    for (int q = 0; q < 8; ++q) buf4[slotC + 8 * q + (t7 ^ q)] = v[q];
    __syncthreads();
    // pass D
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = buf4[slotD + 64 * q];
    b16_levels_q(v);
#pragma unroll
    for (int q = 0; q < 8; ++q) buf4[slotD + 64 * q] = v[q];
    __syncthreads();
    float* zo = z + w * L;  // (col * T + t) * L
    if (staged) {
#pragma unroll 4
      for (int l = tid; l < L; l += blockDim.x) zo[l] = buf[lv_s[l]];
    } else {
      for (int l = tid; l < L; l += blockDim.x) zo[l] = buf[b16_phys(__ldg(lvals + l))];
    }
    __syncthreads();  // buffer b may be refilled from here on
    if (NB == 1 && wn < nitems) {
      if (tid == 0) issue(wn, 0);
      ++iss0;
    }
  }
  if (tid == 0) {
    for (int b = 0; b < 2; ++b)
      if ((b ? iss1 : iss0) > (b ? con1 : con0) &&
          !sk_mbar_wait(sk_smem_u32(&full[b]), (uint32_t)(((b ? iss1 : iss0) - 1) & 1)))
        bad = 1;
    if (bad && err) atomicExch(err, 1);
  }
  __syncthreads();
}

// Buffers of the persistent stage 1: 1 (two CTAs per SM, measured faster on
// GB300) or 2 (RBGS_SRHT_BUFFERS=2, one CTA per SM that prefetches).
int srht_buffers() {
  static int v = []() {
    const char* e = getenv("RBGS_SRHT_BUFFERS");
    const int b = e ? atoi(e) : 1;
    return b == 1 ? 1 : 2;
  }();
  return v;
}

// Stage 2 as a transform across tiles: for each column and distinct low
// index l, the T values z[col, :, l] go through the T-point Hadamard
// transform in registers, which yields entry (i_hi, l) of H (D x) for every
// i_hi; the sampled rows with low index l pick theirs.
template <class TC, class TY, int TT>
__global__ void __launch_bounds__(128) srht_stage2_fwht(const TC* __restrict__ z, int L, const int* __restrict__ off,
                                                        const int* __restrict__ rs, const int* __restrict__ rhi,
                                                        int64_t ncols, int64_t nc0, TC scale, TY* __restrict__ Y1,
                                                        int64_t ldy1, TY* __restrict__ Y2, int64_t ldy2,
                                                        const int* active) {
  if (active && *active == 0) return;
  __shared__ TC sv[TT][129];
  const int64_t col = blockIdx.y;
  const int l = blockIdx.x * 128 + threadIdx.x;
  TC v[TT];
#pragma unroll
  for (int t = 0; t < TT; ++t) v[t] = l < L ? z[((int64_t)col * TT + t) * L + l] : (TC)0;
#pragma unroll
  for (int h = 1; h < TT; h <<= 1) {
#pragma unroll
    for (int e = 0; e < TT; ++e) {
      if ((e & h) == 0) {
        const TC a = v[e], b = v[e + h];
        v[e] = a + b;
        v[e + h] = a - b;
      }
    }
  }
#pragma unroll
  for (int t = 0; t < TT; ++t) sv[t][threadIdx.x] = v[t];
  __syncwarp();
  if (l >= L) return;
  TY* Y = col < nc0 ? Y1 + col * ldy1 : Y2 + (col - nc0) * ldy2;
  for (int q = off[l]; q < off[l + 1]; ++q) {
    const int r = rs[q];
    Y[r] = (TY)(sv[rhi[r]][threadIdx.x] * scale);
  }
}

template <class TC, class TY>
rbgs_status launch_stage2_fwht(int T, int L, const SrhtPlan* plan, const TC* z, int64_t ncols, int64_t nc0, TC scale,
                               TY* Y1, int64_t ldy1, TY* Y2, int64_t ldy2, const int* active, cudaStream_t st,
                               bool* done) {
  *done = true;
  dim3 grid((unsigned)((L + 127) / 128), (unsigned)ncols);
  switch (T) {
#define S2(TT)                                                                                                   \
  case TT:                                                                                                       \
    srht_stage2_fwht<TC, TY, TT><<<grid, 128, 0, st>>>(z, L, plan->d_off, plan->d_rs, plan->d_rhi, ncols, nc0,   \
                                                       scale, Y1, ldy1, Y2, ldy2, active);                      \
    break;
    S2(1) S2(2) S2(4) S2(8) S2(16) S2(32) S2(64)
#undef S2
    default:
      *done = false;
      return RBGS_OK;
  }
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}

// ------------------------------------------------------- Gaussian/Rademacher

constexpr int kDenseRows = 64;   // Theta rows per CTA
constexpr int kDenseJ = 32;      // X rows per step
constexpr int kDenseCols = 64;   // max columns per launch
constexpr int kDenseThreads = 256;

template <int KIND, class TX, class TC, int QN>
__global__ void __launch_bounds__(kDenseThreads) dense_sketch_part(const TX* __restrict__ X, int64_t ldx, int64_t n,
                                                                   int ncols, int64_t k, uint2 key, double scale,
                                                                   int64_t rows_per_split, TC* __restrict__ part,
                                                                   const int* active) {
  if (active && *active == 0) return;
  __shared__ TC th[kDenseRows][kDenseJ + 1];
  __shared__ TC xs[kDenseJ][kDenseCols + 1];
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * kDenseRows;
  const int split = blockIdx.y;
  const int64_t j0 = (int64_t)split * rows_per_split;
  const int64_t j1 = min(n, j0 + rows_per_split);
  const int tr = tid & 15, tc = tid >> 4;
  // QN = ceil(ncols / 16): the column groups of 16 that hold columns of X (a
  // block of 16 columns needs a quarter of the products of a full tile)
  static_assert(QN >= 1 && QN <= 4, "column groups");
  TC acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[i][q] = 0;

  for (int64_t jj0 = j0; jj0 < j1; jj0 += kDenseJ) {
    if (KIND == RBGS_SK_GAUSS) {
      // 32 row pairs x 32 columns of Theta, 4 Box-Muller pairs per thread
      for (int p = tid; p < (kDenseRows / 2) * kDenseJ; p += kDenseThreads) {
        const int rpl = p & 31, jl = p >> 5;
        const int64_t j = jj0 + jl;
        const int64_t rr = r0 + 2 * rpl;
        double z0 = 0.0, z1 = 0.0;
        if (j < j1 && rr < k) gauss_pair(key, j, (uint32_t)(rr >> 1), z0, z1);
        th[2 * rpl][jl] = (TC)(z0 * scale);
        th[2 * rpl + 1][jl] = (TC)(z1 * scale);
      }
    } else if (KIND == RBGS_SK_SPARSE) {
      // 64 rows x 32 columns of Theta: each column's z nonzeros, kept where
      // they fall into this CTA's rows
      if (tid < kDenseJ) {
        const int64_t j = jj0 + tid;
        for (int rl = 0; rl < kDenseRows; ++rl) th[rl][tid] = (TC)0;
        if (j < j1) {
          int64_t rows[8];
          bool neg[8];
          const int z = sparse_column(key, j, k, rows, neg);
#pragma unroll
          for (int s = 0; s < 8; ++s) {
            if (s < z) {
              const int64_t rl = rows[s] - r0;
              if (rl >= 0 && rl < kDenseRows) th[rl][tid] = neg[s] ? (TC)(-scale) : (TC)scale;
            }
          }
        }
      }
    } else {
      if (tid < kDenseJ) {
        const int64_t j = jj0 + tid;
        uint4 bits = make_uint4(0, 0, 0, 0);
        if (j < j1) bits = rademacher_bits(key, j, (uint32_t)(r0 >> 7));
        const int off = (int)(r0 & 127);  // 0 or 64
        for (int rl = 0; rl < kDenseRows; ++rl) {
          const int rb = off + rl;
          const uint32_t b = (word_of(bits, rb >> 5) >> (rb & 31)) & 1u;
          th[rl][tid] = (j < j1) ? (TC)(b ? -scale : scale) : (TC)0;
        }
      }
    }
    for (int e = tid; e < kDenseJ * kDenseCols; e += kDenseThreads) {
      const int jl = e % kDenseJ, c = e / kDenseJ;
      const int64_t j = jj0 + jl;
      xs[jl][c] = (c < ncols && j < j1) ? (TC)X[j + (int64_t)c * ldx] : (TC)0;
    }
    __syncthreads();
#pragma unroll 4
    for (int jl = 0; jl < kDenseJ; ++jl) {
      TC a[4], b[QN];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = th[tr + 16 * i][jl];
#pragma unroll
      for (int q = 0; q < QN; ++q) b[q] = xs[jl][tc + 16 * q];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < QN; ++q) acc[i][q] += a[i] * b[q];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < QN; ++q) {
      const int64_t r = r0 + tr + 16 * i;
      const int c = tc + 16 * q;
      if (r < k && c < ncols) part[((int64_t)split * ncols + c) * k + r] = acc[i][q];
    }
}

template <class TC, class TY>
__global__ void dense_sketch_reduce(const TC* __restrict__ part, int nsplit, int64_t k, int ncols,
                                    TY* __restrict__ Y, int64_t ldy, const int* active) {
  if (active && *active == 0) return;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= k * ncols) return;
  const int64_t r = idx % k;
  const int64_t c = idx / k;
  TC s = 0;
  for (int p = 0; p < nsplit; ++p) s += part[((int64_t)p * ncols + c) * k + r];
  Y[r + c * ldy] = (TY)s;
}

int dense_nsplit(int64_t k, int64_t n) {
  const int64_t rblocks = (k + kDenseRows - 1) / kDenseRows;
  int64_t target = std::max<int64_t>(1, 2 * 152 / std::max<int64_t>(1, rblocks));
  const int64_t maxsplit = std::max<int64_t>(1, (n + 255) / 256);
  return (int)std::min<int64_t>(target, maxsplit);
}

}  // namespace

size_t sketch_scratch_bytes(rbgs_sketch kind, int64_t k, int64_t n, int64_t ncols, bool fp64) {
  const size_t es = fp64 ? 8 : 4;
  if (kind == RBGS_SK_SRHT) {
    int64_t np = 1;
    while (np < n) np <<= 1;
    const int64_t B = std::min<int64_t>(np, kSrhtTile);
    const int64_t T = np / B;
    const int64_t L = std::min<int64_t>(B, k);
    return es * (size_t)(ncols * T * L);
  }
  // the dense sketches accumulate in FP64 whenever the sketch space is FP64
  const int64_t c = std::min<int64_t>(ncols, kDenseCols);
  return 8 * (size_t)(dense_nsplit(k, n) * c * k);
}

template <class TX, class TY>
rbgs_status sketch_apply2_t(rbgs_sketch kind, int64_t k, int64_t n, uint64_t seed, const TX* X1, int64_t ldx1,
                            int64_t nc1, TY* Y1, int64_t ldy1, const TX* X2, int64_t ldx2, int64_t nc2, TY* Y2,
                            int64_t ldy2, void* scratch, size_t scratch_bytes, cudaStream_t st, const int* active) {
  using TC = TX;  // arithmetic follows the input precision
  const int64_t ncols = nc1 + nc2;
  if (ncols == 0 || k == 0) return RBGS_OK;
  if (kind != RBGS_SK_SRHT) {
    rbgs_status s = sketch_apply_t<TX, TY>(kind, k, n, seed, X1, ldx1, nc1, Y1, ldy1, scratch, scratch_bytes, st,
                                           active);
    if (s || nc2 == 0) return s;
    return sketch_apply_t<TX, TY>(kind, k, n, seed, X2, ldx2, nc2, Y2, ldy2, scratch, scratch_bytes, st, active);
  }
  const uint2 key = seed_key(seed);
  const double dscale = 1.0 / std::sqrt((double)k);
  const TC scale = (TC)dscale;
  const SrhtPlan* plan = nullptr;
  rbgs_status s = srht_plan_get(seed, n, k, &plan);
  if (s != RBGS_OK) return s;
  const size_t need = sizeof(TC) * (size_t)(ncols * plan->T) * (size_t)plan->L;
  if (scratch_bytes < need) return RBGS_EINVAL;
  TC* z = reinterpret_cast<TC*>(scratch);
  int logB = 0;
  while ((1 << logB) < plan->B) ++logB;
  const int E = plan->B >= kSrhtThreads ? plan->B / kSrhtThreads : 1;
  if (sizeof(TX) == 4) {
    int dev = 0, nsm = 0;
    RBGS_CUDA_TRY(cudaGetDevice(&dev));
    RBGS_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int64_t nitems = ncols * plan->T;
    const int nb = srht_buffers();
    const int grid = (int)std::min<int64_t>(nitems, (int64_t)nsm * (nb == 1 ? 2 : 1));
    const size_t smem = sizeof(float) * nb * (size_t)plan->B + sizeof(uint32_t) * (size_t)((plan->B + 31) / 32);
    SrhtSrc sd;
    sd.x[0] = reinterpret_cast<const float*>(X1);
    sd.x[1] = reinterpret_cast<const float*>(nc2 ? X2 : X1);
    sd.ld[0] = ldx1;
    sd.ld[1] = nc2 ? ldx2 : ldx1;
    sd.nc0 = nc1;
    float* zf = reinterpret_cast<float*>(z);
    auto go = [&](auto kern) -> rbgs_status {
      RBGS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(float) * nb * kSrhtTile + 4 * kSrhtTile / 32)));
      kern<<<grid, kSrhtThreads, smem, st>>>(sd, n, plan->B, logB, plan->T, key, plan->d_lvals, plan->L, zf, ncols,
                                             active, nullptr);
      RBGS_LAUNCH_CHECK();
      return RBGS_OK;
    };
    if (plan->B == kB16) {
      auto k16 = nb == 1 ? srht_stage1_b16k<1> : srht_stage1_b16k<2>;
      const size_t smem16 = smem + (plan->L <= kB16Staged ? sizeof(int) * (size_t)plan->L : 0);
      RBGS_CUDA_TRY(cudaFuncSetAttribute(k16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem16));
      k16<<<grid, kSrhtThreads, smem16, st>>>(sd, n, plan->T, key, plan->d_lvals, plan->L, zf, ncols, active,
                                              nullptr);
      RBGS_LAUNCH_CHECK();
      s = RBGS_OK;
    } else if (nb == 1) {
      switch (E) {
        case 1: s = go(srht_stage1_persist<1, 1>); break;
        case 2: s = go(srht_stage1_persist<2, 1>); break;
        case 4: s = go(srht_stage1_persist<4, 1>); break;
        case 8: s = go(srht_stage1_persist<8, 1>); break;
        case 16: s = go(srht_stage1_persist<16, 1>); break;
        case 32: s = go(srht_stage1_persist<32, 1>); break;
        default: return RBGS_EINVAL;
      }
    } else {
      switch (E) {
        case 1: s = go(srht_stage1_persist<1, 2>); break;
        case 2: s = go(srht_stage1_persist<2, 2>); break;
        case 4: s = go(srht_stage1_persist<4, 2>); break;
        case 8: s = go(srht_stage1_persist<8, 2>); break;
        case 16: s = go(srht_stage1_persist<16, 2>); break;
        case 32: s = go(srht_stage1_persist<32, 2>); break;
        default: return RBGS_EINVAL;
      }
    }
    if (s) return s;
  } else {
    const size_t smem = sizeof(TC) * (size_t)plan->B + sizeof(uint32_t) * (size_t)((plan->B + 31) / 32);
    for (int src = 0; src < 2; ++src) {
      const TX* X = src ? X2 : X1;
      const int64_t ldx = src ? ldx2 : ldx1;
      const int64_t nc = src ? nc2 : nc1;
      TC* zs = z + (src ? nc1 : 0) * plan->T * plan->L;
      for (int64_t c0 = 0; c0 < nc; c0 += 65535) {
        const int64_t nn = std::min<int64_t>(65535, nc - c0);
        dim3 grid((unsigned)plan->T, (unsigned)nn);
        s = launch_stage1<TX, TC>(grid, smem, st, X + c0 * ldx, ldx, n, plan->B, logB, plan->T, key, plan->d_lvals,
                                  plan->L, zs + c0 * plan->T * plan->L, active);
        if (s) return s;
      }
    }
  }
  bool done = false;
  s = launch_stage2_fwht<TC, TY>(plan->T, plan->L, plan, z, ncols, nc1, scale, Y1, ldy1, Y2, ldy2, active, st, &done);
  if (s) return s;
  if (!done) {
    for (int src = 0; src < 2; ++src) {
      const int64_t nc = src ? nc2 : nc1;
      if (nc == 0) continue;
      const int64_t tot = k * nc;
      srht_stage2<TC, TY><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
          z + (src ? nc1 : 0) * plan->T * plan->L, plan->T, plan->L, plan->d_rhi, plan->d_rl, k, nc, scale,
          src ? Y2 : Y1, src ? ldy2 : ldy1, active);
      RBGS_LAUNCH_CHECK();
    }
  }
  return RBGS_OK;
}

template <class TX, class TY>
rbgs_status sketch_apply_t(rbgs_sketch kind, int64_t k, int64_t n, uint64_t seed, const TX* X, int64_t ldx,
                           int64_t ncols, TY* Y, int64_t ldy, void* scratch, size_t scratch_bytes, cudaStream_t st,
                           const int* active) {
  // The dense sketches (Gaussian, Rademacher, sparse sign) accumulate in the
  // precision of the sketch space TY: FP32 data sketched into an FP64 sketch
  // space are summed in FP64 (steps 1 and 5 at the fine precision, as the
  // paper's precision split has them).  A block that is numerically rank
  // deficient in FP32 needs this: its projected part is of the size of the
  // FP32 rounding, and an FP32 sum would not resolve it.
  using TC = typename std::conditional<sizeof(TY) == 8, double, TX>::type;
  if (ncols == 0 || k == 0) return RBGS_OK;
  if (kind == RBGS_SK_SRHT)
    return sketch_apply2_t<TX, TY>(kind, k, n, seed, X, ldx, ncols, Y, ldy, X, ldx, 0, Y, ldy, scratch,
                                   scratch_bytes, st, active);
  const uint2 key = seed_key(seed);
  const double dscale = 1.0 / std::sqrt((double)(kind == RBGS_SK_SPARSE ? sparse_zeta(k) : k));
  if (kind != RBGS_SK_GAUSS && kind != RBGS_SK_RADEMACHER && kind != RBGS_SK_SPARSE) return RBGS_EINVAL;
  const int nsplit = dense_nsplit(k, n);
  const int64_t rows_per_split = ((n + nsplit - 1) / nsplit + kDenseJ - 1) / kDenseJ * kDenseJ;
  TC* part = reinterpret_cast<TC*>(scratch);
  for (int64_t c0 = 0; c0 < ncols; c0 += kDenseCols) {
    const int nc = (int)std::min<int64_t>(kDenseCols, ncols - c0);
    const size_t need = sizeof(TC) * (size_t)nsplit * nc * (size_t)k;
    if (scratch_bytes < need) return RBGS_EINVAL;
    dim3 grid((unsigned)((k + kDenseRows - 1) / kDenseRows), (unsigned)nsplit);
    auto launch = [&](auto qn) {
      constexpr int QN = decltype(qn)::value;
      if (kind == RBGS_SK_GAUSS)
        dense_sketch_part<RBGS_SK_GAUSS, TX, TC, QN><<<grid, kDenseThreads, 0, st>>>(
            X + c0 * ldx, ldx, n, nc, k, key, dscale, rows_per_split, part, active);
      else if (kind == RBGS_SK_SPARSE)
        dense_sketch_part<RBGS_SK_SPARSE, TX, TC, QN><<<grid, kDenseThreads, 0, st>>>(
            X + c0 * ldx, ldx, n, nc, k, key, dscale, rows_per_split, part, active);
      else
        dense_sketch_part<RBGS_SK_RADEMACHER, TX, TC, QN><<<grid, kDenseThreads, 0, st>>>(
            X + c0 * ldx, ldx, n, nc, k, key, dscale, rows_per_split, part, active);
    };
    switch ((nc + 15) >> 4) {
      case 1: launch(std::integral_constant<int, 1>{}); break;
      case 2: launch(std::integral_constant<int, 2>{}); break;
      case 3: launch(std::integral_constant<int, 3>{}); break;
      default: launch(std::integral_constant<int, 4>{}); break;
    }
    RBGS_LAUNCH_CHECK();
    const int64_t tot = k * nc;
    dense_sketch_reduce<TC, TY><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(part, nsplit, k, nc, Y + c0 * ldy, ldy,
                                                                                       active);
    RBGS_LAUNCH_CHECK();
  }
  return RBGS_OK;
}

template rbgs_status sketch_apply_t<double, double>(rbgs_sketch, int64_t, int64_t, uint64_t, const double*, int64_t,
                                                    int64_t, double*, int64_t, void*, size_t, cudaStream_t,
                                                    const int*);
template rbgs_status sketch_apply_t<float, double>(rbgs_sketch, int64_t, int64_t, uint64_t, const float*, int64_t,
                                                   int64_t, double*, int64_t, void*, size_t, cudaStream_t,
                                                    const int*);
template rbgs_status sketch_apply_t<float, float>(rbgs_sketch, int64_t, int64_t, uint64_t, const float*, int64_t,
                                                  int64_t, float*, int64_t, void*, size_t, cudaStream_t,
                                                  const int*);

template rbgs_status sketch_apply2_t<double, double>(rbgs_sketch, int64_t, int64_t, uint64_t, const double*, int64_t,
                                                     int64_t, double*, int64_t, const double*, int64_t, int64_t,
                                                     double*, int64_t, void*, size_t, cudaStream_t, const int*);
template rbgs_status sketch_apply2_t<float, double>(rbgs_sketch, int64_t, int64_t, uint64_t, const float*, int64_t,
                                                    int64_t, double*, int64_t, const float*, int64_t, int64_t,
                                                    double*, int64_t, void*, size_t, cudaStream_t, const int*);
template rbgs_status sketch_apply2_t<float, float>(rbgs_sketch, int64_t, int64_t, uint64_t, const float*, int64_t,
                                                   int64_t, float*, int64_t, const float*, int64_t, int64_t, float*,
                                                   int64_t, void*, size_t, cudaStream_t, const int*);

}  // namespace rbgs
