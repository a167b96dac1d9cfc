// Tensor-core tall update on sm_103a (tcgen05 + TMA), 3xTF32 split products.
//
//   Qout (n x mb) = [A1 (n x c) | A2 (n x mb)] * G ((c+mb) x mb)
//
// This is step 3 of Alg. 2 fused with the multiplication by R_ii^{-1} of
// Alg. 5 (G = [-R_{1:i-1,i}; I] R_ii^{-1}).  The operation reads the whole
// previous basis once per block, so it is bound by HBM bandwidth; the tensor
// cores are the means to keep up with the bytes at FP32-level accuracy:
//   a = a_hi + a_lo,  g = g_hi + g_lo  (TF32 parts, round to nearest),
//   a g ~ a_hi g_hi + a_hi g_lo + a_lo g_hi     (error ~2^-22 |a g|).
//
// Persistent kernel, one CTA per SM, 128-row tiles, K in chunks of 32:
//   warp 0      TMA producer of the raw ring: A chunk (128 rows x 32 columns
//               of the column-major source, no swizzle, 16 KB), 5 stages
//   warp 1      TMEM allocation and the single MMA-issuing thread
//   warp 2      bulk-copy producer of the pre-split G chunk (hi + lo, 16 KB),
//               4 stages
//   warps 3-6   converters: thread r reads row r of a raw chunk (the raw stage
//               is released as soon as it is read), writes the TF32 hi and lo
//               parts (2 stages) in the K-major no-swizzle core-matrix layout
//               (8 rows x 16 B cores, K-direction core stride 128 B, 8-row
//               group stride 1024 B)
//   warps 7-14  epilogue: drains TMEM into registers, stores the rows
// Accuracy: the tensor cores truncate when they add into an FP32 accumulator,
// so an accumulator that receives every product of a long K loop drifts by
// ~(number of MMAs) * 2^-24.  Each chunk's a_hi g_hi product therefore lands
// in a fresh TMEM slot (4 rotating slots) that the epilogue adds with
// compensated FP32 summation; the two cross terms, 2^-11 smaller, share one
// accumulator per tile (double-buffered across tiles).
// Every mbarrier wait is bounded; on expiry the kernel records an error flag,
// drains its own copies and MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace rbgs {
namespace {

constexpr int TC_M = 128;
constexpr int TC_N = 64;
constexpr int TC_K = 32;        // fp32 elements per chunk
constexpr int RAW_STAGES = 5;   // TMA destinations (raw fp32 A chunks, 16 KB)
constexpr int CV_STAGES = 2;    // converted A (TF32 hi + lo, 32 KB) for the MMA
constexpr int G_STAGES = 4;     // G chunks (TF32 hi + lo, 16 KB)
constexpr int NSLOT = 4;        // TMEM slots for the per-chunk main products
constexpr int TC_THREADS = 480; // 15 warps
constexpr int A_BYTES = TC_M * TC_K * 4;      // 16 KB
constexpr int B_BYTES = TC_N * TC_K * 4;      // 8 KB per part
constexpr int CV_BYTES = 2 * A_BYTES;
constexpr int G_BYTES = 2 * B_BYTES;
constexpr int CV_OFF = RAW_STAGES * A_BYTES;
constexpr int G_OFF = CV_OFF + CV_STAGES * CV_BYTES;
constexpr int SMEM_BAR_OFF = G_OFF + G_STAGES * G_BYTES;
constexpr int SMEM_BYTES = SMEM_BAR_OFF + 512 + 1024;  // + barriers + alignment slack
constexpr uint32_t kMaxSpin = 1u << 26;                // bounded waits (~seconds)
constexpr int TMEM_COLS = 512;                         // 4 main slots + 2 cross accumulators of 64
constexpr int CROSS_COL0 = NSLOT * TC_N;

struct TcParams {
  int64_t n;
  int c, mb, nc1, nc2, ntiles;
  const float* gsplit;
  float* qout;
  int64_t ldo;
  const int* active;
  int* err;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on the phase with the given parity; false on expiry.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t i = 0; i < kMaxSpin; ++i)
    if (mbar_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// Shared-memory matrix descriptor, K-major, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;                // base offset 0, relative LBO, layout SWIZZLE_NONE
}

// Instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                            ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ void umma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    tall_tc_kernel(const __grid_constant__ CUtensorMap tmA1, const __grid_constant__ CUtensorMap tmA2, TcParams p) {
  if (p.active && *p.active == 0) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t bar0 = smem_u32(smem + SMEM_BAR_OFF);
  // barrier slots
  auto raw_full = [&](int s) { return bar0 + 8u * s; };                 // 5
  auto raw_empty = [&](int s) { return bar0 + 8u * (5 + s); };          // 5
  auto cv_full = [&](int s) { return bar0 + 8u * (10 + s); };           // 2
  auto cv_free = [&](int s) { return bar0 + 8u * (12 + s); };           // 2
  auto g_full = [&](int s) { return bar0 + 8u * (14 + s); };            // 4
  auto g_free = [&](int s) { return bar0 + 8u * (18 + s); };            // 4
  auto slot_full = [&](int s) { return bar0 + 8u * (22 + s); };         // 4
  auto slot_free = [&](int s) { return bar0 + 8u * (26 + s); };         // 4
  auto cross_full = [&](int b) { return bar0 + 8u * (30 + b); };        // 2
  auto cross_free = [&](int b) { return bar0 + 8u * (32 + b); };        // 2
  const uint32_t fin_bar = bar0 + 8u * 34;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + SMEM_BAR_OFF + 8 * 36);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + SMEM_BAR_OFF + 8 * 36 + 8);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int nchunks = p.nc1 + p.nc2;

  if (threadIdx.x == 0) {
    for (int s = 0; s < RAW_STAGES; ++s) {
      mbar_init(raw_full(s), 1);
      mbar_init(raw_empty(s), 4);
    }
    for (int s = 0; s < CV_STAGES; ++s) {
      mbar_init(cv_full(s), 4);
      mbar_init(cv_free(s), 1);
    }
    for (int s = 0; s < G_STAGES; ++s) {
      mbar_init(g_full(s), 1);
      mbar_init(g_free(s), 1);
    }
    for (int s = 0; s < NSLOT; ++s) {
      mbar_init(slot_full(s), 1);
      mbar_init(slot_free(s), 8);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(cross_full(b), 1);
      mbar_init(cross_free(b), 8);
    }
    mbar_init(fin_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  auto fail = [&]() {
    *abort_flag = 1;
    atomicExch(p.err, 1);
  };

  if (warp == 0) {
    // ------------------------------------------------- A producer (raw ring)
    if (lane == 0) {
      uint32_t it = 0;
      int armed_phase[RAW_STAGES];
      for (int s = 0; s < RAW_STAGES; ++s) armed_phase[s] = -1;
      for (int tile = blockIdx.x; tile < p.ntiles && !*abort_flag; tile += gridDim.x) {
        const int row0 = tile * TC_M;
        for (int ch = 0; ch < nchunks; ++ch, ++it) {
          const int s = it % RAW_STAGES;
          const uint32_t ph = (it / RAW_STAGES) & 1u;
          if (!mbar_wait(raw_empty(s), ph ^ 1u)) {
            fail();
            break;
          }
          if (*abort_flag) break;
          mbar_expect_tx(raw_full(s), A_BYTES);
          const uint32_t dst = smem_u32(smem + s * A_BYTES);
          if (ch < p.nc1) tma_load_2d(dst, &tmA1, row0, ch * TC_K, raw_full(s));
          else tma_load_2d(dst, &tmA2, row0, (ch - p.nc1) * TC_K, raw_full(s));
          armed_phase[s] = (int)ph;
        }
      }
      // never leave with copies in flight into this CTA's shared memory
      for (int s = 0; s < RAW_STAGES; ++s)
        if (armed_phase[s] >= 0 && !mbar_wait(raw_full(s), (uint32_t)armed_phase[s])) atomicExch(p.err, 2);
    }
  } else if (warp == 2) {
    // -------------------------------------------------------- G producer
    if (lane == 0) {
      uint32_t it = 0;
      int armed_phase[G_STAGES];
      for (int s = 0; s < G_STAGES; ++s) armed_phase[s] = -1;
      for (int tile = blockIdx.x; tile < p.ntiles && !*abort_flag; tile += gridDim.x) {
        for (int ch = 0; ch < nchunks; ++ch, ++it) {
          const int g = it % G_STAGES;
          const uint32_t ph = (it / G_STAGES) & 1u;
          if (!mbar_wait(g_free(g), ph ^ 1u)) {
            fail();
            break;
          }
          if (*abort_flag) break;
          mbar_expect_tx(g_full(g), G_BYTES);
          bulk_load(smem_u32(smem + G_OFF + g * G_BYTES), p.gsplit + (size_t)ch * (2 * TC_N * TC_K), G_BYTES,
                    g_full(g));
          armed_phase[g] = (int)ph;
        }
      }
      for (int s = 0; s < G_STAGES; ++s)
        if (armed_phase[s] >= 0 && !mbar_wait(g_full(s), (uint32_t)armed_phase[s])) atomicExch(p.err, 2);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      uint32_t it = 0, tcount = 0;
      for (int tile = blockIdx.x; tile < p.ntiles && !*abort_flag; tile += gridDim.x, ++tcount) {
        const int b = tcount & 1;
        const uint32_t bph = (tcount >> 1) & 1u;
        if (!mbar_wait(cross_free(b), bph ^ 1u)) {
          fail();
          break;
        }
        tc_fence_after();
        const uint32_t dcross = tmem_base + (uint32_t)(CROSS_COL0 + b * TC_N);
        bool bad = false;
        for (int ch = 0; ch < nchunks; ++ch, ++it) {
          const int c = it % CV_STAGES, g = it % G_STAGES, sl = it % NSLOT;
          const uint32_t cph = (it / CV_STAGES) & 1u, gph = (it / G_STAGES) & 1u, sph = (it / NSLOT) & 1u;
          if (!mbar_wait(slot_free(sl), sph ^ 1u) || !mbar_wait(cv_full(c), cph) || !mbar_wait(g_full(g), gph) ||
              *abort_flag) {
            fail();
            bad = true;
            break;
          }
          tc_fence_after();
          const uint32_t dmain = tmem_base + (uint32_t)(sl * TC_N);
          const uint32_t ahi = smem_u32(smem + CV_OFF + c * CV_BYTES);
          const uint32_t alo = ahi + A_BYTES;
          const uint32_t bhi = smem_u32(smem + G_OFF + g * G_BYTES);
          const uint32_t blo = bhi + B_BYTES;
#pragma unroll
          for (int kk = 0; kk < TC_K / 8; ++kk) {
            const uint32_t off = kk * 256;  // 8 tf32 = two 16-byte cores along K
            const uint64_t dah = umma_desc(ahi + off, 128, 1024);
            const uint64_t dal = umma_desc(alo + off, 128, 1024);
            const uint64_t dbh = umma_desc(bhi + off, 128, 1024);
            const uint64_t dbl = umma_desc(blo + off, 128, 1024);
            umma_tf32(dmain, dah, dbh, kk != 0);              // this chunk's main product, fresh slot
            umma_tf32(dcross, dah, dbl, (ch | kk) != 0);       // small cross terms, whole tile
            umma_tf32(dcross, dal, dbh, 1u);
          }
          umma_commit(cv_free(c));
          umma_commit(g_free(g));
          umma_commit(slot_full(sl));
        }
        if (bad) break;
        umma_commit(cross_full(b));
      }
      // all issued MMAs complete before TMEM is released
      umma_commit(fin_bar);
      if (!mbar_wait(fin_bar, 0)) atomicExch(p.err, 3);
    }
  } else if (warp < 7) {
    // ---------------------------------------------- converters (warps 3..6)
    const int r = threadIdx.x - 96;  // row of the tile
    const int rowoff = (r >> 3) * 1024 + (r & 7) * 16;
    uint32_t it = 0;
    bool stop = false;
    for (int tile = blockIdx.x; tile < p.ntiles && !stop; tile += gridDim.x) {
      for (int ch = 0; ch < nchunks; ++ch, ++it) {
        const int s = it % RAW_STAGES;
        const uint32_t ph = (it / RAW_STAGES) & 1u;
        const int c = it % CV_STAGES;
        const uint32_t cph = (it / CV_STAGES) & 1u;
        const bool ok = __all_sync(0xffffffffu, mbar_wait(raw_full(s), ph) && mbar_wait(cv_free(c), cph ^ 1u));
        if (!ok && lane == 0) fail();
        if (!ok || __shfl_sync(0xffffffffu, (int)*abort_flag, 0)) {
          stop = true;
          break;
        }
        const float* raw = reinterpret_cast<const float*>(smem + s * A_BYTES);
        float v[TC_K];
#pragma unroll
        for (int k = 0; k < TC_K; ++k) v[k] = raw[k * TC_M + r];
        __syncwarp();
        if (lane == 0) mbar_arrive(raw_empty(s));  // the TMA may refill this raw stage now
        unsigned char* hi = smem + CV_OFF + c * CV_BYTES;
        unsigned char* lo = hi + A_BYTES;
#pragma unroll
        for (int c4 = 0; c4 < TC_K / 4; ++c4) {
          uint32_t h[4], l[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float x = v[4 * c4 + q];
            h[q] = tf32_rna(x);
            l[q] = tf32_rna(x - __uint_as_float(h[q]));
          }
          *reinterpret_cast<uint4*>(hi + rowoff + c4 * 128) = make_uint4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<uint4*>(lo + rowoff + c4 * 128) = make_uint4(l[0], l[1], l[2], l[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(cv_full(c));
      }
    }
  } else {
    // ------------------------------------------------ epilogue (warps 7..14)
    // Per chunk: drain the chunk's TMEM slot into compensated FP32 sums;
    // per tile: add the cross-term accumulator and store the rows.  Two
    // warps share each TMEM lane quarter (warp % 4), 32 columns each.
    const int quarter = warp & 3;
    const int half = (warp - 7) >> 2;
    const uint32_t lane_off = (uint32_t)(32 * quarter) << 16;
    const uint32_t col_off = (uint32_t)(32 * half);
    uint32_t it = 0, tcount = 0;
    bool stop = false;
    for (int tile = blockIdx.x; tile < p.ntiles && !stop; tile += gridDim.x, ++tcount) {
      float acc[32], cmp[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        acc[j] = 0.f;
        cmp[j] = 0.f;
      }
      for (int ch = 0; ch < nchunks; ++ch, ++it) {
        const int sl = it % NSLOT;
        const uint32_t sph = (it / NSLOT) & 1u;
        const bool ok = __all_sync(0xffffffffu, mbar_wait(slot_full(sl), sph));
        if (!ok && lane == 0) fail();
        if (!ok || __shfl_sync(0xffffffffu, (int)*abort_flag, 0)) {
          stop = true;
          break;
        }
        tc_fence_after();
        float v[32];
        const uint32_t taddr = tmem_base + lane_off + (uint32_t)(sl * TC_N) + col_off;
        tmem_ld16(taddr, v);
        tmem_ld16(taddr + 16, v + 16);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(slot_free(sl));
#pragma unroll
        for (int j = 0; j < 32; ++j) {  // Kahan-Babuska summation in FP32
          const float y = v[j] - cmp[j];
          const float t = acc[j] + y;
          cmp[j] = (t - acc[j]) - y;
          acc[j] = t;
        }
      }
      if (stop) break;
      const int b = tcount & 1;
      const uint32_t bph = (tcount >> 1) & 1u;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(cross_full(b), bph));
      if (!ok && lane == 0) fail();
      if (!ok || __shfl_sync(0xffffffffu, (int)*abort_flag, 0)) break;
      tc_fence_after();
      float v[32];
      const uint32_t taddr = tmem_base + lane_off + (uint32_t)(CROSS_COL0 + b * TC_N) + col_off;
      tmem_ld16(taddr, v);
      tmem_ld16(taddr + 16, v + 16);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(cross_free(b));
      const int64_t row = (int64_t)tile * TC_M + 32 * quarter + lane;
      if (row < p.n) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if ((int)col_off + j < p.mb) p.qout[row + (int64_t)(col_off + j) * p.ldo] = acc[j] + (v[j] - cmp[j]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                 : "memory");
  }
}

// Split G ((c + mb) x mb, FP64) into per-chunk TF32 hi/lo blocks laid out as
// the B operand (N = 64 rows of K-contiguous cores): chunk ch covers G rows
// [32 ch, 32 ch + 32) of the first c rows for ch < nc1, and rows
// c + 32 (ch - nc1) + [0, 32) of the last mb rows after that; rows outside
// the range and columns >= mb are zero.
__global__ void tc_split_kernel(int c, int mb, int nc1, int nchunks, const double* __restrict__ G, int64_t ldg,
                                float* __restrict__ out, const int* active) {
  if (active && *active == 0) return;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)TC_N * TC_K;
  if (idx >= (int64_t)nchunks * per) return;
  const int ch = (int)(idx / per);
  const int e = (int)(idx % per);
  const int n = e / TC_K, kk = e % TC_K;
  int64_t grow = -1;
  if (ch < nc1) {
    const int kr = ch * TC_K + kk;
    if (kr < c) grow = kr;
  } else {
    const int kr = (ch - nc1) * TC_K + kk;
    if (kr < mb) grow = c + kr;
  }
  const double g = (grow >= 0 && n < mb) ? G[grow + (int64_t)n * ldg] : 0.0;
  const uint32_t hb = tf32_rna((float)g);
  const float h = __uint_as_float(hb);
  const uint32_t lb = tf32_rna((float)(g - (double)h));
  const int off = (n >> 3) * 256 + (kk >> 2) * 32 + (n & 7) * 4 + (kk & 3);  // floats
  float* blk = out + (size_t)ch * (2 * per);
  blk[off] = h;
  blk[per + off] = __uint_as_float(lb);
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  });
  return fn;
}

// 2-D map over a column-major n x cols float matrix, box 128 rows x 32 columns.
bool make_map(CUtensorMap* map, const float* base, int64_t n, int64_t cols, int64_t ld) {
  auto enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)cols};
  cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  cuuint32_t box[2] = {TC_M, TC_K};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

size_t tc_gsplit_floats(int64_t K) { return (size_t)((K + TC_K - 1) / TC_K + 2) * 2 * TC_N * TC_K; }

rbgs_status tc_split_g(int64_t K, int64_t mb, const double* G, int64_t ldg, float* Gsplit, const int* active,
                       cudaStream_t st) {
  if (mb < 1 || mb > TC_N || K < mb) return RBGS_EINVAL;
  const int c = (int)(K - mb);
  const int nc1 = (c + TC_K - 1) / TC_K;
  const int nc2 = ((int)mb + TC_K - 1) / TC_K;
  const int64_t tot = (int64_t)(nc1 + nc2) * TC_N * TC_K;
  tc_split_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(c, (int)mb, nc1, nc1 + nc2, G, ldg, Gsplit, active);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}

rbgs_status tall_update_tc(int64_t n, int64_t c, int64_t mb, const float* A1, int64_t lda1, const float* A2,
                           int64_t lda2, const float* Gsplit, float* Qout, int64_t ldo, const int* active,
                           int* err, cudaStream_t st) {
  if (mb < 1 || mb > TC_N || n < 1 || n >= ((int64_t)1 << 31)) return RBGS_EINVAL;
  if (((uintptr_t)A2 & 15) || (lda2 % 4) || (c > 0 && (((uintptr_t)A1 & 15) || (lda1 % 4)))) return RBGS_EINVAL;
  CUtensorMap m1, m2;
  std::memset(&m1, 0, sizeof(m1));
  if (c > 0 && !make_map(&m1, A1, n, c, lda1)) return RBGS_ECUDA;
  if (!make_map(&m2, A2, n, mb, lda2)) return RBGS_ECUDA;
  if (c == 0) m1 = m2;
  int dev = 0, nsm = 0;
  RBGS_CUDA_TRY(cudaGetDevice(&dev));
  RBGS_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (!err) return RBGS_EINVAL;
  TcParams p;
  p.n = n;
  p.c = (int)c;
  p.mb = (int)mb;
  p.nc1 = (int)((c + TC_K - 1) / TC_K);
  p.nc2 = (int)((mb + TC_K - 1) / TC_K);
  p.ntiles = (int)((n + TC_M - 1) / TC_M);
  p.gsplit = Gsplit;
  p.qout = Qout;
  p.ldo = ldo;
  p.active = active;
  p.err = err;
  RBGS_CUDA_TRY(cudaFuncSetAttribute(tall_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
  const int grid = std::min(p.ntiles, nsm);
  tall_tc_kernel<<<grid, TC_THREADS, SMEM_BYTES, st>>>(m1, m2, p);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}

}  // namespace rbgs
