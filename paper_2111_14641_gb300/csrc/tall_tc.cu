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
//               of the column-major source, no swizzle, 16 KB), 8 stages
//   warp 1      TMEM allocation and the single MMA-issuing thread
//   warp 2      bulk-copy producer of the pre-split G chunk (hi + lo, 16 KB,
//               K-major no-swizzle core-matrix layout), 4 stages
//   warps 3-10  converters: the thread of TMEM lane r reads row r of half a
//               raw chunk (the raw stage is released as soon as it is read),
//               rounds it to TF32 hi and lo parts and stores them into tensor
//               memory (stages of 64 columns), where the MMA reads A
//   warps 11-26 epilogue: drains TMEM into registers, stores the rows
// Keeping A in tensor memory halves the shared-memory traffic per chunk (the
// tensor core would otherwise re-read the 128-row A operand from shared
// memory for each of the 12 MMAs), which bounded the earlier designs.
// Accuracy: the tensor cores truncate when they add into an FP32 accumulator,
// so an accumulator that receives every product of a long K loop drifts by
// ~(number of MMAs) * 2^-24.  Each chunk's products therefore land in a fresh
// TMEM slot (rotating slots), the small cross terms first and the four main
// products last, and the epilogue adds the slots with compensated FP32
// summation.
// Every mbarrier wait is bounded; on expiry the kernel records an error flag,
// drains its own copies and MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace rbgs {
namespace {

constexpr int TC_M = 128;
constexpr int TC_N = 64;
constexpr int TC_K = 32;        // fp32 elements per chunk
constexpr int TC_THREADS = 864; // 27 warps
constexpr int A_BYTES = TC_M * TC_K * 4;      // 16 KB raw fp32 chunk
constexpr int B_BYTES = TC_N * TC_K * 4;      // 8 KB per part
constexpr int G_BYTES = 2 * B_BYTES;
constexpr uint64_t kMaxWaitNs = 2000000000ull;         // bounded waits: 2 s
constexpr uint32_t kSuspendHintNs = 100000u;           // sleep hint per try_wait: 100 us
constexpr int TMEM_COLS = 512;

// Pipeline shape: RAW raw stages (TMA, shared memory), GS G stages (shared
// memory), AS converted-A stages and NS product slots in tensor memory.
// TMEM columns: NS x 64 slots | AS x 64 A stages.
template <int RAW, int GS, int AS, int NS>
struct TcCfg {
  static constexpr int RAW_STAGES = RAW, G_STAGES = GS, A_STAGES = AS, NSLOT = NS;
  static constexpr int G_OFF = RAW * A_BYTES;
  static constexpr int SMEM_BAR_OFF = G_OFF + GS * G_BYTES;
  static constexpr int BAR_BYTES = 1024;  // 65 mbarriers, the TMEM address slot and the abort flag
  static constexpr int SMEM_BYTES = SMEM_BAR_OFF + BAR_BYTES + 1024;  // + alignment slack of the base
  static constexpr int SLOT_COL0 = 0;
  static constexpr int A_COL0 = NS * TC_N;
  static_assert(RAW <= 8 && GS <= 8 && AS <= 8 && NS <= 8, "barrier slots");
  static_assert(A_COL0 + AS * 2 * TC_K <= TMEM_COLS, "TMEM budget");
};

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

// try_wait with a suspend-time hint: a waiting thread sleeps in hardware until
// the phase completes or the hint (ns) elapses, so waiting warps do not take
// issue slots from the converters.
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(kSuspendHintNs)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait on the phase with the given parity: false after kMaxWaitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try(bar, parity)) return true;
    if (global_ns() - t0 > kMaxWaitNs) return false;
  }
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

// Round to TF32 (10 explicit mantissa bits), nearest with ties away from zero,
// on the integer pipes: add half a unit of the kept precision to the
// magnitude bits, then clear the 13 dropped bits (a carry moves into the
// exponent as it should).  For finite inputs this is the same rounding as
// tf32_rna.
__device__ __forceinline__ uint32_t tf32_round_bits(float x) {
  return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
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

// A operand read from tensor memory (rows in lanes, K along columns).
__device__ __forceinline__ void umma_tf32_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(bdesc), "r"(kIdesc), "r"(accum)
      : "memory");
}

// 16 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
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

template <class Cfg>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tall_tc_kernel(const __grid_constant__ CUtensorMap tmA1, const __grid_constant__ CUtensorMap tmA2, TcParams p) {
  constexpr int RAW_STAGES = Cfg::RAW_STAGES, G_STAGES = Cfg::G_STAGES;
  constexpr int A_STAGES = Cfg::A_STAGES, NSLOT = Cfg::NSLOT;
  constexpr int G_OFF = Cfg::G_OFF, SMEM_BAR_OFF = Cfg::SMEM_BAR_OFF;
  constexpr int SLOT_COL0 = Cfg::SLOT_COL0, A_COL0 = Cfg::A_COL0;
  if (p.active && *p.active == 0) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t bar0 = smem_u32(smem + SMEM_BAR_OFF);
  auto raw_full = [&](int s) { return bar0 + 8u * s; };                 // 8 slots
  auto raw_empty = [&](int s) { return bar0 + 8u * (8 + s); };          // 8
  auto a_full = [&](int s) { return bar0 + 8u * (16 + s); };            // 8
  auto a_free = [&](int s) { return bar0 + 8u * (24 + s); };            // 8
  auto g_full = [&](int s) { return bar0 + 8u * (32 + s); };            // 8
  auto g_free = [&](int s) { return bar0 + 8u * (40 + s); };            // 8
  auto slot_full = [&](int s) { return bar0 + 8u * (48 + s); };         // 8
  auto slot_free = [&](int s) { return bar0 + 8u * (56 + s); };         // 8
  const uint32_t fin_bar = bar0 + 8u * 64;
  static_assert(8 * 66 + 16 <= Cfg::BAR_BYTES, "barrier area");
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + SMEM_BAR_OFF + 8 * 66);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + SMEM_BAR_OFF + 8 * 66 + 8);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int nchunks = p.nc1 + p.nc2;

  if (threadIdx.x == 0) {
    for (int s = 0; s < RAW_STAGES; ++s) {
      mbar_init(raw_full(s), 1);
      mbar_init(raw_empty(s), 8);
    }
    for (int s = 0; s < A_STAGES; ++s) {
      mbar_init(a_full(s), 8);
      mbar_init(a_free(s), 1);
    }
    for (int s = 0; s < G_STAGES; ++s) {
      mbar_init(g_full(s), 1);
      mbar_init(g_free(s), 1);
    }
    for (int s = 0; s < NSLOT; ++s) {
      mbar_init(slot_full(s), 1);
      mbar_init(slot_free(s), 16);
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
    // Each chunk's products go to a fresh TMEM slot: the small cross terms
    // a_hi g_lo + a_lo g_hi first, then the four a_hi g_hi products, so the
    // truncating accumulation adds to a small value first and to the large
    // one only four times.
    if (lane == 0) {
      uint32_t it = 0;
      bool bad = false;
      for (int tile = blockIdx.x; tile < p.ntiles && !bad; tile += gridDim.x) {
        for (int ch = 0; ch < nchunks; ++ch, ++it) {
          const int c = it % A_STAGES, g = it % G_STAGES, sl = it % NSLOT;
          const uint32_t cph = (it / A_STAGES) & 1u, gph = (it / G_STAGES) & 1u, sph = (it / NSLOT) & 1u;
          if (!mbar_wait(slot_free(sl), sph ^ 1u) || !mbar_wait(a_full(c), cph) || !mbar_wait(g_full(g), gph) ||
              *abort_flag) {
            fail();
            bad = true;
            break;
          }
          tc_fence_after();
          const uint32_t dslot = tmem_base + (uint32_t)(SLOT_COL0 + sl * TC_N);
          const uint32_t ahi = tmem_base + (uint32_t)(A_COL0 + c * 2 * TC_K);
          const uint32_t alo = ahi + TC_K;
          const uint32_t bhi = smem_u32(smem + G_OFF + g * G_BYTES);
          const uint32_t blo = bhi + B_BYTES;
#pragma unroll
          for (int kk = 0; kk < TC_K / 8; ++kk) {
            umma_tf32_ts(dslot, ahi + 8 * kk, umma_desc(blo + kk * 256, 128, 1024), kk != 0);
            umma_tf32_ts(dslot, alo + 8 * kk, umma_desc(bhi + kk * 256, 128, 1024), 1u);
          }
#pragma unroll
          for (int kk = 0; kk < TC_K / 8; ++kk)
            umma_tf32_ts(dslot, ahi + 8 * kk, umma_desc(bhi + kk * 256, 128, 1024), 1u);
          umma_commit(a_free(c));
          umma_commit(g_free(g));
          umma_commit(slot_full(sl));
        }
      }
      // all issued MMAs complete before TMEM is released
      umma_commit(fin_bar);
      if (!mbar_wait(fin_bar, 0)) atomicExch(p.err, 3);
    }
  } else if (warp < 11) {
    // --------------------------------------------- converters (warps 3..10)
    // A warp may only address TMEM lanes 32 (warp % 4) .. +31, so its rows are
    // those; two warps share each lane quarter, one per half of the chunk's K.
    const int quarter = warp & 3;
    const int khalf = (warp - 3) >> 2;
    const int r = 32 * quarter + lane;  // row of the tile == TMEM lane
    const uint32_t lane_off = (uint32_t)(32 * quarter) << 16;
    constexpr int KH = TC_K / 2;
    uint32_t it = 0;
    bool stop = false;
    for (int tile = blockIdx.x; tile < p.ntiles && !stop; tile += gridDim.x) {
      for (int ch = 0; ch < nchunks; ++ch, ++it) {
        const int s = it % RAW_STAGES;
        const uint32_t ph = (it / RAW_STAGES) & 1u;
        const int c = it % A_STAGES;
        const uint32_t cph = (it / A_STAGES) & 1u;
        const bool ok = __all_sync(0xffffffffu, mbar_wait(raw_full(s), ph) && mbar_wait(a_free(c), cph ^ 1u));
        if (!ok && lane == 0) fail();
        if (!ok || __shfl_sync(0xffffffffu, (int)*abort_flag, 0)) {
          stop = true;
          break;
        }
        tc_fence_after();
        const float* raw = reinterpret_cast<const float*>(smem + s * A_BYTES) + khalf * KH * TC_M;
        uint32_t h[KH], l[KH];
#pragma unroll
        for (int k = 0; k < KH; ++k) {
          const float x = raw[k * TC_M + r];
          h[k] = tf32_round_bits(x);
          l[k] = tf32_round_bits(x - __uint_as_float(h[k]));
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(raw_empty(s));  // the TMA may refill this raw stage now
        const uint32_t abase = tmem_base + lane_off + (uint32_t)(A_COL0 + c * 2 * TC_K + khalf * KH);
        tmem_st16(abase, h);
        tmem_st16(abase + TC_K, l);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(a_full(c));
      }
    }
  } else {
    // ----------------------------------------------- epilogue (warps 11..26)
    // Per chunk: drain its TMEM slot into compensated FP32 sums; per tile:
    // store the rows.  Four warps share each TMEM lane quarter (warp % 4),
    // 16 columns each.
    const int quarter = warp & 3;
    const int part = (warp - 11) >> 2;
    const uint32_t lane_off = (uint32_t)(32 * quarter) << 16;
    const uint32_t col_off = (uint32_t)(16 * part);
    uint32_t it = 0;
    bool stop = false;
    for (int tile = blockIdx.x; tile < p.ntiles && !stop; tile += gridDim.x) {
      float acc[16], cmp[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
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
        float v[16];
        tmem_ld16(tmem_base + lane_off + (uint32_t)(SLOT_COL0 + sl * TC_N) + col_off, v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(slot_free(sl));
#pragma unroll
        for (int j = 0; j < 16; ++j) {  // Kahan-Babuska summation in FP32
          const float y = v[j] - cmp[j];
          const float t = acc[j] + y;
          cmp[j] = (t - acc[j]) - y;
          acc[j] = t;
        }
      }
      if (stop) break;
      const int64_t row = (int64_t)tile * TC_M + 32 * quarter + lane;
      if (row < p.n) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if ((int)col_off + j < p.mb) p.qout[row + (int64_t)(col_off + j) * p.ldo] = acc[j] - cmp[j];
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

// Pipeline configuration (see TcCfg); RBGS_TC_CONFIG=<index> selects another
// shape for tuning measurements.
int tc_config() {
  static int cfg = []() {
    const char* e = getenv("RBGS_TC_CONFIG");
    return e ? atoi(e) : 0;
  }();
  return cfg;
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
  TcParams p{};
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
  const int grid = std::min(p.ntiles, nsm);
  auto go = [&](auto cfg) -> rbgs_status {
    using Cfg = decltype(cfg);
    RBGS_CUDA_TRY(cudaFuncSetAttribute(tall_tc_kernel<Cfg>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Cfg::SMEM_BYTES));
    tall_tc_kernel<Cfg><<<grid, TC_THREADS, Cfg::SMEM_BYTES, st>>>(m1, m2, p);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
  };
  switch (tc_config()) {
    case 1: return go(TcCfg<8, 4, 5, 3>{});
    case 2: return go(TcCfg<8, 4, 6, 2>{});
    case 3: return go(TcCfg<6, 6, 4, 4>{});
    default: return go(TcCfg<8, 4, 4, 4>{});
  }
}

}  // namespace rbgs
