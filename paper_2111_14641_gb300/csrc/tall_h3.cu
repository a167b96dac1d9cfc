// Tensor-core tall update on sm_103a (tcgen05 + TMA) with FP16 hi/lo split
// operands, three products per K step ("F16X3"):
//
//   Qout (n x mb) = [Q_{1:c} | X] * G,   G ((c + mb) x mb)
//
// This is step 3 of Alg. 2 fused with the multiplication by R_ii^{-1} of
// Alg. 5 (G = [-R_{1:i-1,i}; I] R_ii^{-1}).  It streams the whole previous
// basis once per block and is bound by HBM bandwidth.
//
// Operands.  Every column of A = [Q_{1:c} | X] is scaled by a power of two
// s_k and split as s_k a = a_hi + a_lo with a_hi = fp16(s_k a) and
// a_lo = fp16(s_k a - a_hi) (11 + 11 significant bits).  G's columns get a
// power-of-two scale t_j and its rows the inverse scale of A's column:
// b = t_j g / s_k = b_hi + b_lo.  Then
//   sum_k a b = t_j (A G)_j,   a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi,
// with a relative error of about 2^-22 per product, and the epilogue
// multiplies by 1/t_j (exact).  The scales keep every value inside the
// normal FP16 range: the columns of Q are sketch-orthonormal (||Theta q|| = 1,
// so |q| <= ||q|| <= (1 - eps)^{-1/2}) and carry s = 2^9; a raw column x gets
// s = 2^(9 - e) with 2^(e-1) <= ||Theta x|| < 2^e.
//
// Pre-split basis.  The split of the final Q columns is kept in HBM in the
// MMA's own layout (per 128-row tile and 64-column chunk: 16 KB of a_hi then
// 16 KB of a_lo, K-major 8x8 core matrices), written by the kernel that
// produces each block.  It has the same size as FP32, so the previous basis
// streams straight from HBM into shared memory with bulk copies and into the
// tensor core with no conversion.  Only the block's own mb columns (W_i in the
// first pass, the provisional Q'_i in the second) arrive as FP32 through TMA
// and are split by converter warps.
//
// Persistent kernel, one CTA per SM, 128-row tiles, K in chunks of 64:
//   warp 0      bulk-copy producer of the pre-split A chunks (32 KB), AST stages,
//               and the TMA of each tile's raw chunk, RST stages
//   warp 1      TMEM allocation and the single MMA-issuing thread
//   warp 2      bulk-copy producer of the split G chunks (16 KB), BST stages
//   warps 3-10  raw chunk (128 rows x 64 columns FP32, loaded by TMA from
//               warp 0): scaled and split in place into the A layout
//   warps 11-26 epilogue: drains each chunk's TMEM slot into compensated
//               FP32 sums, stores Q (FP32) and, if asked, its split copy
// Accuracy: the tensor core truncates when it adds into an FP32 accumulator,
// so each chunk's 12 products land in a fresh TMEM slot (cross terms first)
// and the epilogue adds the slots with Kahan-Babuska summation.
// Every mbarrier wait is bounded; on expiry the kernel records an error flag,
// drains its own copies and MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace rbgs {
namespace {

constexpr int H_M = 128;                  // rows per tile
constexpr int H_N = 64;                   // output columns (mb <= 64)
constexpr int H_K = 64;                   // K columns per chunk
constexpr int H_THREADS = 864;            // 27 warps
constexpr int H_PART = H_M * H_K * 2;     // 16 KB: one of a_hi / a_lo per chunk
constexpr int H_ACHUNK = 2 * H_PART;      // 32 KB
constexpr int H_BPART = H_N * H_K * 2;    // 8 KB: one of b_hi / b_lo
constexpr int H_BCHUNK = 2 * H_BPART;     // 16 KB
constexpr float kQScale = 512.f;          // 2^9: scale of the sketch-orthonormal Q columns
constexpr uint64_t kMaxWaitNs = 2000000000ull;  // bounded waits: 2 s
constexpr uint32_t kSuspendHintNs = 100000u;

// ATM > 0: the A chunk is copied into ATM tensor-memory stages (tcgen05.cp)
// and the MMAs read A from there; 0: the MMAs read A from shared memory.
template <int AST, int RST, int BST, int NS = 4, int ATM = 0>
struct H3Cfg {
  static constexpr int A_STAGES = AST, R_STAGES = RST, B_STAGES = BST;
  static constexpr int NSLOT = NS;              // TMEM accumulator slots of 64 FP32 columns
  static constexpr int A_TMEM = ATM;
  static constexpr int A_COL0 = NS * 64;        // TMEM A stages: 64 columns each (hi 32 | lo 32)
  static constexpr int TMEM_USED = NS * 64 + ATM * 64;
  static constexpr int TMEM_COLS = TMEM_USED <= 256 ? 256 : 512;
  static_assert(TMEM_USED <= 512, "TMEM budget");
  static_assert(ATM == 0 || ATM == 2 || ATM == 4, "TMEM A stages");
  static constexpr int R_OFF = AST * H_ACHUNK;
  static constexpr int B_OFF = R_OFF + RST * H_ACHUNK;
  static constexpr int BAR_OFF = B_OFF + BST * H_BCHUNK;
  static constexpr int BAR_BYTES = 1024;  // 55 mbarriers, TMEM address, abort flag, 128 scales
  static constexpr int SMEM_BYTES = BAR_OFF + BAR_BYTES + 1024;  // + alignment slack of the base
  static_assert(AST <= 8 && RST <= 2 && BST <= 8, "barrier slots");
  static_assert(SMEM_BYTES <= 232448, "shared memory per CTA");
};

struct H3Params {
  int64_t n;
  int c, mb, qch, ntiles, nch_row;
  const unsigned char* qs;     // pre-split basis (tiled), chunks [0, qch) of each tile are read
  const unsigned char* bsplit; // (qch + 1) chunks of 16 KB
  const float* scales;         // [0, 64): raw column scales; [64, 128): 1/t_j
  float* qout;
  int64_t ldo;
  unsigned char* qs_out;       // where to write the split of Qout (columns cs_out ..), or null
  int cs_out;
  int jsh;                     // TMEM / B column of output column j is j + jsh
  int vec_split;               // (cs_out - jsh) % 8 == 0 and mb + jsh <= 64: vector split stores
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
// Shared-memory matrix descriptor, K-major, no swizzle: lbo = byte distance of
// core matrices adjacent in K, sbo = adjacent in M (or N).
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// Instruction descriptor: kind::f16, D = F32, A = B = F16, both K-major, M = 128, N = 64.
constexpr uint32_t kIdescF16 = (1u << 4) | ((uint32_t)(H_N >> 3) << 17) | ((uint32_t)(H_M >> 4) << 24);
// Byte layout of the A chunk: element (row r, column kk) of a part at
// (kk / 8) * 2048 + (r / 8) * 128 + (r % 8) * 16 + (kk % 8) * 2.
constexpr uint32_t kALbo = 2048, kASbo = 128;
// B chunk: element (output column j, K index kk) at (kk / 8) * 1024 + (j / 8) * 128 + (j % 8) * 16 + (kk % 8) * 2.
constexpr uint32_t kBLbo = 1024, kBSbo = 128;

__device__ __forceinline__ void umma_f16_ss(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdescF16), "r"(accum)
      : "memory");
}
// A operand from tensor memory (rows in lanes, K pairs along the columns).
__device__ __forceinline__ void umma_f16_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(bdesc), "r"(kIdescF16), "r"(accum)
      : "memory");
}
// 128 rows x 256 bits (16 fp16 of K) from shared memory (matrix descriptor) into 8 TMEM columns.
__device__ __forceinline__ void tmem_cp_128x256b(uint32_t taddr, uint64_t sdesc) {
  asm volatile("tcgen05.cp.cta_group::1.128x256b [%0], %1;" ::"r"(taddr), "l"(sdesc) : "memory");
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

// s * x as fp16 hi + lo (s a power of two keeping |s x| inside the fp16 range).
__device__ __forceinline__ void split_f16(float v, unsigned short& hi, unsigned short& lo) {
  const __half h = __float2half_rn(v);
  const __half l = __float2half_rn(v - __half2float(h));
  hi = __half_as_ushort(h);
  lo = __half_as_ushort(l);
}

// Byte offset of (row r, chunk column kk) inside one 16 KB part of an A chunk.
__device__ __forceinline__ uint32_t a_off(int r, int kk) {
  return (uint32_t)((kk >> 3) * 2048 + (r >> 3) * 128 + (r & 7) * 16 + (kk & 7) * 2);
}

template <class Cfg>
__global__ void __launch_bounds__(H_THREADS, 1)
    tall_h3_kernel(const __grid_constant__ CUtensorMap tmRaw, H3Params p) {
  constexpr int AST = Cfg::A_STAGES, RST = Cfg::R_STAGES, BST = Cfg::B_STAGES;
  constexpr int H_NSLOT = Cfg::NSLOT, H_TMEM_COLS = Cfg::TMEM_COLS;
  if (p.active && *p.active == 0) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t bar0 = smem_u32(smem + Cfg::BAR_OFF);
  auto a_full = [&](int s) { return bar0 + 8u * s; };            // 8 slots
  auto a_empty = [&](int s) { return bar0 + 8u * (8 + s); };     // 8
  auto b_full = [&](int s) { return bar0 + 8u * (16 + s); };     // 8
  auto b_empty = [&](int s) { return bar0 + 8u * (24 + s); };    // 8
  auto slot_full = [&](int s) { return bar0 + 8u * (32 + s); };  // 8
  auto slot_free = [&](int s) { return bar0 + 8u * (40 + s); };  // 8
  auto raw_full = [&](int s) { return bar0 + 8u * (48 + s); };   // 2
  auto conv_full = [&](int s) { return bar0 + 8u * (50 + s); };  // 2
  auto raw_empty = [&](int s) { return bar0 + 8u * (52 + s); };  // 2
  const uint32_t fin_bar = bar0 + 8u * 54;
  auto atm_free = [&](int s) { return bar0 + 8u * (55 + s); };   // 4
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + Cfg::BAR_OFF + 8 * 60);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + Cfg::BAR_OFF + 8 * 60 + 8);
  float* sm_scale = reinterpret_cast<float*>(smem + Cfg::BAR_OFF + 8 * 60 + 16);  // 128 floats
  static_assert(8 * 60 + 16 + 128 * 4 <= Cfg::BAR_BYTES, "barrier area");

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int nchunks = p.qch + 1;  // the last chunk of every tile is the raw one

  if (threadIdx.x == 0) {
    for (int s = 0; s < AST; ++s) {
      mbar_init(a_full(s), 1);
      mbar_init(a_empty(s), 1);
    }
    for (int s = 0; s < BST; ++s) {
      mbar_init(b_full(s), 1);
      mbar_init(b_empty(s), 1);
    }
    for (int s = 0; s < H_NSLOT; ++s) {
      mbar_init(slot_full(s), 1);
      mbar_init(slot_free(s), 16);
    }
    for (int s = 0; s < RST; ++s) {
      mbar_init(raw_full(s), 1);
      mbar_init(conv_full(s), 8);
      mbar_init(raw_empty(s), 1);
    }
    mbar_init(fin_bar, 1);
    for (int s = 0; s < 4; ++s) mbar_init(atm_free(s), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 128) sm_scale[threadIdx.x] = p.scales[threadIdx.x];
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(H_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  auto fail = [&](int code) {
    *abort_flag = 1;
    atomicExch(p.err, code);
  };

  if (warp == 0) {
    // ------------------------------------------ pre-split A chunk producer
    // Per tile: the pre-split chunks of the basis, then the TMA of the raw
    // block chunk (FP32) into a raw stage, early enough for the converters.
    if (lane == 0) {
      uint32_t it = 0, rit = 0;
      int armed[AST], rarmed[RST];
      for (int s = 0; s < AST; ++s) armed[s] = -1;
      for (int s = 0; s < RST; ++s) rarmed[s] = -1;
      for (int tile = blockIdx.x; tile < p.ntiles && !*abort_flag; tile += gridDim.x, ++rit) {
        const unsigned char* src = p.qs + (size_t)tile * p.nch_row * H_ACHUNK;
        bool bad = false;
        for (int ch = 0; ch < p.qch; ++ch, ++it) {
          const int s = it % AST;
          const uint32_t ph = (it / AST) & 1u;
          if (!mbar_wait(a_empty(s), ph ^ 1u)) {
            fail(1);
            bad = true;
            break;
          }
          if (*abort_flag) {
            bad = true;
            break;
          }
          mbar_expect_tx(a_full(s), H_ACHUNK);
          bulk_load(smem_u32(smem + s * H_ACHUNK), src + (size_t)ch * H_ACHUNK, H_ACHUNK, a_full(s));
          armed[s] = (int)ph;
        }
        if (bad) break;
        const int rs = (int)(rit % RST);
        const uint32_t rph = (rit / RST) & 1u;
        if (!mbar_wait(raw_empty(rs), rph ^ 1u)) {
          fail(1);
          break;
        }
        if (*abort_flag) break;
        mbar_expect_tx(raw_full(rs), H_ACHUNK);
        tma_load_2d(smem_u32(smem + Cfg::R_OFF + rs * H_ACHUNK), &tmRaw, tile * H_M, 0, raw_full(rs));
        rarmed[rs] = (int)rph;
      }
      // never leave with copies in flight into this CTA's shared memory
      for (int s = 0; s < AST; ++s)
        if (armed[s] >= 0 && !mbar_wait(a_full(s), (uint32_t)armed[s])) atomicExch(p.err, 2);
      for (int s = 0; s < RST; ++s)
        if (rarmed[s] >= 0 && !mbar_wait(raw_full(s), (uint32_t)rarmed[s])) atomicExch(p.err, 2);
    }
  } else if (warp == 2) {
    // ------------------------------------------------------ B chunk producer
    if (lane == 0) {
      uint32_t it = 0;
      int armed[BST];
      for (int s = 0; s < BST; ++s) armed[s] = -1;
      for (int tile = blockIdx.x; tile < p.ntiles && !*abort_flag; tile += gridDim.x) {
        for (int ch = 0; ch < nchunks; ++ch, ++it) {
          const int s = it % BST;
          const uint32_t ph = (it / BST) & 1u;
          if (!mbar_wait(b_empty(s), ph ^ 1u)) {
            fail(1);
            break;
          }
          if (*abort_flag) break;
          mbar_expect_tx(b_full(s), H_BCHUNK);
          bulk_load(smem_u32(smem + Cfg::B_OFF + s * H_BCHUNK), p.bsplit + (size_t)ch * H_BCHUNK, H_BCHUNK,
                    b_full(s));
          armed[s] = (int)ph;
        }
      }
      for (int s = 0; s < BST; ++s)
        if (armed[s] >= 0 && !mbar_wait(b_full(s), (uint32_t)armed[s])) atomicExch(p.err, 2);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t ait = 0, bit = 0, sit = 0, rit = 0;
      bool bad = false;
      for (int tile = blockIdx.x; tile < p.ntiles && !bad; tile += gridDim.x) {
        for (int ch = 0; ch < nchunks; ++ch, ++bit, ++sit) {
          const bool raw = ch == p.qch;
          const int bs = bit % BST, sl = sit % H_NSLOT;
          const uint32_t bph = (bit / BST) & 1u, sph = (sit / H_NSLOT) & 1u;
          const int as = raw ? (int)(rit % RST) : (int)(ait % AST);
          const uint32_t aph = raw ? ((rit / RST) & 1u) : ((ait / AST) & 1u);
          const bool ok = mbar_wait(slot_free(sl), sph ^ 1u) &&
                          mbar_wait(raw ? conv_full(as) : a_full(as), aph) && mbar_wait(b_full(bs), bph);
          if (!ok || *abort_flag) {
            fail(1);
            bad = true;
            break;
          }
          tc_fence_after();
          const uint32_t dslot = tmem_base + (uint32_t)(sl * H_N);
          const uint32_t ahi = smem_u32(smem + (raw ? Cfg::R_OFF + as * H_ACHUNK : as * H_ACHUNK));
          const uint32_t alo = ahi + H_PART;
          const uint32_t bhi = smem_u32(smem + Cfg::B_OFF + bs * H_BCHUNK);
          const uint32_t blo = bhi + H_BPART;
          if constexpr (Cfg::A_TMEM > 0) {
            // A into tensor memory once (tcgen05.cp, 128 rows x 16 K per copy), then
            // the MMAs read it there: the chunk crosses shared memory once, not three times
            const int ts = (int)(sit % Cfg::A_TMEM);
            const uint32_t tph = (sit / Cfg::A_TMEM) & 1u;
            if (!mbar_wait(atm_free(ts), tph ^ 1u)) {  // the MMAs of chunk sit - A_TMEM are done with it
              fail(1);
              bad = true;
              break;
            }
            tc_fence_after();
            const uint32_t ta = tmem_base + (uint32_t)(Cfg::A_COL0 + ts * 64);
#pragma unroll
            for (int kk = 0; kk < H_K / 16; ++kk) {
              tmem_cp_128x256b(ta + 8 * kk, umma_desc(ahi + kk * 2 * kALbo, kALbo, kASbo));
              tmem_cp_128x256b(ta + 32 + 8 * kk, umma_desc(alo + kk * 2 * kALbo, kALbo, kASbo));
            }
#pragma unroll
            for (int kk = 0; kk < H_K / 16; ++kk) {
              umma_f16_ts(dslot, ta + 8 * kk, umma_desc(blo + kk * 2 * kBLbo, kBLbo, kBSbo), kk != 0);
              umma_f16_ts(dslot, ta + 32 + 8 * kk, umma_desc(bhi + kk * 2 * kBLbo, kBLbo, kBSbo), 1u);
            }
#pragma unroll
            for (int kk = 0; kk < H_K / 16; ++kk)
              umma_f16_ts(dslot, ta + 8 * kk, umma_desc(bhi + kk * 2 * kBLbo, kBLbo, kBSbo), 1u);
            umma_commit(atm_free(ts));
          } else {
            // 4 K steps of 16: cross terms first, then the main products
#pragma unroll
            for (int kk = 0; kk < H_K / 16; ++kk) {
              umma_f16_ss(dslot, umma_desc(ahi + kk * 2 * kALbo, kALbo, kASbo),
                          umma_desc(blo + kk * 2 * kBLbo, kBLbo, kBSbo), kk != 0);
              umma_f16_ss(dslot, umma_desc(alo + kk * 2 * kALbo, kALbo, kASbo),
                          umma_desc(bhi + kk * 2 * kBLbo, kBLbo, kBSbo), 1u);
            }
#pragma unroll
            for (int kk = 0; kk < H_K / 16; ++kk)
              umma_f16_ss(dslot, umma_desc(ahi + kk * 2 * kALbo, kALbo, kASbo),
                          umma_desc(bhi + kk * 2 * kBLbo, kBLbo, kBSbo), 1u);
          }
          umma_commit(raw ? raw_empty(as) : a_empty(as));
          umma_commit(b_empty(bs));
          umma_commit(slot_full(sl));
          if (raw) ++rit;
          else ++ait;
        }
      }
      umma_commit(fin_bar);
      if (!mbar_wait(fin_bar, 0)) atomicExch(p.err, 3);
    }
  } else if (warp < 11) {
    // ----------------------------------------- raw chunk (warps 3..10)
    // Thread t splits rows r = t % 128 of column groups g = t / 128 + 2 q
    // (q = 0..3, 8 columns each): reads are conflict-free (consecutive rows),
    // writes are one 16-byte vector per part and group.
    const int t = threadIdx.x - 96;
    const int r = t & 127;
    const int g0 = t >> 7;
    uint32_t it = 0;
    bool stop = false;
    for (int tile = blockIdx.x; tile < p.ntiles && !stop; tile += gridDim.x, ++it) {
      const int s = (int)(it % RST);
      const uint32_t ph = (it / RST) & 1u;
      unsigned char* buf = smem + Cfg::R_OFF + s * H_ACHUNK;
      // one decision for all 256 converter threads (they meet at named barriers below)
      bool ok = mbar_wait(raw_full(s), ph);
      if (!ok) fail(1);
      ok = ok && !*abort_flag;
      uint32_t all_ok;
      asm volatile(
          "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n bar.red.and.pred po, 1, 256, pi;\n"
          " selp.u32 %0, 1, 0, po;\n}\n"
          : "=r"(all_ok)
          : "r"((uint32_t)ok)
          : "memory");
      if (!all_ok) {
        stop = true;
        break;
      }
      // all converter warps read before any writes (in-place split)
      const float* src = reinterpret_cast<const float*>(buf);
      float x[4][8];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int e = 0; e < 8; ++e) x[q][e] = src[(8 * (g0 + 2 * q) + e) * H_M + r];
      asm volatile("bar.sync 1, 256;" ::: "memory");
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int g = g0 + 2 * q;
        uint32_t hv[4], lv[4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
          unsigned short h0, l0, h1, l1;
          split_f16(x[q][e] * sm_scale[8 * g + e], h0, l0);
          split_f16(x[q][e + 1] * sm_scale[8 * g + e + 1], h1, l1);
          hv[e >> 1] = (uint32_t)h0 | ((uint32_t)h1 << 16);
          lv[e >> 1] = (uint32_t)l0 | ((uint32_t)l1 << 16);
        }
        const uint32_t off = a_off(r, 8 * g);
        *reinterpret_cast<uint4*>(buf + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
        *reinterpret_cast<uint4*>(buf + H_PART + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
      }
      // generic-proxy writes become visible to the tensor core (async proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(conv_full(s));
    }
    (void)stop;
  } else {
    // ----------------------------------------------- epilogue (warps 11..26)
    const int quarter = warp & 3;
    const int part = (warp - 11) >> 2;
    const uint32_t lane_off = (uint32_t)(32 * quarter) << 16;
    const int j0 = 16 * part;
    uint32_t it = 0;
    bool stop = false;
    const int r = 32 * quarter + lane;  // row in the tile == TMEM lane
    for (int tile = blockIdx.x; tile < p.ntiles && !stop; tile += gridDim.x) {
      float acc[16], cmp[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        acc[j] = 0.f;
        cmp[j] = 0.f;
      }
      for (int ch = 0; ch < nchunks; ++ch, ++it) {
        const int sl = it % H_NSLOT;
        const uint32_t sph = (it / H_NSLOT) & 1u;
        const bool ok = __all_sync(0xffffffffu, mbar_wait(slot_full(sl), sph));
        if (!ok && lane == 0) fail(1);
        if (!ok || __shfl_sync(0xffffffffu, (int)*abort_flag, 0)) {
          stop = true;
          break;
        }
        tc_fence_after();
        float v[16];
        tmem_ld16(tmem_base + lane_off + (uint32_t)(sl * H_N + j0), v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(slot_free(sl));
#pragma unroll
        for (int j = 0; j < 16; ++j) {  // Kahan-Babuska summation in FP32
          const float y = v[j] - cmp[j];
          const float tt = acc[j] + y;
          cmp[j] = (tt - acc[j]) - y;
          acc[j] = tt;
        }
      }
      if (stop) break;
      const int64_t row = (int64_t)tile * H_M + r;
      // TMEM column jt holds output column jt - jsh (the shift puts 8-column
      // groups of the split copy on 8-aligned columns of the basis)
      float q[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) q[j] = (acc[j] - cmp[j]) * sm_scale[64 + ((j0 + j) & 63)];
      if (row < p.n) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int jo = j0 + j - p.jsh;
          if (jo >= 0 && jo < p.mb) p.qout[row + (int64_t)jo * p.ldo] = q[j];
        }
      }
      if (p.qs_out) {
        // split copy of the new columns, then zeros up to the end of the last chunk they touch
        unsigned char* tb = p.qs_out + (size_t)tile * p.nch_row * H_ACHUNK;
        const int cend = p.cs_out + p.mb;
        const int tail_end = ((cend + H_K - 1) / H_K) * H_K;
        const int gbase = p.cs_out - p.jsh;  // basis column of TMEM column 0
        if (p.vec_split) {
          // gbase % 8 == 0: this thread's two 8-column groups are whole 16-byte vectors
#pragma unroll
          for (int g = 0; g < 2; ++g) {
            const int gc0 = gbase + j0 + 8 * g;
            if (gc0 + 8 <= p.cs_out || gc0 >= tail_end) continue;
            uint32_t hv[4], lv[4];
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
              unsigned short h[2] = {0, 0}, l[2] = {0, 0};
#pragma unroll
              for (int u = 0; u < 2; ++u) {
                const float v = q[8 * g + e + u] * kQScale;
                if (row < p.n && isfinite(v)) split_f16(v, h[u], l[u]);
              }
              hv[e >> 1] = (uint32_t)h[0] | ((uint32_t)h[1] << 16);
              lv[e >> 1] = (uint32_t)l[0] | ((uint32_t)l[1] << 16);
            }
            unsigned char* cb = tb + (size_t)(gc0 >> 6) * H_ACHUNK + a_off(r, gc0 & 63);
            if (gc0 >= p.cs_out) {
              *reinterpret_cast<uint4*>(cb) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
              *reinterpret_cast<uint4*>(cb + H_PART) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
            } else {
              // the group starts inside the previous block: store only this block's columns
#pragma unroll
              for (int e = 0; e < 8; ++e)
                if (gc0 + e >= p.cs_out) {
                  const uint32_t hw = hv[e >> 1] >> (16 * (e & 1)), lw = lv[e >> 1] >> (16 * (e & 1));
                  *reinterpret_cast<unsigned short*>(cb + 2 * e) = (unsigned short)hw;
                  *reinterpret_cast<unsigned short*>(cb + H_PART + 2 * e) = (unsigned short)lw;
                }
            }
          }
          // the rest of the tail (beyond the 64 columns held in TMEM)
          for (int gc0 = gbase + 64 + j0; gc0 < tail_end; gc0 += 64) {
#pragma unroll
            for (int g = 0; g < 2; ++g)
              if (gc0 + 8 * g < tail_end) {
                unsigned char* cb = tb + (size_t)((gc0 + 8 * g) >> 6) * H_ACHUNK + a_off(r, (gc0 + 8 * g) & 63);
                *reinterpret_cast<uint4*>(cb) = make_uint4(0u, 0u, 0u, 0u);
                *reinterpret_cast<uint4*>(cb + H_PART) = make_uint4(0u, 0u, 0u, 0u);
              }
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int jl = j0 + j;
            if (jl < p.mb) {
              unsigned short h = 0, l = 0;
              const float v = q[j] * kQScale;
              if (row < p.n && isfinite(v)) split_f16(v, h, l);
              const int gc = p.cs_out + jl;
              unsigned char* cb = tb + (size_t)(gc >> 6) * H_ACHUNK + a_off(r, gc & 63);
              *reinterpret_cast<unsigned short*>(cb) = h;
              *reinterpret_cast<unsigned short*>(cb + H_PART) = l;
            }
          }
          for (int gc = cend + j0; gc < tail_end; gc += 64) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int c2 = gc + j;
              if (c2 < tail_end) {
                unsigned char* cb = tb + (size_t)(c2 >> 6) * H_ACHUNK + a_off(r, c2 & 63);
                *reinterpret_cast<unsigned short*>(cb) = 0;
                *reinterpret_cast<unsigned short*>(cb + H_PART) = 0;
              }
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(H_TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------- scales --
// One CTA.  Raw column scales from the sketch of the raw block (k x mb,
// column norms ~ the columns' 2-norms) or from given column maxima; output
// column scales t_j from max_k |G_kj| / s_k.  out[0, 64) = s_raw,
// out[64, 128) = 1 / t, out[128, 192) = t.
__device__ __forceinline__ float pow2_scale_for(double v, int target_exp) {
  // 2^(target - e) with 2^(e - 1) <= v < 2^e; 1 for v = 0 or not finite
  if (!(v > 0.0) || !isfinite(v)) return 1.f;
  int e;
  frexp(v, &e);
  int s = target_exp - e;
  s = max(-120, min(120, s));
  return ldexpf(1.f, s);
}

// Per column j (one CTA each): the raw scale s_j from the 2-norm of column j
// of the raw block's sketch (or from the column maximum), and the largest
// |G_kj| / s_k over the basis rows k < c.  tmp[j] = s_raw, tmp[64 + j] = that maximum.
template <class TS>
__global__ void __launch_bounds__(256) h3_colscale_kernel(int64_t c, int mb, const double* __restrict__ G,
                                                          int64_t ldg, const TS* __restrict__ Sraw, int64_t k,
                                                          int64_t lds, const float* __restrict__ rawmax,
                                                          const float* __restrict__ qscale, float* __restrict__ tmp,
                                                          const int* active) {
  if (active && *active == 0) return;
  __shared__ double red[8];
  const int j = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (j >= mb) {
    if (tid == 0) {
      tmp[j] = 1.f;
      tmp[64 + j] = 0.f;
    }
    return;
  }
  double sraw;
  if (rawmax) {
    sraw = (double)pow2_scale_for((double)rawmax[j], 9);
  } else {
    double ss = 0.0;
    const TS* col = Sraw + (int64_t)j * lds;
    for (int64_t r = tid; r < k; r += 256) {
      const double v = (double)col[r];
      ss += v * v;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (lane == 0) red[warp] = ss;
    __syncthreads();
    double tot = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) tot += red[w];
    sraw = (double)pow2_scale_for(sqrt(tot), 9);
    __syncthreads();
  }
  double mx = 0.0;
  const double* gcol = G + (int64_t)j * ldg;
  for (int64_t r = tid; r < c; r += 256) mx = fmax(mx, fabs(gcol[r]) / (qscale ? (double)qscale[r] : (double)kQScale));
#pragma unroll
  for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) red[warp] = mx;
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) m = fmax(m, red[w]);
    tmp[j] = (float)sraw;
    tmp[64 + j] = (float)m;
  }
}

// Output column scales t_j from the basis maxima and the raw rows of G;
// out[0, 64) = s_raw, out[64, 128) = 1 / t, out[128, 192) = t, the t at the
// shifted (TMEM / B) column index.
__global__ void __launch_bounds__(256) h3_tscale_kernel(int64_t c, int mb, int jsh, const double* __restrict__ G,
                                                        int64_t ldg, const float* __restrict__ tmp,
                                                        float* __restrict__ out, const int* active) {
  if (active && *active == 0) return;
  __shared__ double inv_s[64];
  __shared__ double red[4][64];
  __shared__ float tj[64];
  const int tid = threadIdx.x, j = tid & 63, part = tid >> 6;
  if (tid < 64) inv_s[tid] = 1.0 / (double)tmp[tid];  // powers of two: exact
  __syncthreads();
  double mx = part == 0 ? (double)tmp[64 + j] : 0.0;
  if (j < mb) {
    const double* gcol = G + (int64_t)j * ldg + c;
    for (int r = part; r < mb; r += 4) mx = fmax(mx, fabs(gcol[r]) * inv_s[r]);
  }
  red[part][j] = mx;
  __syncthreads();
  if (tid < 64) {
    const double m = fmax(fmax(red[0][tid], red[1][tid]), fmax(red[2][tid], red[3][tid]));
    tj[tid] = tid < mb ? pow2_scale_for(m, 9) : 1.f;
  }
  __syncthreads();
  if (tid < 64) {
    const int jo = tid - jsh;
    const float tt = (jo >= 0 && jo < mb) ? tj[jo] : 1.f;
    out[tid] = tmp[tid];
    out[64 + tid] = 1.f / tt;
    out[128 + tid] = tt;
  }
}

// B chunks: chunk ch < qch holds G rows 64 ch + kk of the Q part (zero at and
// beyond c), chunk qch the mb raw rows c + kk; value t_j g / s_k split into
// fp16 hi (bytes [0, 8K)) and lo ([8K, 16K)) in the K-major core layout.
__global__ void h3_fill_b_kernel(int64_t c, int mb, int qch, int jsh, const double* __restrict__ G, int64_t ldg,
                                 const float* __restrict__ qscale, const float* __restrict__ sc,
                                 unsigned char* __restrict__ B, const int* active) {
  if (active && *active == 0) return;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)H_N * H_K;
  if (idx >= (int64_t)(qch + 1) * per) return;
  const int ch = (int)(idx / per);
  const int e = (int)(idx % per);
  const int j = e / H_K, kk = e % H_K;  // j: B (TMEM) column; output column j - jsh
  const int jo = j - jsh;
  double v = 0.0;
  if (jo >= 0 && jo < mb) {
    if (ch < qch) {
      const int64_t kr = (int64_t)ch * H_K + kk;
      if (kr < c)
        v = G[kr + (int64_t)jo * ldg] * (double)sc[128 + j] / (qscale ? (double)qscale[kr] : (double)kQScale);
    } else if (kk < mb) {
      v = G[c + kk + (int64_t)jo * ldg] * (double)sc[128 + j] / (double)sc[kk];
    }
  }
  const __half h = __double2half(v);
  const __half l = __double2half(v - (double)__half2float(h));
  const uint32_t off = (uint32_t)((kk >> 3) * 1024 + (j >> 3) * 128 + (j & 7) * 16 + (kk & 7) * 2);
  unsigned char* cb = B + (size_t)ch * H_BCHUNK;
  *reinterpret_cast<unsigned short*>(cb + off) = __half_as_ushort(h);
  *reinterpret_cast<unsigned short*>(cb + H_BPART + off) = __half_as_ushort(l);
}

// Column maxima |A_ij| over the rows (as ordered unsigned bits), for the
// stand-alone entry point whose basis carries no sketch.
__global__ void h3_colmax_kernel(int64_t n, int64_t cols, const float* __restrict__ A, int64_t lda,
                                 unsigned int* __restrict__ out) {
  const int64_t j = blockIdx.y;
  float m = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(A[i + j * lda]));
#pragma unroll
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out + j, __float_as_uint(m));
}

// Per-column power-of-two scales from column maxima (2^9 > s max >= 2^8).
__global__ void h3_scale_from_max_kernel(int64_t cols, const unsigned int* __restrict__ mx,
                                         float* __restrict__ scale) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < cols) scale[j] = pow2_scale_for((double)__uint_as_float(mx[j]), 9);
}

// Split A (n x cols, FP32, column-major) into the tiled fp16 hi/lo layout with
// per-column scales; columns [cols, 64 ceil(cols / 64)) and rows >= n are zero.
__global__ void h3_split_kernel(int64_t n, int64_t cols, const float* __restrict__ A, int64_t lda,
                                const float* __restrict__ scale, int nch_row, int64_t ntiles, int64_t groups,
                                unsigned char* __restrict__ qs) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = ntiles * H_M * groups;
  if (idx >= total) return;
  const int64_t rowg = idx % (ntiles * H_M);  // consecutive threads: consecutive rows
  const int64_t gi = idx / (ntiles * H_M);
  const int64_t tile = rowg / H_M;
  const int r = (int)(rowg % H_M);
  uint32_t hv[4], lv[4];
#pragma unroll
  for (int e = 0; e < 8; e += 2) {
    unsigned short h[2] = {0, 0}, l[2] = {0, 0};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t col = gi * 8 + e + u;
      if (rowg < n && col < cols) split_f16(A[rowg + col * lda] * scale[col], h[u], l[u]);
    }
    hv[e >> 1] = (uint32_t)h[0] | ((uint32_t)h[1] << 16);
    lv[e >> 1] = (uint32_t)l[0] | ((uint32_t)l[1] << 16);
  }
  const int64_t ch = gi >> 3;
  const int kk = (int)((gi & 7) * 8);
  unsigned char* cb = qs + ((size_t)tile * nch_row + (size_t)ch) * H_ACHUNK + a_off(r, kk);
  *reinterpret_cast<uint4*>(cb) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
  *reinterpret_cast<uint4*>(cb + H_PART) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode_h3() {
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

// 2-D map over the raw block (n x mb FP32, column-major), box 128 rows x 64
// columns; columns >= mb and rows >= n read as zero.
bool make_raw_map(CUtensorMap* map, const float* base, int64_t n, int64_t mb, int64_t ld) {
  auto enc = get_encode_h3();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)mb};
  cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  cuuint32_t box[2] = {H_M, H_K};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// TMEM slots of the long-K configuration; RBGS_H3_SLOTS=8 selects eight
// (for tuning measurements).
int h3_slots() {
  static int v = []() {
    const char* e = getenv("RBGS_H3_SLOTS");
    return e ? atoi(e) : 4;
  }();
  return v;
}

// RBGS_H3_ATMEM=1: A through tensor memory (tcgen05.cp) in the long-K shape.
int h3_a_tmem() {
  static int v = []() {
    const char* e = getenv("RBGS_H3_ATMEM");
    return e ? atoi(e) : 0;
  }();
  return v;
}

}  // namespace

int64_t h3_nch_row(int64_t m) { return (m + H_K - 1) / H_K; }
size_t h3_qs_bytes(int64_t n, int64_t m) {
  return (size_t)((n + H_M - 1) / H_M) * (size_t)h3_nch_row(m) * H_ACHUNK;
}
size_t h3_b_bytes(int64_t c) { return (size_t)((c + H_K - 1) / H_K + 1) * H_BCHUNK; }

int h3_shift(int64_t cs_out, int64_t mb, bool split_out) {
  const int d = (int)(cs_out % 8);
  return (split_out && mb + d <= H_N) ? d : 0;
}

template <class TS>
rbgs_status h3_prepare(int64_t c, int64_t mb, const double* G, int64_t ldg, const TS* Sraw, int64_t k,
                       const float* rawmax, const float* qscale, int jsh, unsigned char* B, float* scales,
                       const int* active, cudaStream_t st) {
  if (mb < 1 || mb > H_N || c < 0 || jsh < 0 || mb + jsh > H_N) return RBGS_EINVAL;
  // scales[192, 320) is scratch for the per-column pass
  h3_colscale_kernel<TS><<<64, 256, 0, st>>>(c, (int)mb, G, ldg, Sraw, k, k, rawmax, qscale, scales + 192, active);
  RBGS_LAUNCH_CHECK();
  h3_tscale_kernel<<<1, 256, 0, st>>>(c, (int)mb, jsh, G, ldg, scales + 192, scales, active);
  RBGS_LAUNCH_CHECK();
  const int qch = (int)((c + H_K - 1) / H_K);
  const int64_t tot = (int64_t)(qch + 1) * H_N * H_K;
  h3_fill_b_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(c, (int)mb, qch, jsh, G, ldg, qscale, scales,
                                                                  B, active);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}
template rbgs_status h3_prepare<float>(int64_t, int64_t, const double*, int64_t, const float*, int64_t, const float*,
                                       const float*, int, unsigned char*, float*, const int*, cudaStream_t);
template rbgs_status h3_prepare<double>(int64_t, int64_t, const double*, int64_t, const double*, int64_t,
                                        const float*, const float*, int, unsigned char*, float*, const int*,
                                        cudaStream_t);

rbgs_status h3_colmax(int64_t n, int64_t cols, const float* A, int64_t lda, unsigned int* mx, cudaStream_t st) {
  if (cols == 0) return RBGS_OK;
  if (cols > 65535) return RBGS_EINVAL;
  RBGS_CUDA_TRY(cudaMemsetAsync(mx, 0, sizeof(unsigned int) * cols, st));
  dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 64), (unsigned)cols);
  h3_colmax_kernel<<<grid, 256, 0, st>>>(n, cols, A, lda, mx);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}

rbgs_status h3_scales_from_max(int64_t cols, const unsigned int* mx, float* scale, cudaStream_t st) {
  if (cols == 0) return RBGS_OK;
  h3_scale_from_max_kernel<<<(unsigned)((cols + 255) / 256), 256, 0, st>>>(cols, mx, scale);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}

rbgs_status h3_split(int64_t n, int64_t cols, const float* A, int64_t lda, const float* scale, int64_t nch_row,
                     unsigned char* qs, cudaStream_t st) {
  const int64_t ntiles = (n + H_M - 1) / H_M;
  const int64_t nchc = (cols + H_K - 1) / H_K;
  if (nchc > nch_row) return RBGS_EINVAL;
  const int64_t total = ntiles * H_M * nchc * 8;
  if (total == 0) return RBGS_OK;
  h3_split_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(n, cols, A, lda, scale, (int)nch_row, ntiles,
                                                                   nchc * 8, qs);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}

rbgs_status tall_update_h3(int64_t n, int64_t c, int64_t mb, const unsigned char* qs, int64_t nch_row,
                           const float* raw, int64_t ldr, const unsigned char* B, const float* scales, float* Qout,
                           int64_t ldo, unsigned char* qs_out, int64_t cs_out, int jsh, const int* active, int* err,
                           cudaStream_t st) {
  if (mb < 1 || mb > H_N || n < 1 || n >= ((int64_t)1 << 31) || c < 0 || !err) return RBGS_EINVAL;
  if (((uintptr_t)raw & 15) || (ldr % 4)) return RBGS_EINVAL;
  if (jsh < 0 || mb + jsh > H_N || (jsh && !qs_out)) return RBGS_EINVAL;
  const int qch = (int)((c + H_K - 1) / H_K);
  if (qch > 0 && (!qs || qch > nch_row)) return RBGS_EINVAL;
  if (qs_out && (cs_out + mb > nch_row * H_K || cs_out < jsh)) return RBGS_EINVAL;
  CUtensorMap mr;
  std::memset(&mr, 0, sizeof(mr));
  if (!make_raw_map(&mr, raw, n, mb, ldr)) return RBGS_ECUDA;
  int dev = 0, nsm = 0;
  RBGS_CUDA_TRY(cudaGetDevice(&dev));
  RBGS_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  H3Params p{};
  p.n = n;
  p.c = (int)c;
  p.mb = (int)mb;
  p.qch = qch;
  p.ntiles = (int)((n + H_M - 1) / H_M);
  p.nch_row = (int)nch_row;
  p.qs = qs;
  p.bsplit = B;
  p.scales = scales;
  p.qout = Qout;
  p.ldo = ldo;
  p.qs_out = qs_out;
  p.cs_out = (int)cs_out;
  p.jsh = jsh;
  p.vec_split = qs_out && ((cs_out - jsh) % 8 == 0) && (mb + jsh <= H_N);
  p.active = active;
  p.err = err;
  const int grid = std::min(p.ntiles, nsm);
  // pipeline shape by the share of raw chunks: few or no basis chunks per
  // tile want deeper raw staging, long K loops deeper basis staging
  auto go = [&](auto cfg) -> rbgs_status {
    using Cfg = decltype(cfg);
    RBGS_CUDA_TRY(
        cudaFuncSetAttribute(tall_h3_kernel<Cfg>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM_BYTES));
    tall_h3_kernel<Cfg><<<grid, H_THREADS, Cfg::SMEM_BYTES, st>>>(mr, p);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
  };
  if (qch == 0) return go(H3Cfg<1, 2, 2>{});
  if (qch <= 2) return go(H3Cfg<3, 2, 2>{});
  if (h3_slots() == 8) return go(H3Cfg<4, 1, 3, 8>{});
  if (h3_a_tmem() == 2) return go(H3Cfg<4, 1, 3, 4, 2>{});
  if (h3_a_tmem() == 4) return go(H3Cfg<4, 1, 3, 4, 4>{});
  return go(H3Cfg<4, 1, 3>{});
}

}  // namespace rbgs
