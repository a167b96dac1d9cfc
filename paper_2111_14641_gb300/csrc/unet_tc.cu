// Tensor-core 3 x 3 convolution of the U-Net preconditioner on sm_103a
// (tcgen05 kind::f16 with bfloat16 operands, FP32 accumulators in tensor
// memory, TMA halo tiles): the implicit GEMM
//
//   out[p][co] = sum over taps t and input channels ci of in[p + off(t)][ci] * w[t][ci][co]
//
// with M = 128 output pixels (one 128-pixel segment of an image row), N =
// Cout (16..128) and K = 9 Cin taken 16 input channels ("slice") at a time:
// per slice the nine taps are nine MMAs of K = 16 on shifted windows of one
// halo tile.
//
// Halo tile of a slice: two TMA boxes (8 channels x 130 pixels x 3 rows each,
// one per group of 8 channels) of the NHWC bfloat16 input; rows and columns
// outside the image read as zero (the convolution's zero padding).  In shared
// memory a box is [row][pixel][8 channels], 16 bytes per pixel, so pixels
// are the rows of 8 x 16-byte core matrices: the A operand of tap (ox, oy)
// starts at byte (oy 130 + ox) 16 of the tile (core matrices 128 bytes apart
// along M, the second channel group one box, 6240 bytes, away along K).
// Weights: packed once per call into the B operand layout, per slice and tap
// a Cout x 16 block (K-major core matrices), copied with one bulk copy per
// slice.
//
// Persistent kernel, one CTA per SM over (image, row, 128-pixel segment)
// tiles; warp 0 issues the copies, warp 1 owns tensor memory and issues the
// MMAs, warps 2-5 drain the accumulators (bias, ReLU, bfloat16 or FP32
// stores).  Two accumulators in tensor memory let the MMAs of one tile run
// while the previous tile is drained.  Every mbarrier wait is bounded (2 s of
// %globaltimer): on expiry the kernel records an error flag, waits for its
// own copies and MMAs, frees tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace rbgs {
namespace {

constexpr int CT_M = 128;                  // output pixels per tile
constexpr int CT_HALO = CT_M + 2;          // halo pixels per row
constexpr int CT_BOX = 8 * CT_HALO * 3 * 2;  // bytes of one TMA box: 8 ch x 130 px x 3 rows, bf16 = 6240
constexpr int CT_BOX_STRIDE = 6272;        // the second box of a slice starts 128-byte aligned
constexpr int CT_HALO_BYTES = CT_BOX_STRIDE + CT_BOX;  // one halo stage: 12512 bytes
constexpr int CT_STAGE = 12544;            // stage stride (a multiple of 128)
constexpr int CT_THREADS = 192;            // 6 warps
constexpr uint64_t kCtWaitNs = 2000000000ull;
constexpr uint32_t kCtSuspendNs = 100000u;

__device__ __forceinline__ uint32_t ct_smem(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void ct_bar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void ct_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void ct_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool ct_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(kCtSuspendNs)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t ct_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool ct_wait(uint32_t bar, uint32_t parity) {
  if (ct_try(bar, parity)) return true;
  const uint64_t t0 = ct_ns();
  for (;;) {
    if (ct_try(bar, parity)) return true;
    if (ct_ns() - t0 > kCtWaitNs) return false;
  }
}
__device__ __forceinline__ void ct_tma_4d(uint32_t dst, const CUtensorMap* map, int c, int x, int y, int b,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c), "r"(x), "r"(y), "r"(b), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void ct_bulk(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// Shared-memory matrix descriptor, K-major without swizzle.
__device__ __forceinline__ uint64_t ct_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// kind::f16 instruction descriptor: D = F32 (bits 4-5), A = B = BF16 (bits 7-9
// and 10-12), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t ct_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(CT_M >> 4) << 24);
}
__device__ __forceinline__ void ct_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void ct_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void ct_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void ct_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void ct_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct ConvTcParams {
  int N, batch, cin, cout, relu, out_bf16;
  int64_t ld_out;
  int off_out;
  int ntiles, nseg, nslice, stages, wslice_bytes, wbytes;
  const unsigned char* wpack;  // packed weights, nslice x wslice_bytes
  const float* bias;           // or null
  void* out;
  int* err;
};

// Shared memory: the layer's packed weights (resident, loaded once), then
// `stages` halo stages, then the barriers.
template <int MAXST>
__global__ void __launch_bounds__(CT_THREADS, 1)
    conv3x3_tc_kernel(const __grid_constant__ CUtensorMap tmIn, ConvTcParams p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int ST = p.stages;
  unsigned char* halo0 = smem + p.wbytes;
  unsigned char* barea = halo0 + (size_t)ST * CT_STAGE;
  const uint32_t bar0 = ct_smem(barea);
  auto full = [&](int s) { return bar0 + 8u * s; };                       // MAXST
  auto empty = [&](int s) { return bar0 + 8u * (MAXST + s); };            // MAXST
  auto acc_full = [&](int s) { return bar0 + 8u * (2 * MAXST + s); };     // 2
  auto acc_empty = [&](int s) { return bar0 + 8u * (2 * MAXST + 2 + s); };  // 2
  const uint32_t fin = bar0 + 8u * (2 * MAXST + 4);
  const uint32_t wfull = bar0 + 8u * (2 * MAXST + 5);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(barea + 8 * (2 * MAXST + 6));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(barea + 8 * (2 * MAXST + 6) + 8);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      ct_bar_init(full(s), 1);
      ct_bar_init(empty(s), 1);
    }
    for (int s = 0; s < 2; ++s) {
      ct_bar_init(acc_full(s), 1);
      ct_bar_init(acc_empty(s), 4);  // the four epilogue warps
    }
    ct_bar_init(fin, 1);
    ct_bar_init(wfull, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(ct_smem(tmem_slot)),
                 "r"(256)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  ct_fence_before();
  __syncthreads();
  ct_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  auto fail = [&](int code) {
    *abort_flag = 1;
    atomicExch(p.err, code);
  };

  if (warp == 0) {
    // --------------------------------------------------------- copy producer
    if (lane == 0) {
      // the weights, once
      ct_expect_tx(wfull, (uint32_t)(p.nslice * p.wslice_bytes));
      for (int sl = 0; sl < p.nslice; ++sl)
        ct_bulk(ct_smem(smem + (size_t)sl * p.wslice_bytes), p.wpack + (size_t)sl * p.wslice_bytes,
                (uint32_t)p.wslice_bytes, wfull);
      uint32_t it = 0;
      int armed[MAXST];
      for (int s = 0; s < MAXST; ++s) armed[s] = -1;
      bool bad = false;
      for (int tile = blockIdx.x; tile < p.ntiles && !bad; tile += gridDim.x) {
        const int seg = tile % p.nseg;
        const int row = (tile / p.nseg) % p.N;
        const int img = tile / (p.nseg * p.N);
        for (int sl = 0; sl < p.nslice; ++sl, ++it) {
          const int s = (int)(it % (uint32_t)ST);
          const uint32_t ph = (it / (uint32_t)ST) & 1u;
          if (!ct_wait(empty(s), ph ^ 1u) || *abort_flag) {
            fail(1);
            bad = true;
            break;
          }
          unsigned char* st = halo0 + (size_t)s * CT_STAGE;
          ct_expect_tx(full(s), (uint32_t)(2 * CT_BOX));
          ct_tma_4d(ct_smem(st), &tmIn, 16 * sl, CT_M * seg - 1, row - 1, img, full(s));
          ct_tma_4d(ct_smem(st + CT_BOX_STRIDE), &tmIn, 16 * sl + 8, CT_M * seg - 1, row - 1, img, full(s));
          armed[s] = (int)ph;
        }
      }
      // never leave with copies in flight into this CTA's shared memory
      if (!ct_wait(wfull, 0)) atomicExch(p.err, 2);
      for (int s = 0; s < ST; ++s)
        if (armed[s] >= 0 && !ct_wait(full(s), (uint32_t)armed[s])) atomicExch(p.err, 2);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = ct_idesc(p.cout);
      const uint32_t lbo_b = (uint32_t)(16 * p.cout), blk_b = (uint32_t)(32 * p.cout);
      uint32_t it = 0, tcount = 0;
      bool bad = !ct_wait(wfull, 0);
      if (bad) fail(1);
      for (int tile = blockIdx.x; tile < p.ntiles && !bad; tile += gridDim.x, ++tcount) {
        const int ab = (int)(tcount & 1u);
        const uint32_t aph = (tcount >> 1) & 1u;
        if (!ct_wait(acc_empty(ab), aph ^ 1u) || *abort_flag) {
          fail(1);
          break;
        }
        ct_fence_after();
        const uint32_t dacc = tmem_base + (uint32_t)(ab * 128);
        for (int sl = 0; sl < p.nslice; ++sl, ++it) {
          const int s = (int)(it % (uint32_t)ST);
          const uint32_t ph = (it / (uint32_t)ST) & 1u;
          if (!ct_wait(full(s), ph) || *abort_flag) {
            fail(1);
            bad = true;
            break;
          }
          ct_fence_after();
          const uint32_t halo = ct_smem(halo0 + (size_t)s * CT_STAGE);
          const uint32_t wts = ct_smem(smem + (size_t)sl * p.wslice_bytes);
#pragma unroll
          for (int ox = 0; ox < 3; ++ox)
#pragma unroll
            for (int oy = 0; oy < 3; ++oy) {
              const int tap = 3 * ox + oy;
              const uint64_t ad = ct_desc(halo + (uint32_t)((oy * CT_HALO + ox) * 16), CT_BOX_STRIDE, 128);
              const uint64_t bd = ct_desc(wts + (uint32_t)tap * blk_b, lbo_b, 128);
              ct_mma(dacc, ad, bd, idesc, (sl > 0 || tap > 0) ? 1u : 0u);
            }
          ct_commit(empty(s));
        }
        if (bad) break;
        ct_commit(acc_full(ab));
      }
      ct_commit(fin);
      if (!ct_wait(fin, 0)) atomicExch(p.err, 3);
    }
  } else {
    // ------------------------------------------------ epilogue (warps 2..5)
    const int quarter = warp & 3;                 // TMEM lanes 32 quarter .. + 31
    const uint32_t lane_off = (uint32_t)(32 * quarter) << 16;
    const int r = 32 * quarter + lane;            // pixel of the tile
    uint32_t tcount = 0;
    for (int tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x, ++tcount) {
      const int ab = (int)(tcount & 1u);
      const uint32_t aph = (tcount >> 1) & 1u;
      const bool ok = __all_sync(0xffffffffu, ct_wait(acc_full(ab), aph));
      if (!ok && lane == 0) fail(1);
      if (!ok || __shfl_sync(0xffffffffu, (int)*abort_flag, 0)) break;
      ct_fence_after();
      const int seg = tile % p.nseg;
      const int row = (tile / p.nseg) % p.N;
      const int img = tile / (p.nseg * p.N);
      const int64_t pix = ((int64_t)img * p.N + row) * p.N + (int64_t)CT_M * seg + r;
      for (int c0 = 0; c0 < p.cout; c0 += 16) {
        float v[16];
        ct_ld16(tmem_base + lane_off + (uint32_t)(ab * 128 + c0), v);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          float t = v[j] + (p.bias ? p.bias[c0 + j] : 0.f);
          if (p.relu) t = fmaxf(t, 0.f);
          v[j] = t;
        }
        if (p.out_bf16) {
          __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(p.out) + pix * p.ld_out + p.off_out + c0;
          uint32_t w[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
            w[j] = *reinterpret_cast<const uint32_t*>(&h);
          }
          uint4* o4 = reinterpret_cast<uint4*>(o);
          o4[0] = make_uint4(w[0], w[1], w[2], w[3]);
          o4[1] = make_uint4(w[4], w[5], w[6], w[7]);
        } else {
          float4* o4 = reinterpret_cast<float4*>(reinterpret_cast<float*>(p.out) + pix * p.ld_out + p.off_out + c0);
#pragma unroll
          for (int j = 0; j < 4; ++j) o4[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
      }
      ct_fence_before();
      __syncwarp();
      if (lane == 0) ct_arrive(acc_empty(ab));
    }
  }
  __syncthreads();
  ct_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(256) : "memory");
}

// Packed B operand: per slice s (input channels 16 s .. 16 s + 15) and tap t
// a block of 32 Cout bytes, element (kk, co) at (kk / 8) 16 Cout + (co / 8) 128 +
// (co % 8) 16 + (kk % 8) 2, value w[t][16 s + kk][co] (w: FP32 [9][Cin][Cout];
// flip != 0 packs the backward convolution's weights w[8 - t][co][ci] with the
// roles of Cin and Cout exchanged).
__global__ void conv_pack_kernel(int cin, int cout, const float* __restrict__ w, int flip,
                                 __nv_bfloat16* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 9LL * cin * cout) return;
  const int co = (int)(t % cout);
  const int ci = (int)((t / cout) % cin);
  const int tap = (int)(t / ((int64_t)cin * cout));
  float v;
  if (flip) v = w[((int64_t)(8 - tap) * cout + co) * cin + ci];  // original layer: [9][cout][cin] as [tap][ci'][co']
  else v = w[((int64_t)tap * cin + ci) * cout + co];
  const int s = ci >> 4, kk = ci & 15;
  const int64_t byte = (int64_t)s * 288 * cout + (int64_t)tap * 32 * cout + (kk >> 3) * 16 * cout + (co >> 3) * 128 +
                       (co & 7) * 16 + (kk & 7) * 2;
  out[byte / 2] = __float2bfloat16_rn(v);
}

PFN_cuTensorMapEncodeTiled_v12000 ct_encode() {
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

constexpr int kCtMaxStages = 4;

}  // namespace

bool conv_tc_supported(int N, int cin, int cout, int64_t ld_in, int off_in, int64_t ld_out, int off_out) {
  return N >= CT_M && N % CT_M == 0 && cin % 16 == 0 && cin >= 16 && cout % 16 == 0 && cout >= 16 && cout <= 128 &&
         ld_in % 8 == 0 && off_in % 8 == 0 && ld_out % 8 == 0 && off_out % 8 == 0;
}

size_t conv_tc_pack_bytes(int cin, int cout) { return (size_t)18 * cin * cout; }

rbgs_status conv_tc_pack(int cin, int cout, const float* w, int flip, void* packed, cudaStream_t st) {
  const int64_t tot = 9LL * cin * cout;
  conv_pack_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(cin, cout, w, flip, (__nv_bfloat16*)packed);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}

// out = conv3x3(in) on the tensor cores; in: bfloat16 NHWC (channel stride
// ld_in, channels [off_in, off_in + cin)); packed: conv_tc_pack's weights;
// out: bfloat16 (out_bf16) or FP32, channel stride ld_out, offset off_out.
rbgs_status conv_tc(int N, int batch, int cin, int cout, const void* in, int64_t ld_in, int off_in, const void* packed,
                    const float* bias, int relu, void* out, int out_bf16, int64_t ld_out, int off_out, int* err,
                    cudaStream_t st) {
  if (!conv_tc_supported(N, cin, cout, ld_in, off_in, ld_out, off_out) || batch < 1 || !err) return RBGS_EINVAL;
  if (((uintptr_t)in & 15) || ((uintptr_t)packed & 15) || ((uintptr_t)out & 15)) return RBGS_EINVAL;
  auto enc = ct_encode();
  if (!enc) return RBGS_ECUDA;
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  // 4-D map over the input: (channel, x, y, image); the base includes the channel offset
  const __nv_bfloat16* base = reinterpret_cast<const __nv_bfloat16*>(in) + off_in;
  cuuint64_t dims[4] = {(cuuint64_t)cin, (cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)batch};
  cuuint64_t strides[3] = {(cuuint64_t)ld_in * 2, (cuuint64_t)ld_in * 2 * N, (cuuint64_t)ld_in * 2 * N * N};
  cuuint32_t box[4] = {8, (cuuint32_t)CT_HALO, 3, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)base, dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return RBGS_ECUDA;
  ConvTcParams p{};
  p.N = N;
  p.batch = batch;
  p.cin = cin;
  p.cout = cout;
  p.relu = relu;
  p.out_bf16 = out_bf16;
  p.ld_out = ld_out;
  p.off_out = off_out;
  p.nseg = N / CT_M;
  p.ntiles = batch * N * p.nseg;
  p.nslice = cin / 16;
  p.wslice_bytes = 288 * cout;
  p.wbytes = (p.nslice * p.wslice_bytes + 1023) / 1024 * 1024;
  const int budget = 227 * 1024 - 1024 - 256;
  p.stages = std::min(kCtMaxStages, (budget - p.wbytes) / CT_STAGE);
  if (p.stages < 2) return RBGS_EINVAL;
  p.wpack = reinterpret_cast<const unsigned char*>(packed);
  p.bias = bias;
  p.out = out;
  p.err = err;
  // at least 120 KB, so that no SM holds two of these CTAs (each allocates 256
  // tensor-memory columns and stays resident for the whole launch)
  const int smem = std::max(p.wbytes + p.stages * CT_STAGE + 256 + 1024, 120 * 1024);
  int dev = 0, nsm = 0;
  RBGS_CUDA_TRY(cudaGetDevice(&dev));
  RBGS_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  RBGS_CUDA_TRY(cudaFuncSetAttribute(conv3x3_tc_kernel<kCtMaxStages>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem));
  const int grid = std::min(p.ntiles, nsm);
  conv3x3_tc_kernel<kCtMaxStages><<<grid, CT_THREADS, smem, st>>>(map, p);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}

}  // namespace rbgs
