// The learned right preconditioner of randomized block flexible GMRES: an
// L-level U-Net on single-channel N x N images (the residual columns of a
// diffusion problem on an N x N grid), with its forward and backward passes,
// the residual-norm training loss and the Adam update.  None of this is in
// the paper, which preconditions its block GMRES with ILU(0); the Krylov
// layer it serves is the paper's (Alg. 7, Sec. 5.2).
//
// Network (widths c_0 .. c_{L-1}; level l at N / 2^l):
//   encoder l = 0 .. L-1:  a_l = relu(conv(x_l)),  s_l = relu(conv(a_l)),
//                          x_0 = input (1 channel), x_{l+1} = avgpool2(s_l)
//   decoder l = L-2 .. 0:  d_l = relu(conv([upsample2(d_{l+1}); s_l])),  d_{L-1} = s_{L-1}
//   output:                y = conv(d_0)  (c_0 -> 1, linear)
// All convolutions are 3 x 3 with zero padding (cross-correlation).
//
// Precision: activations are stored in bfloat16 and every convolution takes
// bfloat16 operands (its input, rounded on load when that input is FP32, and
// its weights) with FP32 accumulation; biases, the output y, gradients, the
// loss and the optimiser state are FP32.
//
// Layouts.  Image b of a batch is column b of an n = N^2 column-major block
// (pixel (ix, iy) at ix + N iy).  Activations are pixel-major with channels
// innermost: channel ch of pixel p of image b at ((b N^2 + p) ld + off + ch).
// Parameters are one FP32 vector, layer after layer in evaluation order
// (enc0a, enc0b, enc1a, ..., enc{L-1}b, dec{L-2}, ..., dec0, out), each as
// w[tap][ci][co] (tap = 3 ox + oy, ox / oy in {0, 1, 2} the offset + 1 along
// ix / iy) followed by b[co].
//
// Convolutions run on the tensor cores (unet_tc.cu: tcgen05 with bfloat16
// operands and FP32 accumulators) at the levels whose rows are multiples of
// 128 pixels and whose channel counts are multiples of 16, for the forward
// pass and the backward convolution of the input gradient; elsewhere (the
// one-channel input and output layers, the small levels) and for the weight
// gradients they run as direct SIMT kernels (FP32 FMA on bfloat16 operands:
// each CTA computes an 8 x 64-pixel tile for 16 output channels, staging 8
// input channels at a time in shared memory).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace rbgs {
namespace {

constexpr int kTY = 8, kTX = 64;   // output tile: 8 rows x 64 pixels (2 per thread)
constexpr int kCIC = 8;            // input channels staged per step
constexpr int kCOT = 16;           // output channels per CTA
constexpr int kConvThreads = 256;

__device__ __forceinline__ float bf16_round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

template <class T>
__device__ __forceinline__ float load_operand(const T* p);
template <>
__device__ __forceinline__ float load_operand<float>(const float* p) {
  return bf16_round(*p);
}
template <>
__device__ __forceinline__ float load_operand<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}

template <class T>
__device__ __forceinline__ void store_out(T* p, float v);
template <>
__device__ __forceinline__ void store_out<float>(float* p, float v) {
  *p = v;
}
template <>
__device__ __forceinline__ void store_out<__nv_bfloat16>(__nv_bfloat16* p, float v) {
  *p = __float2bfloat16_rn(v);
}

// out = conv3x3(in) (+ bias, relu): in (TIn, ld_in, channels [off_in, off_in +
// Cin)), weights wt[9][Cin][Cout] (bfloat16), out (TOut, ld_out, channels
// [off_out, off_out + Cout)).  Grid (ceil(N / 64), ceil(N / 8), batch *
// ceil(Cout / 16)).
template <class TIn, class TOut>
__global__ void __launch_bounds__(kConvThreads) conv3x3_kernel(int N, int Cin, int Cout, const TIn* __restrict__ in,
                                                               int64_t ld_in, int off_in,
                                                               const __nv_bfloat16* __restrict__ wt,
                                                               const float* __restrict__ bias, int relu,
                                                               TOut* __restrict__ out, int64_t ld_out, int off_out) {
  __shared__ float in_s[kCIC][kTY + 2][kTX + 2];
  __shared__ __align__(16) float w_s[9][kCIC][kCOT];
  const int tid = threadIdx.x;
  const int tx = tid & 31, ty = tid >> 5;  // 8 warps = 8 rows; lanes and lanes + 32 along x
  const int ncog = (Cout + kCOT - 1) / kCOT;
  const int b = blockIdx.z / ncog, co0 = (blockIdx.z % ncog) * kCOT;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  const int64_t img = (int64_t)b * N * N;
  float acc0[kCOT], acc1[kCOT];
#pragma unroll
  for (int c = 0; c < kCOT; ++c) acc0[c] = acc1[c] = 0.f;
  for (int ci0 = 0; ci0 < Cin; ci0 += kCIC) {
    __syncthreads();
    // stage the (8 + 2) x (64 + 2) halo tile of 8 input channels (zero outside)
    for (int t = tid; t < (kTY + 2) * (kTX + 2); t += kConvThreads) {
      const int ry = t / (kTX + 2), rx = t % (kTX + 2);
      const int gy = y0 + ry - 1, gx = x0 + rx - 1;
      const bool inside = gx >= 0 && gx < N && gy >= 0 && gy < N;
      const TIn* src = in + (img + (int64_t)gy * N + gx) * ld_in + off_in + ci0;
#pragma unroll
      for (int c = 0; c < kCIC; ++c)
        in_s[c][ry][rx] = (inside && ci0 + c < Cin) ? load_operand<TIn>(src + c) : 0.f;
    }
    for (int t = tid; t < 9 * kCIC * kCOT; t += kConvThreads) {
      const int tap = t / (kCIC * kCOT), c = (t / kCOT) % kCIC, o = t % kCOT;
      const int ci = ci0 + c, co = co0 + o;
      w_s[tap][c][o] = (ci < Cin && co < Cout) ? __bfloat162float(wt[((int64_t)tap * Cin + ci) * Cout + co]) : 0.f;
    }
    __syncthreads();
#pragma unroll 1
    for (int c = 0; c < kCIC; ++c) {
#pragma unroll
      for (int ox = 0; ox < 3; ++ox) {
#pragma unroll
        for (int oy = 0; oy < 3; ++oy) {
          const float v0 = in_s[c][ty + oy][tx + ox];
          const float v1 = in_s[c][ty + oy][tx + 32 + ox];
          const float4* w4 = reinterpret_cast<const float4*>(&w_s[3 * ox + oy][c][0]);
#pragma unroll
          for (int q = 0; q < kCOT / 4; ++q) {
            const float4 w = w4[q];
            acc0[4 * q] = fmaf(v0, w.x, acc0[4 * q]);
            acc0[4 * q + 1] = fmaf(v0, w.y, acc0[4 * q + 1]);
            acc0[4 * q + 2] = fmaf(v0, w.z, acc0[4 * q + 2]);
            acc0[4 * q + 3] = fmaf(v0, w.w, acc0[4 * q + 3]);
            acc1[4 * q] = fmaf(v1, w.x, acc1[4 * q]);
            acc1[4 * q + 1] = fmaf(v1, w.y, acc1[4 * q + 1]);
            acc1[4 * q + 2] = fmaf(v1, w.z, acc1[4 * q + 2]);
            acc1[4 * q + 3] = fmaf(v1, w.w, acc1[4 * q + 3]);
          }
        }
      }
    }
  }
  const int gy = y0 + ty;
  if (gy >= N) return;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int gx = x0 + tx + 32 * h;
    if (gx >= N) continue;
    TOut* dst = out + (img + (int64_t)gy * N + gx) * ld_out + off_out + co0;
#pragma unroll
    for (int o = 0; o < kCOT; ++o) {
      if (co0 + o >= Cout) break;
      float v = (h ? acc1[o] : acc0[o]) + (bias ? bias[co0 + o] : 0.f);
      if (relu) v = fmaxf(v, 0.f);
      store_out<TOut>(dst + o, v);
    }
  }
}

// dw[tap][ci][co] += sum over the batch's pixels p of in[p + offset(tap)][ci] *
// gz[p][co], both operands rounded to bfloat16.  Each CTA takes 8 input
// channels (blockIdx.y) and a strided share of the 4 x 32-pixel tiles; its
// 256 threads hold (tap, ci) pairs g, g + 16, ... (g = tid / 16) for four
// output channels each (4 (tid % 16) .. + 3), and add into dw once at the end.
constexpr int kWY = 4, kWX = 32;
template <class TIn>
__global__ void __launch_bounds__(256) wgrad3x3_kernel(int N, int batch, int Cin, int Cout,
                                                       const TIn* __restrict__ in, int64_t ld_in, int off_in,
                                                       const float* __restrict__ gz, int64_t ld_g,
                                                       float* __restrict__ dw) {
  __shared__ float in_s[kCIC][kWY + 2][kWX + 2];
  __shared__ __align__(16) float g_s[kWY * kWX][64];
  const int tid = threadIdx.x;
  const int co = 4 * (tid & 15), grp = tid >> 4;
  const int ci0 = blockIdx.y * kCIC;
  float acc[5][4];
#pragma unroll
  for (int q = 0; q < 5; ++q)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[q][e] = 0.f;
  const int tiles_x = (N + kWX - 1) / kWX, tiles_y = (N + kWY - 1) / kWY;
  const int64_t ntiles = (int64_t)batch * tiles_x * tiles_y;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int b = (int)(t / ((int64_t)tiles_x * tiles_y));
    const int r = (int)(t % ((int64_t)tiles_x * tiles_y));
    const int x0 = (r % tiles_x) * kWX, y0 = (r / tiles_x) * kWY;
    const int64_t img = (int64_t)b * N * N;
    __syncthreads();
    for (int u = tid; u < (kWY + 2) * (kWX + 2); u += 256) {
      const int ry = u / (kWX + 2), rx = u % (kWX + 2);
      const int gy = y0 + ry - 1, gx = x0 + rx - 1;
      const bool inside = gx >= 0 && gx < N && gy >= 0 && gy < N;
      const TIn* src = in + (img + (int64_t)gy * N + gx) * ld_in + off_in + ci0;
#pragma unroll
      for (int c = 0; c < kCIC; ++c)
        in_s[c][ry][rx] = (inside && ci0 + c < Cin) ? load_operand<TIn>(src + c) : 0.f;
    }
    for (int u = tid; u < kWY * kWX * 64; u += 256) {
      const int px = u / 64, o = u % 64;
      const int gy = y0 + px / kWX, gx = x0 + px % kWX;
      g_s[px][o] = (gx < N && gy < N && o < Cout) ? bf16_round(gz[(img + (int64_t)gy * N + gx) * ld_g + o]) : 0.f;
    }
    __syncthreads();
    if (co < Cout) {
#pragma unroll 2
      for (int px = 0; px < kWY * kWX; ++px) {
        const float4 g = *reinterpret_cast<const float4*>(&g_s[px][co]);
        const int py = px / kWX, pxx = px % kWX;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          const int pair = grp + 16 * q;
          if (pair < 9 * kCIC) {
            const int tap = pair / kCIC, c = pair % kCIC;
            const float v = in_s[c][py + tap % 3][pxx + tap / 3];
            acc[q][0] = fmaf(v, g.x, acc[q][0]);
            acc[q][1] = fmaf(v, g.y, acc[q][1]);
            acc[q][2] = fmaf(v, g.z, acc[q][2]);
            acc[q][3] = fmaf(v, g.w, acc[q][3]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const int pair = grp + 16 * q;
    if (pair >= 9 * kCIC) continue;
    const int tap = pair / kCIC, ci = ci0 + pair % kCIC;
    if (ci >= Cin) continue;
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (co + e < Cout) atomicAdd(&dw[((int64_t)tap * Cin + ci) * Cout + co + e], acc[q][e]);
  }
}

// db[co] += sum over pixels of gz[p][co].
__global__ void bias_grad_kernel(int64_t npix, int Cout, const float* __restrict__ gz, int64_t ld_g,
                                 float* __restrict__ db) {
  __shared__ float red[256];
  const int co = blockIdx.y;
  float s = 0.f;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x)
    s += gz[p * ld_g + co];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(&db[co], red[0]);
}

// gz = g * (act > 0) over npix pixels and C channels (g and gz: FP32, ld C;
// act: bfloat16 with its own ld and channel offset).
__global__ void relu_mask_kernel(int64_t npix, int C, const float* __restrict__ g, int64_t ld_g,
                                 const __nv_bfloat16* __restrict__ act, int64_t ld_a, int off_a,
                                 float* __restrict__ gz, __nv_bfloat16* __restrict__ gzb) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npix * C) return;
  const int64_t p = t / C;
  const int c = (int)(t % C);
  const float a = __bfloat162float(act[p * ld_a + off_a + c]);
  const float v = a > 0.f ? g[p * ld_g + c] : 0.f;
  gz[p * C + c] = v;
  if (gzb) gzb[p * C + c] = __float2bfloat16_rn(v);  // the operand of a tensor-core backward convolution
}

// x_{l+1} = avgpool2(s_l): out (batch, N/2 x N/2, C, ld C) from in (N x N, ld_in, off_in).
__global__ void avgpool_kernel(int N, int batch, int C, const __nv_bfloat16* __restrict__ in, int64_t ld_in,
                               int off_in, __nv_bfloat16* __restrict__ out) {
  const int H = N / 2;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)batch * H * H * C) return;
  const int c = (int)(t % C);
  const int64_t q = t / C;
  const int ix = (int)(q % H), iy = (int)((q / H) % H);
  const int64_t b = q / ((int64_t)H * H);
  const __nv_bfloat16* s = in + (b * N * N + (int64_t)(2 * iy) * N + 2 * ix) * ld_in + off_in + c;
  const float v = __bfloat162float(s[0]) + __bfloat162float(s[ld_in]) + __bfloat162float(s[(int64_t)N * ld_in]) +
                  __bfloat162float(s[(int64_t)(N + 1) * ld_in]);
  out[t] = __float2bfloat16_rn(0.25f * v);
}

// upsample2: out (N x N, ld_out, channels [0, C)) from in (N/2 x N/2, ld C).
__global__ void upsample_kernel(int N, int batch, int C, const __nv_bfloat16* __restrict__ in,
                                __nv_bfloat16* __restrict__ out, int64_t ld_out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)batch * N * N * C) return;
  const int c = (int)(t % C);
  const int64_t q = t / C;
  const int ix = (int)(q % N), iy = (int)((q / N) % N);
  const int64_t b = q / ((int64_t)N * N);
  const int H = N / 2;
  out[q * ld_out + c] = in[(b * H * H + (int64_t)(iy / 2) * H + ix / 2) * C + c];
}

// g_low (N/2 x N/2, ld C) = sum of the four children of g (N x N, ld_g,
// channels [off_g, off_g + C)): the adjoint of upsample2.
__global__ void upsample_bwd_kernel(int N, int batch, int C, const float* __restrict__ g, int64_t ld_g, int off_g,
                                    float* __restrict__ glow) {
  const int H = N / 2;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)batch * H * H * C) return;
  const int c = (int)(t % C);
  const int64_t q = t / C;
  const int ix = (int)(q % H), iy = (int)((q / H) % H);
  const int64_t b = q / ((int64_t)H * H);
  const float* s = g + (b * N * N + (int64_t)(2 * iy) * N + 2 * ix) * ld_g + off_g + c;
  glow[t] = s[0] + s[ld_g] + s[(int64_t)N * ld_g] + s[(int64_t)(N + 1) * ld_g];
}

// gs (N x N, ld C) = gskip (channels [off_k, off_k + C) of ld_k) + avgpool2
// adjoint of gpool (N/2 x N/2, ld C): gpool / 4 on each of the four children.
__global__ void pool_bwd_add_kernel(int N, int batch, int C, const float* __restrict__ gskip, int64_t ld_k, int off_k,
                                    const float* __restrict__ gpool, float* __restrict__ gs) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)batch * N * N * C) return;
  const int c = (int)(t % C);
  const int64_t q = t / C;
  const int ix = (int)(q % N), iy = (int)((q / N) % N);
  const int64_t b = q / ((int64_t)N * N);
  const int H = N / 2;
  gs[t] = gskip[q * ld_k + off_k + c] + 0.25f * gpool[(b * H * H + (int64_t)(iy / 2) * H + ix / 2) * C + c];
}

// bfloat16 copies of the weights and the transposed, flipped weights of the
// backward convolution: wd[tap][co][ci] = w[8 - tap][ci][co].
__global__ void to_bf16_kernel(int64_t count, const float* __restrict__ p, __nv_bfloat16* __restrict__ q) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) q[t] = __float2bfloat16_rn(p[t]);
}
__global__ void dgrad_weights_kernel(int Cin, int Cout, const float* __restrict__ w, __nv_bfloat16* __restrict__ wd) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 9LL * Cin * Cout) return;
  const int tap = (int)(t / ((int64_t)Cin * Cout));
  const int co = (int)((t / Cin) % Cout), ci = (int)(t % Cin);
  wd[t] = __float2bfloat16_rn(w[((int64_t)(8 - tap) * Cin + ci) * Cout + co]);
}

// Residual loss of a batch (see rbgs_unet_residual_loss): res = (h^2/8) A_f y - x
// per image with its field's face coefficients; loss += 1/2 sum res^2 / total.
__device__ __forceinline__ float diff_apply_scaled(int N, const double* __restrict__ fc, const float* __restrict__ v,
                                                   int ix, int iy) {
  // (h^2 / 8) (A v) at (ix, iy) with A = -div(a grad) (face layout of RBGS_OP_DIFFUSION, nx = ny = N)
  const double* fx = fc;
  const double* fy = fc + (int64_t)(N + 1) * (N + 2);
  const int64_t i = ix + (int64_t)N * iy;
  const float c = v[i];
  const float w = ix > 0 ? v[i - 1] : 0.f, e = ix + 1 < N ? v[i + 1] : 0.f;
  const float s = iy > 0 ? v[i - N] : 0.f, no = iy + 1 < N ? v[i + N] : 0.f;
  const float ae = (float)fx[(ix + 1) + (int64_t)(N + 1) * (iy + 1)], aw = (float)fx[ix + (int64_t)(N + 1) * (iy + 1)];
  const float an = (float)fy[(ix + 1) + (int64_t)(N + 2) * (iy + 1)], as = (float)fy[(ix + 1) + (int64_t)(N + 2) * iy];
  return 0.125f * (ae * (c - e) + aw * (c - w) + an * (c - no) + as * (c - s));
}

__global__ void resid_loss_kernel(int N, int batch, const double* __restrict__ coef, int64_t coef_stride,
                                  const int* __restrict__ field, const float* __restrict__ x, int64_t ldx,
                                  const float* __restrict__ y, int64_t ldy, float* __restrict__ res,
                                  double* __restrict__ loss, double scale) {
  __shared__ double red[8];
  const int64_t n = (int64_t)N * N;
  const int b = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double sq = 0.0;
  if (i < n) {
    const double* fc = coef + (int64_t)field[b] * coef_stride;
    const float r = diff_apply_scaled(N, fc, y + b * ldy, (int)(i % N), (int)(i / N)) - x[b * ldx + i];
    res[b * n + i] = r;
    sq = (double)r * r;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    atomicAdd(loss, 0.5 * scale * t);
  }
}

// gy = (h^2/8) A_f res * scale (A_f symmetric: the gradient of 1/2 ||B y - x||^2 is B^T res).
__global__ void resid_grad_kernel(int N, int batch, const double* __restrict__ coef, int64_t coef_stride,
                                  const int* __restrict__ field, const float* __restrict__ res,
                                  float* __restrict__ gy, int64_t ldg, float scale) {
  const int64_t n = (int64_t)N * N;
  const int b = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* fc = coef + (int64_t)field[b] * coef_stride;
  gy[b * ldg + i] = scale * diff_apply_scaled(N, fc, res + b * n, (int)(i % N), (int)(i / N));
}

// Adam (Kingma and Ba 2015) with bias correction, FP32 state.
__global__ void adam_kernel(int64_t count, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const float gt = g[t];
  const float mt = b1 * m[t] + (1.f - b1) * gt;
  const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
  m[t] = mt;
  v[t] = vt;
  p[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
}

// Column scale of the preconditioner: s_j = ||q_j|| / sqrt(n) (partial sums,
// then the scale), x_j = q_j / s_j in FP32 (0 where s_j = 0).
template <class T>
__global__ void colsq_kernel(int64_t n, const T* __restrict__ Q, int64_t ldq, double* __restrict__ sq) {
  __shared__ double red[8];
  const int j = blockIdx.y;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)Q[i + j * ldq];
    s += v * v;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    atomicAdd(&sq[j], t);
  }
}
template <class T>
__global__ void normalize_kernel(int64_t n, const T* __restrict__ Q, int64_t ldq, const double* __restrict__ sq,
                                 float* __restrict__ X, int64_t ldx) {
  const int j = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double s = sqrt(sq[j] / (double)n);
  X[i + j * ldx] = s > 0.0 ? (float)((double)Q[i + j * ldq] / s) : 0.f;
}
// Z_j = s_j (h^2 / 8) y_j in the basis type.
template <class T>
__global__ void unscale_kernel(int64_t n, const float* __restrict__ Y, int64_t ldy, const double* __restrict__ sq,
                               double hh8, T* __restrict__ Z, int64_t ldz) {
  const int j = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double s = sqrt(sq[j] / (double)n);
  Z[i + j * ldz] = (T)(s * hh8 * (double)Y[i + j * ldy]);
}

// ----------------------------------------------------------------- layout --

struct Layer {
  int cin, cout, relu;
  int64_t w_off, b_off;
};

// The layer list of the network in evaluation order (the parameter layout).
std::vector<Layer> layers_of(const rbgs_unet& net) {
  std::vector<Layer> L;
  int64_t off = 0;
  auto add = [&](int ci, int co, int relu) {
    Layer l{ci, co, relu, off, off + 9LL * ci * co};
    off += 9LL * ci * co + co;
    L.push_back(l);
  };
  const int nl = net.levels;
  for (int l = 0; l < nl; ++l) {
    add(l == 0 ? 1 : net.width[l - 1], net.width[l], 1);
    add(net.width[l], net.width[l], 1);
  }
  for (int l = nl - 2; l >= 0; --l) add(net.width[l + 1] + net.width[l], net.width[l], 1);
  add(net.width[0], 1, 0);
  return L;
}
int64_t num_params(const rbgs_unet& net) {
  const auto L = layers_of(net);
  return L.back().b_off + L.back().cout;
}

bool net_ok(const rbgs_unet* net) {
  if (!net || net->levels < 2 || net->levels > 6 || net->flags < 0 || net->flags > 1) return false;
  for (int l = 0; l < net->levels; ++l)
    if (net->width[l] < 8 || net->width[l] > 64 || net->width[l] % 8) return false;
  return true;
}

// Buffers of one forward (and backward) pass for batch images of N x N.
struct Plan {
  int L = 0, N = 0, batch = 0;
  std::vector<int64_t> npix;  // per level: batch * N_l^2
  // activations (bfloat16)
  std::vector<__nv_bfloat16*> A, CAT, D, X;  // A_l, CAT_l (l < L-1), D_l (l < L-1), X_l (l >= 1)
  __nv_bfloat16* SB = nullptr;              // s_{L-1}
  __nv_bfloat16* wbf = nullptr;             // bfloat16 weights
  __nv_bfloat16* wd = nullptr;              // backward weights of one layer (largest)
  unsigned char* wpk = nullptr;             // tensor-core packed weights, per layer at w_off bytes * 2
  unsigned char* wdpk = nullptr;            // tensor-core packed backward weights of one layer
  std::vector<__nv_bfloat16*> GB;           // per level: bfloat16 copy of the masked gradient
  int* tc_err = nullptr;                    // bounded-wait flag of the tensor-core kernels
  // gradients (FP32)
  std::vector<float*> G1, G2, G3;  // per level: three buffers of npix * cmax_l
  size_t bytes = 0;
};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Lays out (base != null) or sizes (base == null) the buffers.
size_t plan_layout(const rbgs_unet& net, int N, int batch, bool grads, char* base, Plan* P) {
  const int L = net.levels;
  size_t off = 0;
  auto take = [&](size_t b) {
    char* r = base ? base + off : nullptr;
    off += align256(b);
    return r;
  };
  P->L = L;
  P->N = N;
  P->batch = batch;
  P->npix.assign(L, 0);
  P->A.assign(L, nullptr);
  P->CAT.assign(L, nullptr);
  P->D.assign(L, nullptr);
  P->X.assign(L, nullptr);
  P->G1.assign(L, nullptr);
  P->G2.assign(L, nullptr);
  P->G3.assign(L, nullptr);
  for (int l = 0; l < L; ++l) {
    const int Nl = N >> l;
    const int64_t np = (int64_t)batch * Nl * Nl;
    P->npix[l] = np;
    const int c = net.width[l];
    P->A[l] = (__nv_bfloat16*)take(2 * np * c);
    if (l < L - 1) {
      P->CAT[l] = (__nv_bfloat16*)take(2 * np * (net.width[l + 1] + c));
      P->D[l] = (__nv_bfloat16*)take(2 * np * c);
    } else {
      P->SB = (__nv_bfloat16*)take(2 * np * c);
    }
    if (l > 0) P->X[l] = (__nv_bfloat16*)take(2 * np * net.width[l - 1]);
    if (grads) {
      int cmax = c;
      if (l < L - 1) cmax = std::max(cmax, net.width[l + 1] + c);
      if (l > 0) cmax = std::max(cmax, net.width[l - 1]);
      P->G1[l] = (float*)take(4 * np * cmax);
      P->G2[l] = (float*)take(4 * np * cmax);
      P->G3[l] = (float*)take(4 * np * cmax);
    }
  }
  P->wbf = (__nv_bfloat16*)take(2 * num_params(net));
  P->wpk = (unsigned char*)take(2 * num_params(net));
  P->tc_err = (int*)take(256);
  P->GB.assign(L, nullptr);
  if (grads) {
    int64_t wmax = 0;
    for (const auto& ly : layers_of(net)) wmax = std::max<int64_t>(wmax, 9LL * ly.cin * ly.cout);
    P->wd = (__nv_bfloat16*)take(2 * wmax);
    P->wdpk = (unsigned char*)take(2 * wmax);
    for (int l = 0; l < L; ++l) {
      int cmax = net.width[l];
      P->GB[l] = (__nv_bfloat16*)take(2 * P->npix[l] * cmax);
    }
  }
  P->bytes = off;
  return off;
}

// Grow-only device buffers of the U-Net (slot 0: training, saved between the
// forward and the backward call; slot 1: the preconditioner inside FGMRES).
struct NetBuf {
  int dev = -1;
  int slot = 0;
  void* ptr = nullptr;
  size_t bytes = 0;
  Plan plan;
  rbgs_unet net{};
  bool saved = false;
  bool grads = false;
};
std::mutex g_nb_mu;
std::vector<NetBuf> g_nb;

rbgs_status net_buffer(int slot, const rbgs_unet& net, int N, int batch, bool grads, NetBuf** out) {
  int dev = 0;
  RBGS_CUDA_TRY(cudaGetDevice(&dev));
  Plan P;
  const size_t need = plan_layout(net, N, batch, grads, nullptr, &P);
  std::lock_guard<std::mutex> lk(g_nb_mu);
  NetBuf* nb = nullptr;
  for (auto& b : g_nb)
    if (b.dev == dev && b.slot == slot) nb = &b;
  if (!nb) {
    g_nb.push_back(NetBuf{});
    nb = &g_nb.back();
    nb->dev = dev;
    nb->slot = slot;
  }
  if (nb->bytes < need) {
    if (nb->ptr) {
      cudaDeviceSynchronize();
      cudaFree(nb->ptr);
      nb->ptr = nullptr;
      nb->bytes = 0;
    }
    if (cudaMalloc(&nb->ptr, need) != cudaSuccess) {
      cudaGetLastError();
      return RBGS_ENOMEM;
    }
    nb->bytes = need;
  }
  plan_layout(net, N, batch, grads, (char*)nb->ptr, &nb->plan);
  nb->net = net;
  nb->grads = grads;
  *out = nb;
  return RBGS_OK;
}

// Grow-only scratch per device and purpose (2: the preconditioner's FP32
// inputs and outputs, 3: the loss residual, 4: column sums of the input scaling).
struct Scratch {
  int dev = -1, slot = 0;
  void* ptr = nullptr;
  size_t bytes = 0;
};
std::vector<Scratch> g_scr;

rbgs_status scratch(int slot, size_t need, cudaStream_t st, void** out) {
  int dev = 0;
  RBGS_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_nb_mu);
  Scratch* sc = nullptr;
  for (auto& b : g_scr)
    if (b.dev == dev && b.slot == slot) sc = &b;
  if (!sc) {
    g_scr.push_back(Scratch{dev, slot, nullptr, 0});
    sc = &g_scr.back();
  }
  if (sc->bytes < need) {
    if (sc->ptr) {
      cudaStreamSynchronize(st);
      cudaFree(sc->ptr);
      sc->ptr = nullptr;
      sc->bytes = 0;
    }
    if (cudaMalloc(&sc->ptr, need) != cudaSuccess) {
      cudaGetLastError();
      return RBGS_ENOMEM;
    }
    sc->bytes = need;
  }
  *out = sc->ptr;
  return RBGS_OK;
}

unsigned blocks_for(int64_t count, int per = 256) { return (unsigned)((count + per - 1) / per); }

template <class TIn, class TOut>
rbgs_status conv(int N, int batch, int Cin, int Cout, const TIn* in, int64_t ld_in, int off_in,
                 const __nv_bfloat16* w, const float* bias, int relu, TOut* out, int64_t ld_out, int off_out,
                 cudaStream_t st) {
  dim3 grid((unsigned)((N + kTX - 1) / kTX), (unsigned)((N + kTY - 1) / kTY),
            (unsigned)(batch * ((Cout + kCOT - 1) / kCOT)));
  conv3x3_kernel<TIn, TOut><<<grid, kConvThreads, 0, st>>>(N, Cin, Cout, in, ld_in, off_in, w, bias, relu, out,
                                                           ld_out, off_out);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}

template <class TIn>
rbgs_status wgrad(int N, int batch, int Cin, int Cout, const TIn* in, int64_t ld_in, int off_in, const float* gz,
                  float* dw, float* db, cudaStream_t st) {
  const int cic = (Cin + kCIC - 1) / kCIC;
  const int64_t ntiles = (int64_t)batch * ((N + kWX - 1) / kWX) * ((N + kWY - 1) / kWY);
  const unsigned bx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ntiles, 608 / cic + 1));
  wgrad3x3_kernel<TIn><<<dim3(bx, (unsigned)cic), 256, 0, st>>>(N, batch, Cin, Cout, in, ld_in, off_in, gz, Cout,
                                                                 dw);
  RBGS_LAUNCH_CHECK();
  const int64_t npix = (int64_t)batch * N * N;
  bias_grad_kernel<<<dim3((unsigned)std::min<int64_t>(64, (npix + 255) / 256), (unsigned)Cout), 256, 0, st>>>(
      npix, Cout, gz, Cout, db);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}

template <class T>
constexpr int is_bf16() {
  return sizeof(T) == 2 ? 1 : 0;
}

// A forward convolution from bfloat16 activations: on the tensor cores where
// the level and channel counts allow it (rows of a multiple of 128 pixels,
// channels in multiples of 16; rbgs_unet.flags bit 0 turns them off), else the
// SIMT kernel.
template <class TOut>
rbgs_status conv_fwd(const rbgs_unet& net, Plan& P, int N, int B, int cin, int cout, const __nv_bfloat16* in,
                     int64_t ld_in, int off_in, const Layer& ly, const float* params, int relu, TOut* out,
                     int64_t ld_out, int off_out, cudaStream_t st) {
  if (!(net.flags & 1) && conv_tc_supported(N, cin, cout, ld_in, off_in, ld_out, off_out))
    return conv_tc(N, B, cin, cout, in, ld_in, off_in, P.wpk + 2 * ly.w_off, params + ly.b_off, relu, out,
                   is_bf16<TOut>(), ld_out, off_out, P.tc_err, st);
  return conv<__nv_bfloat16, TOut>(N, B, cin, cout, in, ld_in, off_in, P.wbf + ly.w_off, params + ly.b_off, relu,
                                   out, ld_out, off_out, st);
}

// The forward pass into the buffers of nb; y (FP32) column b at y + b ldy.
rbgs_status forward(NetBuf& nb, const float* params, const float* x, int64_t ldx, float* y, int64_t ldy,
                    cudaStream_t st) {
  const rbgs_unet& net = nb.net;
  Plan& P = nb.plan;
  const int L = P.L, N = P.N, B = P.batch;
  const auto lay = layers_of(net);
  const int64_t np = num_params(net);
  to_bf16_kernel<<<blocks_for(np), 256, 0, st>>>(np, params, P.wbf);
  RBGS_LAUNCH_CHECK();
  rbgs_status s;
  RBGS_CUDA_TRY(cudaMemsetAsync(P.tc_err, 0, sizeof(int), st));
  if (!(net.flags & 1)) {  // the tensor-core operand layout of every layer that can use it
    for (const auto& ly : lay)
      if (ly.cin % 16 == 0 && ly.cout % 16 == 0 && ly.cout <= 128)
        if ((s = conv_tc_pack(ly.cin, ly.cout, params + ly.w_off, 0, P.wpk + 2 * ly.w_off, st))) return s;
  }
  int li = 0;
  // the network input x is FP32 with one channel: image b at x + b ldx, i.e.
  // pixel-major with ld 1 only when ldx == N^2; otherwise copy it first
  for (int l = 0; l < L; ++l) {
    const int Nl = N >> l, c = net.width[l];
    const Layer& la = lay[li++];
    const Layer& lb = lay[li++];
    if (l == 0) {
      if (ldx != (int64_t)N * N) return RBGS_EINVAL;
      s = conv<float, __nv_bfloat16>(Nl, B, 1, c, x, 1, 0, P.wbf + la.w_off, params + la.b_off, 1, P.A[0], c, 0, st);
    } else {
      const int cp = net.width[l - 1];
      // x_l = avgpool2(s_{l-1}); s_{l-1} lives in CAT_{l-1} at channel offset c
      avgpool_kernel<<<blocks_for((int64_t)B * Nl * Nl * cp), 256, 0, st>>>(
          Nl * 2, B, cp, P.CAT[l - 1], c + cp, c, P.X[l]);
      RBGS_LAUNCH_CHECK();
      s = conv_fwd<__nv_bfloat16>(net, P, Nl, B, cp, c, P.X[l], cp, 0, la, params, 1, P.A[l], c, 0, st);
    }
    if (s) return s;
    if (l < L - 1) {
      const int cn = net.width[l + 1];
      s = conv_fwd<__nv_bfloat16>(net, P, Nl, B, c, c, P.A[l], c, 0, lb, params, 1, P.CAT[l], cn + c, cn, st);
    } else {
      s = conv_fwd<__nv_bfloat16>(net, P, Nl, B, c, c, P.A[l], c, 0, lb, params, 1, P.SB, c, 0, st);
    }
    if (s) return s;
  }
  for (int l = L - 2; l >= 0; --l) {
    const int Nl = N >> l, c = net.width[l], cn = net.width[l + 1];
    const Layer& ld = lay[li++];
    const __nv_bfloat16* prev = l == L - 2 ? P.SB : P.D[l + 1];
    upsample_kernel<<<blocks_for((int64_t)B * Nl * Nl * cn), 256, 0, st>>>(Nl, B, cn, prev, P.CAT[l], cn + c);
    RBGS_LAUNCH_CHECK();
    s = conv_fwd<__nv_bfloat16>(net, P, Nl, B, cn + c, c, P.CAT[l], cn + c, 0, ld, params, 1, P.D[l], c, 0, st);
    if (s) return s;
  }
  const Layer& lo = lay[li++];
  if (ldy != (int64_t)N * N) return RBGS_EINVAL;
  return conv<__nv_bfloat16, float>(N, B, net.width[0], 1, P.D[0], net.width[0], 0, P.wbf + lo.w_off,
                                    params + lo.b_off, 0, y, 1, 0, st);
}

rbgs_status dgrad(int N, int batch, int Cin, int Cout, const float* w, __nv_bfloat16* wd, const float* gz, float* gx,
                  cudaStream_t st) {
  dgrad_weights_kernel<<<blocks_for(9LL * Cin * Cout), 256, 0, st>>>(Cin, Cout, w, wd);
  RBGS_LAUNCH_CHECK();
  return conv<float, float>(N, batch, Cout, Cin, gz, Cout, 0, wd, nullptr, 0, gx, Cin, 0, st);
}

// The backward convolution gx = conv(gz, flipped transposed w): on the tensor
// cores from the bfloat16 copy gzb of gz where possible, else SIMT from gz.
rbgs_status dgrad_any(const rbgs_unet& net, Plan& P, int N, int batch, int Cin, int Cout, const float* w,
                      const float* gz, const __nv_bfloat16* gzb, float* gx, cudaStream_t st) {
  if (!(net.flags & 1) && gzb && conv_tc_supported(N, Cout, Cin, Cout, 0, Cin, 0)) {
    rbgs_status s = conv_tc_pack(Cout, Cin, w, 1, P.wdpk, st);
    if (s) return s;
    return conv_tc(N, batch, Cout, Cin, gzb, Cout, 0, P.wdpk, nullptr, 0, gx, 0, Cin, 0, P.tc_err, st);
  }
  return dgrad(N, batch, Cin, Cout, w, P.wd, gz, gx, st);
}

// The backward pass of the last forward saved in nb: grads (FP32, the
// parameter layout) = d sum(gy * y) / d params.
rbgs_status backward(NetBuf& nb, const float* params, const float* gy, float* grads, const float* x,
                     cudaStream_t st) {
  const rbgs_unet& net = nb.net;
  Plan& P = nb.plan;
  const int L = P.L, N = P.N, B = P.batch;
  const auto lay = layers_of(net);
  rbgs_status s;
  RBGS_CUDA_TRY(cudaMemsetAsync(grads, 0, sizeof(float) * num_params(net), st));
  RBGS_CUDA_TRY(cudaMemsetAsync(P.tc_err, 0, sizeof(int), st));
  int li = (int)lay.size() - 1;
  // output layer: z = y (linear); input D_0
  {
    const Layer& lo = lay[li--];
    const int c0 = net.width[0];
    if ((s = wgrad<__nv_bfloat16>(N, B, c0, 1, P.D[0], c0, 0, gy, grads + lo.w_off, grads + lo.b_off, st)))
      return s;
    if ((s = dgrad(N, B, c0, 1, params + lo.w_off, P.wd, gy, P.G1[0], st))) return s;  // G1[0] = g(D_0)
  }
  // decoder, l = 0 .. L-2: G1[l] holds g(D_l) on entry
  for (int l = 0; l <= L - 2; ++l) {
    const Layer& ld = lay[li--];
    const int Nl = N >> l, c = net.width[l], cn = net.width[l + 1];
    const int64_t npx = P.npix[l];
    relu_mask_kernel<<<blocks_for(npx * c), 256, 0, st>>>(npx, c, P.G1[l], c, P.D[l], c, 0, P.G2[l], P.GB[l]);
    RBGS_LAUNCH_CHECK();
    if ((s = wgrad<__nv_bfloat16>(Nl, B, cn + c, c, P.CAT[l], cn + c, 0, P.G2[l], grads + ld.w_off,
                                  grads + ld.b_off, st)))
      return s;
    // G3[l] = g(CAT_l): channels [0, cn) go to the upsampled d_{l+1}, [cn, cn + c) to s_l
    if ((s = dgrad_any(net, P, Nl, B, cn + c, c, params + ld.w_off, P.G2[l], P.GB[l], P.G3[l], st))) return s;
    upsample_bwd_kernel<<<blocks_for(P.npix[l + 1] * cn), 256, 0, st>>>(Nl, B, cn, P.G3[l], cn + c, 0, P.G1[l + 1]);
    RBGS_LAUNCH_CHECK();
  }
  // encoder, l = L-1 .. 0: G1[l] = g(s_l) (for l < L-1 the skip part of G3[l] plus the pooled path)
  for (int l = L - 1; l >= 0; --l) {
    const Layer& lb = lay[2 * l + 1];
    const Layer& la = lay[2 * l];
    const int Nl = N >> l, c = net.width[l];
    const int64_t npx = P.npix[l];
    if (l < L - 1) {
      const int cn = net.width[l + 1];
      // G1[l] = G3[l][:, cn:] + avgpool2 adjoint of g(x_{l+1}) (in G2[l+1])
      pool_bwd_add_kernel<<<blocks_for(npx * c), 256, 0, st>>>(Nl, B, c, P.G3[l], cn + c, cn, P.G2[l + 1], P.G1[l]);
      RBGS_LAUNCH_CHECK();
    }
    const __nv_bfloat16* s_act = l < L - 1 ? P.CAT[l] : P.SB;
    const int64_t s_ld = l < L - 1 ? net.width[l + 1] + c : c;
    const int s_off = l < L - 1 ? net.width[l + 1] : 0;
    relu_mask_kernel<<<blocks_for(npx * c), 256, 0, st>>>(npx, c, P.G1[l], c, s_act, s_ld, s_off, P.G2[l], P.GB[l]);
    RBGS_LAUNCH_CHECK();
    if ((s = wgrad<__nv_bfloat16>(Nl, B, c, c, P.A[l], c, 0, P.G2[l], grads + lb.w_off, grads + lb.b_off, st)))
      return s;
    if ((s = dgrad_any(net, P, Nl, B, c, c, params + lb.w_off, P.G2[l], P.GB[l], P.G3[l], st))) return s;  // g(A_l)
    relu_mask_kernel<<<blocks_for(npx * c), 256, 0, st>>>(npx, c, P.G3[l], c, P.A[l], c, 0, P.G1[l], P.GB[l]);
    RBGS_LAUNCH_CHECK();
    if (l == 0) {
      if ((s = wgrad<float>(Nl, B, 1, c, x, 1, 0, P.G1[0], grads + la.w_off, grads + la.b_off, st))) return s;
    } else {
      const int cp = net.width[l - 1];
      if ((s = wgrad<__nv_bfloat16>(Nl, B, cp, c, P.X[l], cp, 0, P.G1[l], grads + la.w_off, grads + la.b_off, st)))
        return s;
      if ((s = dgrad_any(net, P, Nl, B, cp, c, params + la.w_off, P.G1[l], P.GB[l], P.G2[l], st))) return s;
    }
  }
  return RBGS_OK;
}

// With sync: wait, and report an expired bounded wait of the tensor-core
// kernels (their flag) as RBGS_ETIMEOUT.
rbgs_status finish(NetBuf& nb, cudaStream_t st, int sync) {
  if (!sync) return RBGS_OK;
  int herr = 0;
  RBGS_CUDA_TRY(cudaMemcpyAsync(&herr, nb.plan.tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  RBGS_CUDA_TRY(cudaStreamSynchronize(st));
  return herr ? RBGS_ETIMEOUT : RBGS_OK;
}

}  // namespace

// ---------------------------------------------------------------- internal --

void unet_release(int dev) {
  std::lock_guard<std::mutex> lk(g_nb_mu);
  for (auto& b : g_nb)
    if (b.dev == dev && b.ptr) {
      cudaDeviceSynchronize();
      cudaFree(b.ptr);
      b.ptr = nullptr;
      b.bytes = 0;
      b.saved = false;
    }
  for (auto& b : g_scr)
    if (b.dev == dev && b.ptr) {
      cudaDeviceSynchronize();
      cudaFree(b.ptr);
      b.ptr = nullptr;
      b.bytes = 0;
    }
}

// Z (n x mb, basis type T, ldz) = M(Q): per column s = ||q|| / sqrt(n),
// z = s (h^2 / 8) U-Net(q / s), h = 1 / (N + 1) (positively homogeneous).
template <class T>
rbgs_status unet_precondition(const rbgs_unet& net, const float* params, int N, int mb, const T* Q, int64_t ldq,
                              T* Z, int64_t ldz, cudaStream_t st) {
  NetBuf* nb = nullptr;
  rbgs_status s;
  const int64_t n = (int64_t)N * N;
  // scratch: the FP32 inputs and outputs and the column sums, after the plan
  if ((s = net_buffer(1, net, N, mb, false, &nb))) return s;
  void* io = nullptr;
  if ((s = scratch(2, align256(8 * (size_t)n * mb) + align256(8 * (size_t)mb), st, &io))) return s;
  float* xin = (float*)io;
  float* yout = xin + (size_t)n * mb;
  double* sq = (double*)((char*)io + align256(8 * (size_t)n * mb));
  RBGS_CUDA_TRY(cudaMemsetAsync(sq, 0, 8 * (size_t)mb, st));
  const unsigned nbk = (unsigned)std::min<int64_t>(256, (n + 255) / 256);
  colsq_kernel<T><<<dim3(nbk, (unsigned)mb), 256, 0, st>>>(n, Q, ldq, sq);
  RBGS_LAUNCH_CHECK();
  normalize_kernel<T><<<dim3(blocks_for(n), (unsigned)mb), 256, 0, st>>>(n, Q, ldq, sq, xin, n);
  RBGS_LAUNCH_CHECK();
  if ((s = forward(*nb, params, xin, n, yout, n, st))) return s;
  const double h = 1.0 / (double)(N + 1);
  unscale_kernel<T><<<dim3(blocks_for(n), (unsigned)mb), 256, 0, st>>>(n, yout, n, sq, h * h / 8.0, Z, ldz);
  RBGS_LAUNCH_CHECK();
  return RBGS_OK;
}
template rbgs_status unet_precondition<float>(const rbgs_unet&, const float*, int, int, const float*, int64_t, float*,
                                              int64_t, cudaStream_t);
template rbgs_status unet_precondition<double>(const rbgs_unet&, const float*, int, int, const double*, int64_t,
                                               double*, int64_t, cudaStream_t);

bool unet_valid(const rbgs_unet* net, int64_t N) {
  return net_ok(net) && N >= 2 && N % (1 << (net->levels - 1)) == 0 && N < 46341;
}

}  // namespace rbgs

using namespace rbgs;

extern "C" {

int64_t rbgs_unet_num_params(const rbgs_unet* net) { return net_ok(net) ? num_params(*net) : -1; }

rbgs_status rbgs_unet_forward(const rbgs_unet* net, const float* params, int64_t N, int64_t batch, const float* x,
                              float* y, int32_t save, void* stream, int32_t sync) {
  if (!unet_valid(net, N) || !params || !x || !y || batch < 1 || batch * N * N >= ((int64_t)1 << 31))
    return RBGS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  NetBuf* nb = nullptr;
  rbgs_status s;
  if ((s = net_buffer(save ? 0 : 1, *net, (int)N, (int)batch, save != 0, &nb))) return s;
  if ((s = forward(*nb, params, x, N * N, y, N * N, st))) return s;
  nb->saved = save != 0;
  return finish(*nb, st, sync);
}

rbgs_status rbgs_unet_backward(const rbgs_unet* net, const float* params, int64_t N, int64_t batch, const float* x,
                               const float* gy, float* grads, void* stream, int32_t sync) {
  if (!unet_valid(net, N) || !params || !x || !gy || !grads || batch < 1) return RBGS_EINVAL;
  int dev = 0;
  RBGS_CUDA_TRY(cudaGetDevice(&dev));
  NetBuf* nb = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_nb_mu);
    for (auto& b : g_nb)
      if (b.dev == dev && b.slot == 0) nb = &b;
  }
  // the saved forward must be of this network and shape
  if (!nb || !nb->saved || !nb->grads || nb->plan.N != N || nb->plan.batch != batch || nb->net.levels != net->levels)
    return RBGS_EINVAL;
  for (int l = 0; l < net->levels; ++l)
    if (nb->net.width[l] != net->width[l]) return RBGS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  rbgs_status s = backward(*nb, params, gy, grads, x, st);
  if (s) return s;
  return finish(*nb, st, sync);
}

rbgs_status rbgs_unet_residual_loss(int64_t N, int64_t batch, const double* coef, int64_t coef_stride,
                                    const int32_t* field, const float* x, const float* y, float* gy, double* loss,
                                    void* stream, int32_t sync) {
  if (N < 1 || batch < 1 || !coef || !field || !x || !y || !gy || !loss ||
      coef_stride < (N + 1) * (N + 2) + (N + 2) * (N + 1) || batch * N * N >= ((int64_t)1 << 31))
    return RBGS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = N * N;
  // the residual of every image is needed whole before gy = B res: a scratch
  void* scr = nullptr;
  rbgs_status s;
  if ((s = scratch(3, 4 * (size_t)n * batch, st, &scr))) return s;
  float* res = (float*)scr;
  const double total = (double)n * (double)batch;
  RBGS_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(double), st));
  resid_loss_kernel<<<dim3((unsigned)((n + 255) / 256), (unsigned)batch), 256, 0, st>>>(
      (int)N, (int)batch, coef, coef_stride, field, x, n, y, n, res, loss, 1.0 / total);
  RBGS_LAUNCH_CHECK();
  resid_grad_kernel<<<dim3((unsigned)((n + 255) / 256), (unsigned)batch), 256, 0, st>>>(
      (int)N, (int)batch, coef, coef_stride, field, res, gy, n, (float)(1.0 / total));
  RBGS_LAUNCH_CHECK();
  if (sync) RBGS_CUDA_TRY(cudaStreamSynchronize(st));
  return RBGS_OK;
}

rbgs_status rbgs_adam_step(int64_t count, float* params, const float* grads, float* m, float* v, int64_t t,
                           double lr, double beta1, double beta2, double eps, void* stream, int32_t sync) {
  if (count < 0 || !params || !grads || !m || !v || t < 1) return RBGS_EINVAL;
  if (count == 0) return RBGS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const double c1 = 1.0 - std::pow(beta1, (double)t), c2 = 1.0 - std::pow(beta2, (double)t);
  adam_kernel<<<blocks_for(count), 256, 0, st>>>(count, params, grads, m, v, (float)lr, (float)beta1, (float)beta2,
                                                 (float)eps, (float)c1, (float)c2);
  RBGS_LAUNCH_CHECK();
  if (sync) RBGS_CUDA_TRY(cudaStreamSynchronize(st));
  return RBGS_OK;
}

rbgs_status rbgs_unet_scale_inputs(int64_t n, int64_t ncols, int32_t prec, const void* Q, int64_t ldq, float* X,
                                   int64_t ldx, void* stream, int32_t sync) {
  if (n < 1 || ncols < 0 || !Q || !X || ldq < n || ldx < n || ncols > 65535) return RBGS_EINVAL;
  if (ncols == 0) return RBGS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  void* scr = nullptr;
  rbgs_status s;
  if ((s = scratch(4, 8 * (size_t)ncols, st, &scr))) return s;
  double* sq = (double*)scr;
  RBGS_CUDA_TRY(cudaMemsetAsync(sq, 0, 8 * (size_t)ncols, st));
  const unsigned nbk = (unsigned)std::min<int64_t>(256, (n + 255) / 256);
  if (prec == RBGS_P_FP64) {
    colsq_kernel<double><<<dim3(nbk, (unsigned)ncols), 256, 0, st>>>(n, (const double*)Q, ldq, sq);
    RBGS_LAUNCH_CHECK();
    normalize_kernel<double><<<dim3(blocks_for(n), (unsigned)ncols), 256, 0, st>>>(n, (const double*)Q, ldq, sq, X,
                                                                                  ldx);
  } else if (prec >= RBGS_P_FP32 && prec <= RBGS_P_F16X3) {
    colsq_kernel<float><<<dim3(nbk, (unsigned)ncols), 256, 0, st>>>(n, (const float*)Q, ldq, sq);
    RBGS_LAUNCH_CHECK();
    normalize_kernel<float><<<dim3(blocks_for(n), (unsigned)ncols), 256, 0, st>>>(n, (const float*)Q, ldq, sq, X,
                                                                                 ldx);
  } else {
    return RBGS_EINVAL;
  }
  RBGS_LAUNCH_CHECK();
  if (sync) RBGS_CUDA_TRY(cudaStreamSynchronize(st));
  return RBGS_OK;
}

rbgs_status rbgs_unet_precondition(const rbgs_unet* net, const float* params, int64_t N, int32_t prec,
                                   const void* Q, int64_t ldq, int64_t ncols, void* Z, int64_t ldz, void* stream,
                                   int32_t sync) {
  if (!unet_valid(net, N) || !params || !Q || !Z || ncols < 1 || ncols > 64 || ldq < N * N || ldz < N * N)
    return RBGS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  rbgs_status s;
  if (prec == RBGS_P_FP64)
    s = unet_precondition<double>(*net, params, (int)N, (int)ncols, (const double*)Q, ldq, (double*)Z, ldz, st);
  else if (prec >= RBGS_P_FP32 && prec <= RBGS_P_F16X3)
    s = unet_precondition<float>(*net, params, (int)N, (int)ncols, (const float*)Q, ldq, (float*)Z, ldz, st);
  else
    return RBGS_EINVAL;
  if (s) return s;
  if (sync) RBGS_CUDA_TRY(cudaStreamSynchronize(st));
  return RBGS_OK;
}

}  // extern "C"
