// Resolution changes of the U-Net fine stage (Sec. 3.2: a two-stage U-Net after feature
// extraction; two upsampling stages, Sec. 4.2): 2x2 max pooling (stride 2; a window that
// overhangs the last row or column takes the max of its in-frame pixels) and nearest 2x
// upsampling into a channel range of a wider buffer (the concatenation of the level's skip
// features and the upsampled ones).  Both move stored activations unchanged, so BF16 and e4m3
// values stay exactly representable (and e4m3 codes keep their layer's scale); both are
// HBM-bound copies: every thread moves 16-byte chunks, consecutive threads consecutive chunks
// of one output row.
#include <cuda_bf16.h>

#include "sml_internal.h"

namespace sml {

namespace {

constexpr int kResampleThreads = 256;

__device__ __forceinline__ uint4 max4_bf16(uint4 a, uint4 b) {
  uint4 r;
  const __nv_bfloat162* x = reinterpret_cast<const __nv_bfloat162*>(&a);
  const __nv_bfloat162* y = reinterpret_cast<const __nv_bfloat162*>(&b);
  __nv_bfloat162* z = reinterpret_cast<__nv_bfloat162*>(&r);
#pragma unroll
  for (int k = 0; k < 4; ++k) z[k] = __hmax2(x[k], y[k]);
  return r;
}

// e4m3 codes of post-ReLU values are never negative (sign bit clear), and for those the code
// order is the value order, so a bytewise unsigned max is the max of the values.
__device__ __forceinline__ uint4 max16_e4m3(uint4 a, uint4 b) {
  return make_uint4(__vmaxu4(a.x, b.x), __vmaxu4(a.y, b.y), __vmaxu4(a.z, b.z), __vmaxu4(a.w, b.w));
}

__device__ __forceinline__ float4 max4_f32(float4 a, float4 b) {
  return make_float4(fmaxf(a.x, b.x), fmaxf(a.y, b.y), fmaxf(a.z, b.z), fmaxf(a.w, b.w));
}

// One output row (frame t, row r) per blockIdx.y step; its chunks over x.  A "chunk" is 16
// bytes: BF16 row-planar [T][rows][groups][cols][2 chunks], FP8 row-planar
// [T][rows][groups][cols][1 chunk], FP32 NHWC [T][rows][cols][ct/4].
struct ResampleArgs {
  const uint8_t* in;
  uint8_t* out;
  int T, H, W;          // input size
  int Ho, Wo;           // output size
  int in_ct, out_ct;    // channels per pixel of the buffers
  int C, out_off;       // channels moved; first output channel
};

// Row-planar (BF16: NCH = 2 chunks per 16-channel group row, FP8: 1), 2x2 max.
template <int NCH>
__global__ void __launch_bounds__(kResampleThreads) k_pool2_rp(const ResampleArgs a) {
  constexpr int RB = 16 * NCH;  // bytes of a group row
  const int G = a.C / 16, gin = a.in_ct / 16, gout = a.out_ct / 16, g0 = a.out_off / 16;
  const int per_row = G * a.Wo * NCH;
  for (long long row = blockIdx.y; row < (long long)a.T * a.Ho; row += gridDim.y) {
    const int t = (int)(row / a.Ho), io = (int)(row - (long long)t * a.Ho);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < per_row; k += gridDim.x * blockDim.x) {
      const int g = k / (NCH * a.Wo), rem = k - g * NCH * a.Wo, jo = rem / NCH, h = rem - jo * NCH;
      // the window's first pixel (2io, 2jo) is always in the frame
      const uint8_t* p0 = a.in + ((((size_t)t * a.H + 2 * io) * gin + g) * a.W + 2 * jo) * RB + 16 * h;
      const size_t row_step = (size_t)gin * a.W * RB;
      const bool right = 2 * jo + 1 < a.W, down = 2 * io + 1 < a.H;
      auto mx = [](uint4 x, uint4 y) { return NCH == 2 ? max4_bf16(x, y) : max16_e4m3(x, y); };
      uint4 m = __ldg(reinterpret_cast<const uint4*>(p0));
      if (right) m = mx(m, __ldg(reinterpret_cast<const uint4*>(p0 + RB)));
      if (down) m = mx(m, __ldg(reinterpret_cast<const uint4*>(p0 + row_step)));
      if (right && down) m = mx(m, __ldg(reinterpret_cast<const uint4*>(p0 + row_step + RB)));
      *reinterpret_cast<uint4*>(a.out + ((((size_t)t * a.Ho + io) * gout + g0 + g) * a.Wo + jo) * RB + 16 * h) = m;
    }
  }
}

// FP32 NHWC, 2x2 max.
__global__ void __launch_bounds__(kResampleThreads) k_pool2_f32(const ResampleArgs a) {
  const int C4 = a.C / 4;
  const int per_row = a.Wo * C4;
  for (long long row = blockIdx.y; row < (long long)a.T * a.Ho; row += gridDim.y) {
    const int t = (int)(row / a.Ho), io = (int)(row - (long long)t * a.Ho);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < per_row; k += gridDim.x * blockDim.x) {
      const int jo = k / C4, c4 = k - jo * C4;
      // the window's first pixel (2io, 2jo) is always in the frame
      const float4* p0 = reinterpret_cast<const float4*>(a.in) + ((((size_t)t * a.H + 2 * io) * a.W + 2 * jo) * a.in_ct) / 4 + c4;
      const size_t px_step = (size_t)a.in_ct / 4, row_step = (size_t)a.W * a.in_ct / 4;
      const bool right = 2 * jo + 1 < a.W, down = 2 * io + 1 < a.H;
      float4 m = __ldg(p0);
      if (right) m = max4_f32(m, __ldg(p0 + px_step));
      if (down) m = max4_f32(m, __ldg(p0 + row_step));
      if (right && down) m = max4_f32(m, __ldg(p0 + row_step + px_step));
      reinterpret_cast<float4*>(a.out)[((((size_t)t * a.Ho + io) * a.Wo + jo) * a.out_ct + a.out_off) / 4 + c4] = m;
    }
  }
}

// Row-planar (NCH chunks per group row), nearest 2x: out(i, j) = in(i / 2, j / 2).
template <int NCH>
__global__ void __launch_bounds__(kResampleThreads) k_up2_rp(const ResampleArgs a) {
  constexpr int RB = 16 * NCH;
  const int G = a.C / 16, gin = a.in_ct / 16, gout = a.out_ct / 16, g0 = a.out_off / 16;
  const int per_row = G * a.Wo * NCH;
  for (long long row = blockIdx.y; row < (long long)a.T * a.Ho; row += gridDim.y) {
    const int t = (int)(row / a.Ho), io = (int)(row - (long long)t * a.Ho);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < per_row; k += gridDim.x * blockDim.x) {
      const int g = k / (NCH * a.Wo), rem = k - g * NCH * a.Wo, jo = rem / NCH, h = rem - jo * NCH;
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(
          a.in + ((((size_t)t * a.H + (io >> 1)) * gin + g) * a.W + (jo >> 1)) * RB + 16 * h));
      *reinterpret_cast<uint4*>(a.out + ((((size_t)t * a.Ho + io) * gout + g0 + g) * a.Wo + jo) * RB + 16 * h) = v;
    }
  }
}

// FP32 NHWC, nearest 2x.
__global__ void __launch_bounds__(kResampleThreads) k_up2_f32(const ResampleArgs a) {
  const int C4 = a.C / 4;
  const int per_row = a.Wo * C4;
  for (long long row = blockIdx.y; row < (long long)a.T * a.Ho; row += gridDim.y) {
    const int t = (int)(row / a.Ho), io = (int)(row - (long long)t * a.Ho);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < per_row; k += gridDim.x * blockDim.x) {
      const int jo = k / C4, c4 = k - jo * C4;
      const float4 v = __ldg(reinterpret_cast<const float4*>(a.in) +
                             ((((size_t)t * a.H + (io >> 1)) * a.W + (jo >> 1)) * a.in_ct) / 4 + c4);
      reinterpret_cast<float4*>(a.out)[((((size_t)t * a.Ho + io) * a.Wo + jo) * a.out_ct + a.out_off) / 4 + c4] = v;
    }
  }
}

dim3 resample_grid(const ResampleArgs& a, int per_row) {
  const long long rows = (long long)a.T * a.Ho;
  const int bx = (per_row + kResampleThreads - 1) / kResampleThreads;
  return dim3((unsigned)(bx < 64 ? bx : 64), (unsigned)(rows < 65535 ? rows : 65535));
}

bool resample_ok(const ResampleArgs& a, int prec) {
  const int q = prec == kFP32 ? 4 : 16;  // channel granularity of one 16-byte chunk
  return a.T >= 0 && a.H >= 1 && a.W >= 1 && a.Ho >= 1 && a.Wo >= 1 && a.C >= q && a.C % q == 0 && a.in_ct % q == 0 &&
         a.out_ct % q == 0 && a.out_off % q == 0 && a.C <= a.in_ct && a.out_off + a.C <= a.out_ct;
}

}  // namespace

cudaError_t launch_pool2(const void* in, int in_ct, void* out, int out_ct, int out_off, int C, int T, int H, int W,
                         int prec, cudaStream_t s) {
  ResampleArgs a{static_cast<const uint8_t*>(in), static_cast<uint8_t*>(out), T, H, W, (H + 1) / 2, (W + 1) / 2,
                 in_ct, out_ct, C, out_off};
  if (prec != kFP32 && prec != kBF16 && prec != kFP8) return cudaErrorInvalidValue;
  if (!resample_ok(a, prec)) return cudaErrorInvalidValue;
  if (T == 0) return cudaSuccess;
  if (prec == kBF16)
    k_pool2_rp<2><<<resample_grid(a, (C / 16) * a.Wo * 2), kResampleThreads, 0, s>>>(a);
  else if (prec == kFP8)
    k_pool2_rp<1><<<resample_grid(a, (C / 16) * a.Wo), kResampleThreads, 0, s>>>(a);
  else
    k_pool2_f32<<<resample_grid(a, a.Wo * (C / 4)), kResampleThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_upsample2(const void* in, int in_ct, int h, int w, void* out, int out_ct, int out_off, int C, int T,
                             int H, int W, int prec, cudaStream_t s) {
  ResampleArgs a{static_cast<const uint8_t*>(in), static_cast<uint8_t*>(out), T, h, w, H, W, in_ct, out_ct, C, out_off};
  if (prec != kFP32 && prec != kBF16 && prec != kFP8) return cudaErrorInvalidValue;
  if (!resample_ok(a, prec) || (H + 1) / 2 != h || (W + 1) / 2 != w) return cudaErrorInvalidValue;
  if (T == 0) return cudaSuccess;
  if (prec == kBF16)
    k_up2_rp<2><<<resample_grid(a, (C / 16) * W * 2), kResampleThreads, 0, s>>>(a);
  else if (prec == kFP8)
    k_up2_rp<1><<<resample_grid(a, (C / 16) * W), kResampleThreads, 0, s>>>(a);
  else
    k_up2_f32<<<resample_grid(a, W * (C / 4)), kResampleThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace sml
