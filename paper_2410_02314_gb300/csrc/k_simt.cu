// SIMT kernels: first layer (camera transform fused with the Cin=1 dilated 3x3 conv) and
// the FP32 dilated 3x3 conv layers (plain FP32 FMA; the FP32 precision mode).
//
// Layer semantics (dilated convolution, Sec. 3.2.1), per frame and output channel co:
//   a_out[i,j,co] = ReLU(b[co] + sum_{ci,ky,kx} w[co,ci,ky,kx] a_in[i+(ky-1)d, j+(kx-1)d, ci])
// with a_in = 0 outside the frame, at every layer.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cstring>

#include "sml_internal.h"

namespace sml {

namespace {

constexpr int kSimtThreads = 128;


// Layer-1 weights travel by value (kernel parameter); each thread copies the ones it uses
// into registers.
struct L1Params {
  float w[64 * 3 * 9];  // [co][ci][ky*3+kx]
  float b[64];
};

constexpr int kL1Tile = 128;     // pixels of one image row per block (and threads per block)
constexpr int kL1Px = 8;         // pixels per thread: columns pg + 16*p, p < kL1Px
constexpr int kL1ChGroups = 8;   // a thread computes C/8 output channels
constexpr int kL1MaxD = 64;      // largest layer-1 dilation
constexpr int kL1Batch = 4;      // staged rows whose loads are in flight together

// Output rows per block: 16 for the small dilations of a first layer, whose input rows
// overlap (16 + 2d staged rows for 16 output rows), else 4.
__host__ __device__ constexpr int l1_rows(int d) { return d <= 4 ? 16 : 4; }

// Staged input rows of a block: output row r (< R = l1_rows(d)) reads image rows
// i0 + r + (ky-1)d.  For d < R these overlap, and the block stages the R + 2d distinct rows
// i0 - d .. i0 + R - 1 + d once (staged row r + ky d); otherwise all 3R are distinct (staged
// row ky R + r).
__host__ __device__ constexpr int l1_stage_rows(int d) { return d < l1_rows(d) ? l1_rows(d) + 2 * d : 3 * l1_rows(d); }
__device__ __forceinline__ int l1_srow(int r, int ky, int d) {
  return d < l1_rows(d) ? r + ky * d : ky * l1_rows(d) + r;
}
__device__ __forceinline__ int l1_stage_image_row(int sr, int i0, int d) {
  const int R = l1_rows(d);
  return d < R ? i0 - d + sr : i0 + sr % R + (sr / R - 1) * d;
}

// Dynamic shared memory of one block: staged inputs [l1_stage_rows(d)][IN_CH][128 + 2d] as
// float pairs (each value twice, the operand of a packed two-channel FMA), then the padded
// output tile [kL1Tile][C*OB + 16] bytes.
template <int C, int OUT, int IN_CH>
constexpr size_t l1_smem_bytes(int d) {
  return (size_t)l1_stage_rows(d) * IN_CH * (kL1Tile + 2 * d) * 8 +
         (size_t)kL1Tile * (C * (OUT == 0 ? 4 : (OUT == 1 ? 2 : 1)) + 16);
}

// One block: a 128-pixel strip of l1_rows(d) rows of one frame.  Thread (pg = lane % 16,
// cg = 2*warp + lane / 16) computes channels cg*C/8 .. +C/8 for the strip's pixels pg + 16p.
// FMAs take their weights from registers (with constant-bank weight operands they ran at half
// the rate), two channels per packed FMA (__ffma2_rn: each lane one fmaf, so the arithmetic is
// that of the scalar FMA chain).  The distinct dilated input rows of the block (IN_CH input
// channels: the frame itself, or frames t-1, t, t+1) go through the camera transform into
// shared memory first, one global round trip per block, kL1Batch rows of loads in flight at a
// time.  FMA order: bias, then input channel, then taps (ky, kx) row-major.  Outputs are
// staged in shared memory (rows padded by 16 bytes against bank conflicts) so that the stores
// to HBM are whole 16-byte chunks, consecutive across threads.
// (The one-frame BF16 and FP8 cases run k_l1_rp below, which stores from registers.)
template <int C, int OUT, int IN_CH>
__global__ void __launch_bounds__(kL1Tile) k_ingest_l1(const uint16_t* __restrict__ frames, int H, int W, int d,
                                                       int t0, int t_first, int t_last, CamArgs cam,
                                                       const __grid_constant__ L1Params prm, float out_scale,
                                                       void* __restrict__ out, int out_ct) {
  constexpr int CPT = C / kL1ChGroups;
  constexpr int CP = CPT / 2;                             // channel pairs per thread
  constexpr int OB = OUT == 0 ? 4 : (OUT == 1 ? 2 : 1);  // output bytes per channel
  constexpr int OS = C * OB + 16;                        // staged bytes per pixel
  static_assert(CPT % 2 == 0, "channels per thread come in pairs");
  extern __shared__ __align__(16) uint8_t l1_smem[];
  const int span = kL1Tile + 2 * d, nsr = l1_stage_rows(d), R = l1_rows(d);
  float2* xs = reinterpret_cast<float2*>(l1_smem);  // [nsr][IN_CH][span]
  uint8_t* ot = l1_smem + (size_t)nsr * IN_CH * span * 8;
  const int j0 = blockIdx.x * kL1Tile, t = t0 + blockIdx.z, i0 = blockIdx.y * R;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int pg = lane & 15, cg = 2 * warp + (lane >> 4);
  // a staged row is at most 2 * kL1Tile pixels (span <= 256): two elements per thread
#pragma unroll
  for (int ci = 0; ci < IN_CH; ++ci) {
    const int tf = IN_CH == 1 ? t : t + ci - 1;  // source frame of input channel ci
    const bool have = tf >= t_first && tf <= t_last;
    const uint16_t* f = have ? frames + (ptrdiff_t)tf * H * W : frames;  // not read unless have
    for (int sr0 = 0; sr0 < nsr; sr0 += kL1Batch) {
      float adu[kL1Batch][2], g[kL1Batch][2], o[kL1Batch][2];
      bool in[kL1Batch][2];
#pragma unroll
      for (int u = 0; u < kL1Batch; ++u)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int sr = sr0 + u, c = threadIdx.x + k * kL1Tile;
          const int ii = l1_stage_image_row(sr, i0, d), jj = j0 - d + c;
          in[u][k] = have && sr < nsr && c < span && ii >= 0 && ii < H && jj >= 0 && jj < W;
          const size_t px = in[u][k] ? (size_t)ii * W + jj : 0;
          adu[u][k] = in[u][k] ? (float)f[px] : 0.0f;
          g[u][k] = cam.gain_map && in[u][k] ? cam.gain_map[px] : cam.gain;
          o[u][k] = cam.offset_map && in[u][k] ? cam.offset_map[px] : cam.offset;
        }
#pragma unroll
      for (int u = 0; u < kL1Batch; ++u)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int sr = sr0 + u, c = threadIdx.x + k * kL1Tile;
          if (sr < nsr && c < span) {
            // zero outside the frame (the first layer's "same" zero padding)
            const float v = in[u][k] ? cam_transform(adu[u][k], o[u][k], g[u][k], cam.in_scale) : 0.0f;
            xs[((size_t)sr * IN_CH + ci) * span + c] = make_float2(v, v);
          }
        }
    }
  }
  float2 bias[CP];
#pragma unroll
  for (int q = 0; q < CP; ++q) {
    const float* b = prm.b;
    bias[q] = make_float2(b[cg * CPT + 2 * q], b[cg * CPT + 2 * q + 1]);
  }
  // weights of channel pair q, input channel ci, tap k
  auto wpair = [&](int q, int ci, int k) {
    const float* w = prm.w;
    return make_float2(w[((cg * CPT + 2 * q) * IN_CH + ci) * 9 + k], w[((cg * CPT + 2 * q + 1) * IN_CH + ci) * 9 + k]);
  };
  float2 w[IN_CH == 1 ? CP : 1][9];
  if (IN_CH == 1) {
#pragma unroll
    for (int q = 0; q < CP; ++q)
#pragma unroll
      for (int k = 0; k < 9; ++k) w[IN_CH == 1 ? q : 0][k] = wpair(q, 0, k);
  }
  const int npx = W - j0 < kL1Tile ? W - j0 : kL1Tile;  // valid pixels of the strip
  for (int r = 0; r < R; ++r) {
    const int i = i0 + r;
    if (i >= H) break;
    __syncthreads();  // xs is filled; the previous row's ot is written out
    const float2* xr[3];  // staged rows of the three vertical taps
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) xr[ky] = xs + (size_t)l1_srow(r, ky, d) * IN_CH * span;
    // ReLU, quantise and stage one pixel's CPT outputs
    auto stage = [&](int px, const float2 (&acc)[CP]) {
      float a[CPT];
#pragma unroll
      for (int q = 0; q < CP; ++q) {
        a[2 * q] = fmaxf(acc[q].x, 0.0f);
        a[2 * q + 1] = fmaxf(acc[q].y, 0.0f);
      }
      uint8_t* dst = ot + (size_t)px * OS + cg * CPT * OB;
      if (OUT == 0) {
#pragma unroll
        for (int c = 0; c < CPT; ++c) reinterpret_cast<float*>(dst)[c] = a[c];
      } else if (OUT == 1) {
#pragma unroll
        for (int c = 0; c < CPT; c += 2) {
          __nv_bfloat162 h2 = __floats2bfloat162_rn(a[c], a[c + 1]);
          *reinterpret_cast<__nv_bfloat162*>(dst + 2 * c) = h2;
        }
      } else {
#pragma unroll
        for (int c = 0; c < CPT; c += 2)
          *reinterpret_cast<uint16_t*>(dst + c) = __nv_cvt_float2_to_fp8x2(
              make_float2(a[c] * out_scale, a[c + 1] * out_scale), __NV_SATFINITE, __NV_E4M3);
      }
    };
    if (IN_CH == 1) {  // one pixel at a time: its outputs are staged right away
#pragma unroll
      for (int p = 0; p < kL1Px; ++p) {
        const int px = pg + 16 * p;
        float2 x[9];
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
          for (int kx = 0; kx < 3; ++kx) x[ky * 3 + kx] = xr[ky][px + kx * d];
        float2 acc[CP];
#pragma unroll
        for (int q = 0; q < CP; ++q) {
          float2 a = bias[q];
#pragma unroll
          for (int k = 0; k < 9; ++k) a = __ffma2_rn(w[IN_CH == 1 ? q : 0][k], x[k], a);
          acc[q] = a;
        }
        stage(px, acc);
      }
    } else {  // input channel outer, so each channel's weights are loaded once per row
      float2 acc[kL1Px][CP];
#pragma unroll
      for (int p = 0; p < kL1Px; ++p)
#pragma unroll
        for (int q = 0; q < CP; ++q) acc[p][q] = bias[q];
#pragma unroll
      for (int ci = 0; ci < IN_CH; ++ci) {
        float2 wc[CP][9];
#pragma unroll
        for (int q = 0; q < CP; ++q)
#pragma unroll
          for (int k = 0; k < 9; ++k) wc[q][k] = wpair(q, ci, k);
#pragma unroll
        for (int p = 0; p < kL1Px; ++p) {
          const int px = pg + 16 * p;
          float2 x[9];
#pragma unroll
          for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) x[ky * 3 + kx] = xr[ky][(size_t)ci * span + px + kx * d];
#pragma unroll
          for (int q = 0; q < CP; ++q)
#pragma unroll
            for (int k = 0; k < 9; ++k) acc[p][q] = __ffma2_rn(wc[q][k], x[k], acc[p][q]);
        }
      }
#pragma unroll
      for (int p = 0; p < kL1Px; ++p) stage(pg + 16 * p, acc[p]);
    }
    __syncthreads();
    const size_t row = (size_t)t * H + i;
    // index arithmetic below divides by compile-time constants only
    if (OUT == 0) {  // NHWC float: pixels out_ct floats apart, channels 0..C-1 of each
      constexpr int CH = C / 4;  // float4 per pixel
      const int pst = out_ct / 4;
      float4* dst = reinterpret_cast<float4*>(static_cast<float*>(out) + (row * W + j0) * out_ct);
      for (int k = threadIdx.x; k < npx * CH; k += kL1Tile) {
        const int px = k / CH, h = k - px * CH;
        dst[(size_t)px * pst + h] = *reinterpret_cast<const float4*>(ot + (size_t)px * OS + 16 * h);
      }
    } else {  // row-planar [T][H][out_ct/16][W][16 channels]: per group, npx rows of 16*OB bytes
      constexpr int G = C / 16, CH = OB;  // 16-byte chunks per group row
      const int gt = out_ct / 16;         // groups per pixel row of the buffer
      uint8_t* base = static_cast<uint8_t*>(out);
#pragma unroll
      for (int g = 0; g < G; ++g) {
        uint8_t* grow = base + ((row * gt + g) * W + j0) * 16 * OB;
        for (int k = threadIdx.x; k < npx * CH; k += kL1Tile) {
          const int px = k / CH, h = k - px * CH;
          const uint4 v = *reinterpret_cast<const uint4*>(ot + (size_t)px * OS + 16 * g * OB + 16 * h);
          *reinterpret_cast<uint4*>(grow + 16 * k) = v;
        }
      }
    }
  }
}

// The tensor-core precisions' first layer of a one-frame net (OUT = 1: bf16, 2: e4m3 scaled by
// out_scale), stored straight from registers.  A block has G = C/16 warps and covers a
// 128-pixel strip of l1_rows(d) output rows of one frame; warp g writes channel group g: lane
// pair (2u, 2u+1) takes pixels u + 16p (p < 8), the even lane channels 0..7 of the group and
// the odd lane 8..15, so each thread ends a pixel with one 16-byte (bf16) or 8-byte (e4m3)
// store and one warp store covers 16 whole pixel rows of the group.  Staging (camera
// transform of the block's distinct dilated input rows), FMA order (bias, then taps (ky, kx)
// row-major, each lane of the packed FMA one fmaf), ReLU and rounding are those of
// k_ingest_l1, so both give the same bits.  DEVW: weights and bias from device memory.
template <int C, int OUT, bool DEVW>
__global__ void __launch_bounds__(C * 2) k_l1_rp(const uint16_t* __restrict__ frames, int H, int W, int d, int t0,
                                                 CamArgs cam, const __grid_constant__ L1Params prm, float out_scale,
                                                 void* __restrict__ out, int out_ct, const float* __restrict__ wdev,
                                                 const float* __restrict__ bdev) {
  static_assert(OUT == 1 || OUT == 2, "bf16 or e4m3 row-planar output");
  constexpr int NT = C * 2;               // threads: 32 per 16-channel group
  constexpr int OB = OUT == 1 ? 2 : 1;    // output bytes per channel
  extern __shared__ __align__(16) uint8_t l1_smem[];
  const int span = kL1Tile + 2 * d, nsr = l1_stage_rows(d), R = l1_rows(d);
  float2* xs = reinterpret_cast<float2*>(l1_smem);  // [nsr][span]
  const int j0 = blockIdx.x * kL1Tile, t = t0 + blockIdx.z, i0 = blockIdx.y * R;
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int half = lane & 1, u = lane >> 1;
  const uint16_t* f = frames + (ptrdiff_t)t * H * W;
  // staging: kL1Batch elements per thread with their loads in flight together
  const int nst = nsr * span;
  for (int e0 = threadIdx.x; e0 < nst; e0 += kL1Batch * NT) {
    float adu[kL1Batch], gn[kL1Batch], of[kL1Batch];
    bool in[kL1Batch];
#pragma unroll
    for (int k = 0; k < kL1Batch; ++k) {
      const int e = e0 + k * NT, sr = e / span, c = e - sr * span;
      const int ii = l1_stage_image_row(sr, i0, d), jj = j0 - d + c;
      in[k] = e < nst && ii >= 0 && ii < H && jj >= 0 && jj < W;
      const size_t px = in[k] ? (size_t)ii * W + jj : 0;
      adu[k] = in[k] ? (float)f[px] : 0.0f;
      gn[k] = cam.gain_map && in[k] ? cam.gain_map[px] : cam.gain;
      of[k] = cam.offset_map && in[k] ? cam.offset_map[px] : cam.offset;
    }
#pragma unroll
    for (int k = 0; k < kL1Batch; ++k) {
      const int e = e0 + k * NT;
      if (e < nst) {
        // zero outside the frame (the first layer's "same" zero padding)
        const float v = in[k] ? cam_transform(adu[k], of[k], gn[k], cam.in_scale) : 0.0f;
        xs[e] = make_float2(v, v);
      }
    }
  }
  const int c0 = g * 16 + half * 8;  // first channel of this thread
  const float* wsrc = DEVW ? wdev : prm.w;
  const float* bsrc = DEVW ? bdev : prm.b;
  float2 w[4][9], bias[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    bias[q] = make_float2(bsrc[c0 + 2 * q], bsrc[c0 + 2 * q + 1]);
#pragma unroll
    for (int k = 0; k < 9; ++k) w[q][k] = make_float2(wsrc[(c0 + 2 * q) * 9 + k], wsrc[(c0 + 2 * q + 1) * 9 + k]);
  }
  __syncthreads();
  const int npx = W - j0 < kL1Tile ? W - j0 : kL1Tile;  // valid pixels of the strip
  const int gt = out_ct / 16;                            // groups per pixel row of the buffer
  for (int r = 0; r < R; ++r) {
    const int i = i0 + r;
    if (i >= H) break;
    const float2* xr[3];
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) xr[ky] = xs + (size_t)l1_srow(r, ky, d) * span;
    uint8_t* dst = static_cast<uint8_t*>(out) + ((((size_t)t * H + i) * gt + g) * W + j0) * (16 * OB) + half * 8 * OB;
#pragma unroll
    for (int p = 0; p < kL1Px; ++p) {
      const int px = u + 16 * p;
      float2 x[9];
#pragma unroll
      for (int ky = 0; ky < 3; ++ky)
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) x[ky * 3 + kx] = xr[ky][px + kx * d];
      uint32_t ow[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float2 a = bias[q];
#pragma unroll
        for (int k = 0; k < 9; ++k) a = __ffma2_rn(w[q][k], x[k], a);
        const float lo = fmaxf(a.x, 0.0f), hi = fmaxf(a.y, 0.0f);
        if (OUT == 1) {
          __nv_bfloat162 h2 = __floats2bfloat162_rn(lo, hi);
          ow[q] = *reinterpret_cast<uint32_t*>(&h2);
        } else {
          ow[q] = __nv_cvt_float2_to_fp8x2(make_float2(lo * out_scale, hi * out_scale), __NV_SATFINITE, __NV_E4M3);
        }
      }
      if (px < npx) {
        if (OUT == 1)
          *reinterpret_cast<uint4*>(dst + (size_t)px * 32) = make_uint4(ow[0], ow[1], ow[2], ow[3]);
        else
          *reinterpret_cast<uint2*>(dst + (size_t)px * 16) = make_uint2(ow[0] | (ow[1] << 16), ow[2] | (ow[3] << 16));
      }
    }
  }
}

// Heads of one pixel from its CO final activations (one fully unrolled loop per head count).
template <int CO, int NH>
__device__ __forceinline__ void f32_heads_out(const float (&acc)[CO], const float* __restrict__ hw,
                                              const float* __restrict__ hb, int t, size_t px, size_t plane,
                                              float* __restrict__ maps, float* __restrict__ logits) {
#pragma unroll
  for (int k = 0; k < NH; ++k) {
    float h = hb[k];
#pragma unroll
    for (int c = 0; c < CO; ++c) h = fmaf(hw[k * CO + c], acc[c], h);
    if (k == 0) {
      if (logits) logits[(size_t)t * plane + px] = h;
      h = 1.0f / (1.0f + expf(-h));
    } else if (k >= kHeads) {
      h = softplus_f(h);
    }
    maps[((size_t)t * NH + k) * plane + px] = h;
  }
}

// FP32 dilated conv: one thread per pixel, all CO output channels in registers.  Input
// channels 0..ci-1 of pixels in_ct floats apart; outputs at channel out_off of pixels out_ct
// floats apart (a channel range of a dense block's concatenation, or the whole pixel).
// Weights in shared memory as [tap][ci][co]; each float4 read is a warp-wide broadcast.
template <int CO, bool HEADS>
__global__ void __launch_bounds__(kSimtThreads) k_dconv_f32(const F32LayerArgs a, const float* __restrict__ hw,
                                                            const float* __restrict__ hb, int nh,
                                                            float* __restrict__ maps, float* __restrict__ logits) {
  extern __shared__ float4 smem4[];
  float* sw = reinterpret_cast<float*>(smem4);
  const int ci_n = a.ci, H = a.H, W = a.W, d = a.d;
  for (int k = threadIdx.x; k < 9 * ci_n * CO / 4; k += blockDim.x) smem4[k] = reinterpret_cast<const float4*>(a.w)[k];
  __syncthreads();
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long npx = (long long)a.T * H * W;
  if (q >= npx) return;
  int j = (int)(q % W);
  int i = (int)((q / W) % H);
  int t = (int)(q / ((long long)H * W));
  float acc[CO];
#pragma unroll
  for (int co = 0; co < CO; ++co) acc[co] = a.b[co];
  for (int ky = 0; ky < 3; ++ky) {
    int ii = i + (ky - 1) * d;
    if (ii < 0 || ii >= H) continue;
    for (int kx = 0; kx < 3; ++kx) {
      int jj = j + (kx - 1) * d;
      if (jj < 0 || jj >= W) continue;
      const float4* src = reinterpret_cast<const float4*>(a.in + (((size_t)t * H + ii) * W + jj) * a.in_ct);
      const float* wt = sw + (ky * 3 + kx) * ci_n * CO;
#pragma unroll 2
      for (int c4 = 0; c4 < ci_n / 4; ++c4) {
        float4 v = __ldg(src + c4);
        float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float4* wr = reinterpret_cast<const float4*>(wt + (4 * c4 + e) * CO);
#pragma unroll
          for (int o4 = 0; o4 < CO / 4; ++o4) {
            float4 ww = wr[o4];
            acc[4 * o4 + 0] = fmaf(vv[e], ww.x, acc[4 * o4 + 0]);
            acc[4 * o4 + 1] = fmaf(vv[e], ww.y, acc[4 * o4 + 1]);
            acc[4 * o4 + 2] = fmaf(vv[e], ww.z, acc[4 * o4 + 2]);
            acc[4 * o4 + 3] = fmaf(vv[e], ww.w, acc[4 * o4 + 3]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int co = 0; co < CO; ++co) acc[co] = fmaxf(acc[co], 0.0f);
  if (!HEADS) {
    float4* dst = reinterpret_cast<float4*>(a.out + (size_t)q * a.out_ct + a.out_off);
#pragma unroll
    for (int c4 = 0; c4 < CO / 4; ++c4)
      dst[c4] = make_float4(acc[4 * c4], acc[4 * c4 + 1], acc[4 * c4 + 2], acc[4 * c4 + 3]);
  } else {
    // 1x1 heads (Sec. 3.2): h_k = hb[k] + sum_c hw[k,c] a[c]; p = sigmoid(h_0); the
    // uncertainty heads (k >= 5) are softplus(h_k)
    size_t plane = (size_t)H * W;
    size_t px = (size_t)i * W + j;
    if (nh == kHeads)
      f32_heads_out<CO, kHeads>(acc, hw, hb, t, px, plane, maps, logits);
    else
      f32_heads_out<CO, kMaxHeads>(acc, hw, hb, t, px, plane, maps, logits);
  }
}

// Maximum of post-ReLU activations (all >= 0, so float bit patterns order like unsigned) over
// rows of seg consecutive elements, stride elements apart: one layer's output channels inside
// a wider buffer (BF16 row-planar: its groups of every pixel row; FP32 NHWC: its channels of
// every pixel).
template <bool BF16>
__global__ void __launch_bounds__(256) k_amax(const void* __restrict__ x, size_t rows, size_t seg, size_t stride,
                                              unsigned* __restrict__ out) {
  float m = 0.0f;
  const size_t n = rows * seg;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    const size_t r = k / seg, e = r * stride + (k - r * seg);
    float v = BF16 ? __bfloat162float(static_cast<const __nv_bfloat16*>(x)[e]) : static_cast<const float*>(x)[e];
    m = fmaxf(m, v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

inline unsigned grid_for(long long npx) { return (unsigned)((npx + kSimtThreads - 1) / kSimtThreads); }

}  // namespace

// The register-store first layer (k_l1_rp): its staged rows take at most 26 KB.
template <int C, int OUT, bool DEVW>
static cudaError_t launch_l1_rp(const uint16_t* frames, int T, int H, int W, int d, const CamArgs& cam,
                                const L1Params& prm, float out_scale, void* out, int out_ct, const float* wdev,
                                const float* bdev, cudaStream_t s) {
  const size_t smem = (size_t)l1_stage_rows(d) * (kL1Tile + 2 * d) * 8;
  for (int t0 = 0; t0 < T; t0 += 65535) {
    dim3 grid((W + kL1Tile - 1) / kL1Tile, (H + l1_rows(d) - 1) / l1_rows(d), (unsigned)(T - t0 < 65535 ? T - t0 : 65535));
    k_l1_rp<C, OUT, DEVW><<<grid, C * 2, smem, s>>>(frames, H, W, d, t0, cam, prm, out_scale, out, out_ct, wdev, bdev);
  }
  return cudaGetLastError();
}

template <int C, int OUT, int IN_CH>
static cudaError_t launch_l1(const uint16_t* frames, int T, int H, int W, int d, int t_first, int t_last,
                             const CamArgs& cam, const L1Params& prm, float out_scale, void* out, int out_ct,
                             cudaStream_t s) {
  if constexpr (OUT != 0 && IN_CH == 1) {
    return launch_l1_rp<C, OUT, false>(frames, T, H, W, d, cam, prm, out_scale, out, out_ct, nullptr, nullptr, s);
  } else {
    const size_t smem = l1_smem_bytes<C, OUT, IN_CH>(d);
    // opt in to more than 48 KB on the current device, to the largest size any dilation takes
    // (the same value on every launch: no host state, and no race between threads or devices)
    cudaError_t e = cudaFuncSetAttribute(
        k_ingest_l1<C, OUT, IN_CH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)std::max(l1_smem_bytes<C, OUT, IN_CH>(4), l1_smem_bytes<C, OUT, IN_CH>(kL1MaxD)));
    if (e != cudaSuccess) return e;
    for (int t0 = 0; t0 < T; t0 += 65535) {
      dim3 grid((W + kL1Tile - 1) / kL1Tile, (H + l1_rows(d) - 1) / l1_rows(d),
                (unsigned)(T - t0 < 65535 ? T - t0 : 65535)),
          block(kL1Tile);
      k_ingest_l1<C, OUT, IN_CH><<<grid, block, smem, s>>>(frames, H, W, d, t0, t_first, t_last, cam, prm, out_scale,
                                                           out, out_ct);
    }
    return cudaGetLastError();
  }
}

// BF16 training's first layer: weights from device memory, bf16 row-planar output.
template <int C>
static cudaError_t launch_l1_devw(const uint16_t* frames, int T, int H, int W, int d, const CamArgs& cam,
                                  const float* wdev, const float* bdev, void* out, cudaStream_t s) {
  L1Params prm;
  memset(&prm, 0, sizeof(prm));
  return launch_l1_rp<C, 1, true>(frames, T, H, W, d, cam, prm, 1.0f, out, C, wdev, bdev, s);
}

template <int C>
static cudaError_t launch_l1_prec(const uint16_t* frames, int T, int H, int W, int d, int in_ch, int t_first,
                                  int t_last, const CamArgs& cam, const L1Params& prm, int prec, float out_scale,
                                  void* out, int out_ct, cudaStream_t s) {
  if (in_ch == 1) {
    if (prec == kFP32) return launch_l1<C, 0, 1>(frames, T, H, W, d, t_first, t_last, cam, prm, out_scale, out, out_ct, s);
    if (prec == kBF16) return launch_l1<C, 1, 1>(frames, T, H, W, d, t_first, t_last, cam, prm, out_scale, out, out_ct, s);
    return launch_l1<C, 2, 1>(frames, T, H, W, d, t_first, t_last, cam, prm, out_scale, out, out_ct, s);
  }
  if (prec == kFP32) return launch_l1<C, 0, 3>(frames, T, H, W, d, t_first, t_last, cam, prm, out_scale, out, out_ct, s);
  if (prec == kBF16) return launch_l1<C, 1, 3>(frames, T, H, W, d, t_first, t_last, cam, prm, out_scale, out, out_ct, s);
  return launch_l1<C, 2, 3>(frames, T, H, W, d, t_first, t_last, cam, prm, out_scale, out, out_ct, s);
}

cudaError_t launch_ingest_l1_devw(const uint16_t* frames, int T, int H, int W, int d, CamArgs cam, const float* w1_dev,
                                  const float* b1_dev, int C, void* out, cudaStream_t s) {
  if ((long long)T * H * W == 0) return cudaSuccess;
  if (d < 1 || d > kL1MaxD) return cudaErrorInvalidValue;
  switch (C) {
    case 16: return launch_l1_devw<16>(frames, T, H, W, d, cam, w1_dev, b1_dev, out, s);
    case 32: return launch_l1_devw<32>(frames, T, H, W, d, cam, w1_dev, b1_dev, out, s);
    case 48: return launch_l1_devw<48>(frames, T, H, W, d, cam, w1_dev, b1_dev, out, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_ingest_l1(const uint16_t* frames, int T, int H, int W, int d, CamArgs cam, const float* w1,
                             const float* b1, int C, int in_ch, int t_first, int t_last, int prec, float out_scale,
                             void* out, int out_ct, cudaStream_t s) {
  if ((long long)T * H * W == 0) return cudaSuccess;
  if (d < 1 || d > kL1MaxD || C > 64 || (in_ch != 1 && in_ch != 3)) return cudaErrorInvalidValue;
  if (t_first > 0 || t_last < T - 1) return cudaErrorInvalidValue;
  if (out_ct < C || out_ct % 16) return cudaErrorInvalidValue;
  // w1/b1 are host copies here: they travel as a kernel parameter
  L1Params prm;
  memset(&prm, 0, sizeof(prm));
  memcpy(prm.w, w1, sizeof(float) * C * in_ch * 9);
  memcpy(prm.b, b1, sizeof(float) * C);
  switch (C) {
    case 16: return launch_l1_prec<16>(frames, T, H, W, d, in_ch, t_first, t_last, cam, prm, prec, out_scale, out, out_ct, s);
    case 32: return launch_l1_prec<32>(frames, T, H, W, d, in_ch, t_first, t_last, cam, prm, prec, out_scale, out, out_ct, s);
    case 48: return launch_l1_prec<48>(frames, T, H, W, d, in_ch, t_first, t_last, cam, prm, prec, out_scale, out, out_ct, s);
    case 64: return launch_l1_prec<64>(frames, T, H, W, d, in_ch, t_first, t_last, cam, prm, prec, out_scale, out, out_ct, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_amax(const void* x, int prec, int T, int H, int W, int ct, int off, int cnt, unsigned* out,
                        cudaStream_t s) {
  if (T <= 0 || cnt <= 0) return cudaSuccess;
  if (off < 0 || off + cnt > ct) return cudaErrorInvalidValue;
  if (prec == kFP32) {  // NHWC: channels [off, off + cnt) of every pixel
    k_amax<false><<<1024, 256, 0, s>>>(static_cast<const float*>(x) + off, (size_t)T * H * W, (size_t)cnt, (size_t)ct, out);
  } else if (prec == kBF16) {  // row-planar: groups [off / 16, (off + cnt) / 16) of every pixel row
    if (off % 16 || cnt % 16 || ct % 16) return cudaErrorInvalidValue;
    k_amax<true><<<1024, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(x) + (size_t)(off / 16) * W * 16, (size_t)T * H,
                                      (size_t)(cnt / 16) * W * 16, (size_t)(ct / 16) * W * 16, out);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int CO, bool HEADS>
static cudaError_t launch_f32_impl(const F32LayerArgs& a, const float* hw, const float* hb, int nh, float* maps,
                                   float* logits, cudaStream_t s) {
  if (HEADS && nh != kHeads && nh != kMaxHeads) return cudaErrorInvalidValue;
  if (a.ci < 4 || a.ci % 4 || a.ci * CO > kF32MaxWeights || a.in_ct < a.ci || a.in_ct % 4) return cudaErrorInvalidValue;
  if (!HEADS && (a.out_off < 0 || a.out_off % 4 || a.out_off + CO > a.out_ct || a.out_ct % 4)) return cudaErrorInvalidValue;
  size_t smem = sizeof(float) * 9 * a.ci * CO;
  // the weight image may exceed 48 KB: opt in on the current device to the largest image
  // (the same value on every launch)
  cudaError_t e = cudaFuncSetAttribute(k_dconv_f32<CO, HEADS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(float) * 9 * kF32MaxWeights);
  if (e != cudaSuccess) return e;
  long long npx = (long long)a.T * a.H * a.W;
  if (npx == 0) return cudaSuccess;
  k_dconv_f32<CO, HEADS><<<grid_for(npx), kSimtThreads, smem, s>>>(a, hw, hb, nh, maps, logits);
  return cudaGetLastError();
}

cudaError_t launch_dconv_f32(const F32LayerArgs& a, cudaStream_t s) {
  switch (a.co) {
    case 16: return launch_f32_impl<16, false>(a, nullptr, nullptr, 0, nullptr, nullptr, s);
    case 32: return launch_f32_impl<32, false>(a, nullptr, nullptr, 0, nullptr, nullptr, s);
    case 48: return launch_f32_impl<48, false>(a, nullptr, nullptr, 0, nullptr, nullptr, s);
    case 64: return launch_f32_impl<64, false>(a, nullptr, nullptr, 0, nullptr, nullptr, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_dconv_f32_heads(const F32LayerArgs& a, const float* hw, const float* hb, int nh, float* maps,
                                   float* logits, cudaStream_t s) {
  if (a.ci != a.co) return cudaErrorInvalidValue;
  switch (a.co) {
    case 16: return launch_f32_impl<16, true>(a, hw, hb, nh, maps, logits, s);
    case 32: return launch_f32_impl<32, true>(a, hw, hb, nh, maps, logits, s);
    case 48: return launch_f32_impl<48, true>(a, hw, hb, nh, maps, logits, s);
    case 64: return launch_f32_impl<64, true>(a, hw, hb, nh, maps, logits, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace sml
