// Training kernels (FP32, NHWC activations): forward and hand-written backward of the dilated
// 3x3 conv + bias + ReLU layer (dilated convolution, Sec. 3.2.1), and the fused 1x1 heads +
// loss + head gradients (binary cross-entropy on p, Sec. 3.3, plus a masked L2 on the
// offset, z and photon heads).  Weights use the PyTorch layout [Cout][Cin][3][3]; the
// kernels re-lay them out while staging them in shared memory.
//
// Reductions over pixels (weight, bias and head gradients, the loss) go through per-block
// partial sums and a second kernel that adds them in block order, so every result is
// deterministic.
#include <cuda_bf16.h>

#include <cstring>

#include "sml_internal.h"

namespace sml {

namespace {

constexpr int kTThreads = 128;

// Direct conv, one thread per pixel, CO accumulators.
//   forward (DGRAD = false): out[q, o] = ReLU(b[o] + sum_{tap,i} w[o][i][tap] in[q + off(tap), i])
//   dgrad   (DGRAD = true):  out[q, i] = sum_{tap,o} w[o][i][tap] dz[q - off(tap), o],
//                            dz = in * [mask > 0]  (in = dy, mask = the layer's ReLU output)
// In the dgrad case CI is the layer's Cout and CO its Cin; the tap is mirrored.
template <int CI, int CO, bool DGRAD>
__global__ void __launch_bounds__(kTThreads) k_tconv(const float* __restrict__ in, const float* __restrict__ mask,
                                                     const float* __restrict__ w, const float* __restrict__ b,
                                                     float* __restrict__ out, int B, int H, int W, int d) {
  extern __shared__ float sw[];  // [tap][CI][CO]
  for (int k = threadIdx.x; k < 9 * CI * CO; k += blockDim.x) {
    int co = k % CO, ci = (k / CO) % CI, tap = k / (CO * CI);
    // forward: w[co][ci][tap]; dgrad: channels swap roles and the tap is mirrored
    sw[k] = DGRAD ? w[((size_t)ci * CO + co) * 9 + (8 - tap)] : w[((size_t)co * CI + ci) * 9 + tap];
  }
  __syncthreads();
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)B * H * W) return;
  int j = (int)(q % W), i = (int)((q / W) % H), t = (int)(q / ((long long)H * W));
  float acc[CO];
#pragma unroll
  for (int o = 0; o < CO; ++o) acc[o] = DGRAD ? 0.0f : b[o];
  for (int ky = 0; ky < 3; ++ky) {
    int ii = i + (ky - 1) * d;
    if (ii < 0 || ii >= H) continue;
    for (int kx = 0; kx < 3; ++kx) {
      int jj = j + (kx - 1) * d;
      if (jj < 0 || jj >= W) continue;
      size_t src = (((size_t)t * H + ii) * W + jj) * CI;
      const float* wt = sw + (ky * 3 + kx) * CI * CO;
      for (int c = 0; c < CI; ++c) {
        float v = in[src + c];
        if (DGRAD) v = mask[src + c] > 0.0f ? v : 0.0f;
#pragma unroll
        for (int o = 0; o < CO; ++o) acc[o] = fmaf(v, wt[c * CO + o], acc[o]);
      }
    }
  }
  float* dst = out + (size_t)q * CO;
#pragma unroll
  for (int o = 0; o < CO; ++o) dst[o] = DGRAD ? acc[o] : fmaxf(acc[o], 0.0f);
}

// Weight/bias gradient partials: block b owns a contiguous pixel range; thread (co, r) owns
// the k-range [r*KPT, (r+1)*KPT) of k = tap*CI + ci for output channel co.
constexpr int kWgPx = 8;  // pixels staged per step

template <int CI, int CO>
struct WgCfg {
  static constexpr int R = (256 + CO - 1) / CO;
  static constexpr int THREADS = CO * R;
  static constexpr int K = 9 * CI;
  static constexpr int KPT = (((K + R - 1) / R) + 3) & ~3;
  static constexpr int NOUT = CO * K + CO;  // dw then db
};

// RP = true: dy holds dz itself, as bf16 row-planar activations [B][H][CO/16][W][16] (the ReLU
// mask already applied; y unused) -- the first layer's gradient in BF16 training.
template <int CI, int CO, bool RP = false>
__global__ void __launch_bounds__(WgCfg<CI, CO>::THREADS) k_wgrad_partial(const float* __restrict__ x,
                                                                          const void* __restrict__ dy,
                                                                          const float* __restrict__ y, int B, int H,
                                                                          int W, int d, long long px_per_block,
                                                                          float* __restrict__ partial) {
  using Cfg = WgCfg<CI, CO>;
  __shared__ __align__(16) float xs[kWgPx][Cfg::K + 4];
  __shared__ float zs[kWgPx][CO];
  const int co = threadIdx.x % CO, r = threadIdx.x / CO;
  const int k0 = r * Cfg::KPT;
  float acc[Cfg::KPT];
#pragma unroll
  for (int k = 0; k < Cfg::KPT; ++k) acc[k] = 0.0f;
  float accb = 0.0f;
  const long long npx = (long long)B * H * W;
  const long long p0 = (long long)blockIdx.x * px_per_block;
  const long long p1 = p0 + px_per_block < npx ? p0 + px_per_block : npx;
  for (long long base = p0; base < p1; base += kWgPx) {
    __syncthreads();
    for (int e = threadIdx.x; e < kWgPx * (Cfg::K + CO); e += blockDim.x) {
      int p = e / (Cfg::K + CO), k = e - p * (Cfg::K + CO);
      long long q = base + p;
      float v = 0.0f;
      if (q < p1) {
        int j = (int)(q % W), i = (int)((q / W) % H), t = (int)(q / ((long long)H * W));
        if (k < Cfg::K) {
          int tap = k / CI, ci = k - tap * CI;
          int ii = i + (tap / 3 - 1) * d, jj = j + (tap % 3 - 1) * d;
          if (ii >= 0 && ii < H && jj >= 0 && jj < W) v = x[(((size_t)t * H + ii) * W + jj) * CI + ci];
          xs[p][k] = v;
        } else {
          int o = k - Cfg::K;
          if (RP) {
            const size_t src = ((((size_t)t * H + i) * (CO / 16) + o / 16) * W + j) * 16 + (o % 16);
            v = __bfloat162float(static_cast<const __nv_bfloat16*>(dy)[src]);
          } else {
            const size_t src = (size_t)q * CO + o;
            v = y[src] > 0.0f ? static_cast<const float*>(dy)[src] : 0.0f;
          }
          zs[p][o] = v;
        }
      } else {
        if (k < Cfg::K) xs[p][k] = 0.0f;
        else zs[p][k - Cfg::K] = 0.0f;
      }
    }
    __syncthreads();
#pragma unroll 1
    for (int p = 0; p < kWgPx; ++p) {
      const float z = zs[p][co];
      accb += z;
#pragma unroll
      for (int k = 0; k < Cfg::KPT; ++k)
        if (k0 + k < Cfg::K) acc[k] = fmaf(z, xs[p][k0 + k], acc[k]);
    }
  }
  float* dst = partial + (size_t)blockIdx.x * Cfg::NOUT;
#pragma unroll
  for (int k = 0; k < Cfg::KPT; ++k)
    if (k0 + k < Cfg::K) dst[(size_t)co * Cfg::K + k0 + k] = acc[k];
  if (r == 0) dst[CO * Cfg::K + co] = accb;
}

// Sum partials over blocks in block order; write dw in [Cout][Cin][3][3] and db.
template <int CI, int CO>
__global__ void k_wgrad_reduce(const float* __restrict__ partial, int nblocks, float* __restrict__ dw,
                               float* __restrict__ db) {
  using Cfg = WgCfg<CI, CO>;
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= Cfg::NOUT) return;
  float s = 0.0f;
  for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * Cfg::NOUT + o];
  if (o < CO * Cfg::K) {
    int co = o / Cfg::K, k = o - co * Cfg::K, tap = k / CI, ci = k - tap * CI;
    dw[((size_t)co * CI + ci) * 9 + tap] = s;
  } else {
    db[o - CO * Cfg::K] = s;
  }
}

// --- heads + loss --------------------------------------------------------------------
constexpr int kHThreads = 256;

// Number of target pixels (target p > 0.5), per-block partial counts.
__global__ void __launch_bounds__(kHThreads) k_count_targets(const float* __restrict__ tgt, int B, int HW,
                                                             float* __restrict__ partial) {
  __shared__ float s[kHThreads];
  long long n = (long long)B * HW;
  float c = 0.0f;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    long long b = q / HW, px = q - b * HW;
    c += tgt[(size_t)b * kHeads * HW + px] > 0.5f ? 1.0f : 0.0f;
  }
  s[threadIdx.x] = c;
  __syncthreads();
  for (int o = kHThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}

// Per pixel: heads, loss terms and (optionally) gradients.  Partial layout per block:
// [0] BCE sum, [1] L2 sum, [2 .. 2+5C) dhw, [2+5C .. 2+5C+5) dhb.
// RP = true (BF16 training): a holds bf16 row-planar activations [B][H][C/16][W][16], and da
// receives dz = (d loss / d a) * [a > 0] (the last conv layer's ReLU mask applied), rounded to
// bf16, in the same layout.
template <int C, bool RP = false>
__global__ void __launch_bounds__(kHThreads) k_heads_loss(const void* __restrict__ a, const float* __restrict__ tgt,
                                                          int B, int HW, int W, const float* __restrict__ hw,
                                                          const float* __restrict__ hb, float* __restrict__ h,
                                                          const float* __restrict__ nt_partial, int nt_blocks,
                                                          const float* __restrict__ grad_scale, void* __restrict__ da,
                                                          float* __restrict__ partial) {
  extern __shared__ float sm[];
  float* s_a = sm;                       // [kHThreads][C]
  float* s_dh = s_a + kHThreads * C;     // [kHThreads][5]
  float* s_l = s_dh + kHThreads * kHeads;  // [kHThreads][2]
  __shared__ float s_hw[kHeads * C];
  __shared__ float s_hb[kHeads];
  for (int k = threadIdx.x; k < kHeads * C; k += blockDim.x) s_hw[k] = hw[k];
  if (threadIdx.x < kHeads) s_hb[threadIdx.x] = hb[threadIdx.x];
  __syncthreads();
  float nt = 0.0f;
  for (int b = 0; b < nt_blocks; ++b) nt += nt_partial[b];
  const long long npx = (long long)B * HW;
  const float inv_npx = 1.0f / (float)npx;
  const float inv_nt = 1.0f / (nt > 0.0f ? nt : 1.0f);
  const float gs = grad_scale ? *grad_scale : 0.0f;
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float bce = 0.0f, l2 = 0.0f;
  float dh[kHeads] = {0, 0, 0, 0, 0};
  if (q < npx) {
    long long b = q / HW, px = q - b * HW;
    float av[C];
    // row-planar: group g of pixel (b, i, j) at (((b H + i) G + g) W + j) x 16 elements
    const size_t rp0 = RP ? (((size_t)b * (HW / W) + px / W) * (C / 16) * W + px % W) * 16 : 0;
    if (RP) {
      const __nv_bfloat16* ap = static_cast<const __nv_bfloat16*>(a);
#pragma unroll
      for (int c = 0; c < C; ++c) av[c] = __bfloat162float(ap[rp0 + (size_t)(c / 16) * W * 16 + (c % 16)]);
    } else {
      const float* ap = static_cast<const float*>(a) + (size_t)q * C;
#pragma unroll
      for (int c = 0; c < C; ++c) av[c] = ap[c];
    }
    float hv[kHeads];
#pragma unroll
    for (int k = 0; k < kHeads; ++k) {
      float s = s_hb[k];
#pragma unroll
      for (int c = 0; c < C; ++c) s = fmaf(s_hw[k * C + c], av[c], s);
      hv[k] = s;
      h[((size_t)b * kHeads + k) * HW + px] = s;
    }
    const float* tp = tgt + (size_t)b * kHeads * HW + px;
    float y0 = tp[0];
    float h0 = hv[0];
    bce = fmaxf(h0, 0.0f) - h0 * y0 + log1pf(expf(-fabsf(h0)));
    dh[0] = (1.0f / (1.0f + expf(-h0)) - y0) * inv_npx * gs;
    bool m = y0 > 0.5f;
#pragma unroll
    for (int k = 1; k < kHeads; ++k) {
      float e = m ? hv[k] - tp[(size_t)k * HW] : 0.0f;
      l2 = fmaf(e, e, l2);
      dh[k] = 2.0f * e * inv_nt * gs;
    }
    if (da) {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < kHeads; ++k) s = fmaf(s_hw[k * C + c], dh[k], s);
        if (RP)
          static_cast<__nv_bfloat16*>(da)[rp0 + (size_t)(c / 16) * W * 16 + (c % 16)] =
              __float2bfloat16_rn(av[c] > 0.0f ? s : 0.0f);
        else
          static_cast<float*>(da)[(size_t)q * C + c] = s;
      }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) s_a[threadIdx.x * C + c] = av[c];
  } else {
#pragma unroll
    for (int c = 0; c < C; ++c) s_a[threadIdx.x * C + c] = 0.0f;
  }
#pragma unroll
  for (int k = 0; k < kHeads; ++k) s_dh[threadIdx.x * kHeads + k] = dh[k];
  s_l[threadIdx.x * 2] = bce;
  s_l[threadIdx.x * 2 + 1] = l2;
  __syncthreads();
  float* dst = partial + (size_t)blockIdx.x * (2 + kHeads * C + kHeads);
  for (int o = threadIdx.x; o < 2 + kHeads * C + kHeads; o += blockDim.x) {
    float s = 0.0f;
    if (o < 2) {
      for (int p = 0; p < kHThreads; ++p) s += s_l[p * 2 + o];
    } else if (o < 2 + kHeads * C) {
      int k = (o - 2) / C, c = (o - 2) - k * C;
      for (int p = 0; p < kHThreads; ++p) s = fmaf(s_dh[p * kHeads + k], s_a[p * C + c], s);
    } else {
      int k = o - 2 - kHeads * C;
      for (int p = 0; p < kHThreads; ++p) s += s_dh[p * kHeads + k];
    }
    dst[o] = s;
  }
}

__global__ void k_heads_reduce(const float* __restrict__ partial, int nblocks, int C, long long npx,
                               const float* __restrict__ nt_partial, int nt_blocks, float* __restrict__ loss,
                               float* __restrict__ dhw, float* __restrict__ dhb) {
  const int nout = 2 + kHeads * C + kHeads;
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nout) return;
  float s = 0.0f;
  for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * nout + o];
  if (o == 0) {
    float nt = 0.0f;
    for (int b = 0; b < nt_blocks; ++b) nt += nt_partial[b];
    float l2 = 0.0f;
    for (int b = 0; b < nblocks; ++b) l2 += partial[(size_t)b * nout + 1];
    *loss = s / (float)npx + l2 / (nt > 0.0f ? nt : 1.0f);
  } else if (o >= 2 && o < 2 + kHeads * C) {
    if (dhw) dhw[o - 2] = s;
  } else if (o >= 2 + kHeads * C) {
    if (dhb) dhb[o - 2 - kHeads * C] = s;
  }
}

__global__ void k_train_ingest(const uint16_t* __restrict__ f, long long n, float gain, float offset, float in_scale,
                               float* __restrict__ x0) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) x0[q] = __fmul_rn(__fdiv_rn(__fsub_rn((float)f[q], offset), gain), in_scale);
}

constexpr int kWgBlocks = 304;
constexpr int kNtBlocks = 64;

template <int CI, int CO>
cudaError_t conv_fwd_impl(const float* x, int B, int H, int W, int d, const float* w, const float* b, float* y,
                          cudaStream_t s) {
  size_t smem = sizeof(float) * 9 * CI * CO;
  cudaError_t e = cudaFuncSetAttribute(k_tconv<CI, CO, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  long long npx = (long long)B * H * W;
  k_tconv<CI, CO, false><<<(unsigned)((npx + kTThreads - 1) / kTThreads), kTThreads, smem, s>>>(x, nullptr, w, b, y, B,
                                                                                                   H, W, d);
  return cudaGetLastError();
}

template <int CI, int CO>
cudaError_t conv_bwd_impl(const float* x, const float* y, const float* dy, int B, int H, int W, int d, const float* w,
                          float* dx, float* dw, float* db, float* work, cudaStream_t s) {
  long long npx = (long long)B * H * W;
  cudaError_t e;
  if (dx) {
    size_t smem = sizeof(float) * 9 * CI * CO;
    e = cudaFuncSetAttribute(k_tconv<CO, CI, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_tconv<CO, CI, true><<<(unsigned)((npx + kTThreads - 1) / kTThreads), kTThreads, smem, s>>>(dy, y, w, nullptr, dx,
                                                                                                  B, H, W, d);
  }
  using Cfg = WgCfg<CI, CO>;
  long long ppb = (npx + kWgBlocks - 1) / kWgBlocks;
  ppb = (ppb + kWgPx - 1) / kWgPx * kWgPx;
  int nb = (int)((npx + ppb - 1) / ppb);
  k_wgrad_partial<CI, CO><<<nb, Cfg::THREADS, 0, s>>>(x, dy, y, B, H, W, d, ppb, work);
  k_wgrad_reduce<CI, CO><<<(Cfg::NOUT + 255) / 256, 256, 0, s>>>(work, nb, dw, db);
  return cudaGetLastError();
}

template <int C, bool RP = false>
cudaError_t heads_impl(const void* a, const float* tgt, int B, int H, int W, const float* hw, const float* hb,
                       float* h, float* loss, const float* gscale, void* da, float* dhw, float* dhb, float* work,
                       cudaStream_t s) {
  const int HW = H * W;
  long long npx = (long long)B * HW;
  int nb = (int)((npx + kHThreads - 1) / kHThreads);
  float* nt_partial = work;
  float* partial = work + kNtBlocks;
  size_t smem = sizeof(float) * kHThreads * (C + kHeads + 2);
  cudaError_t e = cudaFuncSetAttribute(k_heads_loss<C, RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_count_targets<<<kNtBlocks, kHThreads, 0, s>>>(tgt, B, HW, nt_partial);
  k_heads_loss<C, RP><<<nb, kHThreads, smem, s>>>(a, tgt, B, HW, W, hw, hb, h, nt_partial, kNtBlocks, gscale, da,
                                                  partial);
  int nout = 2 + kHeads * C + kHeads;
  k_heads_reduce<<<(nout + 255) / 256, 256, 0, s>>>(partial, nb, C, npx, nt_partial, kNtBlocks, loss, dhw, dhb);
  return cudaGetLastError();
}

}  // namespace

size_t train_conv_work_bytes(int B, int H, int W, int cin, int cout) {
  (void)B;
  (void)H;
  (void)W;
  return sizeof(float) * (size_t)kWgBlocks * ((size_t)cout * 9 * cin + cout);
}

size_t train_heads_work_bytes(int B, int H, int W, int C) {
  long long npx = (long long)B * H * W;
  long long nb = (npx + kHThreads - 1) / kHThreads;
  return sizeof(float) * ((size_t)kNtBlocks + (size_t)nb * (2 + kHeads * C + kHeads));
}

#define SML_CH_SWITCH(C, CALL) \
  switch (C) {                 \
    case 16: CALL(16); break;  \
    case 32: CALL(32); break;  \
    case 48: CALL(48); break;  \
    case 64: CALL(64); break;  \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t train_conv_fwd(const float* x, int B, int H, int W, int cin, int cout, int d, const float* w,
                           const float* b, float* y, cudaStream_t s) {
  if ((long long)B * H * W == 0) return cudaSuccess;
  if (cin == 1) {
#define F1(CO) return conv_fwd_impl<1, CO>(x, B, H, W, d, w, b, y, s)
    SML_CH_SWITCH(cout, F1)
#undef F1
  }
  if (cin != cout) return cudaErrorInvalidValue;
#define FC(CO) return conv_fwd_impl<CO, CO>(x, B, H, W, d, w, b, y, s)
  SML_CH_SWITCH(cout, FC)
#undef FC
  return cudaErrorInvalidValue;
}

cudaError_t train_conv_bwd(const float* x, const float* y, const float* dy, int B, int H, int W, int cin, int cout,
                           int d, const float* w, float* dx, float* dw, float* db, void* work, cudaStream_t s) {
  if ((long long)B * H * W == 0) return cudaSuccess;
  float* wk = static_cast<float*>(work);
  if (cin == 1) {
    if (dx) return cudaErrorInvalidValue;  // no input gradient for the image
#define B1(CO) return conv_bwd_impl<1, CO>(x, y, dy, B, H, W, d, w, nullptr, dw, db, wk, s)
    SML_CH_SWITCH(cout, B1)
#undef B1
  }
  if (cin != cout) return cudaErrorInvalidValue;
#define BC(CO) return conv_bwd_impl<CO, CO>(x, y, dy, B, H, W, d, w, dx, dw, db, wk, s)
  SML_CH_SWITCH(cout, BC)
#undef BC
  return cudaErrorInvalidValue;
}

cudaError_t train_heads_loss(const float* a, const float* tgt, int B, int H, int W, int C, const float* hw,
                             const float* hb, float* h, float* loss, const float* gscale, float* da, float* dhw,
                             float* dhb, void* work, cudaStream_t s) {
  if ((long long)B * H * W == 0) return cudaErrorInvalidValue;
  float* wk = static_cast<float*>(work);
#define HL(CC) return heads_impl<CC>(a, tgt, B, H, W, hw, hb, h, loss, gscale, da, dhw, dhb, wk, s)
  SML_CH_SWITCH(C, HL)
#undef HL
  return cudaErrorInvalidValue;
}

cudaError_t train_heads_loss_rp(const void* a, const float* tgt, int B, int H, int W, int C, const float* hw,
                                const float* hb, float* h, float* loss, const float* gscale, void* dz, float* dhw,
                                float* dhb, void* work, cudaStream_t s) {
  if ((long long)B * H * W == 0) return cudaErrorInvalidValue;
  float* wk = static_cast<float*>(work);
#define HR(CC) return heads_impl<CC, true>(a, tgt, B, H, W, hw, hb, h, loss, gscale, dz, dhw, dhb, wk, s)
  SML_CH_SWITCH(C, HR)
#undef HR
  return cudaErrorInvalidValue;
}

cudaError_t train_l0_wgrad_rp(const float* x0, const void* dz0, int B, int H, int W, int C, int d, float* dw,
                              float* db, void* work, cudaStream_t s) {
  const long long npx = (long long)B * H * W;
  if (npx == 0) return cudaSuccess;
  float* wk = static_cast<float*>(work);
#define W0(CO)                                                                                     \
  {                                                                                                \
    using Cfg = WgCfg<1, CO>;                                                                      \
    long long ppb = (npx + kWgBlocks - 1) / kWgBlocks;                                             \
    ppb = (ppb + kWgPx - 1) / kWgPx * kWgPx;                                                       \
    const int nb = (int)((npx + ppb - 1) / ppb);                                                   \
    k_wgrad_partial<1, CO, true><<<nb, Cfg::THREADS, 0, s>>>(x0, dz0, nullptr, B, H, W, d, ppb, wk); \
    k_wgrad_reduce<1, CO><<<(Cfg::NOUT + 255) / 256, 256, 0, s>>>(wk, nb, dw, db);                 \
    return cudaGetLastError();                                                                     \
  }
  SML_CH_SWITCH(C, W0)
#undef W0
  return cudaErrorInvalidValue;
}

cudaError_t train_ingest(const uint16_t* f, long long n, float gain, float offset, float in_scale, float* x0,
                         cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_train_ingest<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(f, n, gain, offset, in_scale, x0);
  return cudaGetLastError();
}

}  // namespace sml
