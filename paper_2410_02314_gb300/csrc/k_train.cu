// Training kernels (FP32, NHWC activations): forward and hand-written backward of the dilated
// 3x3 conv + bias + ReLU layer (dilated convolution, Sec. 3.2.1), and the fused 1x1 heads +
// loss + head gradients (binary cross-entropy on p, Sec. 3.3, plus a masked L2 on the
// offset, z and photon heads).  Weights use the PyTorch layout [Cout][Cin][3][3]; the
// kernels re-lay them out while staging them in shared memory.
//
// Reductions over pixels (weight, bias and head gradients, the loss) go through per-block
// partial sums and a second kernel that adds them in an order fixed by the sizes alone, so
// every result is deterministic.
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

template <int CI, int CO>
__global__ void __launch_bounds__(WgCfg<CI, CO>::THREADS) k_wgrad_partial(const float* __restrict__ x,
                                                                          const float* __restrict__ dy,
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
          const size_t src = (size_t)q * CO + o;
          v = y[src] > 0.0f ? dy[src] : 0.0f;
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

// Sum partials over blocks; write dw in [Cout][Cin][3][3] and db.  A block takes 32 outputs;
// warp s adds blocks s, s + 8, ... in order and the eight slice sums are added in slice order
// (a fixed order for given sizes).
constexpr int kRedSlices = 8;

template <int CI, int CO>
__global__ void __launch_bounds__(32 * kRedSlices) k_wgrad_reduce(const float* __restrict__ partial, int nblocks,
                                                                   float* __restrict__ dw, float* __restrict__ db) {
  using Cfg = WgCfg<CI, CO>;
  __shared__ float s_sum[kRedSlices][32];
  const int ol = threadIdx.x & 31, sl = threadIdx.x >> 5;
  const int o = blockIdx.x * 32 + ol;
  float acc = 0.0f;
  if (o < Cfg::NOUT) {
#pragma unroll 4
    for (int b = sl; b < nblocks; b += kRedSlices) acc += partial[(size_t)b * Cfg::NOUT + o];
  }
  s_sum[sl][ol] = acc;
  __syncthreads();
  if (sl != 0 || o >= Cfg::NOUT) return;
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kRedSlices; ++k) s += s_sum[k][ol];
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
  const long long n = (long long)B * HW, stride = (long long)gridDim.x * blockDim.x;
  float c = 0.0f;
  for (long long q0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; q0 < n; q0 += 4 * stride) {
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {  // four loads in flight
      const long long q = q0 + u * stride, b = q / HW, px = q - b * HW;
      v[u] = q < n ? __ldg(tgt + (size_t)b * kHeads * HW + px) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) c += v[u] > 0.5f ? 1.0f : 0.0f;
  }
  s[threadIdx.x] = c;
  __syncthreads();
  for (int o = kHThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}

// Heads, loss terms and (optionally) gradients, one thread per pixel.  A warp takes 32
// consecutive pixels per step: each lane loads its pixel's C activations and 5 targets (all
// loads of the step in flight together), forms the five heads, the loss terms and the head
// gradients dh, and writes its pixel's h and d loss / d a.  The head weight gradient
// dhw[k][c] = sum_p dh[p][k] a[p][c] (and dhb[k] = sum_p dh[p][k], as a column of ones) goes
// through shared memory: the warp's 32 pixels are staged there and lane l adds the pairs
// (k, c) numbered l, l + 32, ... over them, pixel by pixel.  Blocks stride over warp steps; at
// the end the warps are added in warp order, so the result depends only on the sizes.
// Partial layout per block: [0] BCE sum, [1] L2 sum, [2 .. 2+5C) dhw [k][c], [2+5C .. +5) dhb.
// RP = true (BF16 training): a holds bf16 row-planar activations [B][H][C/16][W][16] and da
// receives dz = (d loss / d a) * [a > 0] (the last conv layer's ReLU mask applied), rounded to
// bf16, in the same layout.  RP = false: a and da are FP32 [B][H][W][C], da without the mask.
constexpr int kHLThreads = 128;  // k_heads_loss block: 4 warps, 3 blocks per SM

template <int C>
struct HeadCfg {
  static constexpr int WARPS = kHLThreads / 32;
  static constexpr int NPAIR = kHeads * (C + 1);  // (k, c) pairs, c = C the ones column
  static constexpr int MP = (NPAIR + 31) / 32;    // pairs per lane
  static constexpr int NOUT = 2 + kHeads * C + kHeads;
};
constexpr int kHBlocks = 456;  // grid cap (3 blocks on each of 152 SMs); sizes the partial buffer

template <int C, bool RP = false>
__global__ void __launch_bounds__(kHLThreads, 3) k_heads_loss(const void* __restrict__ a, const float* __restrict__ tgt,
                                                             int B, int HW, int W, const float* __restrict__ hw,
                                                             const float* __restrict__ hb, float* __restrict__ h,
                                                             const float* __restrict__ nt_partial, int nt_blocks,
                                                             const float* __restrict__ grad_scale,
                                                             void* __restrict__ da, float* __restrict__ partial) {
  using Cfg = HeadCfg<C>;
  constexpr int XS = C + 1;  // staged floats per pixel (odd: lanes hit distinct banks)
  __shared__ float s_red[Cfg::WARPS][Cfg::NOUT];
  __shared__ __align__(16) float s_w[kHeads][C];
  __shared__ float s_x[Cfg::WARPS][32 * XS];
  __shared__ float s_dh[Cfg::WARPS][32 * kHeads];
  __shared__ float s_nt;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = threadIdx.x; k < kHeads * C; k += blockDim.x) s_w[k / C][k % C] = hw[k];
  if (warp == 0) {  // target count: integer-valued partial sums, exact in any order
    float nt = 0.0f;
    for (int b = lane; b < nt_blocks; b += 32) nt += nt_partial[b];
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) nt += __shfl_xor_sync(0xffffffffu, nt, m);
    if (lane == 0) s_nt = nt;
  }
  float bias[kHeads];
#pragma unroll
  for (int k = 0; k < kHeads; ++k) bias[k] = hb[k];
  __syncthreads();
  const long long npx = (long long)B * HW;
  const float inv_npx = 1.0f / (float)npx;
  const float inv_nt = 1.0f / (s_nt > 0.0f ? s_nt : 1.0f);
  const float gs = grad_scale ? *grad_scale : 0.0f;
  // this lane's (k, c) pairs as shared-memory offsets into a staged pixel and its dh
  int pk[Cfg::MP], pc[Cfg::MP];
  float acc[Cfg::MP];
#pragma unroll
  for (int m = 0; m < Cfg::MP; ++m) {
    const int P = lane + 32 * m;
    pk[m] = P < Cfg::NPAIR ? P / XS : 0;
    pc[m] = P < Cfg::NPAIR ? P % XS : 0;
    acc[m] = 0.0f;
  }
  float bce = 0.0f, l2 = 0.0f;
  float* xw = s_x[warp];
  float* dw = s_dh[warp];
  const long long nsteps = (npx + 31) / 32;
  for (long long st = (long long)blockIdx.x * Cfg::WARPS + warp; st < nsteps;
       st += (long long)gridDim.x * Cfg::WARPS) {
    const long long q = st * 32 + lane;
    const bool in = q < npx;
    const long long b = in ? q / HW : 0;
    const int px = in ? (int)(q - b * HW) : 0;
    float av[C], tv[kHeads];
    size_t a0 = 0;  // element offset of this pixel's first channel
    if (in) {
      const float* tp = tgt + (size_t)b * kHeads * HW + px;
#pragma unroll
      for (int k = 0; k < kHeads; ++k) tv[k] = __ldg(tp + (size_t)k * HW);
      if (RP) {
        const int i = px / W, j = px - i * W;
        a0 = (((size_t)b * (HW / W) + i) * (C / 16) * W + j) * 16;  // group g at + g W 16
        uint4 u[C / 8];
#pragma unroll
        for (int g = 0; g < C / 16; ++g) {
          const uint4* src = reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(a) + a0 +
                                                            (size_t)g * W * 16);
          u[2 * g] = __ldcs(src);
          u[2 * g + 1] = __ldcs(src + 1);
        }
#pragma unroll
        for (int v = 0; v < C / 8; ++v) {
          const __nv_bfloat162* p2 = reinterpret_cast<const __nv_bfloat162*>(&u[v]);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float2 f = __bfloat1622float2(p2[e]);
            av[8 * v + 2 * e] = f.x;
            av[8 * v + 2 * e + 1] = f.y;
          }
        }
      } else {
        a0 = (size_t)q * C;
        const float4* src = reinterpret_cast<const float4*>(static_cast<const float*>(a) + a0);
#pragma unroll
        for (int v = 0; v < C / 4; ++v) {
          const float4 f = __ldcs(src + v);
          av[4 * v] = f.x, av[4 * v + 1] = f.y, av[4 * v + 2] = f.z, av[4 * v + 3] = f.w;
        }
      }
    } else {
#pragma unroll
      for (int c = 0; c < C; ++c) av[c] = 0.0f;
#pragma unroll
      for (int k = 0; k < kHeads; ++k) tv[k] = 0.0f;
    }
    float dh[kHeads];
#pragma unroll
    for (int k = 0; k < kHeads; ++k) dh[k] = 0.0f;
    if (in) {
      float hv[kHeads];
#pragma unroll
      for (int k = 0; k < kHeads; ++k) {
        float s = bias[k];
#pragma unroll
        for (int c = 0; c < C; ++c) s = fmaf(s_w[k][c], av[c], s);
        hv[k] = s;
        h[((size_t)b * kHeads + k) * HW + px] = s;
      }
      const float y0 = tv[0], h0 = hv[0];
      bce += fmaxf(h0, 0.0f) - h0 * y0 + log1pf(expf(-fabsf(h0)));
      dh[0] = (1.0f / (1.0f + expf(-h0)) - y0) * inv_npx * gs;
      const bool m = y0 > 0.5f;
#pragma unroll
      for (int k = 1; k < kHeads; ++k) {
        const float e = m ? hv[k] - tv[k] : 0.0f;
        l2 = fmaf(e, e, l2);
        dh[k] = 2.0f * e * inv_nt * gs;
      }
      if (da) {
        if (RP) {
#pragma unroll
          for (int g = 0; g < C / 16; ++g) {
            uint4 u[2];
            __nv_bfloat162* p2 = reinterpret_cast<__nv_bfloat162*>(u);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              float s2[2];
#pragma unroll
              for (int t = 0; t < 2; ++t) {
                const int c = 16 * g + 2 * e + t;
                float s = 0.0f;
#pragma unroll
                for (int k = 0; k < kHeads; ++k) s = fmaf(s_w[k][c], dh[k], s);
                s2[t] = av[c] > 0.0f ? s : 0.0f;
              }
              p2[e] = __floats2bfloat162_rn(s2[0], s2[1]);
            }
            uint4* dst = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(da) + a0 + (size_t)g * W * 16);
            __stcs(dst, u[0]);
            __stcs(dst + 1, u[1]);
          }
        } else {
          float4* dst = reinterpret_cast<float4*>(static_cast<float*>(da) + a0);
#pragma unroll
          for (int v = 0; v < C / 4; ++v) {
            float s4[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              float s = 0.0f;
#pragma unroll
              for (int k = 0; k < kHeads; ++k) s = fmaf(s_w[k][4 * v + t], dh[k], s);
              s4[t] = s;
            }
            __stcs(dst + v, make_float4(s4[0], s4[1], s4[2], s4[3]));
          }
        }
      }
    }
    if (!da) continue;  // the loss alone: no head weight gradient (a kernel-uniform branch)
    // stage the warp's pixels, then each lane adds its (k, c) pairs over them
#pragma unroll
    for (int c = 0; c < C; ++c) xw[lane * XS + c] = av[c];
    xw[lane * XS + C] = 1.0f;
#pragma unroll
    for (int k = 0; k < kHeads; ++k) dw[lane * kHeads + k] = dh[k];
    __syncwarp();
#pragma unroll 4
    for (int p = 0; p < 32; ++p) {
#pragma unroll
      for (int m = 0; m < Cfg::MP; ++m) acc[m] = fmaf(dw[p * kHeads + pk[m]], xw[p * XS + pc[m]], acc[m]);
    }
    __syncwarp();
  }
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    bce += __shfl_xor_sync(0xffffffffu, bce, m);
    l2 += __shfl_xor_sync(0xffffffffu, l2, m);
  }
#pragma unroll
  for (int m = 0; m < Cfg::MP; ++m) {
    const int P = lane + 32 * m;
    if (P < Cfg::NPAIR) {
      const int k = P / XS, c = P - k * XS;
      s_red[warp][c < C ? 2 + k * C + c : 2 + kHeads * C + k] = acc[m];
    }
  }
  if (lane == 0) {
    s_red[warp][0] = bce;
    s_red[warp][1] = l2;
  }
  __syncthreads();
  float* dst = partial + (size_t)blockIdx.x * Cfg::NOUT;
  for (int oi = threadIdx.x; oi < Cfg::NOUT; oi += blockDim.x) {
    float s = 0.0f;
#pragma unroll
    for (int wp = 0; wp < Cfg::WARPS; ++wp) s += s_red[wp][oi];
    dst[oi] = s;
  }
}

// One block per output: the block's threads add the per-block partials in a fixed strided
// order and a fixed tree.  Block 0 also adds the L2 column and forms the loss.
__global__ void __launch_bounds__(kHThreads) k_heads_reduce(const float* __restrict__ partial, int nblocks, int C,
                                                            long long npx, const float* __restrict__ nt_partial,
                                                            int nt_blocks, float* __restrict__ loss,
                                                            float* __restrict__ dhw, float* __restrict__ dhb) {
  __shared__ float s0[kHThreads], s1[kHThreads];
  const int nout = 2 + kHeads * C + kHeads;
  const int o = blockIdx.x;
  if (o == 1) return;  // the L2 column is block 0's
  float a0 = 0.0f, a1 = 0.0f;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    a0 += partial[(size_t)b * nout + o];
    if (o == 0) a1 += partial[(size_t)b * nout + 1];
  }
  s0[threadIdx.x] = a0;
  s1[threadIdx.x] = a1;
  __syncthreads();
  for (int m = kHThreads / 2; m > 0; m >>= 1) {
    if (threadIdx.x < m) {
      s0[threadIdx.x] += s0[threadIdx.x + m];
      s1[threadIdx.x] += s1[threadIdx.x + m];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  if (o == 0) {
    float nt = 0.0f;
    for (int b = 0; b < nt_blocks; ++b) nt += nt_partial[b];
    *loss = s0[0] / (float)npx + s1[0] / (nt > 0.0f ? nt : 1.0f);
  } else if (o < 2 + kHeads * C) {
    if (dhw) dhw[o - 2] = s0[0];
  } else if (dhb) {
    dhb[o - 2 - kHeads * C] = s0[0];
  }
}

// First-layer weight and bias gradient of BF16 training: dw[co][tap] = sum_p dz0[p][co]
// x0[p + off(tap)] and db[co] = sum_p dz0[p][co], x0 the FP32 network input [B][H][W], dz0
// bf16 row-planar [B][H][C/16][W][16].  A block runs kL0Slots row slots of C/16 warps; warp w
// of a slot reads channel group w of the slot's pixel rows, lane pair (2u, 2u + 1) pixel
// j = u + 16n (the even lane channels 0..7 of the group, the odd lane 8..15), so one warp load
// covers 16 whole 32-byte pixels.  Each lane keeps 8 x (9 + 1) running sums; at the end the
// lanes of one parity are added with shuffles and the slots in slot order, giving per-block
// partials in k_wgrad_reduce<1, C>'s layout.
constexpr int kL0Slots = 4;

template <int C>
__global__ void __launch_bounds__(C / 16 * 32 * kL0Slots) k_l0_wgrad_rp(const float* __restrict__ x0,
                                                                      const __nv_bfloat16* __restrict__ dz0, int B,
                                                                      int H, int W, int d,
                                                                      float* __restrict__ partial) {
  constexpr int G = C / 16;
  __shared__ float s_red[kL0Slots][C][10];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = warp % G, slot = warp / G;
  const int half = lane & 1, u = lane >> 1;
  float acc[8][9], accb[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    accb[e] = 0.0f;
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[e][k] = 0.0f;
  }
  const long long rows = (long long)B * H;
  for (long long r = (long long)blockIdx.x * kL0Slots + slot; r < rows; r += (long long)gridDim.x * kL0Slots) {
    const int i = (int)(r % H);
    const float* xf = x0 + (size_t)(r / H) * H * W;  // this row's frame
    const __nv_bfloat16* zr = dz0 + ((size_t)r * G + g) * W * 16 + half * 8;
    const bool rv0 = i - d >= 0, rv2 = i + d < H;
#pragma unroll 4
    for (int j = u; j < W; j += 16) {
      const uint4 zz = __ldcs(reinterpret_cast<const uint4*>(zr + (size_t)j * 16));
      const __nv_bfloat162* z2 = reinterpret_cast<const __nv_bfloat162*>(&zz);
      float z[8];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 f = __bfloat1622float2(z2[e]);
        z[2 * e] = f.x;
        z[2 * e + 1] = f.y;
      }
      float xv[9];
#pragma unroll
      for (int ky = 0; ky < 3; ++ky) {
        const bool rv = ky == 0 ? rv0 : (ky == 2 ? rv2 : true);
        const int ii = i + (ky - 1) * d;
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          const int jj = j + (kx - 1) * d;
          xv[ky * 3 + kx] = rv && jj >= 0 && jj < W ? __ldg(xf + (size_t)ii * W + jj) : 0.0f;
        }
      }
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        accb[e] += z[e];
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[e][k] = fmaf(z[e], xv[k], acc[e][k]);
      }
    }
  }
  // lanes of one parity hold the same 8 channels
#pragma unroll
  for (int m = 2; m < 32; m <<= 1) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      accb[e] += __shfl_xor_sync(0xffffffffu, accb[e], m);
#pragma unroll
      for (int k = 0; k < 9; ++k) acc[e][k] += __shfl_xor_sync(0xffffffffu, acc[e][k], m);
    }
  }
  if (lane < 2) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int c = g * 16 + lane * 8 + e;
#pragma unroll
      for (int k = 0; k < 9; ++k) s_red[slot][c][k] = acc[e][k];
      s_red[slot][c][9] = accb[e];
    }
  }
  __syncthreads();
  float* dst = partial + (size_t)blockIdx.x * (10 * C);
  for (int oi = threadIdx.x; oi < 10 * C; oi += blockDim.x) {
    const int c = oi / 10, k = oi - c * 10;
    float s = 0.0f;
#pragma unroll
    for (int sl = 0; sl < kL0Slots; ++sl) s += s_red[sl][c][k];
    if (k < 9)
      dst[c * 9 + k] = s;
    else
      dst[9 * C + c] = s;
  }
}

__global__ void k_train_ingest(const uint16_t* __restrict__ f, long long n, float gain, float offset, float in_scale,
                               float* __restrict__ x0) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) x0[q] = __fmul_rn(__fdiv_rn(__fsub_rn((float)f[q], offset), gain), in_scale);
}

constexpr int kWgBlocks = 304;
constexpr int kNtBlocks = 304;

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
  k_wgrad_reduce<CI, CO><<<(Cfg::NOUT + 31) / 32, 32 * kRedSlices, 0, s>>>(work, nb, dw, db);
  return cudaGetLastError();
}

template <int C, bool RP = false>
cudaError_t heads_impl(const void* a, const float* tgt, int B, int H, int W, const float* hw, const float* hb,
                       float* h, float* loss, const float* gscale, void* da, float* dhw, float* dhb, float* work,
                       cudaStream_t s) {
  using Cfg = HeadCfg<C>;
  const int HW = H * W;
  const long long npx = (long long)B * HW;
  const long long nblk = (npx + 32 * Cfg::WARPS - 1) / (32 * Cfg::WARPS);
  const int nb = (int)(nblk < kHBlocks ? nblk : kHBlocks);
  float* nt_partial = work;
  float* partial = work + kNtBlocks;
  k_count_targets<<<kNtBlocks, kHThreads, 0, s>>>(tgt, B, HW, nt_partial);
  k_heads_loss<C, RP><<<nb, kHLThreads, 0, s>>>(a, tgt, B, HW, W, hw, hb, h, nt_partial, kNtBlocks, gscale, da,
                                               partial);
  k_heads_reduce<<<Cfg::NOUT, kHThreads, 0, s>>>(partial, nb, C, npx, nt_partial, kNtBlocks, loss, dhw, dhb);
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
  (void)B;
  (void)H;
  (void)W;
  return sizeof(float) * ((size_t)kNtBlocks + (size_t)kHBlocks * (2 + kHeads * C + kHeads));
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
#define W0(CO)                                                                                  \
  {                                                                                             \
    const long long rows = (long long)B * H;                                                    \
    const long long nblk = (rows + kL0Slots - 1) / kL0Slots;                                    \
    const int nb = (int)(nblk < kWgBlocks ? nblk : kWgBlocks);                                  \
    k_l0_wgrad_rp<CO><<<nb, CO / 16 * 32 * kL0Slots, 0, s>>>(x0, static_cast<const __nv_bfloat16*>(dz0), B, H, W, d, \
                                                             wk);                               \
    k_wgrad_reduce<1, CO><<<(WgCfg<1, CO>::NOUT + 31) / 32, 32 * kRedSlices, 0, s>>>(wk, nb, dw, db); \
    return cudaGetLastError();                                                                  \
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
