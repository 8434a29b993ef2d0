// Tensor-core kernels of BF16 training (dilated convolution, Sec. 3.2.1): the device-side
// packing of FP32 master weights into the conv kernel's BF16 B images (forward, and mirrored
// for the input gradient), and the weight-gradient contraction on tcgen05.
//
// Weight gradient of a dilated 3x3 layer with C inputs and C outputs:
//   dW[co][ci][ky][kx] = sum_p dZ[p][co] * X[p + ((ky-1)d, (kx-1)d)][ci],   db[co] = sum_p dZ[p][co]
// with dZ the gradient of the layer's pre-activation (ReLU mask applied) and X its input
// (zero outside the frame).  K runs over pixels, so both operands are MN-major: a TMA row
// box of the row-planar activations ([T][H][G][W][16 channels], G = C/16) lands as G planes
// of [pixel][16 channels] with the 32-byte swizzle, which is the canonical MN-major SW32
// operand (planes = atoms along M/N, LBO = plane stride; 8 pixels per atom along K, SBO =
// 256 B).  A = dZ of one 128-pixel row strip (M = 64: the C output channels, the planes
// beyond them zero), B = X of the row i + (ky-1)d, its descriptor started (kx-1)d+d pixel
// lines into a box that begins d pixels left of the strip (the tap shift along K).  The three
// X rows of a unit sit in consecutive planes, so one MMA of N = 3C covers the three vertical
// taps of a horizontal tap; each tap accumulates into its own C TMEM columns (kx-major), and
// one more MMA per K step against a plane of ones accumulates sum_p dZ (the bias gradient).  The accumulators stay in TMEM
// across all the work units of a CTA (a contiguous range of row strips); each CTA writes its
// partial sums, and a second kernel adds the partials in CTA order (deterministic).
#include <cuda_bf16.h>

#include "sml_internal.h"
#include "tc_ptx.cuh"

namespace sml {

namespace {

constexpr int kWgThreads = 128;
constexpr int kWgMaxStages = 8;

// Columns of one CTA's partial sums for a layer of C channels: 9 taps x C, then 16 columns
// holding the bias gradient (the same value 16 times).
__host__ __device__ constexpr int wg_cols(int C) { return 9 * C + 16; }

struct WgKArgs {
  int T, H, W, d;
  int S;                  // pixels per strip (the dZ box): 128, or the frame width rounded up to 32
  int NS;                 // strips per row
  uint32_t units;         // T * H * NS
  uint32_t dz_plane;      // bytes of one plane of a dZ box (S x 32)
  uint32_t x_plane;       // bytes of one plane of an X row box ((S + 2d rounded up to 32) x 32)
  uint32_t x_slot;        // bytes of one X row slot (G planes; the 3 slots are contiguous)
  uint32_t stage_bytes;   // dZ slot (M/16 planes) + 3 X slots
  int nstages;            // ring stages (<= kWgMaxStages)
  float* partial;         // [gridDim.x][C][wg_cols(C)]
  int* err;
};

constexpr int kWgM = 64;  // MMA M: the output channels, padded to 64

template <int C>
__global__ void __launch_bounds__(kWgThreads, 1) k_wgrad_tc(const __grid_constant__ CUtensorMap tm_dz,
                                                            const __grid_constant__ CUtensorMap tm_x, const WgKArgs a) {
  constexpr int G = C / 16;
  constexpr int COLS = wg_cols(C);
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* s_stage = smem;
  uint8_t* s_ones = s_stage + (size_t)a.nstages * a.stage_bytes;  // 1024 B of bf16 1.0
  uint64_t* full_bar = reinterpret_cast<uint64_t*>(s_ones + 1024);
  uint64_t* empty_bar = full_bar + kWgMaxStages;
  uint64_t* done_bar = empty_bar + kWgMaxStages;
  volatile uint32_t* s_tmem = reinterpret_cast<volatile uint32_t*>(done_bar + 1);
  volatile int* s_abort = reinterpret_cast<volatile int*>(s_tmem + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t u_begin = (uint32_t)(((unsigned long long)blockIdx.x * a.units) / gridDim.x);
  const uint32_t u_end = (uint32_t)(((unsigned long long)(blockIdx.x + 1) * a.units) / gridDim.x);

  // set-up: zero the dZ planes beyond the C channels (M padding), the ones plane, barriers, TMEM
  for (int s = 0; s < a.nstages; ++s) {
    uint4* z = reinterpret_cast<uint4*>(s_stage + (size_t)s * a.stage_bytes + (size_t)G * a.dz_plane);
    for (int k = threadIdx.x; k < (int)((kWgM / 16 - G) * a.dz_plane / 16); k += kWgThreads) z[k] = make_uint4(0, 0, 0, 0);
  }
  for (int k = threadIdx.x; k < 1024 / 16; k += kWgThreads)
    reinterpret_cast<uint4*>(s_ones)[k] = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
  if (threadIdx.x == 0) {
    for (int s = 0; s < a.nstages; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    mbar_init(smem_u32(&done_bar[0]), 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32((const void*)s_tmem)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *s_tmem;
  {  // accumulators start at zero
    float z[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) z[k] = 0.0f;
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c = 0; c < COLS; c += 16) tmem_st16(lane_addr + c, z);
    tmem_st_wait();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();

  const uint32_t tx = (uint32_t)G * a.dz_plane + 3u * (uint32_t)G * a.x_plane;
  const uint32_t dz_slot = (uint32_t)(kWgM / 16) * a.dz_plane;
  const uint32_t nst = (uint32_t)a.nstages;
  if (warp == 0 && lane == 0) {
    // ------------------------------------------------ TMA producer
    uint32_t st = 0, ph = 0, issued = 0;
    for (uint32_t u = u_begin; u < u_end; ++u) {
      const uint32_t s_ = u % (uint32_t)a.NS, r = u / (uint32_t)a.NS;
      const int i = (int)(r % (uint32_t)a.H), t = (int)(r / (uint32_t)a.H), j0 = (int)s_ * a.S;
      if (issued >= nst && !mbar_wait(smem_u32(&empty_bar[st]), ph ^ 1u, a.err, s_abort)) break;
      const uint32_t fb = smem_u32(&full_bar[st]);
      mbar_expect_tx(fb, tx);
      uint8_t* base = s_stage + (size_t)st * a.stage_bytes;
      tma_load_5d(smem_u32(base), &tm_dz, 0, j0, 0, i, t, fb);
#pragma unroll
      for (int ky = 0; ky < 3; ++ky)
        tma_load_5d(smem_u32(base + dz_slot + (size_t)ky * a.x_slot), &tm_x, 0, j0 - a.d, 0, i + (ky - 1) * a.d, t, fb);
      ++issued;
      if (++st == nst) {
        st = 0;
        ph ^= 1u;
      }
    }
    // no load of ours may still be landing when the CTA exits
    const uint32_t n_drain = issued < nst ? issued : nst;
    for (uint32_t k = 0; k < n_drain; ++k) {
      const uint32_t back = k + 1;
      const uint32_t s2 = (st + nst - (back % nst)) % nst;
      const uint32_t p2 = (back > st) ? (ph ^ 1u) : ph;
      mbar_wait_own(smem_u32(&full_bar[s2]), p2, a.err, s_abort);
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------ MMA issuer (single thread)
    // bf16 x bf16 -> f32, M = 64, A and B MN-major (instruction descriptor bits 15, 16).  The
    // three X row slots of a stage are contiguous planes (x_slot = G planes), so one B operand
    // of N = 3C spans the rows of all three vertical taps: its 16-channel atoms are (ky, group)
    // in order, x_plane apart.  Per K step: one MMA per horizontal tap, plus the ones MMA.
    const uint32_t idesc_c = instr_desc(kBF16, kWgM, 3 * C) | (1u << 15) | (1u << 16);
    const uint32_t idesc_1 = instr_desc(kBF16, kWgM, 16) | (1u << 15) | (1u << 16);
    const uint64_t ones = smem_desc(smem_u32(s_ones), 256u, 256u, 6u);
    // descriptors of stage 0, K step 0; a K step adds 16 pixel lines (512 B, 32 in the
    // descriptor's 16-byte address field), a stage adds stage_bytes
    const uint64_t a0 = smem_desc(smem_u32(s_stage), a.dz_plane, 256u, 6u);
    uint64_t b0[3];
#pragma unroll
    for (int kx = 0; kx < 3; ++kx) b0[kx] = smem_desc(smem_u32(s_stage) + dz_slot + (uint32_t)(kx * a.d) * 32u, a.x_plane, 256u, 6u);
    uint32_t st = 0, ph = 0;
    bool issued = false;
    for (uint32_t u = u_begin; u < u_end; ++u) {
      if (!mbar_wait(smem_u32(&full_bar[st]), ph, a.err, s_abort)) break;
      fence_after_sync();
      const int j0 = (int)(u % (uint32_t)a.NS) * a.S;
      const int valid = a.W - j0 < a.S ? a.W - j0 : a.S;
      const int nk = (valid + 15) / 16;  // K steps that hold pixels of the frame
      const uint64_t st16 = (uint64_t)((st * a.stage_bytes) >> 4);
      for (int ks = 0; ks < nk; ++ks) {
        const uint64_t off = st16 + (uint64_t)(ks * 32);
        const uint64_t ad = a0 + off;
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) umma<kBF16>(tmem + (uint32_t)(kx * 3 * C), ad, b0[kx] + off, idesc_c, 1u);
        umma<kBF16>(tmem + (uint32_t)(9 * C), ad, ones, idesc_1, 1u);
      }
      umma_commit(smem_u32(&empty_bar[st]));
      issued = true;
      if (++st == nst) {
        st = 0;
        ph ^= 1u;
      }
    }
    umma_commit(smem_u32(&done_bar[0]));  // arrives once every MMA issued above has completed
    (void)issued;
  }
  __syncwarp();
  // ------------------------------------------------ epilogue: TMEM -> partial sums
  const bool ok = mbar_wait_own(smem_u32(&done_bar[0]), 0, a.err, s_abort);
  fence_after_sync();
  if (ok && !*s_abort) {
    // an M = 64 MMA writes D row 16w + t to TMEM lane 32w + t (t < 16): lanes 0-15 of each
    // warp's quarter hold output channels 16w .. 16w + 15
    const int co = warp * 16 + lane;
    const bool mine = lane < 16 && co < C;
    float* dst = a.partial + ((size_t)blockIdx.x * C + (mine ? co : 0)) * COLS;
    for (int c = 0; c < COLS; c += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
      tmem_ld_wait();
      if (mine) {
#pragma unroll
        for (int k = 0; k < 16; ++k) dst[c + k] = v[k];
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

// dW[co][ci][ky][kx] and db[co] from the CTAs' partial sums.  A block takes 32 outputs; warp
// s of it adds CTAs s, s + 8, ... in order, and the eight slice sums are added in slice order:
// a fixed order for given sizes, with eight times the loads in flight of one thread per output.
constexpr int kRedSlices = 8;

template <int C>
__global__ void __launch_bounds__(32 * kRedSlices) k_wgrad_reduce(const float* __restrict__ partial, int nblk,
                                                                   float* __restrict__ dw, float* __restrict__ db) {
  constexpr int COLS = wg_cols(C);
  constexpr int NO = C * (9 * C + 1);  // (co, column) pairs of the partial sums
  __shared__ float s_sum[kRedSlices][32];
  const int ol = threadIdx.x & 31, sl = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + ol;
  const int co = e / (9 * C + 1), c = e % (9 * C + 1);
  float acc = 0.0f;
  if (e < NO) {
#pragma unroll 4
    for (int b = sl; b < nblk; b += kRedSlices) acc += partial[((size_t)b * C + co) * COLS + c];
  }
  s_sum[sl][ol] = acc;
  __syncthreads();
  if (sl != 0 || e >= NO) return;
  float v = 0.0f;
#pragma unroll
  for (int k = 0; k < kRedSlices; ++k) v += s_sum[k][ol];
  if (c == 9 * C) {
    db[co] = v;
  } else {  // column kx * 3C + ky * C + ci
    const int kx = c / (3 * C), ky = (c % (3 * C)) / C, ci = c % C;
    dw[((size_t)co * C + ci) * 9 + ky * 3 + kx] = v;
  }
}

// B images of the tensor-core conv from FP32 weights w [cout][cin][3][3] (PyTorch layout),
// rounded to bf16: the forward image (CI = cin, CO = cout) and, for the input gradient, the
// image of the mirrored, transposed weights w'[ci][co][ky][kx] = w[co][ci][2-ky][2-kx]
// (CI = cout, CO = cin).  Layout as tc_pack_bimg: per (kx, k step) one block of N = 3 CO rows
// (n = ky CO + o) by 16 K elements (i = 16 ks + k), byte (n/8)*256 + (k/8)*128 + (n%8)*16 +
// (k%8)*2.
__global__ void k_pack_bimg_bf16(const float* __restrict__ w, int cin, int cout, __nv_bfloat16* __restrict__ fwd,
                                 __nv_bfloat16* __restrict__ dgrad) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int n_el = 9 * cin * cout;  // elements of one image (K padded to 16 is exact: channels are multiples of 16)
  if (e >= 2 * n_el) return;
  const bool dg = e >= n_el;
  const int q = dg ? e - n_el : e;
  const int CI = dg ? cout : cin, CO = dg ? cin : cout;
  const int nks = CI / 16, N = 3 * CO;
  const int blk = q / (N * 16), r = q % (N * 16);
  const int n = r / 16, k = r % 16;
  const int kx = blk / nks, ks = blk % nks;
  const int ky = n / CO, o = n % CO, i = ks * 16 + k;
  // forward: w[o][i][ky][kx]; input gradient: w'[o][i][ky][kx] = w[i][o][2-ky][2-kx]
  const float v = dg ? w[((size_t)i * cin + o) * 9 + (2 - ky) * 3 + (2 - kx)] : w[((size_t)o * cin + i) * 9 + ky * 3 + kx];
  const size_t off = (size_t)blk * (N / 8) * 256 + (size_t)(n / 8) * 256 + (size_t)(k / 8) * 128 + (size_t)(n % 8) * 16 +
                     (size_t)(k % 8) * 2;
  (dg ? dgrad : fwd)[off / 2] = __float2bfloat16_rn(v);
}

}  // namespace

size_t train_wgrad_tc_work_bytes(int C, int num_sms) { return (size_t)num_sms * C * wg_cols(C) * sizeof(float); }

// Strip width of the weight gradient: 128 pixels, or the frame width rounded up to 32 for
// narrower frames (training patches), so that the boxes carry little beyond the frame.  The X
// box adds the 2d halo, rounded up to 32 pixels (1 KB planes).
void wgrad_tc_boxes(int W, int d, int* dz_px, int* x_px) {
  const int S = W >= kTileM ? kTileM : (W + 31) / 32 * 32;
  *dz_px = S;
  *x_px = (S + 2 * d + 31) / 32 * 32;
}

cudaError_t launch_pack_bimg_bf16(const float* w, int cin, int cout, void* fwd, void* dgrad, cudaStream_t s) {
  if (cin % 16 || cout % 16 || cin < 16 || cout < 16) return cudaErrorInvalidValue;
  const int n = 2 * 9 * cin * cout;
  k_pack_bimg_bf16<<<(n + 255) / 256, 256, 0, s>>>(w, cin, cout, static_cast<__nv_bfloat16*>(fwd),
                                                   static_cast<__nv_bfloat16*>(dgrad));
  return cudaGetLastError();
}

cudaError_t launch_wgrad_tc(const CUtensorMap* tm_dz, const CUtensorMap* tm_x, int T, int H, int W, int C, int d,
                            float* partial, int num_sms, float* dw, float* db, int* err, cudaStream_t s) {
  if (C != 16 && C != 32 && C != 48) return cudaErrorInvalidValue;  // 9 C + 16 TMEM columns <= 512
  WgKArgs a{};
  a.T = T;
  a.H = H;
  a.W = W;
  a.d = d;
  int dz_px = 0, x_px = 0;
  wgrad_tc_boxes(W, d, &dz_px, &x_px);
  a.S = dz_px;
  a.NS = (W + a.S - 1) / a.S;
  const long long units = (long long)T * H * a.NS;
  if (units >= (1LL << 31)) return cudaErrorInvalidValue;
  a.units = (uint32_t)units;
  a.dz_plane = (uint32_t)dz_px * 32u;
  a.x_plane = (uint32_t)x_px * 32u;
  a.x_slot = (uint32_t)(C / 16) * a.x_plane;  // a multiple of 1024 (x_plane is): the slots are contiguous planes
  a.stage_bytes = (uint32_t)(kWgM / 16) * a.dz_plane + 3u * a.x_slot;
  a.partial = partial;
  a.err = err;
  // as many ring stages as fit next to the fixed part (alignment slack, ones plane, barriers)
  const size_t fixed = 1024 + 1024 + 8 * (2 * kWgMaxStages + 1) + 16;
  const size_t avail = 227 * 1024 - fixed;
  a.nstages = (int)std::min<size_t>(kWgMaxStages, avail / a.stage_bytes);
  if (a.nstages < 2) return cudaErrorInvalidConfiguration;
  const size_t smem = fixed + (size_t)a.nstages * a.stage_bytes;
  const int grid = (int)std::min<long long>(units > 0 ? units : 1, num_sms);
  cudaError_t e;
  if (units > 0) {
#define SML_WG(CC)                                                                                           \
  case CC:                                                                                                   \
    e = cudaFuncSetAttribute(k_wgrad_tc<CC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);        \
    if (e != cudaSuccess) return e;                                                                          \
    k_wgrad_tc<CC><<<grid, kWgThreads, smem, s>>>(*tm_dz, *tm_x, a);                                         \
    break;
    switch (C) {
      SML_WG(16)
      SML_WG(32)
      SML_WG(48)
    }
#undef SML_WG
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  } else {
    if ((e = cudaMemsetAsync(partial, 0, (size_t)C * wg_cols(C) * sizeof(float), s)) != cudaSuccess) return e;
  }
  const int nred = (C * (9 * C + 1) + 31) / 32;
  switch (C) {
    case 16: k_wgrad_reduce<16><<<nred, 32 * kRedSlices, 0, s>>>(partial, grid, dw, db); break;
    case 32: k_wgrad_reduce<32><<<nred, 32 * kRedSlices, 0, s>>>(partial, grid, dw, db); break;
    default: k_wgrad_reduce<48><<<nred, 32 * kRedSlices, 0, s>>>(partial, grid, dw, db); break;
  }
  return cudaGetLastError();
}

}  // namespace sml
