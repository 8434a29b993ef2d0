// Decode of per-pixel maps into localizations, on the device (post-processing kept in GPU
// memory, Sec. 2.2; its cost matters, Sec. 4.2.1).  Output format per Sec. 3.2: the
// probability map selects pixels, the offset maps place the emitter inside the pixel.
//
// Detection rule: p > p_min and p is the maximum of its in-frame 3x3 neighbourhood, with
// ties going to the first pixel in raster order (strict > against earlier neighbours,
// >= against later ones).  Readout: x = j + dx, y = i + dy, z = z_scale*zhat,
// photons = ph_scale*Nhat, each a single IEEE rounding (__fadd_rn / __fmul_rn: no FMA).
//
// Order: three kernels give (frame, row, column) order without atomics.  Each block owns
// 1024 consecutive pixels (4 passes of 256 threads); count -> exclusive scan of the block
// counts (plus a running total that carries over chunks) -> write at block offset + rank,
// where the rank inside a block comes from warp ballots.
#include "sml_internal.h"

namespace sml {

namespace {

__device__ __forceinline__ bool dec_flag(const float* __restrict__ maps, int H, int W, long long q, float p_min) {
  long long plane = (long long)H * W;
  int t = (int)(q / plane);
  long long px = q - (long long)t * plane;
  int i = (int)(px / W);
  int j = (int)(px - (long long)i * W);
  const float* p = maps + (size_t)t * kHeads * plane;
  float v = p[px];
  if (!(v > p_min)) return false;
#pragma unroll
  for (int di = -1; di <= 1; ++di) {
    int ii = i + di;
    if (ii < 0 || ii >= H) continue;
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj) {
      if (di == 0 && dj == 0) continue;
      int jj = j + dj;
      if (jj < 0 || jj >= W) continue;
      float nb = p[(size_t)ii * W + jj];
      bool earlier = (di < 0) || (di == 0 && dj < 0);
      if (earlier ? !(v > nb) : !(v >= nb)) return false;
    }
  }
  return true;
}

__global__ void __launch_bounds__(kDecodeThreads) k_decode_count(DecodeArgs a) {
  __shared__ unsigned warp_sum[kDecodeThreads / 32];
  long long npx = (long long)a.T * a.H * a.W;
  long long base = (long long)blockIdx.x * kDecodePxPerBlock;
  unsigned cnt = 0;
  for (int it = 0; it < kDecodePxPerBlock / kDecodeThreads; ++it) {
    long long q = base + it * kDecodeThreads + threadIdx.x;
    bool f = q < npx && dec_flag(a.maps, a.H, a.W, q, a.p_min);
    cnt += __popc(__ballot_sync(0xffffffffu, f));
  }
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) warp_sum[warp] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned s = 0;
    for (int w = 0; w < kDecodeThreads / 32; ++w) s += warp_sum[w];
    a.block_counts[blockIdx.x] = s;
  }
}

// Single block: exclusive scan of block counts, offset by the running total.
__global__ void __launch_bounds__(1024) k_decode_scan(DecodeArgs a, long long nblocks) {
  __shared__ unsigned long long warp_tot[32];
  __shared__ unsigned long long carry;
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = *a.total;
  __syncthreads();
  for (long long start = 0; start < nblocks; start += 1024) {
    long long idx = start + threadIdx.x;
    unsigned long long v = idx < nblocks ? a.block_counts[idx] : 0ull;
    unsigned long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long n = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += n;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      unsigned long long w = warp_tot[lane];
      unsigned long long wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        unsigned long long n = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += n;
      }
      warp_tot[lane] = wi - w;  // exclusive prefix of warp totals
    }
    __syncthreads();
    unsigned long long c = carry;
    if (idx < nblocks) a.block_offsets[idx] = c + warp_tot[warp] + incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry = c + warp_tot[warp] + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *a.total = carry;
}

__global__ void __launch_bounds__(kDecodeThreads) k_decode_write(DecodeArgs a) {
  __shared__ unsigned warp_cnt[kDecodeThreads / 32];
  long long npx = (long long)a.T * a.H * a.W;
  long long plane = (long long)a.H * a.W;
  long long base = (long long)blockIdx.x * kDecodePxPerBlock;
  unsigned long long off = a.block_offsets[blockIdx.x];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned lt_mask = (1u << lane) - 1u;
  for (int it = 0; it < kDecodePxPerBlock / kDecodeThreads; ++it) {
    long long q = base + it * kDecodeThreads + threadIdx.x;
    bool f = q < npx && dec_flag(a.maps, a.H, a.W, q, a.p_min);
    unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) warp_cnt[warp] = __popc(bal);
    __syncthreads();
    unsigned before = 0, total = 0;
    for (int w = 0; w < kDecodeThreads / 32; ++w) {
      unsigned c = warp_cnt[w];
      before += (w < warp) ? c : 0u;
      total += c;
    }
    if (f) {
      unsigned long long idx = off + before + __popc(bal & lt_mask);
      if (idx < a.capacity) {
        int t = (int)(q / plane);
        long long px = q - (long long)t * plane;
        int i = (int)(px / a.W);
        int j = (int)(px - (long long)i * a.W);
        const float* m = a.maps + (size_t)t * kHeads * plane;
        sml_record r;
        r.frame = a.frame0 + t;
        r.x = __fadd_rn((float)j, m[plane + px]);
        r.y = __fadd_rn((float)i, m[2 * plane + px]);
        r.z = __fmul_rn(a.z_scale, m[3 * plane + px]);
        r.photons = __fmul_rn(a.ph_scale, m[4 * plane + px]);
        r.p = m[px];
        a.out[idx] = r;
      }
    }
    off += total;
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_decode(const DecodeArgs& a, cudaStream_t s, int* launches) {
  long long npx = (long long)a.T * a.H * a.W;
  long long nb = decode_blocks(npx);
  if (nb == 0) return cudaSuccess;
  k_decode_count<<<(unsigned)nb, kDecodeThreads, 0, s>>>(a);
  k_decode_scan<<<1, 1024, 0, s>>>(a, nb);
  k_decode_write<<<(unsigned)nb, kDecodeThreads, 0, s>>>(a);
  if (launches) *launches += 3;
  return cudaGetLastError();
}

}  // namespace sml
