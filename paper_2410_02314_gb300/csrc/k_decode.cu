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
// where the rank inside a block comes from warp ballots.  The count pass stores its ballots
// (one bit per pixel) when given room for them, and the write pass then reads them instead of
// evaluating the 3x3 neighbourhoods again.
#include "sml_internal.h"

namespace sml {

namespace {

constexpr int kPxPerThread = kDecodePxPerBlock / kDecodeThreads;

// Location of a pixel of the chunk: frame t, row i, column j (valid = inside the chunk).
struct PxLoc {
  int t, i, j;
  bool valid;
};

// Pixels q0 + k*kDecodeThreads + threadIdx.x (k < kPxPerThread) of the block starting at q0:
// one 64-bit division per thread, then 32-bit arithmetic.
__device__ __forceinline__ void dec_locate(const DecodeArgs& a, long long q0, PxLoc (&loc)[kPxPerThread]) {
  const long long npx = (long long)a.T * a.H * a.W;
  const unsigned plane = (unsigned)a.H * (unsigned)a.W;
  const long long t0 = q0 / plane;
  const unsigned r0 = (unsigned)(q0 - t0 * plane);
#pragma unroll
  for (int k = 0; k < kPxPerThread; ++k) {
    const unsigned off = (unsigned)(k * kDecodeThreads) + threadIdx.x;
    loc[k].valid = q0 + off < npx;
    unsigned r = r0 + off;
    int t = (int)t0;
    if (r >= plane) {  // the block crosses into the next frame(s)
      const unsigned dt = r / plane;
      t += (int)dt;
      r -= dt * plane;
    }
    const unsigned i = r / (unsigned)a.W;
    loc[k].t = t;
    loc[k].i = (int)i;
    loc[k].j = (int)(r - i * (unsigned)a.W);
  }
}

// Detection flags of the thread's pixels.  All centre and neighbour loads are issued before
// any test (out-of-frame neighbours read as -inf, which never blocks a detection), so each
// thread pays one memory round trip instead of two per pixel.
template <int NH>
__device__ __forceinline__ void dec_flags(const DecodeArgs& a, const PxLoc (&loc)[kPxPerThread],
                                          bool (&flag)[kPxPerThread]) {
  const size_t plane = (size_t)a.H * a.W;
  float v[kPxPerThread][9];
#pragma unroll
  for (int k = 0; k < kPxPerThread; ++k) {
    const float* p = a.maps + (size_t)loc[k].t * NH * plane;
#pragma unroll
    for (int di = -1; di <= 1; ++di)
#pragma unroll
      for (int dj = -1; dj <= 1; ++dj) {
        const int ii = loc[k].i + di, jj = loc[k].j + dj;
        const bool in = loc[k].valid && ii >= 0 && ii < a.H && jj >= 0 && jj < a.W;
        v[k][(di + 1) * 3 + dj + 1] = in ? __ldg(p + (size_t)ii * a.W + jj) : -INFINITY;
      }
  }
#pragma unroll
  for (int k = 0; k < kPxPerThread; ++k) {
    const float c = v[k][4];
    bool f = loc[k].valid && c > a.p_min;
#pragma unroll
    for (int n = 0; n < 9; ++n) {
      if (n == 4) continue;
      // strict against earlier neighbours (raster order), >= against later ones
      f = f && (n < 4 ? c > v[k][n] : c >= v[k][n]);
    }
    flag[k] = f;
  }
}

// The same flags as dec_flags, with the horizontal neighbours taken from the adjacent lanes:
// the 32 lanes of a warp hold 32 consecutive pixels in raster order, so each lane loads only
// its own column at rows i-1, i, i+1 and shuffles the columns j-1 and j+1 in; lanes 0 and 31
// load the column just outside the warp's run.  A neighbour outside the frame (j = 0 or
// j = W-1, where the adjacent lane holds the next or previous row) reads as -inf, as in
// dec_flags.
template <int NH>
__device__ __forceinline__ void dec_flags_shfl(const DecodeArgs& a, const PxLoc (&loc)[kPxPerThread],
                                               bool (&flag)[kPxPerThread]) {
  const size_t plane = (size_t)a.H * a.W;
  const int lane = threadIdx.x & 31;
  float col[kPxPerThread][3], edge[kPxPerThread][3];
#pragma unroll
  for (int k = 0; k < kPxPerThread; ++k) {
    const float* p = a.maps + (size_t)loc[k].t * NH * plane;
    const int je = lane == 0 ? loc[k].j - 1 : loc[k].j + 1;
    const bool edge_lane = lane == 0 || lane == 31;
#pragma unroll
    for (int di = -1; di <= 1; ++di) {
      const int ii = loc[k].i + di;
      const bool in = loc[k].valid && ii >= 0 && ii < a.H;
      col[k][di + 1] = in ? __ldg(p + (size_t)ii * a.W + loc[k].j) : -INFINITY;
      edge[k][di + 1] = edge_lane && in && je >= 0 && je < a.W ? __ldg(p + (size_t)ii * a.W + je) : -INFINITY;
    }
  }
#pragma unroll
  for (int k = 0; k < kPxPerThread; ++k) {
    float l[3], r[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      l[q] = __shfl_up_sync(0xffffffffu, col[k][q], 1);
      r[q] = __shfl_down_sync(0xffffffffu, col[k][q], 1);
      if (lane == 0) l[q] = edge[k][q];
      if (lane == 31) r[q] = edge[k][q];
      if (loc[k].j == 0) l[q] = -INFINITY;
      if (loc[k].j == a.W - 1) r[q] = -INFINITY;
    }
    const float c = col[k][1];
    // strict against earlier neighbours (row i-1, and the left one), >= against later ones
    flag[k] = loc[k].valid && c > a.p_min && c > l[0] && c > col[k][0] && c > r[0] && c > l[1] && c >= r[1] &&
              c >= l[2] && c >= col[k][2] && c >= r[2];
  }
}

// NH: channels of the maps (5, or 9 with the uncertainty maps).
template <int NH>
__global__ void __launch_bounds__(kDecodeThreads) k_decode_count(DecodeArgs a) {
  __shared__ unsigned warp_sum[kDecodeThreads / 32];
  const long long q0 = (long long)blockIdx.x * kDecodePxPerBlock;
  PxLoc loc[kPxPerThread];
  bool flag[kPxPerThread];
  dec_locate(a, q0, loc);
  dec_flags_shfl<NH>(a, loc, flag);
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned cnt = 0;
#pragma unroll
  for (int k = 0; k < kPxPerThread; ++k) {
    const unsigned b = __ballot_sync(0xffffffffu, flag[k]);
    cnt += __popc(b);
    if (a.flag_words && lane == 0)
      a.flag_words[((size_t)blockIdx.x * kPxPerThread + k) * (kDecodeThreads / 32) + warp] = b;
  }
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

// SIGMA: also write the uncertainties of each record (9-head maps).  STORED: the detections
// come from the count pass's ballots (a.flag_words) instead of the maps' neighbourhoods.
template <int NH, bool SIGMA, bool STORED>
__global__ void __launch_bounds__(kDecodeThreads) k_decode_write(DecodeArgs a) {
  __shared__ unsigned warp_cnt[kPxPerThread][kDecodeThreads / 32];
  const long long q0 = (long long)blockIdx.x * kDecodePxPerBlock;
  const size_t plane = (size_t)a.H * a.W;
  PxLoc loc[kPxPerThread];
  bool flag[kPxPerThread];
  dec_locate(a, q0, loc);
  if (!STORED) dec_flags<NH>(a, loc, flag);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  unsigned bal[kPxPerThread];
#pragma unroll
  for (int k = 0; k < kPxPerThread; ++k) {
    if (STORED) {
      bal[k] = a.flag_words[((size_t)blockIdx.x * kPxPerThread + k) * (kDecodeThreads / 32) + warp];
      flag[k] = (bal[k] >> lane) & 1u;
    } else {
      bal[k] = __ballot_sync(0xffffffffu, flag[k]);
    }
    if (lane == 0) warp_cnt[k][warp] = __popc(bal[k]);
  }
  __syncthreads();
  // raster order inside the block: pass k, then warp, then lane
  unsigned long long off = a.block_offsets[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kPxPerThread; ++k) {
    unsigned before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kDecodeThreads / 32; ++w) {
      const unsigned c = warp_cnt[k][w];
      before += (w < warp) ? c : 0u;
      total += c;
    }
    if (flag[k]) {
      const unsigned long long idx = off + before + __popc(bal[k] & lt_mask);
      if (idx < a.capacity) {
        const size_t px = (size_t)loc[k].i * a.W + loc[k].j;
        const float* m = a.maps + (size_t)loc[k].t * NH * plane;
        sml_record r;
        r.frame = a.frame0 + loc[k].t;
        r.x = __fadd_rn((float)loc[k].j, m[plane + px]);
        r.y = __fadd_rn((float)loc[k].i, m[2 * plane + px]);
        r.z = __fmul_rn(a.z_scale, m[3 * plane + px]);
        r.photons = __fmul_rn(a.ph_scale, m[4 * plane + px]);
        r.p = m[px];
        a.out[idx] = r;
        if (SIGMA) {  // uncertainty maps 5..8 at the same pixel
          sml_sigma u;
          u.sigma_x = m[5 * plane + px];
          u.sigma_y = m[6 * plane + px];
          u.sigma_z = __fmul_rn(a.z_scale, m[7 * plane + px]);
          u.sigma_photons = __fmul_rn(a.ph_scale, m[8 * plane + px]);
          a.out_sigma[idx] = u;
        }
      }
    }
    off += total;
  }
}

}  // namespace

cudaError_t launch_decode(const DecodeArgs& a, cudaStream_t s, int* launches) {
  if (a.nh != kHeads && a.nh != kMaxHeads) return cudaErrorInvalidValue;
  long long npx = (long long)a.T * a.H * a.W;
  long long nb = decode_blocks(npx);
  if (nb == 0) return cudaSuccess;
  if (a.nh == kMaxHeads)
    k_decode_count<kMaxHeads><<<(unsigned)nb, kDecodeThreads, 0, s>>>(a);
  else
    k_decode_count<kHeads><<<(unsigned)nb, kDecodeThreads, 0, s>>>(a);
  k_decode_scan<<<1, 1024, 0, s>>>(a, nb);
  const bool st = a.flag_words != nullptr;
  if (a.nh == kMaxHeads && a.out_sigma) {
    if (st) k_decode_write<kMaxHeads, true, true><<<(unsigned)nb, kDecodeThreads, 0, s>>>(a);
    else k_decode_write<kMaxHeads, true, false><<<(unsigned)nb, kDecodeThreads, 0, s>>>(a);
  } else if (a.nh == kMaxHeads) {
    if (st) k_decode_write<kMaxHeads, false, true><<<(unsigned)nb, kDecodeThreads, 0, s>>>(a);
    else k_decode_write<kMaxHeads, false, false><<<(unsigned)nb, kDecodeThreads, 0, s>>>(a);
  } else {
    if (st) k_decode_write<kHeads, false, true><<<(unsigned)nb, kDecodeThreads, 0, s>>>(a);
    else k_decode_write<kHeads, false, false><<<(unsigned)nb, kDecodeThreads, 0, s>>>(a);
  }
  if (launches) *launches += 3;
  return cudaGetLastError();
}

}  // namespace sml
