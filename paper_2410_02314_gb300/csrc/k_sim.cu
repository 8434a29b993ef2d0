// Camera-frame simulator on the device (the synthetic workloads' generator; the paper's own
// data are simulated frames, Sec. 4.1).  The definition is in include/sml_sim.h.
//
// Emitters are binned on the host into 16 x 16 pixel tiles per frame (counting sort).  One
// block renders one tile: it stages the emitters of the tiles within the PSF window, computes
// each emitter's pixel-integrated factors for the tile's 16 columns and 16 rows once (the PSF
// is separable), and every thread sums N * Ey(i) * Ex(j) over them for its pixel, then draws
// the Poisson count and converts to ADU.
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/sml_sim.h"
#include "sml_internal.h"

namespace sml {
namespace {

constexpr int kTile = 16;      // tile edge (px); a block of kTile^2 threads renders one tile
constexpr int kSimBatch = 64;  // emitters staged per round

struct SimEmitter {
  float x, y, sx, sy, photons, cx, cy, pad;  // cx, cy: rint of x, y (the PSF window's centre)
};

struct SimArgs {
  const SimEmitter* em;
  const int* bin_off;  // [T * nty * ntx + 1]
  const float* bg;     // [T]
  int T, H, W, ntx, nty, r, reach;
  CamArgs cam;
  unsigned long long seed;
  long long frame0;
  int noise;
  uint16_t* adu;
  float* mu_out;
};

// The i-th output (from 0) of splitmix64 seeded with `seed` (Vigna's published generator:
// the state advances by the golden-ratio increment, each output is the state mixed).
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed, unsigned long long i) {
  unsigned long long z = seed + (i + 1ull) * 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

struct PixelUniforms {
  unsigned long long seed, base;
  int k = 0;
  __device__ double next() {  // u in [0, 1); at most 64 per pixel
    const unsigned long long b = splitmix64_at(seed, base + (unsigned long long)(k < 63 ? k : 63));
    ++k;
    return (double)(b >> 11) * 0x1.0p-53;
  }
};

// Poisson(mu) from the pixel's uniforms: Knuth's multiplication method below 12, Hormann's
// transformed rejection with squeeze (PTRS) from 12 on; draws are bounded (64 per pixel).
__device__ double poisson_draw(double mu, PixelUniforms& u) {
  if (!(mu > 0.0)) return 0.0;
  if (mu < 12.0) {
    const double L = exp(-mu);
    double p = 1.0;
    int k = 0;
    for (; k < 63; ++k) {
      p *= u.next();
      if (p <= L) break;
    }
    return (double)k;
  }
  const double smu = sqrt(mu), b = 0.931 + 2.53 * smu, a = -0.059 + 0.02483 * b;
  const double inv_alpha = 1.1239 + 1.1328 / (b - 3.4), vr = 0.9277 - 3.6224 / (b - 2.0);
  const double log_mu = log(mu);
  double k = floor(mu);
  for (int trial = 0; trial < 31; ++trial) {
    const double U = u.next() - 0.5, V = u.next();
    const double us = 0.5 - fabs(U);
    k = floor((2.0 * a / us + b) * U + mu + 0.43);
    if (us >= 0.07 && V <= vr) return k;
    if (k < 0.0 || (us < 0.013 && V > us)) continue;
    if (log(V) + log(inv_alpha) - log(a / (us * us) + b) <= -mu + k * log_mu - lgamma(k + 1.0)) return k;
  }
  return k < 0.0 ? 0.0 : k;  // 31 rejections in a row: not reached in practice
}

// Pixel-integrated 1-D Gaussian over the pixel centred at integer index c.
__device__ __forceinline__ float pix_integral(float c, float mu, float s2) {
  return 0.5f * (erff((c + 0.5f - mu) / s2) - erff((c - 0.5f - mu) / s2));
}

__global__ void __launch_bounds__(kTile * kTile) k_sim(const SimArgs a) {
  __shared__ SimEmitter s_em[kSimBatch];
  __shared__ float s_ex[kSimBatch][kTile], s_ey[kSimBatch][kTile];
  const int t = blockIdx.z, tx = blockIdx.x, ty = blockIdx.y;
  const int i0 = ty * kTile, j0 = tx * kTile;
  const int li = threadIdx.x / kTile, lj = threadIdx.x % kTile;
  const int i = i0 + li, j = j0 + lj;
  float mu = 0.0f;
  for (int dy = -a.reach; dy <= a.reach; ++dy) {
    const int by = ty + dy;
    if (by < 0 || by >= a.nty) continue;
    for (int dx = -a.reach; dx <= a.reach; ++dx) {
      const int bx = tx + dx;
      if (bx < 0 || bx >= a.ntx) continue;
      const int bin = (t * a.nty + by) * a.ntx + bx;
      const int e0 = a.bin_off[bin], e1 = a.bin_off[bin + 1];
      for (int base = e0; base < e1; base += kSimBatch) {  // uniform across the block
        const int ne = e1 - base < kSimBatch ? e1 - base : kSimBatch;
        if (threadIdx.x < ne) s_em[threadIdx.x] = a.em[base + threadIdx.x];
        __syncthreads();
        for (int p = threadIdx.x; p < ne * 2 * kTile; p += blockDim.x) {
          const int e = p / (2 * kTile), k = p % (2 * kTile);
          const SimEmitter& m = s_em[e];
          if (k < kTile) {  // column factor; zero outside the emitter's window
            const int jj = j0 + k;
            s_ex[e][k] = fabsf((float)jj - m.cx) <= (float)a.r ? pix_integral((float)jj, m.x, 1.41421356f * m.sx) : 0.0f;
          } else {
            const int ii = i0 + k - kTile;
            s_ey[e][k - kTile] =
                fabsf((float)ii - m.cy) <= (float)a.r ? pix_integral((float)ii, m.y, 1.41421356f * m.sy) : 0.0f;
          }
        }
        __syncthreads();
        for (int e = 0; e < ne; ++e) mu = fmaf(s_em[e].photons * s_ey[e][li], s_ex[e][lj], mu);
        __syncthreads();
      }
    }
  }
  if (i >= a.H || j >= a.W) return;
  mu += a.bg[t];
  const size_t q = ((size_t)t * a.H + i) * a.W + j;
  if (a.mu_out) a.mu_out[q] = mu;
  double e = mu;
  if (a.noise) {
    PixelUniforms u{a.seed, ((((unsigned long long)(a.frame0 + t) * a.H + i) * a.W + j) * 64ull)};
    e = poisson_draw((double)mu, u);
  }
  const size_t px = (size_t)i * a.W + j;
  const double g = a.cam.gain_map ? (double)a.cam.gain_map[px] : (double)a.cam.gain;
  const double o = a.cam.offset_map ? (double)a.cam.offset_map[px] : (double)a.cam.offset;
  double v = rint(__dadd_rn(__dmul_rn(e, g), o));  // two roundings, as written (no FMA)
  v = v < 0.0 ? 0.0 : (v > 65535.0 ? 65535.0 : v);
  a.adu[q] = (uint16_t)v;
}

}  // namespace
}  // namespace sml

extern "C" int sml_sim_frames(const int32_t* frame, const float* x, const float* y, const float* z,
                              const float* photons, long long n, const float* bg, int T, int H, int W, int astig,
                              float sigma0, const sml_camera* cam, unsigned long long seed, long long frame0, int noise,
                              uint16_t* d_adu, float* d_mu) {
  using namespace sml;
  if (T < 0 || T > 65535 || H < 1 || W < 1 || H > 16384 || W > 16384 || n < 0 || !(sigma0 > 0.0f) || !cam || !d_adu ||
      (T > 0 && !bg) || frame0 < 0)
    return SML_ERR_BAD_ARG;
  if (n > 0 && (!frame || !x || !y || !photons || (astig && !z))) return SML_ERR_BAD_ARG;
  if (!cam->gain_map && !(cam->gain > 0.0f)) return SML_ERR_BAD_ARG;
  if (T == 0) return SML_OK;
  const int ntx = (W + kTile - 1) / kTile, nty = (H + kTile - 1) / kTile;
  const long long nbins = (long long)T * ntx * nty;
  if (nbins >= (1LL << 31) || n >= (1LL << 31)) return SML_ERR_BAD_ARG;  // tile bins and offsets are 32-bit
  // widths, PSF window and tile bins on the host
  std::vector<SimEmitter> em((size_t)n);
  std::vector<int> key((size_t)n);
  double smax = sigma0;
  for (long long k = 0; k < n; ++k) {
    if (frame[k] < 0 || frame[k] >= T || !std::isfinite(x[k]) || !std::isfinite(y[k]) || !(photons[k] >= 0.0f))
      return SML_ERR_BAD_ARG;
    double sx = sigma0, sy = sigma0;
    if (astig) {
      const double ux = ((double)z[k] + 400.0) / 500.0, uy = ((double)z[k] - 400.0) / 500.0;
      sx = sigma0 * std::sqrt(1.0 + ux * ux);
      sy = sigma0 * std::sqrt(1.0 + uy * uy);
    }
    smax = std::max(smax, std::max(sx, sy));
    SimEmitter& m = em[(size_t)k];
    m.x = x[k];
    m.y = y[k];
    m.sx = (float)sx;
    m.sy = (float)sy;
    m.photons = photons[k];
    m.cx = (float)std::nearbyint((double)x[k]);
    m.cy = (float)std::nearbyint((double)y[k]);
    m.pad = 0.0f;
    const int bx = (int)std::min<double>(std::max<double>(m.cx, 0.0), W - 1) / kTile;
    const int by = (int)std::min<double>(std::max<double>(m.cy, 0.0), H - 1) / kTile;
    key[(size_t)k] = (int)(((long long)frame[k] * nty + by) * ntx + bx);
  }
  const int r = (int)std::ceil(4.0 * smax) + 1;
  const int reach = (r + kTile - 1) / kTile;
  std::vector<int> off((size_t)nbins + 1, 0);
  for (long long k = 0; k < n; ++k) ++off[(size_t)key[(size_t)k] + 1];
  for (long long b = 0; b < nbins; ++b) off[(size_t)b + 1] += off[(size_t)b];
  std::vector<SimEmitter> sorted((size_t)n);
  {
    std::vector<int> fill(off.begin(), off.end() - 1);
    for (long long k = 0; k < n; ++k) sorted[(size_t)fill[(size_t)key[(size_t)k]]++] = em[(size_t)k];
  }
  SimEmitter* d_em = nullptr;
  int* d_off = nullptr;
  float* d_bg = nullptr;
  auto release = [&]() {
    cudaFree(d_em);
    cudaFree(d_off);
    cudaFree(d_bg);
  };
  cudaError_t e;
  if ((e = cudaMalloc(&d_em, std::max<size_t>(1, (size_t)n) * sizeof(SimEmitter))) != cudaSuccess ||
      (e = cudaMalloc(&d_off, off.size() * sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&d_bg, (size_t)T * sizeof(float))) != cudaSuccess) {
    release();
    return e == cudaErrorMemoryAllocation ? SML_ERR_OOM : SML_ERR_CUDA;
  }
  if ((n > 0 && cudaMemcpy(d_em, sorted.data(), (size_t)n * sizeof(SimEmitter), cudaMemcpyHostToDevice) != cudaSuccess) ||
      cudaMemcpy(d_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_bg, bg, (size_t)T * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
    release();
    return SML_ERR_CUDA;
  }
  SimArgs a{};
  a.em = d_em;
  a.bin_off = d_off;
  a.bg = d_bg;
  a.T = T;
  a.H = H;
  a.W = W;
  a.ntx = ntx;
  a.nty = nty;
  a.r = r;
  a.reach = reach;
  a.cam = CamArgs{cam->gain, cam->offset, 1.0f, cam->gain_map, cam->offset_map};
  a.seed = seed;
  a.frame0 = frame0;
  a.noise = noise;
  a.adu = d_adu;
  a.mu_out = d_mu;
  k_sim<<<dim3((unsigned)ntx, (unsigned)nty, (unsigned)T), kTile * kTile>>>(a);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  release();
  return e == cudaSuccess ? SML_OK : SML_ERR_CUDA;
}
