// sml_decode_maps_static: the decode of sml_decode_maps for callers that cannot allocate
// device memory.
//
// Who needs it: code that must not call cudaMalloc / cudaFree while it runs, e.g. an
// acquisition loop that shares the GPU with a live camera stream (cudaFree synchronises the
// whole device and would stall it), or a plugin whose host application reserves all device
// memory in its own pool so that a cudaMalloc from the library would fail.  Such a caller
// passes its own input, output and count buffers; the only scratch (per-block detection
// counts and their prefix offsets) lives in the fixed array below.
//
// The array holds kStaticMaxBlocks entries, enough for kStaticMaxPixels = T*H*W pixels per
// call (16,777,216, e.g. 256 frames of 256 x 256); larger calls are rejected.  Every GPU that
// loads the library keeps this array (192 KiB) until the process exits.  All calls share it:
// two calls whose work overlaps on the GPU (different streams, or different host threads)
// race on it and must be serialised by the caller.  Each call rewrites every scratch entry
// it reads, and zeroes the caller's count before use.
#include <mutex>

#include "../../include/sml.h"
#include "sml_internal.h"

namespace sml {
namespace {

constexpr long long kStaticMaxPixels = 1LL << 24;
constexpr long long kStaticMaxBlocks = kStaticMaxPixels / kDecodePxPerBlock;

struct StaticScratch {
  unsigned long long offsets[kStaticMaxBlocks];
  unsigned counts[kStaticMaxBlocks];
};

static __device__ __align__(256) StaticScratch g_scratch;

// Device address of g_scratch, looked up with the device current on the first call and again
// whenever the current CUDA context's unique ID differs from the one of the last look-up:
// after cudaDeviceReset (or a release of the primary context) the module is loaded anew in a
// new context and the array may live elsewhere.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
StaticScratch* g_addr[kMaxDevices] = {nullptr};
unsigned long long g_addr_ctx[kMaxDevices] = {0};

typedef CUresult (*PFN_ctxGetCurrent_t)(CUcontext*);
typedef CUresult (*PFN_ctxGetId_t)(CUcontext, unsigned long long*);

template <typename F>
F driver_fn(const char* name) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    return reinterpret_cast<F>(p);
  return nullptr;
}

// Unique ID of the calling thread's current context (0 if none is current yet).
bool current_ctx_id(unsigned long long* id) {
  static PFN_ctxGetCurrent_t get_cur = driver_fn<PFN_ctxGetCurrent_t>("cuCtxGetCurrent");
  static PFN_ctxGetId_t get_id = driver_fn<PFN_ctxGetId_t>("cuCtxGetId");
  CUcontext cur = nullptr;
  if (!get_cur || !get_id || get_cur(&cur) != CUDA_SUCCESS) return false;
  *id = 0;
  return !cur || get_id(cur, id) == CUDA_SUCCESS;
}

int scratch_address(StaticScratch** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SML_ERR_CUDA;
  unsigned long long id = 0;
  if (!current_ctx_id(&id)) return SML_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (id == 0 || !g_addr[dev] || g_addr_ctx[dev] != id) {
    // the look-up also makes the device's primary context current when none was
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return SML_ERR_CUDA;
    if (!current_ctx_id(&id) || id == 0) return SML_ERR_CUDA;
    g_addr[dev] = static_cast<StaticScratch*>(p);
    g_addr_ctx[dev] = id;
  }
  *out = g_addr[dev];
  return SML_OK;
}

}  // namespace
}  // namespace sml

extern "C" int sml_decode_maps_static(const float* d_maps, int T, int H, int W, float p_min, float z_scale,
                                      float ph_scale, sml_record* d_out, size_t capacity,
                                      unsigned long long* d_n_out, void* stream) {
  using namespace sml;
  if (!d_n_out || (T > 0 && !d_maps) || (capacity > 0 && !d_out)) return SML_ERR_BAD_ARG;
  if (T < 0 || H < 1 || W < 1 || H > 16384 || W > 16384) return SML_ERR_BAD_ARG;
  if (!(p_min >= 0.0f && p_min < 1.0f)) return SML_ERR_BAD_ARG;
  if ((long long)T * H * W > kStaticMaxPixels) return SML_ERR_UNSUPPORTED;  // beyond the fixed scratch
  StaticScratch* scratch = nullptr;
  int r = scratch_address(&scratch);
  if (r) return r;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(d_n_out, 0, sizeof(unsigned long long), s) != cudaSuccess) return SML_ERR_CUDA;
  if (T == 0) return SML_OK;
  DecodeArgs da{};
  da.maps = d_maps;
  da.T = T;
  da.H = H;
  da.W = W;
  da.frame0 = 0;
  da.p_min = p_min;
  da.z_scale = z_scale;
  da.ph_scale = ph_scale;
  da.out = d_out;
  da.capacity = capacity;
  da.total = d_n_out;
  da.block_counts = scratch->counts;
  da.block_offsets = scratch->offsets;
  return launch_decode(da, s, nullptr) == cudaSuccess ? SML_OK : SML_ERR_CUDA;
}
