// C ABI and host runtime: net-spec parsing, weight upload (BatchNorm folding, layout packing,
// FP8 scaling), per-frame-size plans (workspace, TMA descriptors), chunked execution and
// the host <-> device boundary.  The entry points are documented in include/sml.h.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cctype>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include <chrono>

#include "../../include/sml_debug.h"
#include "../../include/sml_io.h"
#include "../../include/sml_train.h"
#include "sml_internal.h"

using namespace sml;

namespace {

// The training kernels read and write activations 16 bytes at a time.
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// ------------------------------------------------------------------ tiny JSON reader
struct JVal {
  enum Kind { kNull, kNum, kStr, kArr, kObj, kBool } kind = kNull;
  double num = 0;
  std::string str;
  std::vector<JVal> arr;
  std::map<std::string, JVal> obj;
};

struct JParser {
  const char* p;
  bool ok = true;
  void ws() {
    while (*p && isspace((unsigned char)*p)) ++p;
  }
  bool lit(const char* s) {
    size_t n = strlen(s);
    if (strncmp(p, s, n) == 0) {
      p += n;
      return true;
    }
    return false;
  }
  JVal value() {
    JVal v;
    ws();
    if (*p == '{') {
      ++p;
      v.kind = JVal::kObj;
      ws();
      if (*p == '}') {
        ++p;
        return v;
      }
      while (ok) {
        ws();
        JVal k = value();
        if (!ok || k.kind != JVal::kStr) {
          ok = false;
          break;
        }
        ws();
        if (*p != ':') {
          ok = false;
          break;
        }
        ++p;
        v.obj[k.str] = value();
        ws();
        if (*p == ',') {
          ++p;
          continue;
        }
        if (*p == '}') {
          ++p;
          break;
        }
        ok = false;
      }
    } else if (*p == '[') {
      ++p;
      v.kind = JVal::kArr;
      ws();
      if (*p == ']') {
        ++p;
        return v;
      }
      while (ok) {
        v.arr.push_back(value());
        ws();
        if (*p == ',') {
          ++p;
          continue;
        }
        if (*p == ']') {
          ++p;
          break;
        }
        ok = false;
      }
    } else if (*p == '"') {
      ++p;
      v.kind = JVal::kStr;
      while (*p && *p != '"') {
        if (*p == '\\' && p[1]) ++p;
        v.str.push_back(*p++);
      }
      if (*p != '"') ok = false;
      else ++p;
    } else if (lit("true")) {
      v.kind = JVal::kBool;
      v.num = 1;
    } else if (lit("false")) {
      v.kind = JVal::kBool;
    } else if (lit("null")) {
      v.kind = JVal::kNull;
    } else {
      char* end = nullptr;
      v.num = strtod(p, &end);
      if (end == p) ok = false;
      else {
        v.kind = JVal::kNum;
        p = end;
      }
    }
    return v;
  }
};

// ------------------------------------------------------------------ tensor map encoder
typedef CUresult (*PFN_encodeTiled_t)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                      const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                      CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

PFN_encodeTiled_t get_encoder() {
  static PFN_encodeTiled_t fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_encodeTiled_t>(p);
  }
  return fn;
}

std::string g_create_error;

}  // namespace

// ------------------------------------------------------------------ context
constexpr int kMaxBufs = 6;    // activation buffers: 2 at full resolution, 2 per U-Net level
constexpr int kMaxLevels = 2;  // U-Net levels

struct Plan {
  int H = 0, W = 0, Tc = 0;
  unsigned long long last_use = 0;
  void* act[kMaxBufs] = {nullptr};
  float* maps = nullptr;
  unsigned* block_counts = nullptr;
  unsigned long long* block_offsets = nullptr;
  unsigned* flag_words = nullptr;  // decode: the count pass's detection ballots
  uint16_t* frames = nullptr;  // staging for host frames
  float* cam_maps = nullptr;   // staging for host camera maps [2][H][W]
  cudaEvent_t done = nullptr;  // recorded on the stream of every call that used the plan
  size_t bytes = 0;            // device bytes of the buffers above
  CUtensorMap tmap[kMaxLayers];  // per layer, over its input buffer: one box per row (width depends on d)
  bool pair_rows[kMaxLayers] = {false};  // FP8 layers whose map loads 32-byte pixel pairs
};

// One conv layer of the net in execution order: cin -> cout channels at dilation d.  Layer 0
// reads the frames; layer l >= 1 reads channels [0, cin) of activation buffer in_buf and
// (unless it is the last layer, whose output feeds the heads) writes channels
// [out_off, out_off + cout) of buffer out_buf.  Plain stacks alternate between the two buffers.
// A dense block (Sec. 3.2.1) keeps its concatenation in one buffer: the block input in
// channels [0, C), dense layer j reads [0, C + j g) and appends its g outputs at C + j g; the
// transition reads the whole concatenation and writes the next block input into [0, C) of
// the other buffer.
struct LayerDesc {
  int cin = 0, cout = 0, d = 1, in_buf = -1, out_buf = 0, out_off = 0;
  int level = 0;  // resolution: H and W halved (rounded up) level times (U-Net layers)
};

// An activation buffer: its resolution level and channels per pixel.  Buffers 0 and 1 are the
// full-resolution ping-pong pair; a U-Net of L levels adds per level l a skip buffer A_l
// (2C channels: the level's features, then the upsampled ones) and a work buffer B_l (C).
struct BufDesc {
  int level = 0, ct = 0;
};

// One launch of the forward after layer 1, in order: a conv layer (LayerDesc index `layer`),
// or a 2x2 max pool / nearest 2x upsample of channels [0, C) of in_buf into channels
// [out_off, out_off + C) of out_buf.
enum StepKind { kStepConv = 0, kStepPool = 1, kStepUp = 2 };
struct Step {
  int kind = kStepConv, layer = 0;
  int in_buf = 0, out_buf = 0, out_off = 0, C = 0;
};

struct sml_ctx {
  int device = 0, num_sms = 0;
  // spec
  int in_ch = 1, C = 0, L = 0;
  LayerDesc lay[kMaxLayers];
  int growth = 0;  // dense blocks: channels each dense layer adds (0: plain stack)
  int nh = kHeads; // output heads: 5, or 9 with the uncertainty heads
  int unet = 0;    // U-Net fine stage levels before the last layer (0: none)
  BufDesc buf[kMaxBufs];
  int nbuf = 2;
  std::vector<Step> steps;
  int ct = 0;      // channels per pixel of the activation buffers (C, or C + the longest block's k g)
  int prec = kFP32;
  float in_scale = 1e-3f, z_scale = 1000.f, ph_scale = 10000.f;
  float act_scale[kMaxLayers] = {0};
  long long chunk_px = 1 << 24;
  int tc_stages = 0;  // "tc_stages": TMA ring depth, 0 = as deep as shared memory allows
  // failure-path tests ("debug_wait_ns", "debug_poison_cta"): a shorter give-up time of the
  // tensor-core kernels' waits, and one CTA of every conv launch whose producer loads nothing
  unsigned long long debug_wait_ns = 0;
  int debug_poison_cta = -1;
  bool fp8_pair_rows = true;  // "fp8_pair_rows": 0 keeps 16-byte TMA rows for FP8 (comparison runs)
  // device weights
  std::vector<float> w1, b1;  // layer 1 [C][in_ch][9], [C] (host: passed to the kernel by value)
  float* wf32[kMaxLayers] = {nullptr};  // [9][cin][cout]
  float* bias[kMaxLayers] = {nullptr};
  void* bimg[kMaxLayers] = {nullptr};
  float* deq[kMaxLayers] = {nullptr};
  float* head_w = nullptr;  // device copies (FP32 SIMT path)
  float* head_b = nullptr;
  // host copies for the tensor-core path (passed to its kernels by value)
  std::vector<float> h_bias[kMaxLayers], h_deq[kMaxLayers];
  std::vector<float> h_head_w, h_head_b;
  // runtime: plans (workspace + TMA maps) for up to kMaxPlans frame sizes, least recently
  // used evicted first; plan points at the one in use
  std::vector<std::unique_ptr<Plan>> plans;
  Plan* plan = nullptr;
  unsigned long long plan_clock = 0;
  cudaStream_t stream = nullptr;
  unsigned long long* d_total = nullptr;
  int* d_err = nullptr;
  sml_record* d_rec = nullptr;
  size_t d_rec_cap = 0;
  sml_sigma* d_sig = nullptr;  // staging of uncertainty records for host outputs
  size_t d_sig_cap = 0;
  std::vector<void*> owned;
  std::string err;
  int launches = 0;
  // kernel timing (sml_profile_enable)
  bool prof_on = false;
  struct ProfEv {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<ProfEv> prof_events;
  size_t prof_used = 0;
};

namespace {

int fail(sml_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  else g_create_error = buf;
  return code;
}

int cuda_fail(sml_ctx* c, cudaError_t e, const char* where) {
  return fail(c, e == cudaErrorMemoryAllocation ? SML_ERR_OOM : SML_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define SML_CUDA(call, where)                  \
  do {                                         \
    cudaError_t e_ = (call);                   \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

template <typename T>
int dev_alloc(sml_ctx* ctx, T** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc");
  *p = static_cast<T*>(q);
  return SML_OK;
}

template <typename T>
int upload(sml_ctx* ctx, T** dst, const void* src, size_t bytes) {
  int r = dev_alloc(ctx, dst, bytes);
  if (r) return r;
  ctx->owned.push_back(*dst);
  SML_CUDA(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice), "upload");
  return SML_OK;
}

void free_plan(Plan& p) {
  if (p.done) cudaEventDestroy(p.done);
  for (void* a : p.act) cudaFree(a);
  cudaFree(p.maps);
  cudaFree(p.block_counts);
  cudaFree(p.block_offsets);
  cudaFree(p.flag_words);
  cudaFree(p.frames);
  cudaFree(p.cam_maps);
  p = Plan();
}

size_t act_elem_bytes(int prec) { return prec == kFP32 ? 4 : (prec == kBF16 ? 2 : 1); }

// Size of a frame dimension at a U-Net level: halved, rounded up, `level` times.
int level_dim(int n, int level) {
  for (int k = 0; k < level; ++k) n = (n + 1) / 2;
  return n;
}

// Row-planar activations [Tc][H][Gt][W][row bytes], Gt = ct/16 groups of 16 channels (32-byte
// rows in BF16, 16-byte rows in FP8).  A layer reading its first g_in groups sees the 5-D
// tensor (group row, W, g_in, H, Tc) with the buffer's strides and loads boxes (group row,
// tc_box_width(d) pixels, g_in, 1, 1): one input row segment per box, BF16 rows with the
// 32-byte swizzle.  Pixels left of 0 or right of W-1, and rows outside [0,H), are filled with
// zeros by TMA.  FP8 frames of even width are read as 32-byte pixel pairs instead (pairs =
// true): tensor (pair of group rows, W/2, g_in, H, Tc), boxes of tc_box_width(d)/2 pairs,
// which land in shared memory byte for byte as the 16-byte rows would (a TMA row of 16 bytes
// moves a half sector; a pair row a whole one).
int encode_act_map(sml_ctx* ctx, CUtensorMap* m, void* base, int Tc, int H, int W, int d, int g_in, int gt,
                   bool pairs = false) {
  PFN_encodeTiled_t enc = get_encoder();
  if (!enc) return fail(ctx, SML_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  const bool bf16 = ctx->prec == kBF16;
  if (pairs && (bf16 || W % 2)) return fail(ctx, SML_ERR_CUDA, "pixel-pair rows need fp8 and an even width");
  const cuuint64_t rowb = bf16 ? 32 : 16;
  cuuint64_t dims[5] = {pairs ? 32ull : 16ull, (cuuint64_t)(pairs ? W / 2 : W), (cuuint64_t)g_in, (cuuint64_t)H,
                        (cuuint64_t)Tc};
  cuuint64_t strides[4] = {pairs ? 32ull : rowb, rowb * W, rowb * W * gt, rowb * W * gt * H};
  cuuint32_t box[5] = {pairs ? 32u : 16u, (cuuint32_t)(pairs ? tc_box_width(d) / 2 : tc_box_width(d)),
                       (cuuint32_t)g_in, 1u, 1u};
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  CUresult r = enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 5, base, dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, bf16 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, SML_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return SML_OK;
}

// Brackets the launches issued in its scope with an event pair when profiling is on.
struct ProfScope {
  sml_ctx* ctx;
  sml_ctx::ProfEv* ev = nullptr;
  cudaStream_t s;
  ProfScope(sml_ctx* c, int cls, cudaStream_t st) : ctx(c), s(st) {
    if (!ctx->prof_on) return;
    if (ctx->prof_used == ctx->prof_events.size()) {
      sml_ctx::ProfEv e{cls, nullptr, nullptr};
      if (cudaEventCreate(&e.a) != cudaSuccess || cudaEventCreate(&e.b) != cudaSuccess) return;
      ctx->prof_events.push_back(e);
    }
    ev = &ctx->prof_events[ctx->prof_used++];
    ev->cls = cls;
    cudaEventRecord(ev->a, s);
  }
  ~ProfScope() {
    if (ev) cudaEventRecord(ev->b, s);
  }
};

constexpr size_t kMaxPlans = 4;

// Frames per chunk of a call on T frames of H x W: as many as chunk_px pixels hold (at least
// one), and no more than the call has.
int chunk_frames_for(const sml_ctx* ctx, int T, int H, int W) {
  const long long tmax = std::max(1LL, ctx->chunk_px / ((long long)H * W));
  return (int)std::max(1LL, std::min<long long>(T, tmax));
}

// Device buffers of a plan for frames of H x W: the chunk (Tc frames of at most chunk_px
// pixels together), the activation buffers of every resolution level, the maps, the decode
// scratch, and the staging of host frames (with the context frames) and host camera maps.
struct PlanSizes {
  int Tc = 1;
  size_t act[kMaxBufs] = {0};
  size_t maps = 0, counts = 0, offsets = 0, flags = 0, frames = 0, cam = 0;
  size_t total() const {
    size_t t = maps + counts + offsets + flags + frames + cam;
    for (size_t a : act) t += a;
    return t;
  }
};

PlanSizes plan_sizes(const sml_ctx* ctx, int H, int W, int Tc) {
  PlanSizes z;
  const long long hw = (long long)H * W;
  z.Tc = Tc;
  const size_t npx = (size_t)z.Tc * hw;
  for (int b = 0; b < ctx->nbuf; ++b)
    z.act[b] = (size_t)z.Tc * level_dim(H, ctx->buf[b].level) * level_dim(W, ctx->buf[b].level) * ctx->buf[b].ct *
               act_elem_bytes(ctx->prec);
  z.maps = npx * ctx->nh * sizeof(float);
  z.counts = decode_blocks(npx) * sizeof(unsigned);
  z.offsets = decode_blocks(npx) * sizeof(unsigned long long);
  z.flags = decode_blocks(npx) * (kDecodePxPerBlock / 32) * sizeof(unsigned);
  z.frames = (size_t)(z.Tc + 2) * hw * sizeof(uint16_t);  // + context frames
  z.cam = 2 * hw * sizeof(float);
  return z;
}

// Marks the end of a call's use of the current plan on its stream: a later eviction of the
// plan waits for this point only (not for the whole device).
void plan_used(sml_ctx* ctx, cudaStream_t s) {
  if (ctx->plan && ctx->plan->done) cudaEventRecord(ctx->plan->done, s);
}

// The plan for a call on T frames of H x W: the context's plan of that frame size if its
// chunk holds the call's chunk, else a new one (replacing a smaller plan of the size, and
// evicting the least recently used plan beyond kMaxPlans sizes).  A plan's chunk holds
// min(T, chunk_px / (H W)) frames of the call that created it, so small calls get small plans.
int get_plan(sml_ctx* ctx, int H, int W, int T) {
  ++ctx->plan_clock;
  const int want = chunk_frames_for(ctx, T, H, W);
  for (size_t k = 0; k < ctx->plans.size(); ++k) {
    Plan& q = *ctx->plans[k];
    if (q.H != H || q.W != W) continue;
    if (q.Tc >= want) {
      q.last_use = ctx->plan_clock;
      ctx->plan = &q;
      return SML_OK;
    }
    // too small for this call: freed after the last call that used it, then re-planned
    if (q.done) SML_CUDA(cudaEventSynchronize(q.done), "plan resize");
    free_plan(q);
    ctx->plans.erase(ctx->plans.begin() + k);
    break;
  }
  if (ctx->plans.size() >= kMaxPlans) {  // evict the least recently used plan
    size_t victim = 0;
    for (size_t k = 1; k < ctx->plans.size(); ++k)
      if (ctx->plans[k]->last_use < ctx->plans[victim]->last_use) victim = k;
    // its buffers may still be in use by the last call that used it, on that call's stream
    Plan& v = *ctx->plans[victim];
    if (v.done) SML_CUDA(cudaEventSynchronize(v.done), "plan eviction");
    free_plan(v);
    ctx->plans.erase(ctx->plans.begin() + victim);
  }
  std::unique_ptr<Plan> np(new Plan());
  Plan& p = *np;
  const PlanSizes z = plan_sizes(ctx, H, W, want);
  const int Tc = z.Tc;
  int r;
  for (int b = 0; b < ctx->nbuf; ++b) {
    if ((r = dev_alloc(ctx, &p.act[b], z.act[b]))) {
      free_plan(p);
      return r;
    }
  }
  if ((r = dev_alloc(ctx, &p.maps, z.maps)) || (r = dev_alloc(ctx, &p.block_counts, z.counts)) ||
      (r = dev_alloc(ctx, &p.block_offsets, z.offsets)) || (r = dev_alloc(ctx, &p.flag_words, z.flags)) ||
      (r = dev_alloc(ctx, &p.frames, z.frames)) || (r = dev_alloc(ctx, &p.cam_maps, z.cam))) {
    free_plan(p);
    return r;
  }
  cudaError_t e = cudaEventCreateWithFlags(&p.done, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    free_plan(p);
    return cuda_fail(ctx, e, "plan event");
  }
  p.bytes = z.total();
  if (ctx->prec != kFP32) {
    for (int l = 1; l < ctx->L; ++l) {
      const LayerDesc& y = ctx->lay[l];
      const int Wl = level_dim(W, y.level);
      p.pair_rows[l] = ctx->prec == kFP8 && Wl % 2 == 0 && ctx->fp8_pair_rows;
      if ((r = encode_act_map(ctx, &p.tmap[l], p.act[y.in_buf], Tc, level_dim(H, y.level), Wl, y.d, y.cin / 16,
                              ctx->buf[y.in_buf].ct / 16, p.pair_rows[l]))) {
        free_plan(p);
        return r;
      }
    }
  }
  p.H = H;
  p.W = W;
  p.Tc = Tc;
  p.last_use = ctx->plan_clock;
  ctx->plan = np.get();
  ctx->plans.push_back(std::move(np));
  return SML_OK;
}

// The frames a chunk's first layer may read: with three-frame context (in_ch = 3) the frames
// just before and after the chunk, where the stack has them.
struct FrameRange {
  int first, last;  // relative to the chunk's first frame
};
// before / after: the frame just before / after the call's T frames exists too (a stack
// processed in batches, whose neighbours are real frames of the stack).
FrameRange chunk_frames(const sml_ctx* ctx, int T, int t0, int tc, bool before = false, bool after = false) {
  if (ctx->in_ch == 1) return {0, tc - 1};
  return {(t0 > 0 || before) ? -1 : 0, (t0 + tc < T || after) ? tc : tc - 1};
}

// One chunk of frames through the network: maps [tc][5][H][W] (+ optional logits).  d_frames
// points at the chunk's first frame; frames fr.first .. fr.last around it are readable.
int forward_chunk(sml_ctx* ctx, const uint16_t* d_frames, int tc, FrameRange fr, int H, int W, const CamArgs& cam,
                  float* maps, float* logits, cudaStream_t s, unsigned* d_amax = nullptr) {
  Plan& p = *ctx->plan;
  const int L = ctx->L, C = ctx->C;
  float l1_scale = ctx->prec == kFP8 ? 1.0f / ctx->act_scale[1] : 1.0f;
  {
    ProfScope ps(ctx, SML_KERNEL_LAYER1, s);
    const int b0 = ctx->lay[0].out_buf;
    SML_CUDA(launch_ingest_l1(d_frames, tc, H, W, ctx->lay[0].d, cam, ctx->w1.data(), ctx->b1.data(), C, ctx->in_ch,
                              fr.first, fr.last, ctx->prec, l1_scale, p.act[b0], ctx->buf[b0].ct, s),
             "layer 1");
  }
  ++ctx->launches;
  // calibration: the maximum of every stored layer output (d_amax[l + 1] for layer l)
  auto amax_of = [&](int l, void* buf) {
    const LayerDesc& y = ctx->lay[l];
    return launch_amax(buf, ctx->prec, tc, level_dim(H, y.level), level_dim(W, y.level), ctx->buf[y.out_buf].ct,
                       y.out_off, y.cout, d_amax + l + 1, s);
  };
  if (d_amax) SML_CUDA(amax_of(0, p.act[ctx->lay[0].out_buf]), "amax");
  for (const Step& st : ctx->steps) {
    if (st.kind != kStepConv) {  // U-Net resolution change
      const BufDesc& bi = ctx->buf[st.in_buf];
      const BufDesc& bo = ctx->buf[st.out_buf];
      ProfScope ps(ctx, SML_KERNEL_CONV, s);
      if (st.kind == kStepPool)
        SML_CUDA(launch_pool2(p.act[st.in_buf], bi.ct, p.act[st.out_buf], bo.ct, st.out_off, st.C, tc,
                              level_dim(H, bi.level), level_dim(W, bi.level), ctx->prec, s),
                 "pool");
      else
        SML_CUDA(launch_upsample2(p.act[st.in_buf], bi.ct, level_dim(H, bi.level), level_dim(W, bi.level),
                                  p.act[st.out_buf], bo.ct, st.out_off, st.C, tc, level_dim(H, bo.level),
                                  level_dim(W, bo.level), ctx->prec, s),
                 "upsample");
      ++ctx->launches;
      continue;
    }
    const int l = st.layer;
    const bool last = (l == L - 1);
    const LayerDesc& y = ctx->lay[l];
    const int Hl = level_dim(H, y.level), Wl = level_dim(W, y.level);
    void* in = p.act[y.in_buf];
    void* out = last ? nullptr : p.act[y.out_buf];
    const int out_ct = last ? C : ctx->buf[y.out_buf].ct;
    ProfScope ps(ctx, last ? SML_KERNEL_CONV_HEADS : SML_KERNEL_CONV, s);
    if (ctx->prec == kFP32) {
      F32LayerArgs fa{};
      fa.in = static_cast<const float*>(in);
      fa.out = static_cast<float*>(out);
      fa.w = ctx->wf32[l];
      fa.b = ctx->bias[l];
      fa.T = tc;
      fa.H = Hl;
      fa.W = Wl;
      fa.d = y.d;
      fa.ci = y.cin;
      fa.co = y.cout;
      fa.in_ct = ctx->buf[y.in_buf].ct;
      fa.out_ct = out_ct;
      fa.out_off = y.out_off;
      if (last)
        SML_CUDA(launch_dconv_f32_heads(fa, ctx->head_w, ctx->head_b, ctx->nh, maps, logits, s), "fp32 conv+heads");
      else
        SML_CUDA(launch_dconv_f32(fa, s), "fp32 conv");
    } else {
      TcLayerArgs a{};
      a.tmap = &p.tmap[l];
      a.stages = ctx->tc_stages;
      a.bimg = ctx->bimg[l];
      a.bias = ctx->h_bias[l].data();
      a.deq = ctx->h_deq[l].empty() ? nullptr : ctx->h_deq[l].data();
      a.out_inv_scale = (ctx->prec == kFP8 && !last) ? 1.0f / ctx->act_scale[l + 1] : 1.0f;
      a.out = out;
      a.out_g0 = y.out_off / 16;
      a.out_gt = out_ct / 16;
      a.head_w = ctx->h_head_w.data();
      a.head_b = ctx->h_head_b.data();
      a.nh = ctx->nh;
      a.maps = maps;
      a.logits = logits;
      a.T = tc;
      a.H = Hl;
      a.W = Wl;
      a.d = y.d;
      a.ci = y.cin;
      a.co = y.cout;
      a.prec = ctx->prec;
      a.err = ctx->d_err;
      a.wait_ns = ctx->debug_wait_ns;
      a.poison_cta = ctx->debug_poison_cta;
      a.pair_rows = p.pair_rows[l] ? 1 : 0;
      SML_CUDA(launch_dconv_tc(a, last, ctx->num_sms, s), "tensor-core conv");
    }
    ++ctx->launches;
    if (d_amax && !last) SML_CUDA(amax_of(l, out), "amax");
  }
  return SML_OK;
}

int check_device_error(sml_ctx* ctx) {
  int h = 0;
  SML_CUDA(cudaMemcpy(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost), "error word");
  if (h) {
    cudaMemset(ctx->d_err, 0, sizeof(int));
    return fail(ctx, SML_ERR_CUDA, "a device-side wait timed out (kernel gave up and returned)");
  }
  return SML_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int check_dims(sml_ctx* ctx, int T, int H, int W) {
  if (T < 0 || H < 1 || W < 1 || H > 16384 || W > 16384) return fail(ctx, SML_ERR_BAD_ARG, "bad frame dims T=%d H=%d W=%d", T, H, W);
  return SML_OK;
}

int check_thr(sml_ctx* ctx, const sml_thresholds* thr) {
  if (!thr || !(thr->p_min >= 0.0f && thr->p_min < 1.0f)) return fail(ctx, SML_ERR_BAD_ARG, "p_min must be in [0,1)");
  return SML_OK;
}

int make_cam(sml_ctx* ctx, const sml_camera* cam, CamArgs* out) {
  if (!cam) return fail(ctx, SML_ERR_BAD_ARG, "camera is NULL");
  if (!cam->gain_map && !(cam->gain > 0.0f)) return fail(ctx, SML_ERR_BAD_ARG, "gain must be > 0");
  out->gain = cam->gain;
  out->offset = cam->offset;
  out->in_scale = ctx->in_scale;
  out->gain_map = cam->gain_map;
  out->offset_map = cam->offset_map;
  return SML_OK;
}

// Whole call on device-resident frames: chunks of whole frames, one running record count.
int localize_device(sml_ctx* ctx, const uint16_t* d_frames, bool frames_on_host, int T, int H, int W, const CamArgs& cam,
                    float p_min, sml_record* d_out, size_t capacity, unsigned long long* d_n, cudaStream_t s,
                    sml_sigma* d_sigma = nullptr, bool before = false, bool after = false) {
  int r = get_plan(ctx, H, W, T);
  if (r) return r;
  Plan& p = *ctx->plan;
  SML_CUDA(cudaMemsetAsync(d_n, 0, sizeof(unsigned long long), s), "memset count");
  const size_t fpx = (size_t)H * W;
  for (int t0 = 0; t0 < T; t0 += p.Tc) {
    int tc = std::min(p.Tc, T - t0);
    const uint16_t* f = d_frames + (size_t)t0 * fpx;
    const FrameRange fr = chunk_frames(ctx, T, t0, tc, before, after);
    if (frames_on_host) {  // the chunk and its context frames, staged into the plan's buffer
      const size_t n = (size_t)(fr.last - fr.first + 1) * fpx;
      SML_CUDA(cudaMemcpyAsync(p.frames, f + (ptrdiff_t)fr.first * (ptrdiff_t)fpx, n * sizeof(uint16_t),
                               cudaMemcpyHostToDevice, s),
               "H2D frames");
      f = p.frames - (ptrdiff_t)fr.first * (ptrdiff_t)fpx;
    }
    if ((r = forward_chunk(ctx, f, tc, fr, H, W, cam, p.maps, nullptr, s))) return r;
    DecodeArgs da{};
    da.maps = p.maps;
    da.T = tc;
    da.H = H;
    da.W = W;
    da.frame0 = t0;
    da.p_min = p_min;
    da.z_scale = ctx->z_scale;
    da.ph_scale = ctx->ph_scale;
    da.out = d_out;
    da.out_sigma = d_sigma;
    da.nh = ctx->nh;
    da.capacity = capacity;
    da.total = d_n;
    da.block_counts = p.block_counts;
    da.block_offsets = p.block_offsets;
    da.flag_words = p.flag_words;
    ProfScope ps(ctx, SML_KERNEL_DECODE, s);
    SML_CUDA(launch_decode(da, s, &ctx->launches), "decode");
  }
  plan_used(ctx, s);
  return SML_OK;
}

int parse_spec(sml_ctx* ctx, const char* spec) {
  JParser jp{spec};
  JVal root = jp.value();
  if (!jp.ok || root.kind != JVal::kObj) return fail(nullptr, SML_ERR_BAD_SPEC, "net spec is not a JSON object");
  auto num = [&](const char* k, double def) {
    auto it = root.obj.find(k);
    return (it != root.obj.end() && it->second.kind == JVal::kNum) ? it->second.num : def;
  };
  ctx->in_ch = (int)num("in_ch", 1);
  ctx->C = (int)num("channels", 0);
  ctx->in_scale = (float)num("in_scale", 1e-3);
  ctx->z_scale = (float)num("z_scale", 1000.0);
  ctx->ph_scale = (float)num("ph_scale", 10000.0);
  ctx->chunk_px = (long long)num("chunk_px", (double)(1 << 24));
  ctx->tc_stages = (int)num("tc_stages", 0);
  ctx->fp8_pair_rows = num("fp8_pair_rows", 1.0) != 0.0;
  ctx->debug_wait_ns = (unsigned long long)num("debug_wait_ns", 0.0);
  ctx->debug_poison_cta = (int)num("debug_poison_cta", -1.0);
  if (ctx->debug_poison_cta >= 0 && (ctx->debug_wait_ns < 1000000ull || ctx->debug_wait_ns > 2000000000ull))
    return fail(nullptr, SML_ERR_BAD_SPEC, "debug_poison_cta needs debug_wait_ns in [1e6, 2e9]");
  if (ctx->tc_stages < 0 || (ctx->tc_stages > 0 && ctx->tc_stages < 4) || ctx->tc_stages > 16)
    return fail(nullptr, SML_ERR_BAD_SPEC, "tc_stages must be 0 (as deep as shared memory allows) or 4..16");

  if (ctx->in_ch != 1 && ctx->in_ch != 3)
    return fail(nullptr, SML_ERR_BAD_SPEC, "in_ch must be 1 (one frame) or 3 (frames t-1, t, t+1)");
  if (ctx->C != 16 && ctx->C != 32 && ctx->C != 48 && ctx->C != 64)
    return fail(nullptr, SML_ERR_BAD_SPEC, "channels must be 16, 32, 48 or 64");
  if (ctx->chunk_px < 1) return fail(nullptr, SML_ERR_BAD_SPEC, "chunk_px must be >= 1");
  auto it = root.obj.find("dilations");
  if (it == root.obj.end() || it->second.kind != JVal::kArr) return fail(nullptr, SML_ERR_BAD_SPEC, "dilations missing");
  auto dil_of = [](const JVal& v, int* out) {
    if (v.kind != JVal::kNum || v.num < 1 || v.num > 64 || v.num != floor(v.num)) return false;
    *out = (int)v.num;
    return true;
  };
  std::vector<int> dil(it->second.arr.size());
  for (size_t l = 0; l < dil.size(); ++l)
    if (!dil_of(it->second.arr[l], &dil[l]))
      return fail(nullptr, SML_ERR_BAD_SPEC, "dilation %d must be an integer in 1..64", (int)l);
  const int C = ctx->C;
  auto dc = root.obj.find("dcd");
  if (dc == root.obj.end() || dc->second.kind == JVal::kNull) {
    // plain stack: layer l reads buffer (l-1) & 1 and writes buffer l & 1
    ctx->L = (int)dil.size();
    if (ctx->L < 2 || ctx->L > kMaxLayers) return fail(nullptr, SML_ERR_BAD_SPEC, "need 2..%d layers", kMaxLayers);
    ctx->ct = C;
    for (int l = 0; l < ctx->L; ++l) {
      LayerDesc& y = ctx->lay[l];
      y.cin = l ? C : ctx->in_ch;
      y.cout = C;
      y.d = dil[l];
      y.in_buf = l ? (l - 1) & 1 : -1;
      y.out_buf = l & 1;
      y.out_off = 0;
    }
  } else {
    // dense blocks (Sec. 3.2.1): stem (dilations[0]); per block, dense layers and a transition
    // back to C channels (d = 1); then the plain layers dilations[1:] (the last feeds the heads)
    const JVal& o = dc->second;
    auto gi = o.obj.find("growth");
    auto bi = o.obj.find("blocks");
    if (o.kind != JVal::kObj || gi == o.obj.end() || gi->second.kind != JVal::kNum || bi == o.obj.end() ||
        bi->second.kind != JVal::kArr || bi->second.arr.empty())
      return fail(nullptr, SML_ERR_BAD_SPEC, "dcd needs growth and a non-empty list of blocks");
    const int g = (int)gi->second.num;
    if (gi->second.num != g || (g != 16 && g != 32 && g != 48 && g != 64))
      return fail(nullptr, SML_ERR_BAD_SPEC, "dcd growth must be 16, 32, 48 or 64");
    if (dil.size() < 2) return fail(nullptr, SML_ERR_BAD_SPEC, "dcd nets need a stem and at least one plain layer");
    ctx->growth = g;
    int L = 0, cur = 0, widest = C;
    auto add = [&](int cin, int cout, int d, int in_buf, int out_buf, int out_off) {
      if (L < kMaxLayers) {
        LayerDesc& y = ctx->lay[L];
        y.cin = cin;
        y.cout = cout;
        y.d = d;
        y.in_buf = in_buf;
        y.out_buf = out_buf;
        y.out_off = out_off;
      }
      ++L;
    };
    add(ctx->in_ch, C, dil[0], -1, 0, 0);
    for (const JVal& blk : bi->second.arr) {
      if (blk.kind != JVal::kArr || blk.arr.empty()) return fail(nullptr, SML_ERR_BAD_SPEC, "dcd blocks must be non-empty lists");
      const int k = (int)blk.arr.size();
      for (int j = 0; j < k; ++j) {
        int d = 0;
        if (!dil_of(blk.arr[j], &d)) return fail(nullptr, SML_ERR_BAD_SPEC, "dcd dilations must be integers in 1..64");
        add(C + j * g, g, d, cur, cur, C + j * g);
      }
      add(C + k * g, C, 1, cur, 1 - cur, 0);
      cur = 1 - cur;
      widest = std::max(widest, C + k * g);
    }
    for (size_t l = 1; l < dil.size(); ++l) {
      add(C, C, dil[l], cur, 1 - cur, 0);
      cur = 1 - cur;
    }
    if (L > kMaxLayers) return fail(nullptr, SML_ERR_BAD_SPEC, "dcd net has %d conv layers (at most %d)", L, kMaxLayers);
    if (widest > kTcMaxCin)
      return fail(nullptr, SML_ERR_BAD_SPEC, "dcd block concatenation has %d channels (at most %d)", widest, kTcMaxCin);
    ctx->L = L;
    ctx->ct = widest;
  }
  // launches after layer 1: one per conv layer, on the full-resolution ping-pong buffers
  ctx->nbuf = 2;
  ctx->buf[0] = ctx->buf[1] = BufDesc{0, ctx->ct};
  ctx->steps.clear();
  for (int l = 1; l < ctx->L; ++l) ctx->steps.push_back(Step{kStepConv, l, 0, 0, 0, 0});
  auto un = root.obj.find("unet");
  if (un != root.obj.end() && un->second.kind != JVal::kNull) {
    // U-Net fine stage (Sec. 3.2) before the last layer: per level down a 2x2 max pool and a
    // 3x3 conv C -> C; per level up a nearest 2x upsample concatenated after the level's skip
    // features and a 3x3 conv 2C -> C
    const JVal& o = un->second;
    auto li = o.obj.find("levels");
    if (o.kind != JVal::kObj || li == o.obj.end() || li->second.kind != JVal::kNum || li->second.num < 1 ||
        li->second.num > kMaxLevels || li->second.num != floor(li->second.num))
      return fail(nullptr, SML_ERR_BAD_SPEC, "unet needs \"levels\": 1..%d", kMaxLevels);
    const int lv = (int)li->second.num;
    if (ctx->L < 2) return fail(nullptr, SML_ERR_BAD_SPEC, "unet needs a conv layer before the last one");
    if (ctx->L - 1 + 2 * lv + 1 > kMaxLayers)
      return fail(nullptr, SML_ERR_BAD_SPEC, "the net has more than %d conv layers", kMaxLayers);
    ctx->unet = lv;
    LayerDesc last = ctx->lay[ctx->L - 1];
    const int cur = last.in_buf;  // holds the features [0, C) the U-Net starts from
    ctx->steps.pop_back();
    int L = ctx->L - 1;
    ctx->ct = std::max(ctx->ct, 2 * C);  // room for the upsampled features after the skip
    ctx->buf[0] = ctx->buf[1] = BufDesc{0, ctx->ct};
    auto A = [](int l) { return 2 + 2 * (l - 1); };  // skip buffer of level l (2C)
    auto B = [](int l) { return 3 + 2 * (l - 1); };  // work buffer of level l (C)
    for (int l = 1; l <= lv; ++l) {
      ctx->buf[A(l)] = BufDesc{l, 2 * C};
      ctx->buf[B(l)] = BufDesc{l, C};
    }
    ctx->nbuf = 2 + 2 * lv;
    auto conv = [&](int cin, int in_buf, int out_buf, int level) {
      LayerDesc& y = ctx->lay[L];
      y = LayerDesc{};
      y.cin = cin;
      y.cout = C;
      y.d = 1;
      y.in_buf = in_buf;
      y.out_buf = out_buf;
      y.out_off = 0;
      y.level = level;
      ctx->steps.push_back(Step{kStepConv, L, 0, 0, 0, 0});
      ++L;
    };
    int src = cur;
    for (int l = 1; l <= lv; ++l) {  // down: pool, then conv into the level's skip buffer
      ctx->steps.push_back(Step{kStepPool, -1, src, B(l), 0, C});
      conv(C, B(l), A(l), l);
      src = A(l);
    }
    int g = A(lv);  // the deepest level's features
    for (int l = lv; l >= 1; --l) {  // up: upsample after the skip of level l-1, then conv
      const int cat = l - 1 == 0 ? cur : A(l - 1);
      ctx->steps.push_back(Step{kStepUp, -1, g, cat, C, C});
      const int out = l - 1 == 0 ? 1 - cur : B(l - 1);
      conv(2 * C, cat, out, l - 1);
      g = out;
    }
    last.in_buf = g;
    ctx->lay[L] = last;
    ctx->steps.push_back(Step{kStepConv, L, 0, 0, 0, 0});
    ctx->L = L + 1;
  }
  auto pr = root.obj.find("precision");
  std::string prec = (pr != root.obj.end() && pr->second.kind == JVal::kStr) ? pr->second.str : "fp32";
  if (prec == "fp32") ctx->prec = kFP32;
  else if (prec == "bf16") ctx->prec = kBF16;
  else if (prec == "fp8") ctx->prec = kFP8;
  else return fail(nullptr, SML_ERR_BAD_SPEC, "precision must be fp32, bf16 or fp8");
  if (ctx->prec == kFP8) {
    auto as = root.obj.find("act_scales");
    if (as == root.obj.end() || as->second.kind != JVal::kArr || (int)as->second.arr.size() != ctx->L)
      return fail(nullptr, SML_ERR_BAD_SPEC, "fp8 needs act_scales with one entry per layer");
    for (int l = 0; l < ctx->L; ++l) {
      const JVal& v = as->second.arr[l];
      if (v.kind != JVal::kNum || !(v.num > 0)) return fail(nullptr, SML_ERR_BAD_SPEC, "act_scales must be > 0");
      ctx->act_scale[l] = (float)v.num;
    }
  }
  for (int l = 1; l < ctx->L; ++l) {  // every layer must fit its kernel's shared memory
    const LayerDesc& y = ctx->lay[l];
    const bool fits = ctx->prec == kFP32 ? y.cin * y.cout <= kF32MaxWeights : tc_layer_fits(y.cin, y.cout, y.d, ctx->prec);
    if (!fits)
      return fail(nullptr, SML_ERR_UNSUPPORTED, "conv layer %d (%d -> %d channels, d = %d) does not fit shared memory", l,
                  y.cin, y.cout, y.d);
  }
  auto hd = root.obj.find("heads");
  if (hd != root.obj.end()) {
    // 5 position heads, or those and the 4 uncertainty heads, in this order
    static const char* kNames[kMaxHeads] = {"p", "dx", "dy", "z", "N", "sx", "sy", "sz", "sN"};
    const JVal& h = hd->second;
    if (h.kind != JVal::kArr || (h.arr.size() != kHeads && h.arr.size() != kMaxHeads))
      return fail(nullptr, SML_ERR_BAD_SPEC, "heads must list 5 outputs (p, dx, dy, z, N) or 9 (and sx, sy, sz, sN)");
    for (size_t k = 0; k < h.arr.size(); ++k)
      if (h.arr[k].kind != JVal::kStr || h.arr[k].str != kNames[k])
        return fail(nullptr, SML_ERR_BAD_SPEC, "head %d must be \"%s\"", (int)k, kNames[k]);
    ctx->nh = (int)h.arr.size();
  }
  return SML_OK;
}

// Weight blob: header "<8s7I16i" (version 1, plain stacks of up to 16 layers) or "<8s7I32i"
// (version 2: nets with dense blocks or a U-Net, reserved = growth, and plain stacks of 17..32
// layers, reserved = 0; dil[32] = every layer's dilation in execution order);
// then per layer W[cout][cin][3][3], b[cout] (+ BatchNorm, version 1 only) and the heads.
// Checks the header against the spec and the size; host only (runs before any device call).
int check_blob(const sml_ctx* ctx, const void* blob, size_t bytes, size_t* hdr_out, int* has_bn_out) {
  const uint8_t* b = static_cast<const uint8_t*>(blob);
  const bool v2 = ctx->growth > 0 || ctx->unet > 0 || ctx->L > 16;  // plain stacks of 17..32 layers: version 2
  const int ndil = v2 ? 32 : 16;
  const size_t hdr_bytes = 8 + 7 * 4 + (size_t)ndil * 4;
  if (!blob || bytes < hdr_bytes || memcmp(b, "SMLW0001", 8) != 0)
    return fail(nullptr, SML_ERR_BAD_WEIGHTS, "weight blob: bad magic or too short");
  uint32_t h[7];
  int32_t dil[32];
  memcpy(h, b + 8, sizeof(h));
  memcpy(dil, b + 8 + sizeof(h), (size_t)ndil * 4);
  const int L = (int)h[1], C = (int)h[2], in_ch = (int)h[3], nh = (int)h[4], has_bn = (int)h[5];
  if (h[0] != (v2 ? 2u : 1u) || L != ctx->L || C != ctx->C || in_ch != ctx->in_ch || nh != ctx->nh ||
      (v2 && ((int)h[6] != ctx->growth || has_bn)))
    return fail(nullptr, SML_ERR_BAD_WEIGHTS, "weight blob header does not match the net spec");
  for (int l = 0; l < L; ++l)
    if (dil[l] != ctx->lay[l].d) return fail(nullptr, SML_ERR_BAD_WEIGHTS, "weight blob dilations do not match the net spec");
  size_t need = hdr_bytes;
  for (int l = 0; l < L; ++l) {
    const LayerDesc& y = ctx->lay[l];
    need += 4 * ((size_t)y.cout * y.cin * 9 + y.cout + (has_bn ? 4 * (size_t)y.cout + 1 : 0));
  }
  need += 4 * ((size_t)ctx->nh * C + ctx->nh);
  if (bytes != need) return fail(nullptr, SML_ERR_BAD_WEIGHTS, "weight blob has %zu bytes, expected %zu", bytes, need);
  if (hdr_out) *hdr_out = hdr_bytes;
  if (has_bn_out) *has_bn_out = has_bn;
  return SML_OK;
}

// The conv layer that produced each input channel of every layer (-1: the frames), from the
// step list: a conv step writes its output channels, a pool or upsample step moves channels
// with their producer.  Layers of dense blocks (Sec. 3.2.1) and of the U-Net (Sec. 3.2) read
// channels of several producers.
std::vector<std::vector<int>> input_producers(const sml_ctx* ctx) {
  std::vector<std::vector<int>> prov(ctx->nbuf), prod(ctx->L);
  for (int b = 0; b < ctx->nbuf; ++b) prov[b].assign(ctx->buf[b].ct, -1);
  prod[0].assign(ctx->lay[0].cin, -1);
  for (int c = 0; c < ctx->lay[0].cout; ++c) prov[ctx->lay[0].out_buf][ctx->lay[0].out_off + c] = 0;
  for (const Step& st : ctx->steps) {
    if (st.kind == kStepConv) {
      const LayerDesc& y = ctx->lay[st.layer];
      prod[st.layer].assign(prov[y.in_buf].begin(), prov[y.in_buf].begin() + y.cin);
      if (st.layer < ctx->L - 1)
        for (int c = 0; c < y.cout; ++c) prov[y.out_buf][y.out_off + c] = st.layer;
    } else {
      for (int c = 0; c < st.C; ++c) prov[st.out_buf][st.out_off + c] = prov[st.in_buf][c];
    }
  }
  return prod;
}

int load_weights(sml_ctx* ctx, const void* blob, size_t bytes) {
  size_t hdr_bytes = 0;
  int has_bn = 0;
  int r = check_blob(ctx, blob, bytes, &hdr_bytes, &has_bn);
  if (r) return r;
  const uint8_t* b = static_cast<const uint8_t*>(blob);
  const int L = ctx->L, C = ctx->C;
  const float* f = reinterpret_cast<const float*>(b + hdr_bytes);  // blob offsets are 4-byte aligned
  std::vector<float> tmp;
  size_t off = 0;
  auto take = [&](size_t n) {
    tmp.assign(n, 0.f);
    memcpy(tmp.data(), reinterpret_cast<const uint8_t*>(f) + off * 4, n * 4);
    off += n;
    return tmp;
  };
  // FP8 nets with dense blocks or a U-Net fold the scale of each input channel into the weights
  const bool fold = ctx->prec == kFP8 && (ctx->growth || ctx->unet);
  const std::vector<std::vector<int>> prod = fold ? input_producers(ctx) : std::vector<std::vector<int>>();
  for (int l = 0; l < L; ++l) {
    const int cin = ctx->lay[l].cin, cout = ctx->lay[l].cout;
    std::vector<float> w = take((size_t)cout * cin * 9);
    std::vector<float> bias = take(cout);
    if (has_bn) {
      std::vector<float> bn = take(4 * (size_t)cout);
      float eps = take(1)[0];
      for (int co = 0; co < cout; ++co) {  // fold: W' = W g/sqrt(v+e); b' = (b-m) g/sqrt(v+e) + beta
        double sc = (double)bn[co] / sqrt((double)bn[3 * cout + co] + (double)eps);
        for (int k = 0; k < cin * 9; ++k) w[(size_t)co * cin * 9 + k] = (float)(w[(size_t)co * cin * 9 + k] * sc);
        bias[co] = (float)(((double)bias[co] - bn[2 * cout + co]) * sc + bn[cout + co]);
      }
    }
    if (!std::all_of(w.begin(), w.end(), [](float x) { return std::isfinite(x); }) ||
        !std::all_of(bias.begin(), bias.end(), [](float x) { return std::isfinite(x); }))
      return fail(nullptr, SML_ERR_BAD_WEIGHTS, "layer %d has non-finite weights", l);
    if (l == 0) {
      ctx->w1 = w;
      ctx->b1 = bias;
      continue;
    }
    // [co][ci][ky][kx] -> [tap][ci][co]
    std::vector<float> t((size_t)9 * cin * cout);
    for (int co = 0; co < cout; ++co)
      for (int ci = 0; ci < cin; ++ci)
        for (int tap = 0; tap < 9; ++tap) t[((size_t)tap * cin + ci) * cout + co] = w[((size_t)co * cin + ci) * 9 + tap];
    if (ctx->prec == kFP32) {
      if ((r = upload(ctx, &ctx->wf32[l], t.data(), t.size() * 4)) || (r = upload(ctx, &ctx->bias[l], bias.data(), cout * 4)))
        return r;
    } else {
      std::vector<float> wscale(cout, 1.0f), deq(cout, 1.0f);
      if (ctx->prec == kFP8 && fold) {
        // input channels of several producers (dense blocks, U-Net): each weight carries the
        // scale of its input channel, w' = w s_in[ci]; the per-output-channel scale is taken
        // over w', and the epilogue's dequantisation is that scale alone
        std::vector<float> s_in(cin);
        for (int ci = 0; ci < cin; ++ci) s_in[ci] = ctx->act_scale[prod[l][ci] + 1];
        for (int tap = 0; tap < 9; ++tap)
          for (int ci = 0; ci < cin; ++ci)
            for (int co = 0; co < cout; ++co) t[((size_t)tap * cin + ci) * cout + co] *= s_in[ci];
        for (int co = 0; co < cout; ++co) {
          float amax = 0.f;
          for (int k = 0; k < 9 * cin; ++k) amax = std::max(amax, fabsf(t[(size_t)k * cout + co]));
          wscale[co] = amax > 0.f ? amax / 448.0f : 1.0f;
          deq[co] = wscale[co];
        }
      } else if (ctx->prec == kFP8) {
        for (int co = 0; co < cout; ++co) {
          float amax = 0.f;
          for (int k = 0; k < 9 * cin; ++k) amax = std::max(amax, fabsf(t[(size_t)k * cout + co]));
          wscale[co] = amax > 0.f ? amax / 448.0f : 1.0f;
          deq[co] = ctx->act_scale[l] * wscale[co];
        }
      }
      std::vector<uint8_t> img(tc_bimg_bytes(cin, cout, ctx->prec));
      tc_pack_bimg(t.data(), cin, cout, ctx->prec, wscale.data(), img.data());
      if ((r = upload(ctx, &ctx->bimg[l], img.data(), img.size()))) return r;
      ctx->h_bias[l] = bias;
      if (ctx->prec == kFP8) ctx->h_deq[l] = deq;
    }
  }
  std::vector<float> hw = take((size_t)ctx->nh * C);
  if ((r = upload(ctx, &ctx->head_w, hw.data(), hw.size() * 4))) return r;
  ctx->h_head_w = hw;
  std::vector<float> hb = take(ctx->nh);
  if ((r = upload(ctx, &ctx->head_b, hb.data(), hb.size() * 4))) return r;
  ctx->h_head_b = hb;
  return SML_OK;
}

}  // namespace

// ------------------------------------------------------------------ entry points
extern "C" {

int sml_create(const char* net_spec, const void* weights, size_t weights_bytes, sml_ctx** out) {
  g_create_error.clear();
  if (!net_spec || !out) return fail(nullptr, SML_ERR_BAD_ARG, "net_spec and out must be non-NULL");
  *out = nullptr;
  std::unique_ptr<sml_ctx> ctx(new sml_ctx());
  int r = parse_spec(ctx.get(), net_spec);
  if (r) return r;
  if ((r = check_blob(ctx.get(), weights, weights_bytes, nullptr, nullptr))) return r;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(nullptr, SML_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
  cudaDeviceProp prop;
  if ((e = cudaGetDeviceProperties(&prop, dev)) != cudaSuccess)
    return fail(nullptr, SML_ERR_CUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
  if (prop.major != 10 || prop.minor != 3)
    return fail(nullptr, SML_ERR_CUDA, "device %d is sm_%d%d; this build targets sm_103a", dev, prop.major, prop.minor);
  ctx->device = dev;
  ctx->num_sms = prop.multiProcessorCount;
  r = load_weights(ctx.get(), weights, weights_bytes);
  if (r) {
    if (g_create_error.empty()) g_create_error = ctx->err;
    for (void* p : ctx->owned) cudaFree(p);
    return r;
  }
  sml_ctx* c = ctx.get();
  if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaMalloc(&c->d_total, sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMalloc(&c->d_err, sizeof(int))) != cudaSuccess || (e = cudaMemset(c->d_err, 0, sizeof(int))) != cudaSuccess) {
    for (void* p : c->owned) cudaFree(p);
    return fail(nullptr, SML_ERR_CUDA, "context set-up: %s", cudaGetErrorString(e));
  }
  *out = ctx.release();
  return SML_OK;
}

void sml_destroy(sml_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto& q : ctx->plans) free_plan(*q);
  ctx->plans.clear();
  for (void* p : ctx->owned) cudaFree(p);
  cudaFree(ctx->d_total);
  cudaFree(ctx->d_err);
  cudaFree(ctx->d_rec);
  cudaFree(ctx->d_sig);
  for (auto& e : ctx->prof_events) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char* sml_last_error(const sml_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

int sml_last_launch_count(const sml_ctx* ctx) { return ctx ? ctx->launches : 0; }

}  // extern "C"

namespace {

// Device staging buffer of at least n elements (grown on demand, kept by the context).
template <typename T>
int staging(sml_ctx* ctx, T** buf, size_t* cap, size_t n) {
  if (*buf && *cap >= n) return SML_OK;
  cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  int r = dev_alloc(ctx, buf, std::max<size_t>(n, 1) * sizeof(T));
  if (r) return r;
  *cap = std::max<size_t>(n, 1);
  return SML_OK;
}

// sml_localize and sml_localize_sigma: out_sigma NULL for records only.
int localize_sync(sml_ctx* ctx, const uint16_t* frames, int T, int H, int W, const sml_camera* cam,
                  const sml_thresholds* thr, sml_record* out, sml_sigma* out_sigma, size_t capacity, size_t* n_out) {
  ctx->launches = 0;
  int r;
  if (!n_out || (T > 0 && !frames) || (capacity > 0 && !out)) return fail(ctx, SML_ERR_BAD_ARG, "NULL argument");
  if ((r = check_dims(ctx, T, H, W)) || (r = check_thr(ctx, thr))) return r;
  CamArgs ca;
  if ((r = make_cam(ctx, cam, &ca))) return r;
  *n_out = 0;
  if (T == 0) return SML_OK;
  SML_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
  if ((r = get_plan(ctx, H, W, T))) return r;
  cudaStream_t s = ctx->stream;
  const size_t hw = (size_t)H * W;
  // camera maps given in host memory are staged once per call
  if (ca.gain_map && !is_device_ptr(ca.gain_map)) {
    SML_CUDA(cudaMemcpyAsync(ctx->plan->cam_maps, ca.gain_map, hw * 4, cudaMemcpyHostToDevice, s), "H2D gain map");
    ca.gain_map = ctx->plan->cam_maps;
  }
  if (ca.offset_map && !is_device_ptr(ca.offset_map)) {
    SML_CUDA(cudaMemcpyAsync(ctx->plan->cam_maps + hw, ca.offset_map, hw * 4, cudaMemcpyHostToDevice, s), "H2D offset map");
    ca.offset_map = ctx->plan->cam_maps + hw;
  }
  const bool out_dev = capacity > 0 && is_device_ptr(out);
  sml_record* d_out = out;
  if (!out_dev) {
    if ((r = staging(ctx, &ctx->d_rec, &ctx->d_rec_cap, capacity))) return r;
    d_out = ctx->d_rec;
  }
  const bool sig_dev = out_sigma && capacity > 0 && is_device_ptr(out_sigma);
  sml_sigma* d_sig = out_sigma;
  if (out_sigma && !sig_dev) {
    if ((r = staging(ctx, &ctx->d_sig, &ctx->d_sig_cap, capacity))) return r;
    d_sig = ctx->d_sig;
  }
  const bool host_frames = !is_device_ptr(frames);
  if ((r = localize_device(ctx, frames, host_frames, T, H, W, ca, thr->p_min, d_out, capacity, ctx->d_total, s, d_sig)))
    return r;
  unsigned long long total = 0;
  SML_CUDA(cudaMemcpyAsync(&total, ctx->d_total, sizeof(total), cudaMemcpyDeviceToHost, s), "D2H count");
  SML_CUDA(cudaStreamSynchronize(s), "localize");
  if ((r = check_device_error(ctx))) return r;
  *n_out = (size_t)total;
  if (total > capacity) return fail(ctx, SML_ERR_CAPACITY, "%llu detections exceed capacity %zu", total, capacity);
  if (!out_dev && total > 0)
    SML_CUDA(cudaMemcpyAsync(out, d_out, (size_t)total * sizeof(sml_record), cudaMemcpyDeviceToHost, s), "D2H records");
  if (out_sigma && !sig_dev && total > 0)
    SML_CUDA(cudaMemcpyAsync(out_sigma, d_sig, (size_t)total * sizeof(sml_sigma), cudaMemcpyDeviceToHost, s),
             "D2H uncertainties");
  SML_CUDA(cudaStreamSynchronize(s), "D2H records");
  return SML_OK;
}

}  // namespace

extern "C" {

int sml_localize(sml_ctx* ctx, const uint16_t* frames, int T, int H, int W, const sml_camera* cam,
                 const sml_thresholds* thr, sml_record* out, size_t capacity, size_t* n_out) {
  if (!ctx) return SML_ERR_BAD_ARG;
  return localize_sync(ctx, frames, T, H, W, cam, thr, out, nullptr, capacity, n_out);
}

int sml_num_heads(const sml_ctx* ctx) { return ctx ? ctx->nh : 0; }

int sml_num_layers(const sml_ctx* ctx) { return ctx ? ctx->L : 0; }

int sml_workspace_bytes(const sml_ctx* ctx, int T, int H, int W, size_t* plan_bytes, int* plan_resident,
                        size_t* resident_bytes) {
  if (!ctx || T < 1 || H < 1 || W < 1 || H > 16384 || W > 16384) return SML_ERR_BAD_ARG;
  const int want = chunk_frames_for(ctx, T, H, W);
  if (plan_bytes) *plan_bytes = plan_sizes(ctx, H, W, want).total();
  int res = 0;
  size_t tot = 0;
  for (const auto& q : ctx->plans) {
    tot += q->bytes;
    if (q->H == H && q->W == W && q->Tc >= want) res = 1;
  }
  if (plan_resident) *plan_resident = res;
  if (resident_bytes) *resident_bytes = tot;
  return SML_OK;
}

int sml_error_word(sml_ctx* ctx, int* d_word, void* stream) {
  if (!ctx || !d_word) return SML_ERR_BAD_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SML_CUDA(cudaMemcpyAsync(d_word, ctx->d_err, sizeof(int), cudaMemcpyDeviceToDevice, s), "error word");
  SML_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), s), "clear error word");
  return SML_OK;
}

int sml_localize_sigma(sml_ctx* ctx, const uint16_t* frames, int T, int H, int W, const sml_camera* cam,
                       const sml_thresholds* thr, sml_record* out, sml_sigma* out_sigma, size_t capacity,
                       size_t* n_out) {
  if (!ctx) return SML_ERR_BAD_ARG;
  if (ctx->nh != kMaxHeads) return fail(ctx, SML_ERR_UNSUPPORTED, "the net has no uncertainty heads");
  if (capacity > 0 && !out_sigma) return fail(ctx, SML_ERR_BAD_ARG, "NULL argument");
  return localize_sync(ctx, frames, T, H, W, cam, thr, out, out_sigma, capacity, n_out);
}

int sml_localize_async(sml_ctx* ctx, const uint16_t* d_frames, int T, int H, int W, const sml_camera* cam,
                       const sml_thresholds* thr, sml_record* d_out, size_t capacity, unsigned long long* d_n_out,
                       void* stream) {
  if (!ctx) return SML_ERR_BAD_ARG;
  ctx->launches = 0;
  int r;
  if (!d_n_out || (T > 0 && !d_frames) || (capacity > 0 && !d_out)) return fail(ctx, SML_ERR_BAD_ARG, "NULL argument");
  if ((r = check_dims(ctx, T, H, W)) || (r = check_thr(ctx, thr))) return r;
  CamArgs ca;
  if ((r = make_cam(ctx, cam, &ca))) return r;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (T == 0) {
    SML_CUDA(cudaMemsetAsync(d_n_out, 0, sizeof(unsigned long long), s), "memset count");
    return SML_OK;
  }
  return localize_device(ctx, d_frames, false, T, H, W, ca, thr->p_min, d_out, capacity, d_n_out, s);
}

int sml_forward_maps(sml_ctx* ctx, const uint16_t* d_frames, int T, int H, int W, const sml_camera* cam, float* d_maps,
                     float* d_logits, void* stream) {
  if (!ctx) return SML_ERR_BAD_ARG;
  ctx->launches = 0;
  int r;
  if ((T > 0 && (!d_frames || !d_maps))) return fail(ctx, SML_ERR_BAD_ARG, "NULL argument");
  if ((r = check_dims(ctx, T, H, W))) return r;
  CamArgs ca;
  if ((r = make_cam(ctx, cam, &ca))) return r;
  if (T == 0) return SML_OK;
  if ((r = get_plan(ctx, H, W, T))) return r;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t fpx = (size_t)H * W;
  for (int t0 = 0; t0 < T; t0 += ctx->plan->Tc) {
    int tc = std::min(ctx->plan->Tc, T - t0);
    if ((r = forward_chunk(ctx, d_frames + (size_t)t0 * fpx, tc, chunk_frames(ctx, T, t0, tc), H, W, ca,
                           d_maps + (size_t)t0 * ctx->nh * fpx, d_logits ? d_logits + (size_t)t0 * fpx : nullptr, s)))
      return r;
  }
  plan_used(ctx, s);
  return SML_OK;
}

int sml_decode_maps(sml_ctx* ctx, const float* d_maps, int T, int H, int W, const sml_thresholds* thr, sml_record* d_out,
                    size_t capacity, unsigned long long* d_n_out, void* stream) {
  if (!ctx) return SML_ERR_BAD_ARG;
  ctx->launches = 0;
  int r;
  if (!d_n_out || (T > 0 && !d_maps) || (capacity > 0 && !d_out)) return fail(ctx, SML_ERR_BAD_ARG, "NULL argument");
  if ((r = check_dims(ctx, T, H, W)) || (r = check_thr(ctx, thr))) return r;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SML_CUDA(cudaMemsetAsync(d_n_out, 0, sizeof(unsigned long long), s), "memset count");
  if (T == 0) return SML_OK;
  if ((r = get_plan(ctx, H, W, T))) return r;
  Plan& p = *ctx->plan;
  const size_t fpx = (size_t)H * W;
  for (int t0 = 0; t0 < T; t0 += p.Tc) {
    int tc = std::min(p.Tc, T - t0);
    DecodeArgs da{};
    da.maps = d_maps + (size_t)t0 * ctx->nh * fpx;
    da.nh = ctx->nh;
    da.T = tc;
    da.H = H;
    da.W = W;
    da.frame0 = t0;
    da.p_min = thr->p_min;
    da.z_scale = ctx->z_scale;
    da.ph_scale = ctx->ph_scale;
    da.out = d_out;
    da.capacity = capacity;
    da.total = d_n_out;
    da.block_counts = p.block_counts;
    da.block_offsets = p.block_offsets;
    da.flag_words = p.flag_words;
    ProfScope ps(ctx, SML_KERNEL_DECODE, s);
    SML_CUDA(launch_decode(da, s, &ctx->launches), "decode");
  }
  plan_used(ctx, s);
  return SML_OK;
}

int sml_profile_enable(sml_ctx* ctx, int on) {
  if (!ctx) return SML_ERR_BAD_ARG;
  if (on) {
    for (size_t k = 0; k < ctx->prof_used; ++k) cudaEventSynchronize(ctx->prof_events[k].b);
    ctx->prof_used = 0;
  }
  ctx->prof_on = on != 0;
  return SML_OK;
}

int sml_profile_read(sml_ctx* ctx, int kernel_class, double* total_ms, int* launches) {
  if (!ctx || !total_ms || !launches) return SML_ERR_BAD_ARG;
  double sum = 0.0;
  int n = 0;
  for (size_t k = 0; k < ctx->prof_used; ++k) {
    sml_ctx::ProfEv& e = ctx->prof_events[k];
    if (e.cls != kernel_class) continue;
    float ms = 0.f;
    SML_CUDA(cudaEventSynchronize(e.b), "profile sync");
    SML_CUDA(cudaEventElapsedTime(&ms, e.a, e.b), "profile elapsed");
    sum += ms;
    ++n;
  }
  *total_ms = sum;
  *launches = n;
  return SML_OK;
}

int sml_activation_amax(sml_ctx* ctx, const uint16_t* d_frames, int T, int H, int W, const sml_camera* cam,
                        float* amax) {
  if (!ctx) return SML_ERR_BAD_ARG;
  ctx->launches = 0;
  int r;
  if (!amax || (T > 0 && !d_frames)) return fail(ctx, SML_ERR_BAD_ARG, "NULL argument");
  if (ctx->prec == kFP8) return fail(ctx, SML_ERR_UNSUPPORTED, "activation maxima need an fp32 or bf16 context");
  if ((r = check_dims(ctx, T, H, W))) return r;
  CamArgs ca;
  if ((r = make_cam(ctx, cam, &ca))) return r;
  for (int l = 0; l < ctx->L; ++l) amax[l] = 0.0f;
  if (T == 0) return SML_OK;
  if ((r = get_plan(ctx, H, W, T))) return r;
  cudaStream_t s = ctx->stream;
  unsigned* d_amax = nullptr;
  if ((r = dev_alloc(ctx, &d_amax, kMaxLayers * sizeof(unsigned)))) return r;
  std::unique_ptr<unsigned, decltype(&cudaFree)> guard(d_amax, &cudaFree);
  SML_CUDA(cudaMemsetAsync(d_amax, 0, kMaxLayers * sizeof(unsigned), s), "memset amax");
  const size_t fpx = (size_t)H * W;
  for (int t0 = 0; t0 < T; t0 += ctx->plan->Tc) {
    int tc = std::min(ctx->plan->Tc, T - t0);
    if ((r = forward_chunk(ctx, d_frames + (size_t)t0 * fpx, tc, chunk_frames(ctx, T, t0, tc), H, W, ca, ctx->plan->maps,
                           nullptr, s, d_amax)))
      return r;
  }
  plan_used(ctx, s);
  unsigned h[kMaxLayers];
  SML_CUDA(cudaMemcpyAsync(h, d_amax, sizeof(h), cudaMemcpyDeviceToHost, s), "D2H amax");
  SML_CUDA(cudaStreamSynchronize(s), "amax");
  for (int l = 1; l < ctx->L; ++l) memcpy(&amax[l], &h[l], sizeof(float));
  return check_device_error(ctx);
}

int sml_calibrate_fp8(sml_ctx* ctx, const uint16_t* d_frames, int T, int H, int W, const sml_camera* cam, float margin,
                      float* act_scales) {
  if (!ctx) return SML_ERR_BAD_ARG;
  if (!act_scales || !(margin > 0.0f) || !std::isfinite(margin)) return fail(ctx, SML_ERR_BAD_ARG, "bad argument");
  if (T < 1) return fail(ctx, SML_ERR_BAD_ARG, "calibration needs at least one frame");
  float amax[kMaxLayers] = {0};
  int r = sml_activation_amax(ctx, d_frames, T, H, W, cam, amax);
  if (r) return r;
  // e4m3 holds magnitudes up to 448: scale = margin * amax / 448, with amax floored at 1e-6
  // (a layer input that is zero on every calibration frame keeps a usable scale)
  act_scales[0] = 1.0f;  // layer 0 reads the frames, not stored activations
  for (int l = 1; l < ctx->L; ++l) act_scales[l] = std::max(amax[l], 1e-6f) * margin / 448.0f;
  return SML_OK;
}

// ------------------------------------------------------------------ training (sml_train.h)
static int train_status(cudaError_t e) { return e == cudaSuccess ? SML_OK : (e == cudaErrorInvalidValue ? SML_ERR_BAD_ARG : SML_ERR_CUDA); }

int sml_train_ingest(const uint16_t* frames, long long n, float gain, float offset, float in_scale, float* x0,
                     void* stream) {
  if (n < 0 || (n > 0 && (!frames || !x0)) || !(gain > 0.0f)) return SML_ERR_BAD_ARG;
  return train_status(train_ingest(frames, n, gain, offset, in_scale, x0, static_cast<cudaStream_t>(stream)));
}

int sml_train_conv_fwd(const float* x, int B, int H, int W, int cin, int cout, int d, const float* w, const float* b,
                       float* y, void* stream) {
  if (B < 0 || H < 1 || W < 1 || d < 1 || !x || !w || !b || !y) return SML_ERR_BAD_ARG;
  return train_status(train_conv_fwd(x, B, H, W, cin, cout, d, w, b, y, static_cast<cudaStream_t>(stream)));
}

size_t sml_train_conv_bwd_work_bytes(int B, int H, int W, int cin, int cout) {
  return train_conv_work_bytes(B, H, W, cin, cout);
}

int sml_train_conv_bwd(const float* x, const float* y, const float* dy, int B, int H, int W, int cin, int cout, int d,
                       const float* w, float* dx, float* dw, float* db, void* work, size_t work_bytes, void* stream) {
  if (B < 0 || H < 1 || W < 1 || d < 1 || !x || !y || !dy || !w || !dw || !db || !work) return SML_ERR_BAD_ARG;
  if (work_bytes < train_conv_work_bytes(B, H, W, cin, cout)) return SML_ERR_BAD_ARG;
  return train_status(train_conv_bwd(x, y, dy, B, H, W, cin, cout, d, w, dx, dw, db, work,
                                     static_cast<cudaStream_t>(stream)));
}

size_t sml_train_heads_work_bytes(int B, int H, int W, int C) { return train_heads_work_bytes(B, H, W, C); }

int sml_train_heads_loss(const float* a, const float* tgt, int B, int H, int W, int C, const float* hw,
                         const float* hb, float* h, float* loss, const float* grad_scale, float* da, float* dhw,
                         float* dhb, void* work, size_t work_bytes, void* stream) {
  if (B < 1 || H < 1 || W < 1 || !a || !tgt || !hw || !hb || !h || !loss || !work) return SML_ERR_BAD_ARG;
  if (da && (!grad_scale || !dhw || !dhb)) return SML_ERR_BAD_ARG;
  if (!aligned16(a) || (da && !aligned16(da))) return SML_ERR_BAD_ARG;
  if (work_bytes < train_heads_work_bytes(B, H, W, C)) return SML_ERR_BAD_ARG;
  return train_status(train_heads_loss(a, tgt, B, H, W, C, hw, hb, h, loss, da ? grad_scale : nullptr, da, dhw, dhb,
                                       work, static_cast<cudaStream_t>(stream)));
}

// ------------------------------------------------------------------ BF16 training (sml_train.h)
}  // extern "C"

namespace {

// SMs of the current device (cached per device).
int current_num_sms() {
  static int sms[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (!sms[dev]) cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
  return sms[dev];
}

// TMA map over row-planar bf16 activations [B][H][C/16][W][16] with one box per image row:
// `box_px` pixels (128 + 2d rounded up to 32 for the conv's input rows; the weight
// gradient's strip and halo widths from wgrad_tc_boxes) by all C/16 groups; 32-byte swizzle;
// zero fill out of bounds.
bool encode_rp_map(CUtensorMap* m, const void* base, int B, int H, int W, int C, int box_px) {
  PFN_encodeTiled_t enc = get_encoder();
  if (!enc) return false;
  const int G = C / 16;
  cuuint64_t dims[5] = {16ull, (cuuint64_t)W, (cuuint64_t)G, (cuuint64_t)H, (cuuint64_t)B};
  cuuint64_t strides[4] = {32ull, 32ull * W, 32ull * W * G, 32ull * W * G * H};
  cuuint32_t box[5] = {16u, (cuuint32_t)box_px, (cuuint32_t)G, 1u, 1u};
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool train_bf16_dims_ok(int B, int H, int W, int C, int d) {
  return B >= 0 && H >= 1 && W >= 1 && H <= 16384 && W <= 16384 && d >= 1 && d <= 64 &&
         (C == 16 || C == 32 || C == 48) && (long long)B * H * W < (1LL << 31);
}

// The plain-layer conv of BF16 training: forward (bias from b_dev) or input gradient.
int train_bf16_conv(const void* in, const void* mask, int B, int H, int W, int C, int d, const void* bimg,
                    const float* b_dev, void* out, int* d_err, bool dgrad, void* stream) {
  if (!in || !bimg || !out || !d_err || (dgrad ? !mask : !b_dev) || !train_bf16_dims_ok(B, H, W, C, d))
    return SML_ERR_BAD_ARG;
  if (B == 0) return SML_OK;
  CUtensorMap tm;
  if (!encode_rp_map(&tm, in, B, H, W, C, tc_box_width(d))) return SML_ERR_CUDA;
  TcLayerArgs a{};
  a.tmap = &tm;
  a.stages = 0;
  a.bimg = bimg;
  a.bias = nullptr;
  a.bias_dev = dgrad ? nullptr : b_dev;
  a.mask = mask;
  a.out_inv_scale = 1.0f;
  a.out = out;
  a.out_g0 = 0;
  a.out_gt = C / 16;
  a.T = B;
  a.H = H;
  a.W = W;
  a.d = d;
  a.prec = kBF16;
  a.ci = a.co = C;
  a.err = d_err;
  return train_status(launch_dconv_tc_train(a, dgrad, current_num_sms(), static_cast<cudaStream_t>(stream)));
}

}  // namespace

extern "C" {

size_t sml_train_bf16_bimg_bytes(int C) { return (C == 16 || C == 32 || C == 48) ? tc_bimg_bytes(C, C, kBF16) : 0; }

int sml_train_bf16_pack(const float* w, int C, void* bimg_fwd, void* bimg_dgrad, void* stream) {
  if (!w || !bimg_fwd || !bimg_dgrad || (C != 16 && C != 32 && C != 48)) return SML_ERR_BAD_ARG;
  return train_status(launch_pack_bimg_bf16(w, C, C, bimg_fwd, bimg_dgrad, static_cast<cudaStream_t>(stream)));
}

int sml_train_bf16_layer0(const uint16_t* frames, int B, int H, int W, float gain, float offset, float in_scale,
                          const float* w0, const float* b0, int C, int d, void* a0, void* stream) {
  if (!frames || !w0 || !b0 || !a0 || !(gain > 0.0f) || !train_bf16_dims_ok(B, H, W, C, d)) return SML_ERR_BAD_ARG;
  if (B == 0) return SML_OK;
  CamArgs cam{gain, offset, in_scale, nullptr, nullptr};
  return train_status(launch_ingest_l1_devw(frames, B, H, W, d, cam, w0, b0, C, a0, static_cast<cudaStream_t>(stream)));
}

int sml_train_bf16_conv_fwd(const void* x, int B, int H, int W, int C, int d, const void* bimg_fwd, const float* b,
                            void* y, int* d_err, void* stream) {
  return train_bf16_conv(x, nullptr, B, H, W, C, d, bimg_fwd, b, y, d_err, false, stream);
}

int sml_train_bf16_conv_dgrad(const void* dz, const void* x, int B, int H, int W, int C, int d, const void* bimg_dgrad,
                              void* dz_in, int* d_err, void* stream) {
  return train_bf16_conv(dz, x, B, H, W, C, d, bimg_dgrad, nullptr, dz_in, d_err, true, stream);
}

size_t sml_train_bf16_wgrad_work_bytes(int C) {
  const int sms = current_num_sms();
  return (C == 16 || C == 32 || C == 48) && sms > 0 ? train_wgrad_tc_work_bytes(C, sms) : 0;
}

int sml_train_bf16_conv_wgrad(const void* x, const void* dz, int B, int H, int W, int C, int d, float* dw, float* db,
                              void* work, size_t work_bytes, int* d_err, void* stream) {
  if (!x || !dz || !dw || !db || !work || !d_err || !train_bf16_dims_ok(B, H, W, C, d)) return SML_ERR_BAD_ARG;
  const int sms = current_num_sms();
  if (sms <= 0) return SML_ERR_CUDA;
  if (work_bytes < train_wgrad_tc_work_bytes(C, sms)) return SML_ERR_BAD_ARG;
  CUtensorMap tm_dz, tm_x;
  int dz_px = 0, x_px = 0;
  wgrad_tc_boxes(W, d, &dz_px, &x_px);
  if (!encode_rp_map(&tm_dz, dz, B > 0 ? B : 1, H, W, C, dz_px) ||
      !encode_rp_map(&tm_x, x, B > 0 ? B : 1, H, W, C, x_px))
    return SML_ERR_CUDA;
  return train_status(launch_wgrad_tc(&tm_dz, &tm_x, B, H, W, C, d, static_cast<float*>(work), sms, dw, db, d_err,
                                      static_cast<cudaStream_t>(stream)));
}

int sml_train_bf16_heads_loss(const void* a, const float* tgt, int B, int H, int W, int C, const float* hw,
                              const float* hb, float* h, float* loss, const float* grad_scale, void* dz, float* dhw,
                              float* dhb, void* work, size_t work_bytes, void* stream) {
  if (B < 1 || H < 1 || W < 1 || !a || !tgt || !hw || !hb || !h || !loss || !work) return SML_ERR_BAD_ARG;
  if (C != 16 && C != 32 && C != 48 && C != 64) return SML_ERR_BAD_ARG;
  if (dz && (!grad_scale || !dhw || !dhb)) return SML_ERR_BAD_ARG;
  if (!aligned16(a) || (dz && !aligned16(dz))) return SML_ERR_BAD_ARG;
  if (work_bytes < train_heads_work_bytes(B, H, W, C)) return SML_ERR_BAD_ARG;
  return train_status(train_heads_loss_rp(a, tgt, B, H, W, C, hw, hb, h, loss, dz ? grad_scale : nullptr, dz, dhw, dhb,
                                          work, static_cast<cudaStream_t>(stream)));
}

int sml_train_bf16_l0_wgrad(const float* x0, const void* dz0, int B, int H, int W, int C, int d, float* dw, float* db,
                            void* work, size_t work_bytes, void* stream) {
  if (!x0 || !dz0 || !dw || !db || !work || !train_bf16_dims_ok(B, H, W, C, d) || !aligned16(dz0)) return SML_ERR_BAD_ARG;
  if (work_bytes < train_conv_work_bytes(B, H, W, 1, C)) return SML_ERR_BAD_ARG;
  return train_status(train_l0_wgrad_rp(x0, dz0, B, H, W, C, d, dw, db, work, static_cast<cudaStream_t>(stream)));
}

// Debug entry (include/sml_debug.h): one UMMA with both operands MN-major.
int sml_debug_umma_mn(const void* d_a, const void* d_b, float* d_d, int m, int n, int k, int a_bytes, int b_bytes,
                      int a_plane, int b_plane, int b_shift, void* stream) {
  static int* d_err = nullptr;
  if (!d_a || !d_b || !d_d) return SML_ERR_BAD_ARG;
  if (!d_err && cudaMalloc(&d_err, sizeof(int)) != cudaSuccess) return SML_ERR_OOM;
  cudaMemset(d_err, 0, sizeof(int));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = launch_umma_mn_selftest(d_a, d_b, d_d, m, n, k, a_bytes, b_bytes, a_plane, b_plane, b_shift, d_err, s);
  if (e == cudaErrorInvalidValue) return SML_ERR_BAD_ARG;
  if (e != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return SML_ERR_CUDA;
  int h = 0;
  cudaMemcpy(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost);
  return h ? SML_ERR_CUDA : SML_OK;
}

// Debug entry (include/sml_debug.h): host-side injection of a device-side failure report.
int sml_debug_set_error_word(sml_ctx* ctx, int value) {
  if (!ctx) return SML_ERR_BAD_ARG;
  SML_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
  SML_CUDA(cudaMemcpy(ctx->d_err, &value, sizeof(int), cudaMemcpyHostToDevice), "set error word");
  return SML_OK;
}

// Debug entry (include/sml_debug.h): one UMMA tile through the conv kernel's descriptor helpers.
int sml_debug_umma(const void* d_a, const void* d_b, float* d_d, int n, int k, int kind, int d_col, void* stream) {
  static int* d_err = nullptr;
  if (!d_err && cudaMalloc(&d_err, sizeof(int)) != cudaSuccess) return SML_ERR_OOM;
  cudaMemset(d_err, 0, sizeof(int));
  if (n % 16 || n < 16 || n > 256 || k % 32 || k < 32 || d_col < 0 || d_col % 16 || d_col + n > 512) return SML_ERR_BAD_ARG;
  if (kind < 0 || kind > 2) return SML_ERR_BAD_ARG;
  cudaError_t e = launch_umma_selftest(d_a, d_b, d_d, n, k, kind == 1 ? kFP8 : (kind == 2 ? kTF32 : kBF16), d_col, d_err,
                                       static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return SML_ERR_CUDA;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return SML_ERR_CUDA;
  int h = 0;
  cudaMemcpy(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost);
  return h ? SML_ERR_CUDA : SML_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------- stack files

namespace {

// Device-side resources of one sml_localize_file call, released on every exit path.
struct FilePipe {
  sml_reader* reader = nullptr;
  cudaStream_t copy = nullptr;
  cudaEvent_t h2d[2] = {nullptr, nullptr}, cnt[2] = {nullptr, nullptr}, d2h[2] = {nullptr, nullptr},
              comp[2] = {nullptr, nullptr};
  uint8_t* dev = nullptr;                 // frames[2] | records[2] | counts[2]
  unsigned long long* h_cnt = nullptr;    // pinned, 2 counts
  ~FilePipe() {
    if (copy) cudaStreamSynchronize(copy);
    for (int k = 0; k < 2; ++k) {
      if (h2d[k]) cudaEventDestroy(h2d[k]);
      if (cnt[k]) cudaEventDestroy(cnt[k]);
      if (d2h[k]) cudaEventDestroy(d2h[k]);
      if (comp[k]) cudaEventDestroy(comp[k]);
    }
    if (copy) cudaStreamDestroy(copy);
    if (dev) cudaFree(dev);
    if (h_cnt) cudaFreeHost(h_cnt);
    if (reader) sml_reader_close(reader);
  }
};

}  // namespace

extern "C" int sml_localize_file(sml_ctx* ctx, const char* path, long long offset, int T, int H, int W,
                                 const sml_camera* cam, const sml_thresholds* thr, int batch, sml_record* out,
                                 size_t capacity, size_t* n_out, sml_io_stats* stats) {
  if (!ctx) return SML_ERR_BAD_ARG;
  ctx->launches = 0;
  int r;
  if (!path || !n_out || (capacity > 0 && !out) || batch < 1 || offset < 0) return fail(ctx, SML_ERR_BAD_ARG, "bad argument");
  if ((r = check_dims(ctx, T, H, W)) || (r = check_thr(ctx, thr))) return r;
  CamArgs ca;
  if ((r = make_cam(ctx, cam, &ca))) return r;
  *n_out = 0;
  if (stats) memset(stats, 0, sizeof(*stats));
  if (T == 0) return SML_OK;
  const auto t_start = std::chrono::steady_clock::now();
  SML_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
  if ((r = get_plan(ctx, H, W, std::min(T, batch)))) return r;
  cudaStream_t s = ctx->stream;
  const size_t hw = (size_t)H * W;
  if (ca.gain_map && !is_device_ptr(ca.gain_map)) {
    SML_CUDA(cudaMemcpyAsync(ctx->plan->cam_maps, ca.gain_map, hw * 4, cudaMemcpyHostToDevice, s), "H2D gain map");
    ca.gain_map = ctx->plan->cam_maps;
  }
  if (ca.offset_map && !is_device_ptr(ca.offset_map)) {
    SML_CUDA(cudaMemcpyAsync(ctx->plan->cam_maps + hw, ca.offset_map, hw * 4, cudaMemcpyHostToDevice, s), "H2D offset map");
    ca.offset_map = ctx->plan->cam_maps + hw;
  }
  // Three-frame nets (in_ch = 3) need the frame before and after each batch.  Each frame slot
  // then holds [previous batch's last frame | the batch | next batch's first frame], the two
  // context frames copied on the device from the neighbouring slot, and a batch is localized
  // one batch later, once its successor has arrived.
  const bool ctx3 = ctx->in_ch == 3;
  const int ext = ctx3 ? 2 : 0;  // context frames per slot
  FilePipe fp;
  const size_t frame_bytes = (size_t)(batch + ext) * hw * sizeof(uint16_t);
  // a detection is a strict local maximum: at most one per 2x2 block of a frame
  const size_t rec_cap = (size_t)batch * ((H + 1) / 2) * ((W + 1) / 2);
  const size_t rec_bytes = rec_cap * sizeof(sml_record);
  if ((r = dev_alloc(ctx, &fp.dev, 2 * frame_bytes + 2 * rec_bytes + 2 * sizeof(unsigned long long)))) return r;
  uint16_t* d_frames[2] = {reinterpret_cast<uint16_t*>(fp.dev), reinterpret_cast<uint16_t*>(fp.dev + frame_bytes)};
  sml_record* d_rec[2] = {reinterpret_cast<sml_record*>(fp.dev + 2 * frame_bytes),
                          reinterpret_cast<sml_record*>(fp.dev + 2 * frame_bytes + rec_bytes)};
  unsigned long long* d_n = reinterpret_cast<unsigned long long*>(fp.dev + 2 * frame_bytes + 2 * rec_bytes);
  SML_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&fp.h_cnt), 2 * sizeof(unsigned long long), cudaHostAllocDefault),
           "pinned counts");
  SML_CUDA(cudaStreamCreateWithFlags(&fp.copy, cudaStreamNonBlocking), "copy stream");
  for (int k = 0; k < 2; ++k) {
    SML_CUDA(cudaEventCreateWithFlags(&fp.h2d[k], cudaEventDisableTiming), "event");
    SML_CUDA(cudaEventCreateWithFlags(&fp.cnt[k], cudaEventDisableTiming), "event");
    SML_CUDA(cudaEventCreateWithFlags(&fp.d2h[k], cudaEventDisableTiming), "event");
    SML_CUDA(cudaEventCreateWithFlags(&fp.comp[k], cudaEventDisableTiming), "event");
  }
  // one batch more in flight when batches wait for their successor
  if ((r = sml_reader_open(path, offset, T, H, W, batch, ctx3 ? 4 : 3, &fp.reader)))
    return fail(ctx, r, "cannot read %d frames of %dx%d from %s at offset %lld", T, H, W, path, offset);

  struct Done {
    long long first;
    size_t at, n;
  };
  std::vector<Done> done;
  size_t total = 0, written = 0;
  struct Batch {
    int slot = -1, nf = 0;
    long long k = 0, first = 0;
    const uint16_t* host = nullptr;
  };
  Batch wait_comp, wait_fin;  // read but not yet localized (three-frame nets); localized, records pending
  // records of a finished batch: count (host waits for its compute), then an async D2H on
  // the copy stream, which overlaps the next batch's compute
  auto finish = [&](const Batch& p) -> int {
    SML_CUDA(cudaEventSynchronize(fp.cnt[p.slot]), "batch count");
    int rr = sml_reader_release(fp.reader, p.host);  // its H2D finished before its compute
    if (rr) return fail(ctx, rr, "reader release");
    const size_t n = (size_t)fp.h_cnt[p.slot];
    const size_t m = written < capacity ? std::min(n, capacity - written) : 0;
    if (m) SML_CUDA(cudaMemcpyAsync(out + written, d_rec[p.slot], m * sizeof(sml_record), cudaMemcpyDeviceToHost, fp.copy),
                    "D2H records");
    SML_CUDA(cudaEventRecord(fp.d2h[p.slot], fp.copy), "event");
    done.push_back({p.first, written, m});
    written += m;
    total += n;
    return SML_OK;
  };
  // localize a batch whose frames (and context frames) are on the device; `after`: the
  // frame after the batch is in its slot
  auto compute = [&](const Batch& b, bool after) -> int {
    SML_CUDA(cudaStreamWaitEvent(s, fp.h2d[b.slot], 0), "wait H2D");
    if (b.k >= 2) SML_CUDA(cudaStreamWaitEvent(s, fp.d2h[b.slot], 0), "wait D2H");
    const uint16_t* f = d_frames[b.slot] + (ctx3 ? hw : 0);
    int rr = localize_device(ctx, f, false, b.nf, H, W, ca, thr->p_min, d_rec[b.slot], rec_cap, d_n + b.slot, s, nullptr,
                             ctx3 && b.first > 0, after);
    if (rr) return rr;
    SML_CUDA(cudaMemcpyAsync(fp.h_cnt + b.slot, d_n + b.slot, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s),
             "D2H count");
    SML_CUDA(cudaEventRecord(fp.cnt[b.slot], s), "event");
    SML_CUDA(cudaEventRecord(fp.comp[b.slot], s), "event");
    if (wait_fin.slot >= 0 && (rr = finish(wait_fin))) return rr;
    wait_fin = b;
    return SML_OK;
  };
  for (long long k = 0;; ++k) {
    const uint16_t* hp = nullptr;
    int nf = 0;
    long long first = 0;
    if ((r = sml_reader_next(fp.reader, &hp, &nf, &first, 60000)))
      return fail(ctx, r, "reading %s failed or timed out", path);
    if (nf == 0) break;
    const int slot = (int)(k & 1);
    // the slot's previous batch (k - 2) has been localized before its frames are replaced
    if (k >= 2) SML_CUDA(cudaStreamWaitEvent(fp.copy, fp.comp[slot], 0), "wait compute");
    // the copy stream is in order: this H2D follows the D2H that last read d_rec[slot]
    SML_CUDA(cudaMemcpyAsync(d_frames[slot] + (ctx3 ? hw : 0), hp, (size_t)nf * hw * sizeof(uint16_t),
                             cudaMemcpyHostToDevice, fp.copy),
             "H2D frames");
    if (ctx3 && wait_comp.slot >= 0) {  // context frames between this batch and the previous one
      uint16_t* prev = d_frames[wait_comp.slot];
      SML_CUDA(cudaMemcpyAsync(d_frames[slot], prev + (size_t)wait_comp.nf * hw, hw * sizeof(uint16_t),
                               cudaMemcpyDeviceToDevice, fp.copy),
               "context frame");
      SML_CUDA(cudaMemcpyAsync(prev + (size_t)(wait_comp.nf + 1) * hw, d_frames[slot] + hw, hw * sizeof(uint16_t),
                               cudaMemcpyDeviceToDevice, fp.copy),
               "context frame");
    }
    SML_CUDA(cudaEventRecord(fp.h2d[slot], fp.copy), "event");
    Batch b;
    b.slot = slot;
    b.nf = nf;
    b.k = k;
    b.first = first;
    b.host = hp;
    if (!ctx3) {
      if ((r = compute(b, false))) return r;
      continue;
    }
    if (wait_comp.slot >= 0) {
      // its tail frame came with this batch's copies (later on the copy stream)
      SML_CUDA(cudaStreamWaitEvent(s, fp.h2d[slot], 0), "wait context");
      if ((r = compute(wait_comp, true))) return r;
    }
    wait_comp = b;
  }
  if (ctx3 && wait_comp.slot >= 0 && (r = compute(wait_comp, false))) return r;
  if (wait_fin.slot >= 0 && (r = finish(wait_fin))) return r;
  SML_CUDA(cudaStreamSynchronize(fp.copy), "D2H records");
  SML_CUDA(cudaStreamSynchronize(s), "localize");
  if ((r = check_device_error(ctx))) return r;
  for (const Done& d : done)  // frame index within the batch -> index in the stack
    for (size_t i = d.at; i < d.at + d.n; ++i) out[i].frame += (int32_t)d.first;
  if (stats) {
    sml_reader_stats(fp.reader, stats);
    stats->wall_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    stats->frames = T;
  }
  *n_out = total;
  if (total > capacity) return fail(ctx, SML_ERR_CAPACITY, "%zu detections exceed capacity %zu", total, capacity);
  return SML_OK;
}

