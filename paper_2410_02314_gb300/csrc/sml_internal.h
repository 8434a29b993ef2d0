// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sml.h"

namespace sml {

constexpr int kHeads = 5;     // position heads: p logit, dx, dy, zhat, Nhat (the training heads)
constexpr int kMaxHeads = 9;  // + the uncertainty heads sx, sy, sz, sN (Sec. 3.2)
constexpr int kMaxLayers = 32;  // conv layers of a net (plain stacks: 16)
constexpr int kTcMaxCin = 128;   // widest tensor-core conv input (8 groups of 16 channels)
constexpr int kTileM = 128;  // pixels per MMA tile (one row segment)

enum Precision { kFP32 = 0, kBF16 = 1, kFP8 = 2, kTF32 = 3 /* MMA operand kind of the self-test only */ };

// Decode parameters shared by the fused path and sml_decode_maps.
struct DecodeArgs {
  const float* maps;  // [Tc][5][H][W]
  int T, H, W;
  int frame0;  // frame index of the chunk's first frame
  float p_min, z_scale, ph_scale;
  sml_record* out;
  sml_sigma* out_sigma = nullptr;  // uncertainties of each record (9-head maps) or NULL
  int nh = kHeads;                 // channels of the maps: 5, or 9 with the uncertainty maps
  unsigned long long capacity;
  unsigned long long* total;  // running count (device); updated by the scan kernel
  unsigned int* block_counts;  // [nblocks]
  unsigned long long* block_offsets;  // [nblocks]
  // [nblocks][kDecodePxPerBlock / 32] detection ballots of the count pass, reused by the write
  // pass; NULL: the write pass evaluates the detections again
  unsigned int* flag_words = nullptr;
};

constexpr int kDecodeThreads = 256;
constexpr int kDecodePxPerBlock = 1024;

inline long long decode_blocks(long long npx) { return (npx + kDecodePxPerBlock - 1) / kDecodePxPerBlock; }

// Launchers (return cudaError_t of the launch).
cudaError_t launch_decode(const DecodeArgs& a, cudaStream_t s, int* launches);

// Camera parameters for the first layer (device pointers or NULL maps).
struct CamArgs {
  float gain, offset, in_scale;
  const float* gain_map;
  const float* offset_map;
};

#ifdef __CUDACC__
// Uncertainty-head activation: softplus(h) = log(1 + exp(h)), by its defining formula below
// h = 20 (where exp(h) is still far from overflow) and h itself above (the rest is < 2e-9 h).
__device__ __forceinline__ float softplus_f(float h) { return h > 20.0f ? h : log1pf(expf(h)); }

// Network input of one pixel from its ADU value and its camera offset and gain:
// (adu - offset) / gain * in_scale, each step one IEEE rounding.
__device__ __forceinline__ float cam_transform(float adu, float offset, float gain, float in_scale) {
  return __fmul_rn(__fdiv_rn(__fsub_rn(adu, offset), gain), in_scale);
}
#endif

// --- layer 1: camera transform + Cin=1 dilated 3x3 conv, bias, ReLU -------------------
// prec kFP32 writes float NHWC [T][H][W][out_ct] channels 0..C-1; kBF16 / kFP8 write row-planar
// activations [T][H][out_ct/16][W][row bytes] groups 0..C/16-1 (16 channels per group:
// 32-byte bf16 rows, 16-byte e4m3 rows).  out_ct = C except for nets with dense blocks, whose
// buffers hold the block's concatenation (out_ct > C, a multiple of 16).  out_scale
// multiplies the FP8 output before rounding (1 / activation scale).  w1 [C][in_ch][9] and
// b1 [C] are HOST pointers (the weights are passed to the kernel by value).  in_ch = 3 takes
// frames t-1, t, t+1 as the input channels; frames[k] exists for t_first <= k <= t_last
// (t_first in {-1, 0}, t_last in {T-1, T}) and is zero outside that range.
cudaError_t launch_ingest_l1(const uint16_t* frames, int T, int H, int W, int d, CamArgs cam, const float* w1,
                             const float* b1, int C, int in_ch, int t_first, int t_last, int prec, float out_scale,
                             void* out, int out_ct, cudaStream_t s);

// BF16 training: the same first layer (in_ch = 1, bf16 row-planar output with C channels)
// with w1 [C][1][9] and b1 [C] in DEVICE memory.
cudaError_t launch_ingest_l1_devw(const uint16_t* frames, int T, int H, int W, int d, CamArgs cam, const float* w1_dev,
                                  const float* b1_dev, int C, void* out, cudaStream_t s);

// Maximum of one layer's stored output: channels [off, off + cnt) of a buffer of ct channels
// per pixel holding T frames of H x W (atomicMax of the float bits into *out).
cudaError_t launch_amax(const void* x, int prec, int T, int H, int W, int ct, int off, int cnt, unsigned* out,
                        cudaStream_t s);

// --- SIMT FP32 path (NHWC float activations) ------------------------------------------
// Reads channels 0..ci-1 of pixels in_ct floats apart; writes channels out_off..out_off+co-1
// of pixels out_ct floats apart.  w [9][ci][co] (tap, ci, co), b [co] (device).
struct F32LayerArgs {
  const float* in;
  float* out;
  const float* w;
  const float* b;
  int T, H, W, d;
  int ci, co, in_ct, out_ct, out_off;
};
cudaError_t launch_dconv_f32(const F32LayerArgs& a, cudaStream_t s);
// Last layer (ci == co == C) with the fused heads.
cudaError_t launch_dconv_f32_heads(const F32LayerArgs& a, const float* hw, const float* hb, int nh, float* maps,
                                   float* logits, cudaStream_t s);
// Largest ci * co whose FP32 weights fit in shared memory.
constexpr int kF32MaxWeights = 227 * 1024 / (9 * 4);

// --- U-Net resolution changes (k_resample.cu) ------------------------------------------
// 2x2 max pool (stride 2, ceil: output ceil(H/2) x ceil(W/2)) of channels [0, C) of `in`
// ([T][H][W] pixels, in_ct channels each) into channels [out_off, out_off + C) of `out`
// (out_ct channels per pixel).  prec kFP32 (NHWC float, C, cts, offset multiples of 4) or
// kBF16 (row-planar, multiples of 16).
cudaError_t launch_pool2(const void* in, int in_ct, void* out, int out_ct, int out_off, int C, int T, int H, int W,
                         int prec, cudaStream_t s);
// Nearest 2x upsample of channels [0, C) of `in` (h x w, h = ceil(H/2), w = ceil(W/2)) into
// channels [out_off, out_off + C) of `out` (H x W): out(i, j) = in(i/2, j/2).
cudaError_t launch_upsample2(const void* in, int in_ct, int h, int w, void* out, int out_ct, int out_off, int C, int T,
                             int H, int W, int prec, cudaStream_t s);

// --- tensor-core path (row-planar activations) -------------------------------------
struct TcLayerArgs {
  const CUtensorMap* tmap;  // input activations, one box per row (5-D map for this dilation)
  int stages;               // TMA ring depth (0 = as many as shared memory allows)
  const void* bimg;         // device: packed B operand image for this layer
  const float* bias;        // HOST [co] (passed to the kernel by value)
  const float* deq;         // HOST [co] per-output-channel dequant factor (FP8) or NULL
  float out_inv_scale;      // FP8: 1 / scale of the output activations
  void* out;                // row-planar output activations (middle layers)
  int out_g0, out_gt;       // output: first group written, groups per pixel row of the buffer
  const float* head_w;      // last layer: HOST [nh][C]
  const float* head_b;      // last layer: HOST [nh]
  int nh;                   // last layer: heads (5, or 9 with the uncertainty heads)
  float* maps;              // last layer: [T][nh][H][W]
  float* logits;            // last layer: optional [T][H][W]
  int T, H, W, d, prec;
  int ci, co;               // input channels read (groups 0..ci/16-1 of the input buffer), outputs
  int* err;                 // device error word (wait timeouts)
  const float* bias_dev = nullptr;  // BF16 training: device bias [co], used instead of `bias`
  const void* mask = nullptr;       // input gradient: the lower layer's activations (layout of out)
  unsigned long long wait_ns = 0;   // failure-path tests: give-up time of the waits (0 = 2 s)
  int poison_cta = -1;              // failure-path tests: a CTA whose producer loads nothing
  int pair_rows = 0;                // FP8: the map loads 32-byte pixel pairs (even W; see encode_act_map)
};
cudaError_t launch_dconv_tc(const TcLayerArgs& a, bool last, int num_sms, cudaStream_t s);
// BF16 training, plain C -> C layers: the forward conv (bias from a.bias_dev) or, with dgrad,
// the input gradient dz_in = conv(dz; mirrored transposed weights) * [a.mask > 0] (no bias).
cudaError_t launch_dconv_tc_train(const TcLayerArgs& a, bool dgrad, int num_sms, cudaStream_t s);
size_t tc_bimg_bytes(int ci, int co, int prec);
void tc_pack_bimg(const float* w_tap_ci_co /*[9][ci][co]*/, int ci, int co, int prec, const float* w_scale, void* dst);
int tc_box_width(int d);
// Whether a ci -> co layer at dilation d fits the tensor-core conv's shared memory.
bool tc_layer_fits(int ci, int co, int d, int prec);

// --- BF16 training on the tensor cores (k_train_tc.cu) -----------------------------------
size_t train_wgrad_tc_work_bytes(int C, int num_sms);
// Box widths (pixels) of the weight gradient's dZ and X tensor maps for frames W wide.
void wgrad_tc_boxes(int W, int d, int* dz_px, int* x_px);
// FP32 w [cout][cin][3][3] -> bf16 B images of the conv: forward and mirrored-transposed (dgrad).
cudaError_t launch_pack_bimg_bf16(const float* w, int cin, int cout, void* fwd, void* dgrad, cudaStream_t s);
// dw [C][C][3][3], db [C] of a C -> C layer from dz (tm_dz: 128-pixel row boxes) and the
// layer input x (tm_x: the conv's row boxes for dilation d); partial: train_wgrad_tc_work_bytes.
cudaError_t launch_wgrad_tc(const CUtensorMap* tm_dz, const CUtensorMap* tm_x, int T, int H, int W, int C, int d,
                            float* partial, int num_sms, float* dw, float* db, int* err, cudaStream_t s);

// --- training (k_train.cu) -------------------------------------------------------------
size_t train_conv_work_bytes(int B, int H, int W, int cin, int cout);
size_t train_heads_work_bytes(int B, int H, int W, int C);
cudaError_t train_conv_fwd(const float* x, int B, int H, int W, int cin, int cout, int d, const float* w,
                           const float* b, float* y, cudaStream_t s);
cudaError_t train_conv_bwd(const float* x, const float* y, const float* dy, int B, int H, int W, int cin, int cout,
                           int d, const float* w, float* dx, float* dw, float* db, void* work, cudaStream_t s);
cudaError_t train_heads_loss(const float* a, const float* tgt, int B, int H, int W, int C, const float* hw,
                             const float* hb, float* h, float* loss, const float* gscale, float* da, float* dhw,
                             float* dhb, void* work, cudaStream_t s);
cudaError_t train_ingest(const uint16_t* f, long long n, float gain, float offset, float in_scale, float* x0,
                         cudaStream_t s);
// BF16 training: heads + loss from bf16 row-planar activations, writing dz (masked, bf16
// row-planar); first-layer weight gradient from bf16 row-planar dz0 and the fp32 input x0.
cudaError_t train_heads_loss_rp(const void* a, const float* tgt, int B, int H, int W, int C, const float* hw,
                                const float* hb, float* h, float* loss, const float* gscale, void* dz, float* dhw,
                                float* dhb, void* work, cudaStream_t s);
cudaError_t train_l0_wgrad_rp(const float* x0, const void* dz0, int B, int H, int W, int C, int d, float* dw,
                              float* db, void* work, cudaStream_t s);

// Debug: one 128 x N x K UMMA through the same descriptor helpers (exposed for tests).
cudaError_t launch_umma_selftest(const void* a, const void* b, float* d, int N, int K, int prec, int d_col, int* err,
                                 cudaStream_t s);
// Debug: one M x N x K product with both operands MN-major (32-byte-swizzled planes).
cudaError_t launch_umma_mn_selftest(const void* A, const void* B, float* D, int M, int N, int K, int a_bytes,
                                    int b_bytes, int a_plane, int b_plane, int b_shift, int* err, cudaStream_t s);

}  // namespace sml
