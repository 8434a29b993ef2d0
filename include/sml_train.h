/*
 * sml_train.h -- training entry points of the GB300 localization library.
 *
 * Hand-written forward and backward kernels for training the dilated-conv localization
 * network on simulated frames (dilated convolution, Sec. 3.2.1; per-pixel heads, Sec. 3.2;
 * loss = binary cross-entropy on p, Sec. 3.3, plus a masked L2 on the dx, dy, z and photon
 * heads).  The calls before the BF16 section use FP32 arithmetic, NHWC activations
 * [B][H][W][C], PyTorch weight layout [Cout][Cin][3][3].  Every pointer is device memory
 * unless stated otherwise; every call is stream ordered and
 * returns SML_OK or SML_ERR_BAD_ARG / SML_ERR_CUDA (see sml.h).  Reductions over pixels are
 * deterministic (fixed block order).  Supported widths: Cin = Cout in {16,32,48,64}, or
 * Cin = 1 for the first layer.
 */
#ifndef SML_TRAIN_H
#define SML_TRAIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* x0[q] = (frames[q] - offset) / gain * in_scale for n = B*H*W uint16 pixels. */
int sml_train_ingest(const uint16_t* frames, long long n, float gain, float offset, float in_scale, float* x0,
                     void* stream);

/* y = ReLU(b + dilated_conv_d(x; w)) with "same" zero padding: x [B][H][W][cin],
 * w [cout][cin][3][3], b [cout], y [B][H][W][cout]. */
int sml_train_conv_fwd(const float* x, int B, int H, int W, int cin, int cout, int d, const float* w, const float* b,
                       float* y, void* stream);

/* Scratch bytes sml_train_conv_bwd needs for these sizes. */
size_t sml_train_conv_bwd_work_bytes(int B, int H, int W, int cin, int cout);

/* Backward of sml_train_conv_fwd.  dy = d loss / d y.  With dz = dy * [y > 0]:
 *   dx [B][H][W][cin] (may be NULL; must be NULL when cin = 1) = transposed dilated conv of dz;
 *   dw [cout][cin][3][3] = sum over pixels of dz x (overwritten); db [cout] = sum of dz.
 * work: caller scratch of sml_train_conv_bwd_work_bytes bytes (contents not preserved). */
int sml_train_conv_bwd(const float* x, const float* y, const float* dy, int B, int H, int W, int cin, int cout, int d,
                       const float* w, float* dx, float* dw, float* db, void* work, size_t work_bytes, void* stream);

/* Scratch bytes sml_train_heads_loss needs for these sizes. */
size_t sml_train_heads_work_bytes(int B, int H, int W, int C);

/* Heads, loss and head gradients.  a [B][H][W][C] (last conv layer output), targets
 * tgt [B][5][H][W] (channel 0 in {0,1}, channels 1..4 the dx, dy, zhat, Nhat targets).
 *   h [B][5][H][W] = hb + hw a (raw heads: logit, dx, dy, zhat, Nhat);
 *   loss (one float) = mean over pixels of BCE(sigmoid(h0), t0)
 *                      + sum over target pixels of sum_k (h_k - t_k)^2 / max(1, #targets).
 * If da is non-NULL the gradients of (*grad_scale) * loss are written too: da [B][H][W][C],
 * dhw [5][C], dhb [5] (grad_scale: one device float, e.g. the incoming gradient). */
int sml_train_heads_loss(const float* a, const float* tgt, int B, int H, int W, int C, const float* hw,
                         const float* hb, float* h, float* loss, const float* grad_scale, float* da, float* dhw,
                         float* dhb, void* work, size_t work_bytes, void* stream);

/*
 * ---------------------------------------------------------------------------------------
 * BF16 training on the tensor cores: BF16 activations, weights and activation gradients,
 * FP32 accumulation, FP32 weight and bias gradients (the caller keeps FP32 master weights).
 * Plain C -> C layers with C in {16, 32, 48} (the first layer 1 -> C; heads 5 x C, C up to 64).
 * Activations and activation gradients are row-planar bf16 tensors [B][H][C/16][W][16]
 * (16 channels of one pixel in 32 bytes, pixel rows of one 16-channel group contiguous),
 * the layout of the inference path's tensor-core layers.  Every conv layer is
 *   a_l = ReLU(b_l + dilated_conv_d(a_{l-1}; w_l)),  "same" zero padding (Sec. 3.2.1);
 * its gradient is carried as dz_l = d loss / d (pre-activation of layer l), i.e. with the
 * ReLU mask applied.  d_err: a caller-owned device int that a tensor-core kernel sets to
 * nonzero if one of its bounded waits (2 s) gave up (its outputs are then incomplete).
 * Every call is stream ordered; reductions are deterministic (fixed order).
 * ---------------------------------------------------------------------------------------
 */

/* Bytes of one packed bf16 B image of a C -> C layer (0 for unsupported C). */
size_t sml_train_bf16_bimg_bytes(int C);

/* Packs FP32 weights w [C][C][3][3] into the conv kernel's bf16 B images: bimg_fwd for the
 * forward, bimg_dgrad for the input gradient (weights mirrored in (ky, kx), in and out
 * channels swapped).  Call after every update of the master weights. */
int sml_train_bf16_pack(const float* w, int C, void* bimg_fwd, void* bimg_dgrad, void* stream);

/* First layer: camera transform of the uint16 frames [B][H][W] ((adu - offset) / gain *
 * in_scale), 3x3 conv 1 -> C at dilation d with w0 [C][1][3][3] and b0 [C] (device FP32),
 * ReLU, stored as bf16 row-planar a0. */
int sml_train_bf16_layer0(const uint16_t* frames, int B, int H, int W, float gain, float offset, float in_scale,
                          const float* w0, const float* b0, int C, int d, void* a0, void* stream);

/* Forward of a C -> C layer: y = ReLU(b + dilated_conv_d(x; w)), x and y row-planar bf16,
 * bimg_fwd from sml_train_bf16_pack, b device FP32 [C]. */
int sml_train_bf16_conv_fwd(const void* x, int B, int H, int W, int C, int d, const void* bimg_fwd, const float* b,
                            void* y, int* d_err, void* stream);

/* Input gradient of a C -> C layer: dz_in = (transposed dilated conv of dz with w) * [x > 0],
 * i.e. the pre-activation gradient of the layer below (x = that layer's ReLU output, this
 * layer's input).  dz, x, dz_in row-planar bf16; bimg_dgrad from sml_train_bf16_pack. */
int sml_train_bf16_conv_dgrad(const void* dz, const void* x, int B, int H, int W, int C, int d, const void* bimg_dgrad,
                              void* dz_in, int* d_err, void* stream);

/* Scratch bytes of sml_train_bf16_conv_wgrad on the current device. */
size_t sml_train_bf16_wgrad_work_bytes(int C);

/* Weight and bias gradient of a C -> C layer: dw [C][C][3][3] = sum over pixels of
 * dz[p][co] x[p + tap offset][ci] (overwritten), db [C] = sum of dz; x the layer's input and
 * dz its pre-activation gradient, both row-planar bf16.  work: sml_train_bf16_wgrad_work_bytes. */
int sml_train_bf16_conv_wgrad(const void* x, const void* dz, int B, int H, int W, int C, int d, float* dw, float* db,
                              void* work, size_t work_bytes, int* d_err, void* stream);

/* Heads, loss and head gradients as sml_train_heads_loss, from the last layer's row-planar
 * bf16 output a; if dz is non-NULL it receives (d ((*grad_scale) * loss) / d a) * [a > 0] as
 * row-planar bf16 (the last layer's pre-activation gradient), with dhw [5][C] and dhb [5].
 * work: sml_train_heads_work_bytes. */
int sml_train_bf16_heads_loss(const void* a, const float* tgt, int B, int H, int W, int C, const float* hw,
                              const float* hb, float* h, float* loss, const float* grad_scale, void* dz, float* dhw,
                              float* dhb, void* work, size_t work_bytes, void* stream);

/* Weight and bias gradient of the first layer: dw [C][1][3][3], db [C] from its FP32 input
 * x0 [B][H][W] (sml_train_ingest) and its pre-activation gradient dz0 (row-planar bf16, from
 * sml_train_bf16_conv_dgrad of the second layer).  work: sml_train_conv_bwd_work_bytes(B, H,
 * W, 1, C). */
int sml_train_bf16_l0_wgrad(const float* x0, const void* dz0, int B, int H, int W, int C, int d, float* dw, float* db,
                            void* work, size_t work_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif
