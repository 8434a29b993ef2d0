/*
 * sml_train.h -- training entry points of the GB300 localization library.
 *
 * Hand-written forward and backward kernels for training the dilated-conv localization
 * network on simulated frames (dilated convolution, Sec. 3.2.1; per-pixel heads, Sec. 3.2;
 * loss = binary cross-entropy on p, Sec. 3.3, plus a masked L2 on the dx, dy, z and photon
 * heads).  FP32 arithmetic, NHWC activations [B][H][W][C], PyTorch weight layout
 * [Cout][Cin][3][3].  Every pointer is device memory; every call is stream ordered and
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

#ifdef __cplusplus
}
#endif

#endif
