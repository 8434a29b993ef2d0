/*
 * sml_sim.h -- camera-frame simulator of the GB300 localization library.
 *
 * The paper evaluates on simulated single-molecule frames (Sec. 4.1) without giving the
 * simulator; this is the synthetic workloads' generator run on the device, so that large
 * stacks (thousands of 2048 x 2048 frames) can be made in place of the paper's datasets.
 *
 * Per frame t and pixel (i, j) (pixel (i, j) covers [j-1/2, j+1/2) x [i-1/2, i+1/2)):
 *   mu = bg[t] + sum over emitters e of frame t with |i - rint(y_e)| <= r and
 *        |j - rint(x_e)| <= r of  N_e * Ex_e(j) * Ey_e(i),
 *   Ex_e(j) = (erf((j + 1/2 - x_e) / (sqrt(2) sx_e)) - erf((j - 1/2 - x_e) / (sqrt(2) sx_e))) / 2
 *   (Ey likewise with y_e, sy_e), the pixel-integrated Gaussian PSF;
 *   sx = sy = sigma0, or with astig the astigmatic widths
 *   sx = sigma0 sqrt(1 + ((z + 400 nm) / 500 nm)^2), sy = sigma0 sqrt(1 + ((z - 400 nm) / 500 nm)^2);
 *   r = ceil(4 max(sx, sy) over the call's emitters) + 1 (the PSF window);
 *   e = Poisson(mu) (or e = mu with noise = 0);
 *   adu = rint(gain * e + offset) clamped to [0, 65535] (gain/offset scalars or [H][W] maps).
 * mu is computed in float32.  The Poisson draws of pixel q = ((frame0 + t) H + i) W + j use
 * the uniform numbers u_k = (S(q * 64 + k) >> 11) * 2^-53, k < 64, where S(m) is output m
 * (counting from 0) of splitmix64 seeded with `seed` (Vigna's generator: S(m) is the mix of
 * seed + (m + 1) * 0x9e3779b97f4a7c15): Knuth's multiplication method for mu < 12,
 * Hormann's transformed rejection with squeeze (PTRS, 1993) otherwise.
 */
#ifndef SML_SIM_H
#define SML_SIM_H

#include <stddef.h>
#include <stdint.h>

#include "sml.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * sml_sim_frames -- T frames of H x W (1 <= H, W <= 16384) into d_adu (device uint16
 * [T][H][W]) and, if d_mu is not NULL, the expected image mu (device float32 [T][H][W]).
 * Emitters: n entries of HOST arrays frame (int32, 0..T-1), x, y (px), z (nm; ignored
 * without astig), photons (e-); bg: HOST float32 [T] (e- per pixel).  cam: gain (> 0) and
 * offset, or device maps [H][W].  noise = 0 gives adu from mu without Poisson noise.
 * frame0: index of the call's first frame in its stack (the noise of a frame depends only
 * on seed, frame0 + t and the pixel).  Synchronous.  Errors: SML_ERR_BAD_ARG (sizes, frame
 * indices, NULL pointers, non-positive sigma0 or gain, 2^31 or more emitters or 16 x 16 tiles
 * in one call), SML_ERR_OOM, SML_ERR_CUDA.
 */
int sml_sim_frames(const int32_t* frame, const float* x, const float* y, const float* z, const float* photons,
                   long long n, const float* bg, int T, int H, int W, int astig, float sigma0, const sml_camera* cam,
                   unsigned long long seed, long long frame0, int noise, uint16_t* d_adu, float* d_mu);

#ifdef __cplusplus
}
#endif

#endif
