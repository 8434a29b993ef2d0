/*
 * CPU oracle for the dilated-convolution localization path (test infrastructure).
 *
 * This file is test infrastructure: only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline leg may load it.  It shares no code, header or table with the CUDA
 * library; the two only see the same seeded inputs.
 *
 * It is the plain definition of what the path computes, written slowly and directly:
 *   - forward of the plain dilated 3x3 stack (dilated convolution, Sec. 3.2.1) with
 *     "same" zero padding at every layer, optional BatchNorm applied unfolded, ReLU,
 *     then 1x1 heads (per-pixel probability and offsets, DECODE-style outputs, Sec. 3.2;
 *     optionally the four uncertainty heads, activated by softplus), all in float64;
 *   - the decode of per-pixel maps into a localization list (post-processing of
 *     Sec. 2.2 / Sec. 4.2.1), in float32 with every operation rounded once
 *     (compiled with -ffp-contract=off);
 *   - the training loss (binary cross-entropy on p, Sec. 3.3, plus a masked L2 on the
 *     offset / z / photon heads) and its exact gradient by reverse accumulation, float64.
 *
 * OpenMP splits the outer loops over independent outputs; it never changes the order in
 * which any single output is summed.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NH 5 /* heads: logit p, dx, dy, z, photons */

typedef struct {
  int32_t frame;
  float x, y, z, photons, p;
} orc_record; /* 24 bytes */

typedef struct {
  float sx, sy, sz, sN; /* uncertainties of x, y (px), z (nm), photons */
} orc_sigma;

/* ------------------------------------------------------------------ rounding to narrow formats */

/* float32 -> bfloat16 (8 significant bits), round to nearest, ties to even; returned as double. */
double orc_round_bf16(double v) {
  float f = (float)v;
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (double)f; /* inf / nan unchanged */
  uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  u &= 0xffff0000u;
  memcpy(&f, &u, 4);
  return (double)f;
}

/* float32 -> e4m3 (1 sign, 4 exponent bits with bias 7, 3 mantissa bits, no infinities;
 * largest finite 448, smallest normal 2^-6, subnormal spacing 2^-9), round to nearest even,
 * values beyond the largest finite saturate to +-448.  Returned as double. */
double orc_round_e4m3(double v) {
  float f = (float)v;
  double a = fabs((double)f);
  if (a != a) return (double)f;
  double sgn = f < 0 ? -1.0 : 1.0;
  if (a >= 448.0) return sgn * 448.0;
  int e;
  frexp(a, &e); /* a = m * 2^e, m in [0.5, 1) */
  int ex = e - 1; /* a in [2^ex, 2^(ex+1)) */
  if (ex < -6) ex = -6; /* subnormal range shares the spacing of the smallest binade */
  double spacing = ldexp(1.0, ex - 3);
  double q = nearbyint(a / spacing) * spacing; /* default rounding mode: ties to even */
  if (q > 448.0) q = 448.0;
  return sgn * q;
}

/* Round activations the way the tensor-core path stores them: quant 1 = bf16,
 * quant 2 = e4m3 of a / scale (then multiplied back by scale). */
static void round_acts(double* a, size_t n, int quant, double scale) {
  if (quant == 1)
    for (size_t k = 0; k < n; ++k) a[k] = orc_round_bf16(a[k]);
  else if (quant == 2) {
    float inv = (float)(1.0 / scale);
    for (size_t k = 0; k < n; ++k) a[k] = orc_round_e4m3((double)((float)a[k] * inv)) * scale;
  }
}

/* Round every element of a (fmt 1 = bf16, 2 = e4m3) in place. */
void orc_round_array(double* a, size_t n, int fmt) {
  for (size_t k = 0; k < n; ++k) a[k] = fmt == 1 ? orc_round_bf16(a[k]) : orc_round_e4m3(a[k]);
}

/* ------------------------------------------------------------------ helpers */

static size_t conv_w_count(int layer, int in_ch, int C) {
  return (size_t)C * (size_t)(layer == 0 ? in_ch : C) * 9u;
}

static size_t conv_w_offset(int layer, int in_ch, int C) {
  size_t off = 0;
  for (int l = 0; l < layer; ++l) off += conv_w_count(l, in_ch, C);
  return off;
}

/* ADU -> electrons -> network input: x = (adu - offset) / gain * in_scale. */
void orc_ingest(const uint16_t* frames, int T, int H, int W, const double* gain_map,
                const double* offset_map, double gain, double offset, double in_scale,
                double* x0 /* [T,H,W] */) {
  for (int t = 0; t < T; ++t)
    for (int i = 0; i < H; ++i)
      for (int j = 0; j < W; ++j) {
        size_t px = (size_t)i * W + j;
        double g = gain_map ? gain_map[px] : gain;
        double o = offset_map ? offset_map[px] : offset;
        double adu = (double)frames[(size_t)t * H * W + px];
        x0[(size_t)t * H * W + px] = (adu - o) / g * in_scale;
      }
}

/*
 * One dilated 3x3 conv layer on one frame, planar layout [c][i][j]:
 *   z[co,i,j] = b[co] + sum_{ci,ky,kx} w[co,ci,ky,kx] * a[ci, i+(ky-1)d, j+(kx-1)d]
 * with a = 0 outside the frame.  Optional BN (gamma, beta, mean, var rows of bn[4][Cout])
 * is applied to z before the ReLU.  pre (optional) receives z after BN, out gets ReLU(z).
 */
static void conv_layer(const double* a, int cin, int H, int W, const double* w, const double* b,
                       const double* bn, double eps, int cout, int d, double* pre, double* out) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int co = 0; co < cout; ++co)
    for (int i = 0; i < H; ++i)
      for (int j = 0; j < W; ++j) {
        double s = b[co];
        for (int ci = 0; ci < cin; ++ci)
          for (int ky = 0; ky < 3; ++ky) {
            int ii = i + (ky - 1) * d;
            if (ii < 0 || ii >= H) continue;
            for (int kx = 0; kx < 3; ++kx) {
              int jj = j + (kx - 1) * d;
              if (jj < 0 || jj >= W) continue;
              s += w[((size_t)co * cin + ci) * 9 + ky * 3 + kx] * a[((size_t)ci * H + ii) * W + jj];
            }
          }
        if (bn) {
          double g = bn[co], be = bn[cout + co], mu = bn[2 * cout + co], var = bn[3 * cout + co];
          s = g * (s - mu) / sqrt(var + eps) + be;
        }
        size_t o = ((size_t)co * H + i) * W + j;
        if (pre) pre[o] = s;
        out[o] = s > 0.0 ? s : 0.0;
      }
}

/*
 * One conv layer (Sec. 3.2.1 dilated convolution, "same" zero padding, bias, ReLU) of one
 * frame: in [cin][H][W] -> out [cout][H][W]; w [cout][cin][3][3], b [cout].  The forward of
 * nets with dense connection dilated blocks (Sec. 3.2.1) is this layer applied to channel
 * ranges of concatenated buffers (oracle/__init__.py).
 */
void orc_conv(const double* in, int cin, int H, int W, const double* w, const double* b, int cout, int d, double* out) {
  conv_layer(in, cin, H, W, w, b, NULL, 0.0, cout, d, NULL, out);
}

/*
 * Forward of the stack on network inputs x0 [T, in_ch, H, W] (float64).
 *   conv_w: concatenated per-layer [Cout][Cin][3][3]; conv_b: [L][C];
 *   bn: NULL or [L][4][C]; head_w [nh][C]; head_b [nh].
 *   heads out: [T,nh,H,W] raw head values (logit of p, dx, dy, z/z_scale, N/ph_scale, and with
 *   nh = 9 the four uncertainty heads).
 *   acts (optional): [T][L][C][H][W] post-ReLU activations of every layer.
 */
void orc_forward_xqh(const double* x0, int T, int H, int W, int L, int C, int in_ch, const int* dil,
                     const double* conv_w, const double* conv_b, const double* bn, double bn_eps, int nh,
                     const double* head_w, const double* head_b, double* heads, double* acts, int quant,
                     const double* act_scales) {
  size_t plane = (size_t)H * W;
  double* bufA = (double*)malloc(sizeof(double) * C * plane);
  double* bufB = (double*)malloc(sizeof(double) * C * plane);
  for (int t = 0; t < T; ++t) {
    const double* in = x0 + (size_t)t * in_ch * plane;
    int cin = in_ch;
    double* cur = bufA;
    for (int l = 0; l < L; ++l) {
      const double* w = conv_w + conv_w_offset(l, in_ch, C);
      const double* bnl = bn ? bn + (size_t)l * 4 * C : NULL;
      if (l > 0 && quant) round_acts((double*)in, (size_t)C * plane, quant, act_scales ? act_scales[l] : 1.0);
      conv_layer(in, cin, H, W, w, conv_b + (size_t)l * C, bnl, bn_eps, C, dil[l], NULL, cur);
      if (acts) memcpy(acts + ((size_t)t * L + l) * C * plane, cur, sizeof(double) * C * plane);
      in = cur;
      cin = C;
      cur = (cur == bufA) ? bufB : bufA;
    }
    /* 1x1 heads: h[k] = head_b[k] + sum_c head_w[k,c] * a_L[c] */
    for (int k = 0; k < nh; ++k)
      for (size_t px = 0; px < plane; ++px) {
        double s = head_b[k];
        for (int c = 0; c < C; ++c) s += head_w[(size_t)k * C + c] * in[(size_t)c * plane + px];
        heads[((size_t)t * nh + k) * plane + px] = s;
      }
  }
  free(bufA);
  free(bufB);
}

void orc_forward_xq(const double* x0, int T, int H, int W, int L, int C, int in_ch, const int* dil,
                    const double* conv_w, const double* conv_b, const double* bn, double bn_eps,
                    const double* head_w, const double* head_b, double* heads, double* acts, int quant,
                    const double* act_scales) {
  orc_forward_xqh(x0, T, H, W, L, C, in_ch, dil, conv_w, conv_b, bn, bn_eps, NH, head_w, head_b, heads, acts, quant,
                  act_scales);
}

void orc_forward_x(const double* x0, int T, int H, int W, int L, int C, int in_ch, const int* dil,
                   const double* conv_w, const double* conv_b, const double* bn, double bn_eps,
                   const double* head_w, const double* head_b, double* heads, double* acts) {
  orc_forward_xq(x0, T, H, W, L, C, in_ch, dil, conv_w, conv_b, bn, bn_eps, head_w, head_b, heads, acts, 0, NULL);
}

/* Ingest + forward from uint16 frames. */
void orc_forward(const uint16_t* frames, int T, int H, int W, const double* gain_map,
                 const double* offset_map, double gain, double offset, double in_scale, int L, int C,
                 const int* dil, const double* conv_w, const double* conv_b, const double* bn,
                 double bn_eps, const double* head_w, const double* head_b, double* heads) {
  double* x0 = (double*)malloc(sizeof(double) * (size_t)T * H * W);
  orc_ingest(frames, T, H, W, gain_map, offset_map, gain, offset, in_scale, x0);
  orc_forward_x(x0, T, H, W, L, C, 1, dil, conv_w, conv_b, bn, bn_eps, head_w, head_b, heads, NULL);
  free(x0);
}

/* p = 1 / (1 + exp(-logit)), float64. */
void orc_sigmoid(const double* h, size_t n, double* p) {
  for (size_t k = 0; k < n; ++k) p[k] = 1.0 / (1.0 + exp(-h[k]));
}

/* ------------------------------------------------------------------ decode (float32) */

/*
 * Decode per-pixel maps [T,nh,H,W] float32 (channel 0 = p, then dx, dy, zhat, Nhat; with
 * nh = 9 then the uncertainty maps sx, sy, sz, sN) into records ordered by (frame, row,
 * column).  Pixel (t,i,j) is kept iff
 *   p > p_min, and
 *   p > p[n] for each in-frame 8-neighbour n earlier in raster order, and
 *   p >= p[n] for each in-frame 8-neighbour n later in raster order.
 * Readout: x = j + dx, y = i + dy (pixels, centre of pixel = its index), z = z_scale*zhat,
 * photons = ph_scale*Nhat, p.  With sig (nh = 9): sigma_x = sx, sigma_y = sy,
 * sigma_z = z_scale*sz, sigma_photons = ph_scale*sN at the same pixel.  Each value is one
 * float32 operation.  Returns the number of detections; writes at most cap records.
 */
long orc_decode_h(const float* maps, int T, int nh, int H, int W, float p_min, float z_scale, float ph_scale,
                  orc_record* out, orc_sigma* sig, long cap) {
  long n = 0;
  size_t plane = (size_t)H * W;
  for (int t = 0; t < T; ++t) {
    const float* p = maps + (size_t)t * nh * plane;
    for (int i = 0; i < H; ++i)
      for (int j = 0; j < W; ++j) {
        float v = p[(size_t)i * W + j];
        if (!(v > p_min)) continue;
        int keep = 1;
        for (int di = -1; di <= 1 && keep; ++di)
          for (int dj = -1; dj <= 1; ++dj) {
            if (di == 0 && dj == 0) continue;
            int ii = i + di, jj = j + dj;
            if (ii < 0 || ii >= H || jj < 0 || jj >= W) continue;
            float q = p[(size_t)ii * W + jj];
            int earlier = (di < 0) || (di == 0 && dj < 0);
            if (earlier ? !(v > q) : !(v >= q)) {
              keep = 0;
              break;
            }
          }
        if (!keep) continue;
        if (n < cap) {
          size_t px = (size_t)i * W + j;
          orc_record r;
          r.frame = t;
          r.x = (float)j + maps[((size_t)t * nh + 1) * plane + px];
          r.y = (float)i + maps[((size_t)t * nh + 2) * plane + px];
          r.z = z_scale * maps[((size_t)t * nh + 3) * plane + px];
          r.photons = ph_scale * maps[((size_t)t * nh + 4) * plane + px];
          r.p = v;
          out[n] = r;
          if (sig && nh >= 9) {
            orc_sigma u;
            u.sx = maps[((size_t)t * nh + 5) * plane + px];
            u.sy = maps[((size_t)t * nh + 6) * plane + px];
            u.sz = z_scale * maps[((size_t)t * nh + 7) * plane + px];
            u.sN = ph_scale * maps[((size_t)t * nh + 8) * plane + px];
            sig[n] = u;
          }
        }
        ++n;
      }
  }
  return n;
}

long orc_decode(const float* maps, int T, int H, int W, float p_min, float z_scale, float ph_scale,
                orc_record* out, long cap) {
  return orc_decode_h(maps, T, NH, H, W, p_min, z_scale, ph_scale, out, NULL, cap);
}

/* Uncertainty-head activation: softplus(h) = log(1 + exp(h)), float64, in the form
 * max(h, 0) + log1p(exp(-|h|)) (the same value, without overflow of exp for large h). */
void orc_softplus(const double* h, size_t n, double* out) {
  for (size_t k = 0; k < n; ++k) {
    double a = fabs(h[k]);
    out[k] = (h[k] > 0 ? h[k] : 0.0) + log1p(exp(-a));
  }
}

/* ------------------------------------------------------------------ training loss + gradient */

/*
 * Loss on raw heads h [B,5,H,W] against targets y [B,5,H,W] (channel 0 in {0,1}):
 *   loss = (1/Npx) sum_px BCE(sigmoid(h0), y0)
 *        + (1/max(1,Nt)) sum_{px: y0=1} sum_{k=1..4} (h_k - y_k)^2
 * with BCE(p, y) = -(y log p + (1-y) log(1-p)) (Sec. 3.3), evaluated in its stable
 * logit form max(h,0) - h*y + log(1 + exp(-|h|)).  dh receives d loss / d h.
 */
double orc_loss(const double* h, const double* y, int B, int H, int W, double* dh) {
  size_t plane = (size_t)H * W;
  double npx = (double)B * plane;
  long nt = 0;
  for (int b = 0; b < B; ++b)
    for (size_t px = 0; px < plane; ++px) nt += y[((size_t)b * NH) * plane + px] > 0.5;
  double inv_nt = 1.0 / (nt > 0 ? (double)nt : 1.0);
  double bce = 0.0, l2 = 0.0;
  for (int b = 0; b < B; ++b)
    for (size_t px = 0; px < plane; ++px) {
      double h0 = h[((size_t)b * NH) * plane + px], y0 = y[((size_t)b * NH) * plane + px];
      bce += (h0 > 0 ? h0 : 0) - h0 * y0 + log1p(exp(-fabs(h0)));
      if (dh) dh[((size_t)b * NH) * plane + px] = (1.0 / (1.0 + exp(-h0)) - y0) / npx;
      int m = y0 > 0.5;
      for (int k = 1; k < NH; ++k) {
        size_t o = ((size_t)b * NH + k) * plane + px;
        double e = m ? h[o] - y[o] : 0.0;
        l2 += e * e;
        if (dh) dh[o] = 2.0 * e * inv_nt;
      }
    }
  return bce / npx + l2 * inv_nt;
}

/*
 * Gradient of orc_loss through heads and the conv stack (no BN: training uses plain
 * conv + bias), by reverse accumulation of the forward's definition:
 *   dZ_l = dA_l * [A_l > 0]
 *   dW_l[co,ci,ky,kx] = sum_px dZ_l[co,px] * A_{l-1}[ci, px + ((ky-1)d, (kx-1)d)]
 *   db_l[co] = sum_px dZ_l[co,px]
 *   dA_{l-1}[ci,q] = sum_{co,ky,kx} W_l[co,ci,ky,kx] * dZ_l[co, q - ((ky-1)d, (kx-1)d)]
 * Outputs are float64 with the same layouts as the parameters.  Returns the loss.
 */
double orc_loss_grad(const double* x0, const double* y, int B, int H, int W, int L, int C,
                     int in_ch, const int* dil, const double* conv_w, const double* conv_b,
                     const double* head_w, const double* head_b, double* g_conv_w, double* g_conv_b,
                     double* g_head_w, double* g_head_b, double* heads_out) {
  size_t plane = (size_t)H * W;
  size_t nw = conv_w_offset(L, in_ch, C);
  double* acts = (double*)malloc(sizeof(double) * (size_t)B * L * C * plane);
  double* h = (double*)malloc(sizeof(double) * (size_t)B * NH * plane);
  double* dh = (double*)malloc(sizeof(double) * (size_t)B * NH * plane);
  double* dA = (double*)malloc(sizeof(double) * C * plane);
  double* dZ = (double*)malloc(sizeof(double) * C * plane);
  orc_forward_x(x0, B, H, W, L, C, in_ch, dil, conv_w, conv_b, NULL, 0.0, head_w, head_b, h, acts);
  double loss = orc_loss(h, y, B, H, W, dh);
  if (heads_out) memcpy(heads_out, h, sizeof(double) * (size_t)B * NH * plane);
  memset(g_conv_w, 0, sizeof(double) * nw);
  memset(g_conv_b, 0, sizeof(double) * (size_t)L * C);
  memset(g_head_w, 0, sizeof(double) * NH * C);
  memset(g_head_b, 0, sizeof(double) * NH);
  for (int b = 0; b < B; ++b) {
    const double* aL = acts + ((size_t)b * L + (L - 1)) * C * plane;
    const double* dhb = dh + (size_t)b * NH * plane;
    for (int k = 0; k < NH; ++k)
      for (size_t px = 0; px < plane; ++px) {
        double g = dhb[(size_t)k * plane + px];
        g_head_b[k] += g;
        for (int c = 0; c < C; ++c) g_head_w[(size_t)k * C + c] += g * aL[(size_t)c * plane + px];
      }
    for (int c = 0; c < C; ++c)
      for (size_t px = 0; px < plane; ++px) {
        double s = 0.0;
        for (int k = 0; k < NH; ++k) s += head_w[(size_t)k * C + c] * dhb[(size_t)k * plane + px];
        dA[(size_t)c * plane + px] = s;
      }
    for (int l = L - 1; l >= 0; --l) {
      const double* al = acts + ((size_t)b * L + l) * C * plane;
      const double* ain = l > 0 ? acts + ((size_t)b * L + (l - 1)) * C * plane : x0 + (size_t)b * in_ch * plane;
      int cin = l > 0 ? C : in_ch, d = dil[l];
      const double* w = conv_w + conv_w_offset(l, in_ch, C);
      double* gw = g_conv_w + conv_w_offset(l, in_ch, C);
      for (size_t q = 0; q < (size_t)C * plane; ++q) dZ[q] = al[q] > 0.0 ? dA[q] : 0.0;
#pragma omp parallel for schedule(static)
      for (int co = 0; co < C; ++co) {
        double sb = 0.0;
        for (size_t px = 0; px < plane; ++px) sb += dZ[(size_t)co * plane + px];
        g_conv_b[(size_t)l * C + co] += sb;
        for (int ci = 0; ci < cin; ++ci)
          for (int ky = 0; ky < 3; ++ky)
            for (int kx = 0; kx < 3; ++kx) {
              double s = 0.0;
              for (int i = 0; i < H; ++i) {
                int ii = i + (ky - 1) * d;
                if (ii < 0 || ii >= H) continue;
                for (int j = 0; j < W; ++j) {
                  int jj = j + (kx - 1) * d;
                  if (jj < 0 || jj >= W) continue;
                  s += dZ[((size_t)co * H + i) * W + j] * ain[((size_t)ci * H + ii) * W + jj];
                }
              }
              gw[((size_t)co * cin + ci) * 9 + ky * 3 + kx] += s;
            }
      }
      if (l == 0) break;
#pragma omp parallel for collapse(2) schedule(static)
      for (int ci = 0; ci < C; ++ci)
        for (int i = 0; i < H; ++i)
          for (int j = 0; j < W; ++j) {
            double s = 0.0;
            for (int co = 0; co < C; ++co)
              for (int ky = 0; ky < 3; ++ky) {
                int oi = i - (ky - 1) * d;
                if (oi < 0 || oi >= H) continue;
                for (int kx = 0; kx < 3; ++kx) {
                  int oj = j - (kx - 1) * d;
                  if (oj < 0 || oj >= W) continue;
                  s += w[((size_t)co * C + ci) * 9 + ky * 3 + kx] * dZ[((size_t)co * H + oi) * W + oj];
                }
              }
            dA[((size_t)ci * H + i) * W + j] = s;
          }
    }
  }
  free(acts);
  free(h);
  free(dh);
  free(dA);
  free(dZ);
  return loss;
}
