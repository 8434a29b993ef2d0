/*
 * sml.h -- C ABI of the GB300 single-molecule localization library.
 *
 * The library runs the hot path of the DilatedLoc-style method on one GPU: a stack of
 * dilated 3x3 convolutions (dilated convolution, Sec. 3.2.1) over uint16 camera frames,
 * DECODE-style per-pixel output heads (probability p and sub-pixel offsets, Sec. 3.2),
 * and the post-processing of those maps into a list of localizations on the device
 * (Sec. 2.2: post-processing kept in GPU memory; Sec. 4.2.1: post-processing cost).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Return value: SML_OK (0) or a negative SML_ERR_* code.  sml_last_error() gives a
 *    one-line message for the most recent failure of a context (or of sml_create when
 *    called with NULL).
 *  - Frames are uint16 ADU, layout [T][H][W] (row-major, W fastest).  1 <= H, W <= 16384.
 *  - The camera transform is e = (adu - offset) / gain (photo-electrons), and the network
 *    input is e * in_scale (in_scale from the net spec).
 *  - Pixel (i, j) covers [j-1/2, j+1/2) x [i-1/2, i+1/2): its centre is the integer index.
 *    x and y are reported in pixels, z in nm (z_scale * zhat), photons in e- (ph_scale * Nhat).
 *  - A pixel is a detection iff p > p_min, p > p of every in-frame 8-neighbour that comes
 *    earlier in raster order and p >= p of every in-frame 8-neighbour that comes later.
 *    Records are ordered by (frame, row, column); results are deterministic and do not
 *    depend on batch composition or chunking.
 *  - A context is bound to the CUDA device that was current at sml_create.  It is not
 *    thread safe: use one context per host thread.
 *  - No entry point falls back to the CPU.  Without a usable sm_103 device, sml_create
 *    fails with SML_ERR_CUDA.
 */
#ifndef SML_H
#define SML_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SML_OK 0
#define SML_ERR_BAD_ARG -1     /* a NULL pointer, a size out of range, a bad threshold */
#define SML_ERR_BAD_SPEC -2    /* the JSON net spec is malformed or unsupported */
#define SML_ERR_BAD_WEIGHTS -3 /* the weight blob is malformed or does not match the spec */
#define SML_ERR_OOM -4         /* a device or pinned-host allocation failed */
#define SML_ERR_CUDA -5        /* a CUDA runtime or driver call failed */
#define SML_ERR_CAPACITY -6    /* more detections than the output capacity (see below) */
#define SML_ERR_UNSUPPORTED -7 /* valid request the build does not support */

typedef struct sml_ctx sml_ctx;

/* One localization, 24 bytes.  frame is the index within the T frames of the call. */
typedef struct {
  int32_t frame;
  float x, y;    /* pixels */
  float z;       /* nm */
  float photons; /* photo-electrons */
  float p;       /* detection probability at the peak pixel */
} sml_record;

/* Uncertainties of one detection (nets with the four uncertainty heads, Sec. 3.2): the
 * predicted standard deviations of x and y (pixels), z (nm) and photons (e-), read at the
 * detection's pixel: sigma_x = sx, sigma_y = sy, sigma_z = z_scale * sz,
 * sigma_photons = ph_scale * sN, each one float32 rounding. */
typedef struct {
  float sigma_x, sigma_y; /* pixels */
  float sigma_z;          /* nm */
  float sigma_photons;    /* photo-electrons */
} sml_sigma;

/* Camera model.  If gain_map / offset_map are non-NULL they hold per-pixel values [H][W]
 * (float32) and override the scalars.  Their memory space must match the call: host or
 * device for sml_localize, device for the *_async entry points. */
typedef struct {
  float gain;   /* ADU per photo-electron, > 0 */
  float offset; /* ADU */
  const float* gain_map;
  const float* offset_map;
} sml_camera;

typedef struct {
  float p_min; /* detection threshold on p, in [0, 1) */
} sml_thresholds;

/*
 * sml_create -- parse a net spec and a weight blob and upload the network.
 *
 * net_spec: NUL-terminated JSON object, e.g.
 *   {"in_ch":1,"channels":48,"dilations":[1,2,4,8,16,8,4,1],"precision":"bf16",
 *    "in_scale":0.001,"z_scale":1000,"ph_scale":10000}
 *   in_ch 1 (one frame per output frame) or 3 (frames t-1, t, t+1 as the first layer's
 *   input channels, the three-frame temporal context of Sec. 3.1; zero where t-1 or t+1 lies
 *   outside the frames of the call; chunk edges inside a call read the neighbouring frames);
 *   channels in {16,32,48,64}; 2..32 layers with dilations 1..64;
 *   "heads": 5 names (p, dx, dy, z, N: probability logit, sub-pixel offsets, zhat, Nhat) or
 *   9 (those and the uncertainty heads sx, sy, sz, sN, Sec. 3.2; each sigma map is
 *   softplus(h) = log(1 + exp(h)) of its raw head); default 5;
 *   "dcd": dense connection dilated blocks (Sec. 3.2.1), {"growth": g, "blocks": [[d, ...],
 *   ...]} with g in {16,32,48,64}: a stem conv (dilations[0], in_ch -> C), per block one
 *   dense layer per listed dilation (input: the block input and every earlier output of the
 *   block, concatenated; g outputs) and a transition (d = 1, C + k g -> C), then the plain
 *   layers dilations[1:] (at least one); concatenations up to 128 channels, at most 32 conv
 *   layers (SML_ERR_UNSUPPORTED for a layer whose weights do not fit one CTA's shared
 *   memory);
 *   precision "fp32" (SIMT FP32 FMA), "bf16" (tensor cores, FP32 accumulation) or
 *   "fp8" (e4m3 activations and weights, FP32 accumulation; needs "act_scales": one
 *   positive float per conv layer in execution order, act_scales[l] for l >= 1 being the
 *   scale of the activations layer l-1 stores (act_scales[0] is unused); layer l stores
 *   e4m3(a / act_scales[l+1]); weights are rounded per output channel, w / s[co] with
 *   s[co] = max |w[co,:,:,:]| / 448; in nets with dense blocks or a U-Net, whose layers read
 *   channels stored by several layers, each weight is first multiplied by the scale of its
 *   input channel and s[co] is taken over those products).
 *   Optional tuning: "chunk_px": pixels per device chunk (default 2^24); "tc_stages": TMA
 *   ring depth of the tensor-core conv (0 = as deep as shared memory allows, else 4..16);
 *   "fp8_pair_rows": 1 (default) loads FP8 activations of even-width frames as 32-byte pixel
 *   pairs, 0 as 16-byte rows (the same bytes land in shared memory; results are identical).
 *   Failure-path tests only: "debug_poison_cta": c makes CTA c of every tensor-core conv
 *   launch load no data, so that its waits run out after "debug_wait_ns" (1e6..2e9)
 *   nanoseconds and the call reports SML_ERR_CUDA (the kernels' give-up path, with no copy of
 *   that CTA in flight).
 * weights: an SMLW blob (host memory, read during the call only):
 *   header "<8s7I16i": magic "SMLW0001", version 1, L, C, in_ch, n_heads (5 or 9), has_bn,
 *   reserved, dilations[16]; then per layer l: W[C][Cin_l][3][3] f32, b[C] f32 and, if
 *   has_bn, gamma[C], beta[C], mean[C], var[C] f32 and eps f32; then the heads
 *   Wh[n_heads][C] f32 and bh[n_heads] f32 (head order: p logit, dx, dy, zhat, Nhat, then
 *   sx, sy, sz, sN).  BatchNorm is folded into the conv weights here.
 *   Nets with dense blocks or a U-Net, and plain stacks of more than 16 layers, use version 2:
 *   header "<8s7I32i" with reserved = growth (0 without dense blocks) and the 32 dilations of
 *   every conv layer in execution order; layer l's W is [Cout_l][Cin_l][3][3]
 *   with the channel counts of the dcd plan; no BatchNorm.
 * out: receives the context (owned by the caller, freed with sml_destroy).
 * Errors: SML_ERR_BAD_SPEC, SML_ERR_BAD_WEIGHTS, SML_ERR_UNSUPPORTED, SML_ERR_OOM, SML_ERR_CUDA.
 * The spec and the blob are checked on the host before any device call.
 */
int sml_create(const char* net_spec, const void* weights, size_t weights_bytes, sml_ctx** out);

/* Release every device and host resource of the context.  NULL is ignored. */
void sml_destroy(sml_ctx* ctx);

/* Message for the last failure of ctx (or of sml_create if ctx is NULL).  Owned by the
 * library, valid until the next call on the same context. */
const char* sml_last_error(const sml_ctx* ctx);

/*
 * sml_localize -- frames in, localizations out; synchronous.
 *
 * frames: [T][H][W] uint16, host (pageable or pinned) or device memory (detected).
 * cam, thr: host structs; the camera maps may be host or device pointers.
 * out: host or device array of capacity records (detected).  n_out: host.
 * Work is split into chunks of whole frames; records keep (frame, row, column) order.
 * On SML_OK, *n_out records were written.  If the detections exceed capacity, the call
 * returns SML_ERR_CAPACITY, sets *n_out to the number needed and leaves out unspecified.
 * T = 0 is valid and yields *n_out = 0.
 */
int sml_localize(sml_ctx* ctx, const uint16_t* frames, int T, int H, int W, const sml_camera* cam,
                 const sml_thresholds* thr, sml_record* out, size_t capacity, size_t* n_out);

/* Number of output heads of the context's net: 5, or 9 with the uncertainty heads. */
int sml_num_heads(const sml_ctx* ctx);

/* Number of conv layers of the context's net in execution order (the length of an fp8 net
 * spec's "act_scales"; dense blocks and a U-Net add their layers to the spec's dilations). */
int sml_num_layers(const sml_ctx* ctx);

/*
 * sml_workspace_bytes -- device memory of the context's per-frame-size workspace ("plan":
 * activation buffers of one chunk, maps, decode scratch, staging of host frames and camera
 * maps).  A call on T frames of H x W uses a plan whose chunk holds min(T, chunk_px / (H W))
 * frames (at least one): it keeps the plan of that frame size if its chunk is at least that
 * large, and otherwise allocates one (freeing a smaller plan of the size, and the least
 * recently used plan when it holds 4 sizes, each after its last call's work on that call's
 * stream).  Host only, no device call.
 * plan_bytes (or NULL): bytes of the plan a call on T frames of H x W uses; plan_resident (or
 * NULL): 1 if the context holds it now (no allocation), else 0; resident_bytes (or NULL):
 * bytes of all plans the context holds.  Weights and the per-call record staging of host
 * outputs are not counted.  Errors: SML_ERR_BAD_ARG.
 */
int sml_workspace_bytes(const sml_ctx* ctx, int T, int H, int W, size_t* plan_bytes, int* plan_resident,
                        size_t* resident_bytes);

/*
 * sml_error_word -- the stream-ordered status of the context's asynchronous work.  Every
 * mbarrier wait of the tensor-core conv kernels is bounded (2 s); a kernel that gives up sets
 * the context's device error word and returns early, leaving its outputs incomplete.  The
 * synchronous calls check the word and fail with SML_ERR_CUDA; sml_localize_async,
 * sml_forward_maps and sml_decode_maps cannot.  This call enqueues on `stream`, after the work
 * already enqueued there, a copy of the word into d_word (device int: 0 = every kernel of the
 * context finished its work, nonzero = one gave up) and clears the word.  Call it after the
 * asynchronous calls whose results are about to be used, on their stream.
 * Errors: SML_ERR_BAD_ARG, SML_ERR_CUDA.
 */
int sml_error_word(sml_ctx* ctx, int* d_word, void* stream);

/*
 * sml_localize_sigma -- sml_localize plus the uncertainties of every detection, for nets
 * with 9 heads: out_sigma[k] belongs to out[k].  out_sigma is host or device memory
 * (detected) of capacity entries.  Capacity and errors as in sml_localize; a 5-head net
 * returns SML_ERR_UNSUPPORTED.
 */
int sml_localize_sigma(sml_ctx* ctx, const uint16_t* frames, int T, int H, int W, const sml_camera* cam,
                       const sml_thresholds* thr, sml_record* out, sml_sigma* out_sigma, size_t capacity,
                       size_t* n_out);

/*
 * sml_localize_async -- device-resident variant, stream ordered, no host synchronisation.
 *
 * d_frames: device [T][H][W] uint16.  cam maps (if any) are device pointers.
 * d_out: device array of capacity records.  d_n_out: device uint64, overwritten with the
 * number of detections (records beyond capacity are not written; compare on the host).
 * stream: a cudaStream_t (NULL = the legacy default stream).  Every buffer must stay valid
 * until the stream reaches the end of this call's work.  One call at a time per context:
 * calls on different streams that overlap on the GPU would share the context's workspace.
 */
int sml_localize_async(sml_ctx* ctx, const uint16_t* d_frames, int T, int H, int W, const sml_camera* cam,
                       const sml_thresholds* thr, sml_record* d_out, size_t capacity,
                       unsigned long long* d_n_out, void* stream);

/*
 * sml_forward_maps -- the network alone (no decode), device-resident, stream ordered.
 *
 * d_maps: device float32 [T][n_heads][H][W] (n_heads = sml_num_heads): channel 0 = p =
 * sigmoid(logit), channels 1..4 = dx, dy, zhat, Nhat (raw head outputs), channels 5..8 (9-head
 * nets) = softplus of the uncertainty heads sx, sy, sz, sN.  d_logits: device float32
 * [T][H][W] or NULL.
 * These are exactly the maps that sml_localize decodes.
 */
int sml_forward_maps(sml_ctx* ctx, const uint16_t* d_frames, int T, int H, int W, const sml_camera* cam,
                     float* d_maps, float* d_logits, void* stream);

/*
 * sml_decode_maps -- decode caller-supplied maps [T][n_heads][H][W] (device float32, layout
 * of sml_forward_maps) into records, stream ordered; the decode half of sml_localize.
 * z_scale and ph_scale come from the context's net spec.  d_out / d_n_out as in
 * sml_localize_async.
 */
int sml_decode_maps(sml_ctx* ctx, const float* d_maps, int T, int H, int W, const sml_thresholds* thr,
                    sml_record* d_out, size_t capacity, unsigned long long* d_n_out, void* stream);

/*
 * sml_activation_amax -- calibration for the "fp8" precision.  Runs the network of an fp32 or
 * bf16 context over d_frames (device [T][H][W] uint16, camera as in sml_localize with device
 * maps) and writes to amax (host float[L]): amax[l], l = 1..L-1, is the largest activation
 * that layer l-1 stores (its ReLU output, over its output channels; for a plain stack the
 * input of layer l); amax[0] = 0.  An fp8 net spec then uses act_scales[l] = amax[l] / 448
 * (the largest finite e4m3 value).  Synchronous.
 * Errors: SML_ERR_UNSUPPORTED on an fp8 context, SML_ERR_BAD_ARG, SML_ERR_CUDA.
 */
int sml_activation_amax(sml_ctx* ctx, const uint16_t* d_frames, int T, int H, int W, const sml_camera* cam,
                        float* amax);

/*
 * sml_calibrate_fp8 -- activation scales for the "fp8" precision (per-layer activation scale,
 * per-output-channel weight scales).  Runs sml_activation_amax on an fp32 or bf16 context of
 * the net over the calibration frames (d_frames: device [T][H][W] uint16, T >= 1; camera as in
 * sml_activation_amax) and writes to act_scales (host float[L], L = the net's conv layers):
 * act_scales[0] = 1 (layer 0 reads the frames) and, for l >= 1,
 * act_scales[l] = max(amax[l], 1e-6) * margin / 448 (448 = the largest finite e4m3 value;
 * margin > 0 leaves headroom above the calibration maximum, 1 = none), in float32.  These
 * are the "act_scales" of an fp8 net spec of the same net.  Synchronous.
 * Errors: SML_ERR_BAD_ARG (T < 1, margin <= 0), and those of sml_activation_amax.
 */
int sml_calibrate_fp8(sml_ctx* ctx, const uint16_t* d_frames, int T, int H, int W, const sml_camera* cam,
                      float margin, float* act_scales);

/*
 * sml_decode_maps_static -- the decode of sml_decode_maps for callers that cannot allocate
 * device memory.  This entry point has no counterpart in the paper; it exists for callers
 * that must not call cudaMalloc/cudaFree while they run: an acquisition loop sharing the GPU
 * with a live camera stream (cudaFree synchronises the whole device), or a plugin whose host
 * application keeps all device memory in its own pool.  It needs no context and allocates
 * nothing; the caller passes the maps, the output records and the count.
 *
 * d_maps: device float32 [T][5][H][W] in the layout of sml_forward_maps.  z_scale, ph_scale:
 * the readout scales (z = z_scale*zhat, photons = ph_scale*Nhat).  d_out, capacity, d_n_out
 * and stream as in sml_decode_maps; *d_n_out is zeroed, then set to the detection count.
 * Records are identical to those of sml_decode_maps on the same maps.
 *
 * Scratch: a fixed array of 192 KiB in device global memory, declared in the library and
 * kept by every GPU that loads it until the process exits.  It bounds a call to
 * T*H*W <= 16,777,216 pixels (e.g. 256 frames of 256 x 256); larger calls return
 * SML_ERR_UNSUPPORTED without touching any buffer.  The first call on a device looks up the
 * array's device address (with that device current); make that first call before any stream
 * capture.  A call in a new CUDA context of the device (after cudaDeviceReset, for instance)
 * looks the address up again; make that call before any capture too.  All calls share the array: calls whose work overlaps on the GPU (other streams,
 * other host threads) race and must be serialised by the caller.
 * Errors: SML_ERR_BAD_ARG, SML_ERR_UNSUPPORTED, SML_ERR_CUDA.
 */
int sml_decode_maps_static(const float* d_maps, int T, int H, int W, float p_min, float z_scale, float ph_scale,
                           sml_record* d_out, size_t capacity, unsigned long long* d_n_out, void* stream);

/* Number of kernels the last localize / forward / decode call launched (for profiling). */
int sml_last_launch_count(const sml_ctx* ctx);

/*
 * Kernel timing.  sml_profile_enable(ctx, 1) clears the counters and makes every later call
 * bracket each kernel launch with a pair of CUDA events recorded on the launching stream;
 * sml_profile_enable(ctx, 0) stops recording.  sml_profile_read synchronises the recorded
 * events and returns, for one kernel class, the summed device time in milliseconds and the
 * number of timed launches since the last enable.  Classes: SML_KERNEL_LAYER1 (camera
 * transform + first conv), SML_KERNEL_CONV (middle dilated conv layers), SML_KERNEL_CONV_HEADS
 * (last conv layer with the fused heads), SML_KERNEL_DECODE (count + scan + write, timed as
 * one interval).  Timing adds one event pair per launch; leave it off outside profiling.
 */
#define SML_KERNEL_LAYER1 0
#define SML_KERNEL_CONV 1
#define SML_KERNEL_CONV_HEADS 2
#define SML_KERNEL_DECODE 3
int sml_profile_enable(sml_ctx* ctx, int on);
int sml_profile_read(sml_ctx* ctx, int kernel_class, double* total_ms, int* launches);

#ifdef __cplusplus
}
#endif

#endif /* SML_H */
